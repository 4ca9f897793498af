// Batching, graph replay and the lanes-per-cell autotuner.
//
// A batch is the disjoint union of several meshes: one mesh whose cells, faces and vertices are the
// meshes' own, renumbered with offsets. A step over the union processes the interface cells of all
// meshes in the same launches (cells binned by tetrahedron count, each bin with its own lanes per
// cell); per-mesh totals are pairwise trees over each mesh's contiguous segment of the interface
// list, the same tree a single-mesh step builds. vof_step_graph captures a whole step into a CUDA
// graph and replays it, so a step costs one graph launch on the host.
#include <algorithm>
#include <cstring>
#include <vector>

#include "vof_internal.cuh"

struct vof_batch {
  vof_mesh* mesh = nullptr;
  int n = 0;
  std::vector<int64_t> cell_off, face_off, vert_off;
  int64_t* d_cell_off = nullptr;
};

namespace vof {
namespace {

constexpr int kChunk = 2048;

__device__ double seg_tree(const double* x, int64_t lo, int64_t n, int64_t base, double* s) {
  // pairwise tree over the kChunk leaves x[lo + base ..), zeros past lo + n
  const int t = threadIdx.x;  // blockDim.x == kChunk / 2
  const int64_t i0 = base + 2 * t, i1 = i0 + 1;
  s[t] = (i0 < n ? x[lo + i0] : 0.0) + (i1 < n ? x[lo + i1] : 0.0);
  __syncthreads();
  for (int w = kChunk / 4; w > 0; w >>= 1) {
    double v = 0;
    if (t < w) v = s[2 * t] + s[2 * t + 1];
    __syncthreads();
    if (t < w) s[t] = v;
    __syncthreads();
  }
  const double r = s[0];
  __syncthreads();
  return r;
}

__device__ int64_t lower_bound(const int32_t* a, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One block per mesh: its interface cells form the segment [s, e) of the interface list.
__global__ void __launch_bounds__(kChunk / 2) k_totals_seg(Workspace W, const int64_t* cell_off, double* totals) {
  __shared__ double s[kChunk / 2];
  __shared__ double part[2][kChunk];
  __shared__ int64_t seg[2];
  const int m = blockIdx.x;
  const int64_t n_iface = W.counters->n_iface;
  if (threadIdx.x == 0) {
    seg[0] = lower_bound(W.iface_idx, n_iface, cell_off[m]);
    seg[1] = lower_bound(W.iface_idx, n_iface, cell_off[m + 1]);
  }
  __syncthreads();
  const int64_t lo = seg[0], n = seg[1] - seg[0];
  const int64_t nch = (n + kChunk - 1) / kChunk;  // <= kChunk (at most 4.2 M interface cells per mesh)
  for (int64_t c = 0; c < nch && c < kChunk; ++c) {
    const double a = seg_tree(W.mdotV, lo, n, c * kChunk, s);
    const double b = seg_tree(W.QV, lo, n, c * kChunk, s);
    if (threadIdx.x == 0) {
      part[0][c] = a;
      part[1][c] = b;
    }
  }
  __syncthreads();
  for (int q = 0; q < 2; ++q) {
    const double r = nch <= 1 ? (nch ? part[q][0] : 0.0) : seg_tree(part[q], 0, nch, 0, s);
    if (threadIdx.x == 0) totals[2 * m + q] = r;
  }
}

bool same_key(const std::vector<unsigned char>& a, const std::vector<unsigned char>& b) {
  return a.size() == b.size() && std::memcmp(a.data(), b.data(), a.size()) == 0;
}

}  // namespace
}  // namespace vof

using namespace vof;

extern "C" {

vof_status vof_step_graph(vof_mesh* m, const double* d_alpha, const double* d_T, const double* d_T_bnd,
                          const vof_props* props, const vof_options* opt, double* d_mdot, double* d_Q, double* d_totals,
                          void* stream) {
  if (!m || !props || !opt) { set_error("null argument"); return VOF_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) { set_error("vof_step_graph needs a non-default stream"); return VOF_EINVAL; }
  // the captured graph is valid while every argument it bakes in is unchanged
  std::vector<unsigned char> key;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    key.insert(key.end(), c, c + n);
  };
  const void* ptrs[7] = {d_alpha, d_T, d_T_bnd, d_mdot, d_Q, d_totals, (const void*)m->mlp};
  put(ptrs, sizeof(ptrs));
  put(props, sizeof(vof_props));
  put(opt, sizeof(vof_options));
  put(m->bin_G, sizeof(m->bin_G));
  GraphCache& g = m->graph;
  if (!g.exec || !same_key(key, g.key)) {
    const bool timing = m->timing.on;
    m->timing.on = false;  // no event records inside the graph
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { m->timing.on = timing; return cuda_fail(e, "cudaStreamBeginCapture"); }
    vof_status st = vof_step(m, d_alpha, d_T, d_T_bnd, props, opt, d_mdot, d_Q, d_totals, stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    m->timing.on = timing;
    if (st != VOF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    if (g.exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(g.exec, graph, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
      }
    }
    if (!g.exec) {
      e = cudaGraphInstantiate(&g.exec, graph, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        g.exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
      }
    }
    cudaGraphDestroy(graph);
    g.key = key;
    g.captures += 1;
  }
  cudaError_t e = cudaGraphLaunch(g.exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return VOF_OK;
}

vof_status vof_set_group_sizes(vof_mesh* m, const int* h_G) {
  if (!m || !h_G) { set_error("null argument"); return VOF_EINVAL; }
  for (int b = 0; b < kBins; ++b)
    if (!(h_G[b] == 0 || h_G[b] == 1 || h_G[b] == 2 || h_G[b] == 4 || h_G[b] == 8 || h_G[b] == 16 || h_G[b] == 32)) {
      set_error("group size must be 0, 1, 2, 4, 8, 16 or 32");
      return VOF_EINVAL;
    }
  for (int b = 0; b < kBins; ++b) m->bin_G[b] = h_G[b];
  return VOF_OK;
}

vof_status vof_autotune(vof_mesh* m, const double* d_alpha, const vof_options* opt, int reps, int* h_G_out,
                        void* stream) {
  if (!m || !d_alpha || !opt || reps < 1 || reps > 1000) { set_error("bad argument"); return VOF_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  vof_status st = vof_reconstruct(m, d_alpha, opt, stream);
  if (st) return st;
  Counters cn;
  cudaError_t e = cudaMemcpyAsync(&cn, m->ws.counters, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune readback");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // Coordinate descent over the populated bins, largest first: each candidate G of a bin is timed
  // as reps whole reconstructions (selection, learned guess, every bin's root search as parallel
  // branches), the other bins at their current choice, so that the choice accounts for the bins
  // sharing the GPU.
  vof_options o = *opt;
  o.group_size = 0;
  int order[kBins], nb = 0;
  for (int b = 0; b < kBins; ++b)
    if (m->bin_cells[b] && cn.bin_count[b]) order[nb++] = b;
  for (int i = 1; i < nb; ++i)
    for (int j = i; j > 0 && cn.bin_count[order[j]] > cn.bin_count[order[j - 1]]; --j) std::swap(order[j], order[j - 1]);
  for (int b = 0; b < kBins; ++b)
    if (!m->bin_cells[b] || !cn.bin_count[b]) m->bin_G[b] = 0;
  for (int i = 0; i < nb; ++i) {
    const int b = order[i];
    float best = 1e30f;
    int best_G = m->bin_G[b];
    for (int G = 1; G <= 32; G *= 2) {
      m->bin_G[b] = G;
      // warm-up reconstruction (also rejects infeasible shapes)
      if (launch_reconstruct(m, d_alpha, o, s) != VOF_OK) {
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) launch_reconstruct(m, d_alpha, o, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_G = G; }
    }
    m->bin_G[b] = best_G;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (h_G_out)
    for (int b = 0; b < kBins; ++b) h_G_out[b] = m->bin_G[b];
  // leave a consistent reconstruction (and counters) behind
  st = vof_reconstruct(m, d_alpha, opt, stream);
  if (st) return st;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune");
  return VOF_OK;
}

vof_status vof_batch_create(const vof_mesh_desc* d, int n, void* stream, vof_batch** out) {
  if (!d || !out || n < 1) { set_error("bad argument"); return VOF_EINVAL; }
  *out = nullptr;
  vof_batch* b = new (std::nothrow) vof_batch;
  if (!b) { set_error("host allocation failed"); return VOF_ENOMEM; }
  b->n = n;
  b->cell_off.assign(n + 1, 0);
  b->face_off.assign(n + 1, 0);
  b->vert_off.assign(n + 1, 0);
  std::vector<int64_t> cf_off(n + 1, 0), fv_off(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    if (d[i].n_cells <= 0 || d[i].n_faces <= 0 || d[i].n_verts <= 0 || !d[i].cell_face_off || !d[i].face_vert_off) {
      delete b;
      set_error("bad mesh description in batch");
      return VOF_EINVAL;
    }
    b->cell_off[i + 1] = b->cell_off[i] + d[i].n_cells;
    b->face_off[i + 1] = b->face_off[i] + d[i].n_faces;
    b->vert_off[i + 1] = b->vert_off[i] + d[i].n_verts;
    cf_off[i + 1] = cf_off[i] + d[i].cell_face_off[d[i].n_cells];
    fv_off[i + 1] = fv_off[i] + d[i].face_vert_off[d[i].n_faces];
  }
  if (b->cell_off[n] > INT32_MAX || b->face_off[n] > INT32_MAX || b->vert_off[n] > INT32_MAX) {
    delete b;
    set_error("batch too large");
    return VOF_EINVAL;
  }
  std::vector<int64_t> cfo(b->cell_off[n] + 1), fvo(b->face_off[n] + 1);
  std::vector<int32_t> cf(cf_off[n]), fv(fv_off[n]), own(b->face_off[n]), nei(b->face_off[n]);
  std::vector<double> vx(b->vert_off[n]), vy(b->vert_off[n]), vz(b->vert_off[n]);
  for (int i = 0; i < n; ++i) {
    const vof_mesh_desc& m = d[i];
    for (int64_t c = 0; c <= m.n_cells; ++c) cfo[b->cell_off[i] + c] = cf_off[i] + m.cell_face_off[c];
    for (int64_t k = 0; k < m.cell_face_off[m.n_cells]; ++k) {
      const int32_t e = m.cell_face[k];
      cf[cf_off[i] + k] = (int32_t)(((e & 0x7fffffff) + b->face_off[i]) | (e & (int32_t)0x80000000u));
    }
    for (int64_t f = 0; f <= m.n_faces; ++f) fvo[b->face_off[i] + f] = fv_off[i] + m.face_vert_off[f];
    for (int64_t k = 0; k < m.face_vert_off[m.n_faces]; ++k) fv[fv_off[i] + k] = (int32_t)(m.face_vert[k] + b->vert_off[i]);
    for (int64_t f = 0; f < m.n_faces; ++f) {
      own[b->face_off[i] + f] = (int32_t)(m.face_owner[f] + b->cell_off[i]);
      nei[b->face_off[i] + f] = m.face_neigh[f] < 0 ? -1 : (int32_t)(m.face_neigh[f] + b->cell_off[i]);
    }
    std::memcpy(vx.data() + b->vert_off[i], m.vx, 8 * m.n_verts);
    std::memcpy(vy.data() + b->vert_off[i], m.vy, 8 * m.n_verts);
    std::memcpy(vz.data() + b->vert_off[i], m.vz, 8 * m.n_verts);
  }
  vof_mesh_desc u{b->cell_off[n], b->face_off[n], b->vert_off[n], cfo.data(), cf.data(), fvo.data(), fv.data(),
                  own.data(), nei.data(), vx.data(), vy.data(), vz.data()};
  vof_status st = vof_mesh_create(&u, stream, &b->mesh);
  if (st) { delete b; return st; }
  cudaError_t e = cudaMalloc(&b->d_cell_off, (n + 1) * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_cell_off, b->cell_off.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    vof_mesh_destroy(b->mesh);
    delete b;
    return cuda_fail(e, "vof_batch_create");
  }
  *out = b;
  return VOF_OK;
}

vof_status vof_batch_destroy(vof_batch* b) {
  if (!b) return VOF_EINVAL;
  if (b->mesh) vof_mesh_destroy(b->mesh);
  cudaFree(b->d_cell_off);
  delete b;
  return VOF_OK;
}

vof_status vof_batch_mesh(vof_batch* b, vof_mesh** out) {
  if (!b || !out) { set_error("null argument"); return VOF_EINVAL; }
  *out = b->mesh;
  return VOF_OK;
}

vof_status vof_batch_offsets(const vof_batch* b, int64_t* h_cells, int64_t* h_faces, int64_t* h_verts) {
  if (!b) { set_error("null argument"); return VOF_EINVAL; }
  for (int i = 0; i <= b->n; ++i) {
    if (h_cells) h_cells[i] = b->cell_off[i];
    if (h_faces) h_faces[i] = b->face_off[i];
    if (h_verts) h_verts[i] = b->vert_off[i];
  }
  return VOF_OK;
}

vof_status vof_batch_totals(vof_batch* b, double* d_totals, void* stream) {
  if (!b || !d_totals) { set_error("null argument"); return VOF_EINVAL; }
  k_totals_seg<<<b->n, kChunk / 2, 0, (cudaStream_t)stream>>>(b->mesh->ws, b->d_cell_off, d_totals);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "vof_batch_totals");
  return VOF_OK;
}

}  // extern "C"

// C ABI: field access, counters and the host-buffer step.
#include <cstring>

#include "vof_internal.cuh"

using namespace vof;

namespace {

struct FieldDesc {
  const void* ptr;
  int64_t count;
  int bytes;
};

FieldDesc field_of(vof_mesh* m, int f, int64_t n_iface) {
  const Workspace& W = m->ws;
  const MeshView& M = m->view;
  const int64_t nc = m->n_cells, nf = m->n_faces, nv = m->n_verts;
  switch (f) {
    case VOF_F_IFACE_IDX: return {W.iface_idx, n_iface, 4};
    case VOF_F_PHI_V: return {W.phi_v, nv, 8};
    case VOF_F_ISO: return {W.iso, nc, 8};
    case VOF_F_A_INT: return {W.A_int, nc, 8};
    case VOF_F_N_INT: return {W.n_int, 3 * nc, 8};
    case VOF_F_X_GAMMA: return {W.x_gamma, 3 * nc, 8};
    case VOF_F_STATUS: return {W.status, nc, 4};
    case VOF_F_EVALS: return {W.evals, nc, 4};
    case VOF_F_GRAD: return {W.grad, 3 * nc, 8};
    case VOF_F_GRAD_L: return {W.grad_l, 3 * nc, 8};
    case VOF_F_GRAD_V: return {W.grad_v, 3 * nc, 8};
    case VOF_F_Q_L: return {W.q_l, nc, 8};
    case VOF_F_Q_V: return {W.q_v, nc, 8};
    case VOF_F_X_F: return {W.x_f, 3 * nf, 8};
    case VOF_F_D_OWN: return {W.d_own, nf, 8};
    case VOF_F_D_NEIGH: return {W.d_neigh, nf, 8};
    case VOF_F_A_INT_F: return {W.A_int_f, nf, 8};
    case VOF_F_FACE_STAMP: return {W.face_stamp, nf, 4};
    case VOF_F_CELL_VOL: return {M.cell_vol, nc, 8};
    case VOF_F_CELL_CEN: return {M.cell_cen, 3 * nc, 8};
    case VOF_F_FACE_AREA: return {M.face_area, 3 * nf, 8};
    case VOF_F_FACE_CEN: return {M.face_cen, 3 * nf, 8};
    case VOF_F_IFACE_STAMP: return {W.iface_stamp, nc, 4};
    case VOF_F_BAND_STAMP: return {W.band_stamp, nc, 4};
    case VOF_F_A_OWN: return {W.a_own, nf, 8};
    case VOF_F_A_NEIGH: return {W.a_neigh, nf, 8};
    case VOF_F_DTAU: return {W.ex_dtau, 1, 8};
    case VOF_F_LSQ_COND: return {W.lsq_cond, nc, 8};
    case VOF_F_HTC_DIAG: return {W.htc_diag, nc, 8};
    case VOF_F_HTC_RHS: return {W.htc_rhs, nc, 8};
    default: return {nullptr, 0, 0};
  }
}

vof_status read_counters(vof_mesh* m, Counters* c, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(c, m->ws.counters, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "counter readback");
  return VOF_OK;
}

// dst[idx[i]] = src[idx[i]]: the boundary entries of a per-face array, read through a
// device-accessible view of pinned host memory
__global__ void k_gather_faces(int64_t n, const int32_t* idx, const double* src, double* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int32_t f = idx[i];
    dst[f] = src[f];
  }
}

// The device view of host memory that CUDA maps (pinned allocations), else null.
const double* mapped_view(const void* p) {
  cudaPointerAttributes pa;
  const double* v = nullptr;
  if (cudaPointerGetAttributes(&pa, p) == cudaSuccess && pa.type == cudaMemoryTypeHost)
    v = static_cast<const double*>(pa.devicePointer);
  cudaGetLastError();
  return v;
}

// The host-buffer step, enqueued on s without synchronising: alpha on s; T and T_bnd on the
// mesh's copy stream, overlapping the reconstruction (the source stage waits for them); T_bnd
// gathered at the boundary faces through tb_view when there is one; mdot and the totals back.
vof_status host_step_enqueue(vof_mesh* m, const double* h_alpha, const double* h_T, const double* h_T_bnd,
                             const double* tb_view, const vof_props* props, const vof_options* opt, double* h_mdot,
                             double* h_totals, cudaStream_t s) {
  Workspace& W = m->ws;
  const size_t nc = (size_t)m->n_cells, nf = (size_t)m->n_faces;
  cudaError_t e = cudaEventRecord(m->ev_io_start, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(W.io_alpha, h_alpha, nc * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(m->io_stream, m->ev_io_start, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(W.io_T, h_T, nc * 8, cudaMemcpyHostToDevice, m->io_stream);
  if (e == cudaSuccess && h_T_bnd) {
    if (tb_view) {
      if (m->n_bnd > 0) {
        k_gather_faces<<<(unsigned)((m->n_bnd + 255) / 256), 256, 0, m->io_stream>>>(m->n_bnd, m->bnd_faces, tb_view,
                                                                                      W.io_Tb);
        e = cudaGetLastError();
      }
    } else {
      e = cudaMemcpyAsync(W.io_Tb, h_T_bnd, nf * 8, cudaMemcpyHostToDevice, m->io_stream);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(m->ev_io_done, m->io_stream);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  m->io_pending = true;
  vof_status st = vof_step(m, W.io_alpha, W.io_T, h_T_bnd ? W.io_Tb : nullptr, props, opt, W.io_mdot, W.io_Q,
                           W.io_totals, s);
  if (st) {
    if (m->io_pending) {  // the step stopped before its source stage: join the copy stream
      cudaStreamWaitEvent(s, m->ev_io_done, 0);
      m->io_pending = false;
    }
    return st;
  }
  e = cudaMemcpyAsync(h_mdot, W.io_mdot, nc * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_totals, W.io_totals, 2 * 8, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  return VOF_OK;
}

}  // namespace

extern "C" {

vof_status vof_field_size(vof_mesh* m, int field, int64_t* count, int* elem_bytes) {
  if (!m || !count || !elem_bytes || field < 0 || field >= VOF_F_N) { set_error("bad argument"); return VOF_EINVAL; }
  int64_t n_iface = 0;
  if (field == VOF_F_IFACE_IDX) {
    Counters c;
    if (vof_status st = read_counters(m, &c, 0)) return st;
    n_iface = c.n_iface;
  }
  const FieldDesc d = field_of(m, field, n_iface);
  *count = d.count;
  *elem_bytes = d.bytes;
  return VOF_OK;
}

vof_status vof_copy_field(vof_mesh* m, int field, void* d_dst, int64_t count, void* stream) {
  if (!m || field < 0 || field >= VOF_F_N || count < 0) { set_error("bad argument"); return VOF_EINVAL; }
  const FieldDesc d = field_of(m, field, m->n_cells);
  if (count > d.count) { set_error("count exceeds the field size"); return VOF_EINVAL; }
  if (count == 0) return VOF_OK;
  if (!d_dst) { set_error("null destination"); return VOF_EINVAL; }
  cudaError_t e = cudaMemcpyAsync(d_dst, d.ptr, (size_t)count * d.bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vof_copy_field");
  return VOF_OK;
}

vof_status vof_get_counts(vof_mesh* m, vof_counts* out, void* stream) {
  if (!m || !out) { set_error("null argument"); return VOF_EINVAL; }
  Counters c;
  if (vof_status st = read_counters(m, &c, (cudaStream_t)stream)) return st;
  out->step = c.step;
  out->n_iface = c.n_iface;
  out->n_band = c.n_band;
  out->n_crossing = c.n_crossing;
  out->n_degenerate = c.n_degenerate;
  out->n_not_converged = c.n_not_converged;
  out->n_fallback = c.n_fallback;
  out->n_singular = c.n_singular;
  out->n_no_side = c.n_no_side;
  out->n_mlp_skipped = c.n_mlp_skipped;
  out->evals_total = c.evals_total;
  out->tet_evals = c.tet_evals;
  out->tets_prepared = c.tets_prepared;
  out->tets_sectioned = c.tets_sectioned;
  out->evals32_total = c.evals32_total;
  for (int k = 0; k < 6; ++k) out->extrap_iters[k] = c.extrap_iters[k];
  return VOF_OK;
}

vof_status vof_timing_enable(vof_mesh* m, int on) {
  if (!m) { set_error("null argument"); return VOF_EINVAL; }
  Timing& t = m->timing;
  if (on && t.ev.empty()) {
    t.cap = 8192;
    t.ev.resize(2 * (size_t)t.cap);
    t.cls.resize(t.cap);
    for (auto& e : t.ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return cuda_fail(r, "cudaEventCreate");
    }
  }
  t.on = on != 0;
  t.used = 0;
  return VOF_OK;
}

vof_status vof_timing_read(vof_mesh* m, double* ms, int64_t* launches, int n, void* stream) {
  if (!m || !ms || !launches || n < 1) { set_error("bad argument"); return VOF_EINVAL; }
  Timing& t = m->timing;
  for (int k = 0; k < n; ++k) { ms[k] = 0; launches[k] = 0; }
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "vof_timing_read");
  for (int i = 0; i < t.used; ++i) {
    if (t.cls[i] >= n) continue;
    float f = 0;
    e = cudaEventElapsedTime(&f, t.ev[2 * i], t.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms[t.cls[i]] += f;
    launches[t.cls[i]] += 1;
  }
  t.used = 0;
  return VOF_OK;
}

vof_status vof_step_host(vof_mesh* m, const double* h_alpha, const double* h_T, const double* h_T_bnd,
                         const vof_props* props, const vof_options* opt, double* h_mdot, double* h_totals,
                         void* stream) {
  if (!m || !h_alpha || !h_T || !h_mdot || !h_totals || !props || !opt) {
    set_error("null argument");
    return VOF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // only the boundary entries of T_bnd are ever read: a mapped (pinned) h_T_bnd is gathered there
  const double* tb_view = h_T_bnd ? mapped_view(h_T_bnd) : nullptr;
  const bool pinned = mapped_view(h_alpha) && mapped_view(h_T) && mapped_view(h_mdot) && mapped_view(h_totals) &&
                      (!h_T_bnd || tb_view);
  if (!s || !pinned) {
    vof_status st = host_step_enqueue(m, h_alpha, h_T, h_T_bnd, tb_view, props, opt, h_mdot, h_totals, s);
    if (st) {
      cudaStreamSynchronize(s);  // the copies in flight still read the caller's buffers
      return st;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "host-buffer step");
    return VOF_OK;
  }
  // pinned buffers on a stream of the caller's: the copies, the gather and the step are captured
  // once and replayed, valid while the arguments they bake in are unchanged
  std::vector<unsigned char> key;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    key.insert(key.end(), c, c + n);
  };
  const void* ptrs[6] = {h_alpha, h_T, h_T_bnd, h_mdot, h_totals, (const void*)m->mlp};
  put(ptrs, sizeof(ptrs));
  put(props, sizeof(vof_props));
  put(opt, sizeof(vof_options));
  put(m->bin_G, sizeof(m->bin_G));
  GraphCache& g = m->host_graph;
  if (!g.exec || g.key.size() != key.size() || std::memcmp(g.key.data(), key.data(), key.size()) != 0) {
    const bool timing = m->timing.on;
    m->timing.on = false;  // no event records inside the graph
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { m->timing.on = timing; return cuda_fail(e, "cudaStreamBeginCapture"); }
    const vof_status st = host_step_enqueue(m, h_alpha, h_T, h_T_bnd, tb_view, props, opt, h_mdot, h_totals, s);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    m->timing.on = timing;
    m->io_pending = false;
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
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "host-buffer step");
  return VOF_OK;
}

}  // extern "C"

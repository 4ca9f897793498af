// Mesh creation and the C ABI entry points of libvof_gb300.so.
//
// Host side: validation of the mesh arrays, the cell tetrahedralisation by the cell's own
// vertices (faces fanned from their lowest-id vertex, the cell fanned from its lowest-id
// vertex), the vertex->cell table. Device side: face and cell geometry, tetrahedron volumes and
// inverse-distance weights (kernels below), then the step workspace.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "vof_internal.cuh"

namespace vof {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
vof_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return VOF_ECUDA;
}

namespace {

// Face area vector (outward from owner) and area-weighted centroid: fan about the vertex mean.
__global__ void k_face_geom(int64_t nf, const int64_t* fvo, const int32_t* fv, const double* vx, const double* vy,
                            const double* vz, double* area, double* cen) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int64_t o = fvo[f];
  const int n = (int)(fvo[f + 1] - o);
  double mx = 0, my = 0, mz = 0;
  for (int i = 0; i < n; ++i) {
    const int32_t v = fv[o + i];
    mx += vx[v]; my += vy[v]; mz += vz[v];
  }
  mx /= n; my /= n; mz /= n;
  double ax = 0, ay = 0, az = 0, cx = 0, cy = 0, cz = 0, at = 0;
  for (int i = 0; i < n; ++i) {
    const int32_t p = fv[o + i], q = fv[o + (i + 1) % n];
    const double ux = vx[p] - mx, uy = vy[p] - my, uz = vz[p] - mz;
    const double wx = vx[q] - mx, wy = vy[q] - my, wz = vz[q] - mz;
    const double tx = 0.5 * (uy * wz - uz * wy), ty = 0.5 * (uz * wx - ux * wz), tz = 0.5 * (ux * wy - uy * wx);
    ax += tx; ay += ty; az += tz;
    const double ar = sqrt(tx * tx + ty * ty + tz * tz);
    cx += ar * (mx + vx[p] + vx[q]) / 3; cy += ar * (my + vy[p] + vy[q]) / 3; cz += ar * (mz + vz[p] + vz[q]) / 3;
    at += ar;
  }
  area[3 * f] = ax; area[3 * f + 1] = ay; area[3 * f + 2] = az;
  cen[3 * f] = at > 0 ? cx / at : mx;
  cen[3 * f + 1] = at > 0 ? cy / at : my;
  cen[3 * f + 2] = at > 0 ? cz / at : mz;
}

// Tetrahedron volumes (apex = local vertex 0), cell volume = their sum, centroid.
__global__ void k_cell_geom(int64_t nc, const int64_t* cvo, const int32_t* cv, const int64_t* cto, const uint32_t* ct,
                            const double* vx, const double* vy, const double* vz, double* tvol, float* tvf,
                            double* vol, double* ivol, double* cen, int32_t* bad) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int32_t* V = cv + cvo[c];
  const double ax = vx[V[0]], ay = vy[V[0]], az = vz[V[0]];
  double sv = 0, sx = 0, sy = 0, sz = 0;
  for (int64_t t = cto[c]; t < cto[c + 1]; ++t) {
    const uint32_t pk = ct[t];
    const int32_t i0 = V[pk & 255], i1 = V[(pk >> 8) & 255], i2 = V[(pk >> 16) & 255];
    const double ux = vx[i0] - ax, uy = vy[i0] - ay, uz = vz[i0] - az;
    const double wx = vx[i1] - ax, wy = vy[i1] - ay, wz = vz[i1] - az;
    const double qx = vx[i2] - ax, qy = vy[i2] - ay, qz = vz[i2] - az;
    const double v6 = ux * (wy * qz - wz * qy) - uy * (wx * qz - wz * qx) + uz * (wx * qy - wy * qx);
    const double v = v6 / 6.0;
    const double scale = sqrt((ux * ux + uy * uy + uz * uz) * (wx * wx + wy * wy + wz * wz) * (qx * qx + qy * qy + qz * qz));
    if (v6 < -1e-12 * scale) atomicAdd(bad, 1);
    tvol[t] = v;
    sv += v;
    sx += v * (ax + vx[i0] + vx[i1] + vx[i2]) * 0.25;
    sy += v * (ay + vy[i0] + vy[i1] + vy[i2]) * 0.25;
    sz += v * (az + vz[i0] + vz[i1] + vz[i2]) * 0.25;
  }
  vol[c] = sv;
  ivol[c] = 1.0 / sv;
  cen[3 * c] = sx / sv; cen[3 * c + 1] = sy / sv; cen[3 * c + 2] = sz / sv;
  // volume fractions (FP32) for the FP32 refinement of the learned root search
  for (int64_t t = cto[c]; t < cto[c + 1]; ++t) tvf[t] = (float)(tvol[t] / sv);
}

// Vertex positions relative to the cell's apex (local vertex 0), split into (hi, lo) float pairs
// (hi = x rounded to FP32, lo = the rest rounded to FP32): the interface geometry of a step runs
// on the FP32 pipe in pair arithmetic.
__global__ void k_rel_pos(int64_t nc, const int64_t* cvo, const int32_t* cv, const double* vx, const double* vy,
                          const double* vz, float2* rel) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int32_t a = cv[cvo[c]];
  for (int64_t k = cvo[c]; k < cvo[c + 1]; ++k) {
    const int32_t v = cv[k];
    const double d[3] = {vx[v] - vx[a], vy[v] - vy[a], vz[v] - vz[a]};
    for (int q = 0; q < 3; ++q) {
      const float h = __double2float_rn(d[q]);
      rel[3 * k + q] = make_float2(h, __double2float_rn(d[q] - (double)h));
    }
  }
}

// Inverse-distance weights of the cells around each vertex, normalised to sum 1.
// |d_f| of each face: owner centroid to neighbour centroid, or to the face centroid on a boundary
// face; the minimum over the faces by atomicMin on the raw bits.
__global__ void k_dtau_init(double* out) { *out = INFINITY; }
__global__ void k_dtau(int64_t nf, const int32_t* own, const int32_t* nei, const double* cen, const double* fcen,
                       double* out) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int32_t o = own[f], n = nei[f];
  const double* xn = n >= 0 ? cen + 3 * n : fcen + 3 * f;
  const double dx = xn[0] - cen[3 * o], dy = xn[1] - cen[3 * o + 1], dz = xn[2] - cen[3 * o + 2];
  const double d = sqrt(dx * dx + dy * dy + dz * dz);
  atomicMin((unsigned long long*)out, (unsigned long long)__double_as_longlong(d));
}

// Per face: the owner-to-neighbour centroid distance (0 on a boundary face) and the reciprocal of
// the face's area, for the crossing points of the steps.
__global__ void k_face_static(int64_t nf, const int32_t* own, const int32_t* nei, const double* cen, const double* fa,
                              double* len, double* iarea) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int32_t o = own[f], n = nei[f];
  double L = 0;
  if (n >= 0) {
    const double dx = cen[3 * n] - cen[3 * o], dy = cen[3 * n + 1] - cen[3 * o + 1], dz = cen[3 * n + 2] - cen[3 * o + 2];
    L = sqrt(dx * dx + dy * dy + dz * dz);
  }
  len[f] = L;
  const double ax = fa[3 * f], ay = fa[3 * f + 1], az = fa[3 * f + 2];
  iarea[f] = 1.0 / sqrt(ax * ax + ay * ay + az * az);
}

__global__ void k_idw(int64_t nv, const int64_t* vco, const int32_t* vc, const double* vx, const double* vy,
                      const double* vz, const double* cen, double* w) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= nv) return;
  double s = 0;
  for (int64_t k = vco[v]; k < vco[v + 1]; ++k) {
    const int32_t c = vc[k];
    const double dx = vx[v] - cen[3 * c], dy = vy[v] - cen[3 * c + 1], dz = vz[v] - cen[3 * c + 2];
    const double d = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    w[k] = d;
    s += d;
  }
  for (int64_t k = vco[v]; k < vco[v + 1]; ++k) w[k] /= s;
}

template <typename T>
vof_status dev_alloc(vof_mesh* m, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    return VOF_ENOMEM;
  }
  m->allocs.push_back(q);
  *p = (T*)q;
  return VOF_OK;
}

template <typename T>
vof_status upload(vof_mesh* m, T** p, const T* h, size_t n, cudaStream_t s) {
  vof_status st = dev_alloc(m, p, n);
  if (st) return st;
  if (n) {
    cudaError_t e = cudaMemcpyAsync(*p, h, n * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload");
  }
  return VOF_OK;
}

#define TRY(x)                     \
  do {                             \
    vof_status _s = (x);           \
    if (_s != VOF_OK) return _s;   \
  } while (0)

vof_status create(const vof_mesh_desc* d, cudaStream_t s, vof_mesh* m) {
  const int64_t nc = d->n_cells, nf = d->n_faces, nv = d->n_verts;
  if (nc <= 0 || nf <= 0 || nv <= 0 || nc > INT32_MAX || nf > INT32_MAX || nv > INT32_MAX) {
    set_error("mesh sizes out of range");
    return VOF_EINVAL;
  }
  if (!d->cell_face_off || !d->cell_face || !d->face_vert_off || !d->face_vert || !d->face_owner ||
      !d->face_neigh || !d->vx || !d->vy || !d->vz) {
    set_error("null mesh array");
    return VOF_EINVAL;
  }
  // ---- validation
  if (d->cell_face_off[0] != 0 || d->face_vert_off[0] != 0) { set_error("offsets must start at 0"); return VOF_EMESH; }
  for (int64_t c = 0; c < nc; ++c)
    if (d->cell_face_off[c + 1] < d->cell_face_off[c] + 4) { set_error("cell with fewer than 4 faces"); return VOF_EMESH; }
  for (int64_t f = 0; f < nf; ++f) {
    if (d->face_vert_off[f + 1] < d->face_vert_off[f] + 3) { set_error("face with fewer than 3 vertices"); return VOF_EMESH; }
    if (d->face_owner[f] < 0 || d->face_owner[f] >= nc || d->face_neigh[f] < -1 || d->face_neigh[f] >= nc ||
        d->face_neigh[f] == d->face_owner[f]) {
      set_error("face owner/neighbour out of range");
      return VOF_EMESH;
    }
  }
  for (int64_t k = 0; k < d->face_vert_off[nf]; ++k)
    if (d->face_vert[k] < 0 || d->face_vert[k] >= nv) { set_error("face vertex id out of range"); return VOF_EMESH; }
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t k = d->cell_face_off[c]; k < d->cell_face_off[c + 1]; ++k) {
      const int32_t e = d->cell_face[k];
      const int32_t f = e & 0x7fffffff;
      if (f >= nf) { set_error("cell face id out of range"); return VOF_EMESH; }
      const bool rev = e < 0;
      if ((!rev && d->face_owner[f] != c) || (rev && d->face_neigh[f] != c)) {
        set_error("cell_face orientation bit disagrees with face owner/neighbour");
        return VOF_EMESH;
      }
    }
  for (int64_t v = 0; v < nv; ++v)
    if (!std::isfinite(d->vx[v]) || !std::isfinite(d->vy[v]) || !std::isfinite(d->vz[v])) {
      set_error("non-finite vertex coordinate");
      return VOF_EMESH;
    }
  // ---- cell vertices and tetrahedra
  std::vector<int64_t> cvo(nc + 1, 0), cto(nc + 1, 0);
  std::vector<std::vector<int32_t>> cvl(nc);
  std::vector<std::vector<uint32_t>> ctl(nc);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : bad)
  for (int64_t c = 0; c < nc; ++c) {
    std::vector<int32_t>& vs = cvl[c];
    for (int64_t k = d->cell_face_off[c]; k < d->cell_face_off[c + 1]; ++k) {
      const int32_t f = d->cell_face[k] & 0x7fffffff;
      for (int64_t j = d->face_vert_off[f]; j < d->face_vert_off[f + 1]; ++j) vs.push_back(d->face_vert[j]);
    }
    std::sort(vs.begin(), vs.end());
    vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
    if ((int)vs.size() > VOF_MAX_CELL_VERTS) { bad++; continue; }
    auto local = [&](int32_t g) { return (uint32_t)(std::lower_bound(vs.begin(), vs.end(), g) - vs.begin()); };
    const int32_t apex = vs[0];
    std::vector<int32_t> L;
    for (int64_t k = d->cell_face_off[c]; k < d->cell_face_off[c + 1]; ++k) {
      const int32_t e = d->cell_face[k];
      const int32_t f = e & 0x7fffffff;
      L.assign(d->face_vert + d->face_vert_off[f], d->face_vert + d->face_vert_off[f + 1]);
      if (e < 0) std::reverse(L.begin(), L.end());
      const size_t n = L.size();
      const size_t s0 = std::min_element(L.begin(), L.end()) - L.begin();
      for (size_t i = 1; i + 1 < n; ++i) {
        const int32_t t0 = L[s0], t1 = L[(s0 + i) % n], t2 = L[(s0 + i + 1) % n];
        if (t0 == apex || t1 == apex || t2 == apex) continue;
        ctl[c].push_back(local(t0) | (local(t1) << 8) | (local(t2) << 16));
      }
    }
    if ((int)ctl[c].size() > VOF_MAX_CELL_TETS || ctl[c].empty()) bad++;
  }
  if (bad) { set_error("cell exceeds the vertex/tetrahedron limits"); return VOF_EMESH; }
  int max_cv = 0, max_ct = 0;
  for (int64_t c = 0; c < nc; ++c) {
    cvo[c + 1] = cvo[c] + (int64_t)cvl[c].size();
    cto[c + 1] = cto[c] + (int64_t)ctl[c].size();
    max_cv = std::max(max_cv, (int)cvl[c].size());
    max_ct = std::max(max_ct, (int)ctl[c].size());
  }
  std::vector<int32_t> cv(cvo[nc]);
  std::vector<uint32_t> ct(cto[nc]);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    std::copy(cvl[c].begin(), cvl[c].end(), cv.begin() + cvo[c]);
    std::copy(ctl[c].begin(), ctl[c].end(), ct.begin() + cto[c]);
  }
  cvl.clear(); cvl.shrink_to_fit();
  ctl.clear(); ctl.shrink_to_fit();
  // vertex -> cell table
  std::vector<int64_t> vco(nv + 1, 0);
  for (int64_t k = 0; k < cvo[nc]; ++k) vco[cv[k] + 1]++;
  for (int64_t v = 0; v < nv; ++v) vco[v + 1] += vco[v];
  std::vector<int32_t> vc(vco[nv]);
  {
    std::vector<int64_t> pos(vco.begin(), vco.end() - 1);
    for (int64_t c = 0; c < nc; ++c)
      for (int64_t k = cvo[c]; k < cvo[c + 1]; ++k) vc[pos[cv[k]]++] = (int32_t)c;
  }
  for (int64_t v = 0; v < nv; ++v)
    if (vco[v + 1] == vco[v]) { set_error("vertex used by no cell"); return VOF_EMESH; }

  m->n_cells = nc; m->n_faces = nf; m->n_verts = nv;
  m->max_cv = max_cv; m->max_ct = max_ct;
  for (int64_t c = 0; c < nc; ++c) m->max_cf = std::max(m->max_cf, (int)(d->cell_face_off[c + 1] - d->cell_face_off[c]));
  m->mean_ct = (double)cto[nc] / (double)nc;
  for (int64_t c = 0; c < nc; ++c) {
    const int nt = (int)(cto[c + 1] - cto[c]);
    const int b = bin_of(nt);
    m->bin_cells[b]++;
    m->bin_max_ct[b] = std::max(m->bin_max_ct[b], nt);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, dev);
  {
    cudaError_t es = cudaEventCreateWithFlags(&m->ev_fork, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaStreamCreateWithFlags(&m->xm_stream, cudaStreamNonBlocking);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_xfork, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_xjoin, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaStreamCreateWithFlags(&m->io_stream, cudaStreamNonBlocking);
    if (es == cudaSuccess) es = cudaStreamCreateWithFlags(&m->z_stream, cudaStreamNonBlocking);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_zfork, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_zjoin, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_io_start, cudaEventDisableTiming);
    if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_io_done, cudaEventDisableTiming);
    for (int b = 0; b < kBins && es == cudaSuccess; ++b) {
      es = cudaStreamCreateWithFlags(&m->bin_stream[b], cudaStreamNonBlocking);
      if (es == cudaSuccess) es = cudaEventCreateWithFlags(&m->ev_join[b], cudaEventDisableTiming);
    }
    if (es != cudaSuccess) return cuda_fail(es, "bin streams");
  }
  MeshView& V = m->view;
  V.n_cells = nc; V.n_faces = nf; V.n_verts = nv;
  int64_t *d_cfo, *d_fvo, *d_cvo, *d_cto, *d_vco;
  int32_t *d_cf, *d_fv, *d_own, *d_nei, *d_cv, *d_vc;
  uint32_t* d_ct;
  double *d_vx, *d_vy, *d_vz;
  TRY(upload(m, &d_cfo, d->cell_face_off, nc + 1, s));
  TRY(upload(m, &d_cf, d->cell_face, (size_t)d->cell_face_off[nc], s));
  TRY(upload(m, &d_fvo, d->face_vert_off, nf + 1, s));
  TRY(upload(m, &d_fv, d->face_vert, (size_t)d->face_vert_off[nf], s));
  TRY(upload(m, &d_own, d->face_owner, nf, s));
  TRY(upload(m, &d_nei, d->face_neigh, nf, s));
  TRY(upload(m, &d_vx, d->vx, nv, s));
  TRY(upload(m, &d_vy, d->vy, nv, s));
  TRY(upload(m, &d_vz, d->vz, nv, s));
  TRY(upload(m, &d_cvo, cvo.data(), nc + 1, s));
  TRY(upload(m, &d_cv, cv.data(), cv.size(), s));
  TRY(upload(m, &d_cto, cto.data(), nc + 1, s));
  TRY(upload(m, &d_ct, ct.data(), ct.size(), s));
  TRY(upload(m, &d_vco, vco.data(), nv + 1, s));
  TRY(upload(m, &d_vc, vc.data(), vc.size(), s));
  double *d_tvol, *d_vol, *d_cen, *d_fa, *d_fc, *d_w;
  float* d_tvf;
  float2* d_rel;
  double* d_ivol;
  TRY(dev_alloc(m, &d_ivol, nc));
  TRY(dev_alloc(m, &d_rel, 3 * cv.size()));
  int32_t* d_bad;
  TRY(dev_alloc(m, &d_tvol, ct.size()));
  TRY(dev_alloc(m, &d_tvf, ct.size()));
  TRY(dev_alloc(m, &d_vol, nc));
  TRY(dev_alloc(m, &d_cen, 3 * nc));
  TRY(dev_alloc(m, &d_fa, 3 * nf));
  TRY(dev_alloc(m, &d_fc, 3 * nf));
  TRY(dev_alloc(m, &d_w, vc.size()));
  double *d_flen, *d_fia;
  TRY(dev_alloc(m, &d_flen, nf));
  TRY(dev_alloc(m, &d_fia, nf));
  TRY(dev_alloc(m, &d_bad, 1));
  cudaMemsetAsync(d_bad, 0, sizeof(int32_t), s);
  k_face_geom<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(nf, d_fvo, d_fv, d_vx, d_vy, d_vz, d_fa, d_fc);
  k_cell_geom<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(nc, d_cvo, d_cv, d_cto, d_ct, d_vx, d_vy, d_vz, d_tvol,
                                                            d_tvf, d_vol, d_ivol, d_cen, d_bad);
  k_rel_pos<<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(nc, d_cvo, d_cv, d_vx, d_vy, d_vz, d_rel);
  k_idw<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, d_vco, d_vc, d_vx, d_vy, d_vz, d_cen, d_w);
  k_face_static<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(nf, d_own, d_nei, d_cen, d_fa, d_flen, d_fia);
  int32_t h_bad = 0;
  cudaMemcpyAsync(&h_bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "mesh geometry");
  if (h_bad) { set_error("negative tetrahedron volume: cell not convex or faces not outward"); return VOF_EMESH; }
  V.cell_face_off = d_cfo; V.cell_face = d_cf; V.face_owner = d_own; V.face_neigh = d_nei;
  V.vx = d_vx; V.vy = d_vy; V.vz = d_vz;
  V.cell_vert_off = d_cvo; V.cell_vert = d_cv; V.cell_tet_off = d_cto; V.cell_tet = d_ct; V.tet_vol = d_tvol;
  V.tet_vfrac = d_tvf;
  V.rel_pos = d_rel;
  V.vert_cell_off = d_vco; V.vert_cell = d_vc; V.vert_w = d_w;
  V.cell_vol = d_vol; V.cell_ivol = d_ivol; V.cell_cen = d_cen; V.face_area = d_fa; V.face_cen = d_fc;
  V.face_len = d_flen; V.face_iarea = d_fia;
  // ---- workspace
  Workspace& W = m->ws;
  m->n_sel_blocks = (int)((nc + kSelTile - 1) / kSelTile);
  TRY(dev_alloc(m, &W.counters, 1));
  TRY(dev_alloc(m, &W.iface_idx, nc));
  TRY(dev_alloc(m, &W.iface_stamp, nc));
  TRY(dev_alloc(m, &W.band_stamp, nc));
  TRY(dev_alloc(m, &W.vert_stamp, nv));
  TRY(dev_alloc(m, &W.face_stamp, nf));
  TRY(dev_alloc(m, &W.sel_mask, (size_t)m->n_sel_blocks * (kSelTile / 32)));
  TRY(dev_alloc(m, &W.sel_tot, kMaxSelGrid));
  TRY(dev_alloc(m, &W.tile_part, 2 * (size_t)((nc + kSrcTile - 1) / kSrcTile)));
  TRY(dev_alloc(m, &W.band_idx, nc));
  TRY(dev_alloc(m, &W.phi_v, nv));
  TRY(dev_alloc(m, &W.phi_ff, nv));
  TRY(dev_alloc(m, &W.iso, nc));
  TRY(dev_alloc(m, &W.A_int, nc));
  TRY(dev_alloc(m, &W.n_int, 3 * nc));
  TRY(dev_alloc(m, &W.x_gamma, 3 * nc));
  TRY(dev_alloc(m, &W.status, nc));
  TRY(dev_alloc(m, &W.evals, nc));
  TRY(dev_alloc(m, &W.grad, 3 * nc));
  TRY(dev_alloc(m, &W.grad_l, 3 * nc));
  TRY(dev_alloc(m, &W.grad_v, 3 * nc));
  TRY(dev_alloc(m, &W.q_l, nc));
  TRY(dev_alloc(m, &W.q_v, nc));
  TRY(dev_alloc(m, &W.x_f, 3 * nf));
  TRY(dev_alloc(m, &W.d_own, nf));
  TRY(dev_alloc(m, &W.d_neigh, nf));
  TRY(dev_alloc(m, &W.A_int_f, nf));
  TRY(dev_alloc(m, &W.a_own, nf));
  TRY(dev_alloc(m, &W.a_neigh, nf));
  TRY(dev_alloc(m, &W.htc_diag, nc));
  TRY(dev_alloc(m, &W.htc_rhs, nc));
  TRY(dev_alloc(m, &W.xface_list, nf));
  TRY(dev_alloc(m, &W.mdotV, nc));
  TRY(dev_alloc(m, &W.QV, nc));
  TRY(dev_alloc(m, &W.partial, 4 * kMaxPartials));
  TRY(dev_alloc(m, &W.io_alpha, nc));
  TRY(dev_alloc(m, &W.io_T, nc));
  TRY(dev_alloc(m, &W.io_Tb, nf));
  {  // boundary faces, for the host-buffer step's gather of T_bnd
    std::vector<int32_t> bf;
    for (int64_t f = 0; f < nf; ++f)
      if (d->face_neigh[f] < 0) bf.push_back((int32_t)f);
    m->n_bnd = (int64_t)bf.size();
    TRY(upload(m, &m->bnd_faces, bf.data(), bf.size(), s));
  }
  TRY(dev_alloc(m, &W.io_mdot, nc));
  TRY(dev_alloc(m, &W.io_Q, nc));
  TRY(dev_alloc(m, &W.io_totals, 2));
  TRY(dev_alloc(m, &W.mlp_out, nc));
  TRY(dev_alloc(m, &W.bin_list, (size_t)kBins * nc));
  TRY(dev_alloc(m, &W.slow_list, (size_t)kBins * nc));
  TRY(dev_alloc(m, &W.iface_slot, nc));
  TRY(dev_alloc(m, &W.ex_x, 8 * (size_t)nc));
  TRY(dev_alloc(m, &W.ex_k, 5 * (size_t)nc));
  TRY(dev_alloc(m, &W.ex_nb, kExCap * (size_t)nc));
  TRY(dev_alloc(m, &W.ex_g, kExCap * (size_t)nc));
  TRY(dev_alloc(m, &W.ex_mask, nc));
  TRY(dev_alloc(m, &W.ex_itmax, 6 * (size_t)(kExMaxIter + 1)));
  TRY(dev_alloc(m, &W.ex_dtau, 1));
  TRY(dev_alloc(m, &W.lsq_cond, nc));
  // pseudo-time step of the extrapolation: min over faces of |d_f|, by an atomic minimum of the
  // raw bits (non-negative doubles order as their bit patterns)
  k_dtau_init<<<1, 1, 0, s>>>(W.ex_dtau);
  k_dtau<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(nf, d_own, d_nei, d_cen, d_fc, W.ex_dtau);
  cudaMemsetAsync(W.counters, 0, sizeof(Counters), s);
  cudaMemsetAsync(W.iface_stamp, 0, nc * sizeof(uint32_t), s);
  cudaMemsetAsync(W.band_stamp, 0, nc * sizeof(uint32_t), s);
  cudaMemsetAsync(W.vert_stamp, 0, nv * sizeof(uint32_t), s);
  cudaMemsetAsync(W.face_stamp, 0, nf * sizeof(uint32_t), s);
  cudaMemsetAsync(W.status, 0, nc * sizeof(int32_t), s);
  cudaMemsetAsync(W.evals, 0, nc * sizeof(int32_t), s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "workspace init");
  return VOF_OK;
}

void destroy(vof_mesh* m) {
  if (m->graph.exec) cudaGraphExecDestroy(m->graph.exec);
  m->graph.exec = nullptr;
  if (m->host_graph.exec) cudaGraphExecDestroy(m->host_graph.exec);
  m->host_graph.exec = nullptr;
  for (cudaEvent_t e : m->timing.ev) cudaEventDestroy(e);
  m->timing.ev.clear();
  for (void* p : m->allocs) cudaFree(p);
  m->allocs.clear();
  for (int b = 0; b < kBins; ++b) {
    if (m->bin_stream[b]) cudaStreamDestroy(m->bin_stream[b]);
    if (m->ev_join[b]) cudaEventDestroy(m->ev_join[b]);
    m->bin_stream[b] = nullptr;
    m->ev_join[b] = nullptr;
  }
  if (m->ev_fork) cudaEventDestroy(m->ev_fork);
  m->ev_fork = nullptr;
  if (m->xm_stream) cudaStreamDestroy(m->xm_stream);
  if (m->ev_xfork) cudaEventDestroy(m->ev_xfork);
  if (m->ev_xjoin) cudaEventDestroy(m->ev_xjoin);
  m->xm_stream = nullptr;
  m->ev_xfork = m->ev_xjoin = nullptr;
  if (m->z_stream) cudaStreamDestroy(m->z_stream);
  if (m->ev_zfork) cudaEventDestroy(m->ev_zfork);
  if (m->ev_zjoin) cudaEventDestroy(m->ev_zjoin);
  m->z_stream = nullptr;
  m->ev_zfork = m->ev_zjoin = nullptr;
  if (m->io_stream) cudaStreamDestroy(m->io_stream);
  if (m->ev_io_start) cudaEventDestroy(m->ev_io_start);
  if (m->ev_io_done) cudaEventDestroy(m->ev_io_done);
  m->io_stream = nullptr;
  m->ev_io_start = m->ev_io_done = nullptr;
}

}  // namespace
}  // namespace vof

using namespace vof;

extern "C" {

const char* vof_last_error(void) { return g_err.c_str(); }

void vof_default_options(vof_options* o) {
  if (!o) return;
  o->alpha_eps = 1e-12;
  o->tol_alpha = 1e-12;
  o->max_bisect = 100;
  o->root_mode = VOF_ROOT_BISECT;
  o->alpha_iso = 0.5;
  o->htc = 0;
  o->max_secant = 2;
  o->xf_mode = VOF_XF_RECON;
  o->vertex_mode = 0;
  o->group_size = 0;
  o->extrap = 0;
  o->extrap_max_iter = 120;
  o->extrap_tol = 1e-3;
  o->lsq_variant = 0;
  o->guess = 0;
  o->extrap_poll_limit = 1 << 22;
  o->root_narrow = 0x1p-20;
}

vof_status vof_mesh_create(const vof_mesh_desc* desc, void* stream, vof_mesh** out) {
  if (!desc || !out) { set_error("null argument"); return VOF_EINVAL; }
  *out = nullptr;
  vof_mesh* m = new (std::nothrow) vof_mesh;
  if (!m) { set_error("host allocation failed"); return VOF_ENOMEM; }
  vof_status st;
  try {
    st = create(desc, (cudaStream_t)stream, m);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    st = VOF_ENOMEM;
  } catch (...) {
    set_error("unexpected host exception in vof_mesh_create");
    st = VOF_EINVAL;
  }
  if (st != VOF_OK) {
    destroy(m);
    delete m;
    return st;
  }
  *out = m;
  return VOF_OK;
}

vof_status vof_mesh_destroy(vof_mesh* m) {
  if (!m) return VOF_EINVAL;
  destroy(m);
  delete m;
  return VOF_OK;
}

vof_status vof_mesh_info(const vof_mesh* m, int64_t* out5) {
  if (!m || !out5) { set_error("null argument"); return VOF_EINVAL; }
  out5[0] = m->n_cells; out5[1] = m->n_faces; out5[2] = m->n_verts; out5[3] = m->max_cv; out5[4] = m->max_ct;
  return VOF_OK;
}

vof_status vof_mesh_bins(const vof_mesh* m, int64_t* cells5) {
  if (!m || !cells5) { set_error("null argument"); return VOF_EINVAL; }
  for (int b = 0; b < vof::kBins; ++b) cells5[b] = m->bin_cells[b];
  return VOF_OK;
}

static vof_status check_opt(const vof_options* o) {
  if (!o) { set_error("null options"); return VOF_EINVAL; }
  if (!(o->alpha_eps >= 0 && o->alpha_eps < 0.5) || !(o->tol_alpha > 0) || o->max_bisect < 1 || o->max_bisect > 1000 ||
      o->root_mode < VOF_ROOT_BISECT || o->root_mode > VOF_ROOT_FIXED || !(o->alpha_iso > 0.0 && o->alpha_iso < 1.0) ||
      o->max_secant < 0 || o->max_secant > 8 || o->htc < 0 || o->htc > 1 || o->extrap < 0 || o->extrap > 1 ||
      o->extrap_max_iter < 1 || o->extrap_max_iter > kExMaxIter || !(o->extrap_tol > 0) ||
      !std::isfinite(o->extrap_tol) || o->lsq_variant < 0 || o->lsq_variant > 15 || o->guess < 0 || o->guess > 1 ||
      o->extrap_poll_limit < 1 || o->extrap_poll_limit > (1 << 30) ||
      !(o->root_narrow >= 0x1p-20 && o->root_narrow <= 2.0) ||
      o->xf_mode < 0 || o->xf_mode > 2 || o->vertex_mode < 0 || o->vertex_mode > 1 ||
      !(o->group_size == 0 || o->group_size == 1 || o->group_size == 2 || o->group_size == 4 || o->group_size == 8 ||
        o->group_size == 16 || o->group_size == 32)) {
    set_error("option out of range");
    return VOF_EINVAL;
  }
  return VOF_OK;
}

vof_status vof_reconstruct(vof_mesh* m, const double* d_alpha, const vof_options* opt, void* stream) {
  if (!m || !d_alpha) { set_error("null argument"); return VOF_EINVAL; }
  if (vof_status st = check_opt(opt)) return st;
  vof_status st = launch_reconstruct(m, d_alpha, *opt, (cudaStream_t)stream);
  if (st == VOF_OK) m->recon_done = true;
  return st;
}

static vof_status check_source_args(const vof_mesh* m, const double* d_alpha, const double* d_T, const vof_props* props,
                                    const vof_options* opt, const double* d_mdot, const double* d_Q,
                                    const double* d_totals) {
  if (!m || !d_alpha || !d_T || !props || !d_mdot || !d_Q || !d_totals) { set_error("null argument"); return VOF_EINVAL; }
  if (vof_status st = check_opt(opt)) return st;
  if (opt->extrap && m->max_cf > kExMaxFaces) {
    set_error("options.extrap = 1 needs cells of at most 64 faces");
    return VOF_EINVAL;
  }
  if (!(props->h_lv > 0) || !(props->k_l >= 0) || !(props->k_v >= 0) || !std::isfinite(props->T_sat)) {
    set_error("bad properties");
    return VOF_EINVAL;
  }
  return VOF_OK;
}

vof_status vof_phase_change_source(vof_mesh* m, const double* d_alpha, const double* d_T, const double* d_T_bnd,
                                   const vof_props* props, const vof_options* opt, double* d_mdot, double* d_Q,
                                   double* d_totals, void* stream) {
  if (vof_status st = check_source_args(m, d_alpha, d_T, props, opt, d_mdot, d_Q, d_totals)) return st;
  if (!m->recon_done) { set_error("vof_phase_change_source called before vof_reconstruct"); return VOF_ESTATE; }
  StepArgs a{d_alpha, d_T, d_T_bnd, d_mdot, d_Q, d_totals, *props, *opt};
  return launch_source(m, a, (cudaStream_t)stream);
}

vof_status vof_step(vof_mesh* m, const double* d_alpha, const double* d_T, const double* d_T_bnd,
                    const vof_props* props, const vof_options* opt, double* d_mdot, double* d_Q, double* d_totals,
                    void* stream) {
  // both stages see the same alpha, so the crossing-face list runs on a side branch
  if (vof_status st = check_source_args(m, d_alpha, d_T, props, opt, d_mdot, d_Q, d_totals)) return st;
  vof_status st = launch_reconstruct(m, d_alpha, *opt, (cudaStream_t)stream, true);
  if (st) return st;
  m->recon_done = true;
  StepArgs a{d_alpha, d_T, d_T_bnd, d_mdot, d_Q, d_totals, *props, *opt};
  return launch_source(m, a, (cudaStream_t)stream, true);
}

}  // extern "C"

// Step kernels of the hot path: interface selection, vertex field, isovalue root search (bisection,
// learned guess with secant steps, interval cubic, or a fixed isovalue), interface geometry,
// crossing faces and their heat-transfer coefficients, interface-modified least squares, per-side
// gradients and phase-change source, deterministic totals.
//
// Cut volume (paper Sec. 2.1, Eq. edge_intersection; reading: tetrahedralisation by the cell's
// own vertices, phi linear per tetrahedron): for a tetrahedron with corner values p_i and k corners
// at or above c the wet fraction is
//   k = 1 (wet a):         (p_a - c)^3 / prod_{j != a} (p_a - p_j)
//   k = 3 (dry d):     1 - (c - p_d)^3 / prod_{j != d} (p_j - p_d)
//   k = 2 (wet a, b):  [wa^2 wb^2 + (uc + ud) wa wb (wa + wb) + uc ud (wa^2 + wa wb + wb^2)]
//                       / [(p_a - p_c)(p_a - p_d)(p_b - p_c)(p_b - p_d)]
// with w = p - c on wet corners and u = c - p on dry corners: every denominator is a product of
// (wet - dry) differences, so no term is singular and nothing cancels.
#include <cooperative_groups.h>
#include <math_constants.h>
#include <cstring>

#include "vof_internal.cuh"

namespace vof {
namespace {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;

// |x| as an order-preserving integer key, so that magnitude tests stay off the FP64 pipe (an
// FP64 compare costs a warp instruction on the 1/64-rate pipe, like an FMA)
__device__ __forceinline__ uint64_t mag(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool positive(double x) { return __double_as_longlong(x) > 0; }  // x > 0
__device__ __forceinline__ double flip_if(double x, bool f) {  // -x when f, by the sign bit
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(x) ^ ((unsigned long long)f << 63)));
}
__device__ __forceinline__ bool inside(double x, double L, double H) {  // L < x < H
  const uint64_t k = okey(x);
  return k > okey(L) && k < okey(H);
}
__device__ __forceinline__ double dmax(double a, double b) { return okey(a) >= okey(b) ? a : b; }
__device__ __forceinline__ double dmin(double a, double b) { return okey(a) <= okey(b) ? a : b; }

template <int G>
__device__ __forceinline__ uint64_t group_umin(uint64_t v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = min(v, (uint64_t)__shfl_xor_sync(mask, (unsigned long long)v, o));
  return v;
}
template <int G>
__device__ __forceinline__ uint64_t group_umax(uint64_t v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = max(v, (uint64_t)__shfl_xor_sync(mask, (unsigned long long)v, o));
  return v;
}

template <int G>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}
template <int G>
__device__ __forceinline__ double group_min(double v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(mask, v, o));
  return v;
}
template <int G>
__device__ __forceinline__ double group_max(double v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(mask, v, o));
  return v;
}

struct Vec3 {
  double x, y, z;
};
__device__ __forceinline__ Vec3 v3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Vec3 operator*(Vec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// First work of a step: step stamp, counters reset (run by one thread of the first kernel).
__device__ __forceinline__ void begin_step(Counters* cn) {
  cn->step += 1;
  cn->reduce_done = 0;
  cn->n_iface = cn->n_band = cn->n_crossing = cn->n_uvert = 0;
  cn->n_degenerate = cn->n_not_converged = cn->n_fallback = cn->n_singular = cn->n_no_side = cn->n_mlp_skipped = 0;
  cn->evals_total = 0;
  cn->tet_evals = cn->tets_prepared = cn->tets_sectioned = cn->evals32_total = 0;
  for (int b = 0; b < kBins; ++b) cn->bin_count[b] = cn->bin_next[b] = cn->slow_count[b] = cn->slow_next[b] = 0;
  for (int k = 0; k < 6; ++k) cn->extrap_iters[k] = 0;
}

__device__ __forceinline__ bool is_iface(double a, double eps) { return a > eps && a < 1.0 - eps; }

// Phase tests of alpha on its bits (integer pipe; same results as the FP64 comparisons): liquid
// iff alpha > 1/2, vapour iff alpha < 1/2; NaN is neither, and so is alpha = 1/2.
constexpr uint64_t kKeyHalf = 0xbfe0000000000000ull;  // okey(0.5)
__device__ __forceinline__ bool not_nan(double a) {
  return ((uint64_t)__double_as_longlong(a) & 0x7fffffffffffffffull) <= 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool liquid(double a) { return okey(a) > kKeyHalf && not_nan(a); }
__device__ __forceinline__ bool vapour(double a) { return okey(a) < kKeyHalf && not_nan(a); }
// (alpha_P - 1/2)(alpha_Q - 1/2) < 0: one strictly above 1/2, the other strictly below
__device__ __forceinline__ bool crossing_pair(double aP, double aQ) {
  return (liquid(aP) && vapour(aQ)) || (vapour(aP) && liquid(aQ));
}
// eps < alpha < 1 - eps on the bits, with the two bounds' keys computed once per thread
struct IfaceKeys {
  uint64_t lo, hi;
};
__device__ __forceinline__ IfaceKeys iface_keys(double eps) { return {okey(eps), okey(1.0 - eps)}; }
__device__ __forceinline__ bool is_iface_k(double a, IfaceKeys k) {
  const uint64_t x = okey(a);
  return x > k.lo && x < k.hi && not_nan(a);
}

// ---- the step's selection as one cooperative kernel ----------------------------------------------
// Three phases separated by grid-wide barriers (the launch is cooperative, so every block is
// resident). Each block owns a contiguous range of tiles of kSelTile cells (each thread takes
// kSelTile / kThreads consecutive cells of a tile). (1) Step stamp and counters; the interface
// flags of the block's tiles, kept as ballot masks, and the block's count. (2) The block's offset
// from the counts of the blocks before it, then its tiles in order: the order-preserving scatter of
// the interface list and the tetrahedron-count bins (block-aggregated appends). (3) Band and vertex
// stamps, the band list, and the vertex field of each vertex of an interface cell, computed by the
// block that stamps the vertex first.
constexpr int kSelLanes = 8;  // lanes per interface cell in the selection's phase 3

__device__ __forceinline__ int64_t block_sum(int64_t v, int64_t* s8) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s8[threadIdx.x >> 5] = v;
  __syncthreads();
  int64_t t = 0;
  for (int w = 0; w < kThreads / 32; ++w) t += s8[w];
  return t;
}

__global__ void __launch_bounds__(kThreads) k_select(MeshView M, const double* alpha, double eps, int vertex_mode,
                                                     int max_cf, Workspace W) {
  cg::grid_group grid = cg::this_grid();
  constexpr int kPer = kSelTile / kThreads;  // consecutive cells per thread in a tile
  static_assert(kPer >= 1 && kPer <= 32 && kSelTile % kThreads == 0, "tile layout");
  // (kThreads / kSelLanes) * (1 + max faces per cell) band cells, then as many times the maximum
  // vertices per cell
  extern __shared__ int32_t band_buf[];
  __shared__ int64_t s8[kThreads / 32];
  __shared__ int wpre[kThreads / 32 + 1];
  __shared__ int s_bin[kBins], s_nb;
  __shared__ unsigned long long s_binbase[kBins], s_gb;
  const int64_t nc = M.n_cells;
  const int64_t ntiles = (nc + kSelTile - 1) / kSelTile;
  // each block takes a contiguous range of tiles, so that one prefix over the blocks' totals
  // places every tile
  const int64_t tpb = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_lo = min((int64_t)blockIdx.x * tpb, ntiles), t_hi = min(t_lo + tpb, ntiles);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const IfaceKeys ik = iface_keys(eps);
  // (1) interface flags of this thread's kPer consecutive cells (kept as one ballot mask per warp
  // and cell position, so that phase 2 does not read alpha again), counts per tile and per block
  if (blockIdx.x == 0 && threadIdx.x == 0) begin_step(W.counters);
  int64_t mine = 0;
  for (int64_t t = t_lo; t < t_hi; ++t) {
    const int64_t c0 = t * kSelTile + (int64_t)threadIdx.x * kPer;
    unsigned f = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (c0 + k < nc && is_iface_k(alpha[c0 + k], ik)) f |= 1u << k;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const unsigned b = __ballot_sync(0xffffffffu, (f >> k) & 1u);
      if (lane == 0) W.sel_mask[(t * (kThreads / 32) + wid) * kPer + k] = b;
    }
    mine += __popc(f);
  }
  const int64_t btot = block_sum(mine, s8);
  if (threadIdx.x == 0) W.sel_tot[blockIdx.x] = btot;
  grid.sync();
  // (2) this block's offset from the totals of the blocks before it; the tiles in order
  const uint32_t step = W.counters->step;
  int64_t pos = 0;
  {
    int64_t before = 0, all = 0;
    for (int64_t u = threadIdx.x; u < gridDim.x; u += blockDim.x) {
      const int64_t v = W.sel_tot[u];
      all += v;
      if (u < blockIdx.x) before += v;
    }
    pos = block_sum(before, s8);
    const int64_t total = block_sum(all, s8);
    if (blockIdx.x == 0 && threadIdx.x == 0) W.counters->n_iface = total;
  }
  for (int64_t t = t_lo; t < t_hi; ++t) {
    unsigned f = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) f |= ((W.sel_mask[(t * (kThreads / 32) + wid) * kPer + k] >> lane) & 1u) << k;
    // exclusive scan of the per-thread counts: within the warp, then over the warps
    const int cnt = __popc(f);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wpre[wid + 1] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      wpre[0] = 0;
      for (int w = 1; w <= kThreads / 32; ++w) wpre[w] += wpre[w - 1];
    }
    if (threadIdx.x < kBins) s_bin[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p = pos + wpre[wid] + incl - cnt;
    // bins: slots within the block from shared counters, one global atomic per bin and tile
    const int64_t c0 = t * kSelTile + (int64_t)threadIdx.x * kPer;
    int bslot[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      bslot[k] = -1;
      if ((f >> k) & 1u) {
        const int64_t c = c0 + k;
        const int64_t slot = p + __popc(f & ((1u << k) - 1u));
        W.iface_idx[slot] = (int32_t)c;
        W.iface_slot[c] = (int32_t)slot;
        W.iface_stamp[c] = step;
        const int b = bin_of((int)(M.cell_tet_off[c + 1] - M.cell_tet_off[c]));
        bslot[k] = (b << 24) | atomicAdd(&s_bin[b], 1);
      }
    }
    __syncthreads();
    if (threadIdx.x < kBins)
      s_binbase[threadIdx.x] =
          s_bin[threadIdx.x] ? atomicAdd((unsigned long long*)&W.counters->bin_count[threadIdx.x],
                                         (unsigned long long)s_bin[threadIdx.x]) : 0ull;
    pos += wpre[kThreads / 32];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (bslot[k] >= 0) {
        const int b = bslot[k] >> 24;
        W.bin_list[(size_t)b * nc + s_binbase[b] + (bslot[k] & 0xffffff)] = (int32_t)(p + __popc(f & ((1u << k) - 1u)));
      }
  }
  grid.sync();
  // (3) kSelLanes lanes per interface cell, kThreads / kSelLanes cells per block pass: lane j takes
  // face j and vertex j (and j + kSelLanes, ...). New band cells and newly stamped vertices go to
  // shared buffers; one atomic per pass appends the band cells to the band list, and the block then
  // computes the field value of each vertex it stamped first, a thread per vertex (full warps on
  // the FP64 pipe).
  {
    int32_t* vert_buf = band_buf + (kThreads / kSelLanes) * (1 + max_cf);
    __shared__ int s_nv;
    const int sl = threadIdx.x % kSelLanes, scell = threadIdx.x / kSelLanes;
    const int64_t n = W.counters->n_iface;
    for (int64_t base = (int64_t)blockIdx.x * (kThreads / kSelLanes); base < n;
         base += (int64_t)gridDim.x * (kThreads / kSelLanes)) {
      if (threadIdx.x == 0) s_nb = s_nv = 0;
      __syncthreads();
      const int64_t i = base + scell;
      if (i < n) {
        const int32_t c = W.iface_idx[i];
        if (sl == 0 && atomicExch(&W.band_stamp[c], step) != step) band_buf[atomicAdd(&s_nb, 1)] = c;
        const int64_t f0 = M.cell_face_off[c], f1 = M.cell_face_off[c + 1];
        const int64_t v0 = M.cell_vert_off[c], v1 = M.cell_vert_off[c + 1];
        for (int64_t j = sl; j < max(f1 - f0, v1 - v0); j += kSelLanes) {
          if (f0 + j < f1) {
            const int32_t fc = M.cell_face[f0 + j] & 0x7fffffff;
            const int32_t q = M.face_owner[fc] == c ? M.face_neigh[fc] : M.face_owner[fc];
            if (q >= 0 && atomicExch(&W.band_stamp[q], step) != step) band_buf[atomicAdd(&s_nb, 1)] = q;
          }
          if (v0 + j < v1) {
            const int32_t v = M.cell_vert[v0 + j];
            if (atomicExch(&W.vert_stamp[v], step) != step) vert_buf[atomicAdd(&s_nv, 1)] = v;
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_gb = s_nb ? atomicAdd((unsigned long long*)&W.counters->n_band, (unsigned long long)s_nb) : 0ull;
      // vertex field (R1): inverse-distance weights, or the plain mean
      for (int k = threadIdx.x; k < s_nv; k += blockDim.x) {
        const int32_t v = vert_buf[k];
        const int64_t k0 = M.vert_cell_off[v], k1 = M.vert_cell_off[v + 1];
        double sum = 0;
        if (vertex_mode == 0) {
          // four cells' loads in flight at a time; the sum keeps the cell order
          int64_t e = k0;
          for (; e + 4 <= k1; e += 4) {
            const int32_t ca = M.vert_cell[e], cb = M.vert_cell[e + 1], cc = M.vert_cell[e + 2], cd = M.vert_cell[e + 3];
            const double wa = M.vert_w[e], wb = M.vert_w[e + 1], wc = M.vert_w[e + 2], wd = M.vert_w[e + 3];
            const double aa = alpha[ca], ab = alpha[cb], ac = alpha[cc], ad = alpha[cd];
            sum = fma(wa, aa, sum);
            sum = fma(wb, ab, sum);
            sum = fma(wc, ac, sum);
            sum = fma(wd, ad, sum);
          }
          for (; e < k1; ++e) sum = fma(M.vert_w[e], alpha[M.vert_cell[e]], sum);
        } else {
          for (int64_t e = k0; e < k1; ++e) sum += alpha[M.vert_cell[e]];
          sum /= (double)(k1 - k0);
        }
        W.phi_v[v] = sum;
        const float h = __double2float_rn(sum);
        W.phi_ff[v] = make_float2(h, __double2float_rn(sum - (double)h));
      }
      __syncthreads();
      for (int k = threadIdx.x; k < s_nb; k += blockDim.x) W.band_idx[s_gb + k] = band_buf[k];
      __syncthreads();
    }
  }
}

// ---- isovalue root search (R2, R3); the interface geometry follows in k_geom -----------------------
// Once per cell and step every tetrahedron's corner values are sorted (s0 >= s1 >= s2 >= s3) and
// its wet volume is written, for each number k of corners at or above c, as a cubic in a local
// variable x = ref_k - c:
//   k = 1: x = s0 - c,  V x^3 / (d01 d02 d03)
//   k = 2: x = s1 - c,  V [a^2 e f + 3 a e f x + 3 e f x^2 - (a + e + f) x^3] / [e f (a + e)(a + f)]
//          with a = s0 - s1, e = s1 - s2, f = s1 - s3 (the expansion of the bracket in the header)
//   k = 3: x = s3 - c,  V + V x^3 / (d03 d13 d23)
//   k = 0: 0, k = 4: V
// so an evaluation is one integer classification, selects, and the same three FMAs (Horner) in
// every lane: no division and no divergent FP64 code. Every term is bounded by V.
struct TetRow {
  double s0, s1, s2, s3;      // corner values, descending
  double a2, b2, c2, d2;      // k = 2 cubic (times V)
  double d1, d3, v;           // k = 1 and k = 3 cubic coefficients, V
};

__device__ __forceinline__ void cswap(uint64_t& ka, double& va, uint64_t& kb, double& vb) {
  // descending order by key
  const bool sw = ka < kb;
  const uint64_t tk = sw ? kb : ka;
  kb = sw ? ka : kb;
  ka = tk;
  const double tv = sw ? vb : va;
  vb = sw ? va : vb;
  va = tv;
}

__device__ __forceinline__ TetRow tet_prepare(double p0, double p1, double p2, double p3, double vt) {
  uint64_t k0 = okey(p0), k1 = okey(p1), k2 = okey(p2), k3 = okey(p3);
  cswap(k0, p0, k1, p1);
  cswap(k2, p2, k3, p3);
  cswap(k0, p0, k2, p2);
  cswap(k1, p1, k3, p3);
  cswap(k1, p1, k2, p2);
  const double d01 = p0 - p1, d02 = p0 - p2, d03 = p0 - p3, d12 = p1 - p2, d13 = p1 - p3, d23 = p2 - p3;
  TetRow r;
  r.s0 = p0; r.s1 = p1; r.s2 = p2; r.s3 = p3;
  r.v = vt;
  // One division per tetrahedron: R = vt / (product of the six differences, a zero difference
  // entering as 1); each coefficient is R times the differences missing from its own
  // denominator. A zero denominator means the case cannot occur (its interval is empty), so its
  // coefficients are 0.
  // corner values differ exactly when their keys do (keys sorted descending)
  const bool n01 = k0 > k1, n02 = k0 > k2, n12 = k1 > k2, n23 = k2 > k3;
  const double e01 = n01 ? d01 : 1.0, e02 = n02 ? d02 : 1.0, e03 = k0 > k3 ? d03 : 1.0;
  const double e12 = n12 ? d12 : 1.0, e13 = k1 > k3 ? d13 : 1.0, e23 = n23 ? d23 : 1.0;
  const double f1213 = e12 * e13, fA = f1213 * e23, fB = e01 * e02, fC = e01 * e23;
  const double prod = fA * (fB * e03);  // >= 0
  double d1, d3, vk, vke;
  if (__double_as_longlong(prod) > __double_as_longlong(1e-280)) {
    const double R = vt / prod;
    d1 = R * fA;             // vt / (d01 d02 d03)
    d3 = R * (fB * e12);     // vt / (d03 d13 d23)
    vk = R * (fC * f1213);   // vt / (d02 d03)
    vke = R * fC;            // vt / (d02 d03 d12 d13)
  } else {
    d1 = vt / (e01 * (e02 * e03));
    d3 = vt / (e03 * (e13 * e23));
    vk = vt / (e02 * e03);
    vke = vk / f1213;
  }
  r.d1 = n01 ? d1 : 0.0;
  r.d3 = n23 ? d3 : 0.0;
  if (n02 && n12) {
    r.a2 = vk * (d01 * d01);
    r.b2 = 3.0 * vk * d01;
    r.c2 = 3.0 * vk;
    r.d2 = -vke * (d01 + d12 + d13);
  } else {
    r.a2 = r.b2 = r.c2 = r.d2 = 0.0;
  }
  return r;
}

// Wet volume of a prepared tetrahedron at c (kc = okey(c)).
__device__ __forceinline__ double tet_wet_volume(const TetRow& r, uint64_t kc, double c) {
  const int k = (okey(r.s0) >= kc) + (okey(r.s1) >= kc) + (okey(r.s2) >= kc) + (okey(r.s3) >= kc);
  const double ref = k == 1 ? r.s0 : (k == 2 ? r.s1 : r.s3);
  const double A = k == 2 ? r.a2 : (k >= 3 ? r.v : 0.0);
  const double B = k == 2 ? r.b2 : 0.0;
  const double C = k == 2 ? r.c2 : 0.0;
  const double D = k == 1 ? r.d1 : (k == 2 ? r.d2 : (k == 3 ? r.d3 : 0.0));
  const double x = ref - c;
  return fma(fma(fma(D, x, C), x, B), x, A);
}

// The piece of a tetrahedron that straddles a vertex interval (va, vb] of its cell (kvb =
// okey(vb)): its wet volume there is one cubic A + B x + C x^2 + D x^3 in x = ref - c (the case
// of its nk corners at or above vb), added to q0..q3 expanded about cm (x = (ref - cm) - y). Only
// that case's coefficients are formed, by selecting its difference factors before one division:
// wet corners lie at or above vb and dry ones at or below va, so every denominator is a product of
// (wet - dry) differences, all positive.
__device__ __forceinline__ void tet_piece(double p0, double p1, double p2, double p3, double vt, uint64_t kvb,
                                          double cm, double& q0, double& q1, double& q2, double& q3) {
  uint64_t k0 = okey(p0), k1 = okey(p1), k2 = okey(p2), k3 = okey(p3);
  cswap(k0, p0, k1, p1);
  cswap(k2, p2, k3, p3);
  cswap(k0, p0, k2, p2);
  cswap(k1, p1, k3, p3);
  cswap(k1, p1, k2, p2);
  const int nk = (k0 >= kvb) + (k1 >= kvb) + (k2 >= kvb) + (k3 >= kvb);  // 1, 2 or 3
  const bool one = nk == 1, two = nk == 2;
  // denominators: nk = 1: d01 d02 d03; nk = 2: d02 d03 d12 d13; nk = 3: d03 d13 d23
  const double X = (one ? p0 : (two ? p0 : p1)) - (one ? p1 : (two ? p2 : p3));  // d01 | d02 | d13
  const double Y = (one ? p0 : (two ? p1 : p2)) - (one ? p2 : (two ? p2 : p3));  // d02 | d12 | d23
  const double Z = (two ? p1 : 1.0) - (two ? p3 : 0.0);                          // 1   | d13 | 1
  const double d03 = p0 - p3;
  const double YZ = Y * Z;
  const double R = vt / ((d03 * X) * YZ);
  // nk = 2: a = d01, e = d12 (= Y), f = d13 (= Z); vk = vt / (d02 d03) = R e f
  const double a = p0 - p1;
  const double vk = R * YZ;
  const double A = two ? vk * (a * a) : (one ? 0.0 : vt);
  const double B = two ? 3.0 * (vk * a) : 0.0;
  const double C = two ? 3.0 * vk : 0.0;
  const double D = two ? -R * (a + (Y + Z)) : R;
  const double dl = (one ? p0 : (two ? p1 : p3)) - cm;
  q0 += fma(fma(fma(D, dl, C), dl, B), dl, A);
  const double D3 = 3.0 * D;
  q1 -= fma(fma(D3, dl, 2.0 * C), dl, B);
  q2 += fma(D3, dl, C);
  q3 -= D;
}

template <int G>
__device__ __forceinline__ double liquid_volume(const TetRow* rows, int nt, int lane, unsigned mask, double c) {
  const uint64_t kc = okey(c);
  double part = 0;
  for (int t = lane; t < nt; t += G) part += tet_wet_volume(rows[t], kc, c);
  return group_sum<G>(part, mask);
}

// FP32 rows in normalised values (u = (phi - lo)/(hi - lo), volumes / V): the same cubics on
// the FP32 pipe, used only to refine the learned guess before the FP64 phase.
struct TetRow32 {
  float s0, s1, s2, s3, a2, b2, c2, d2, d1, d3, v;
};

__device__ __forceinline__ uint32_t okey32(float x) {
  uint32_t b = __float_as_uint(x);
  b = b == 0x80000000u ? 0u : b;
  return (b >> 31) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ void cswap32(uint32_t& ka, float& va, uint32_t& kb, float& vb) {
  const bool sw = ka < kb;
  const uint32_t tk = sw ? kb : ka;
  kb = sw ? ka : kb;
  ka = tk;
  const float tv = sw ? vb : va;
  vb = sw ? va : vb;
  va = tv;
}

__device__ __forceinline__ TetRow32 tet_prepare32(float p0, float p1, float p2, float p3, float vt) {
  uint32_t k0 = okey32(p0), k1 = okey32(p1), k2 = okey32(p2), k3 = okey32(p3);
  cswap32(k0, p0, k1, p1);
  cswap32(k2, p2, k3, p3);
  cswap32(k0, p0, k2, p2);
  cswap32(k1, p1, k3, p3);
  cswap32(k1, p1, k2, p2);
  const float d01 = p0 - p1, d02 = p0 - p2, d03 = p0 - p3, d12 = p1 - p2, d13 = p1 - p3, d23 = p2 - p3;
  TetRow32 r;
  r.s0 = p0; r.s1 = p1; r.s2 = p2; r.s3 = p3;
  r.v = vt;
  const float P1 = d01 * (d02 * d03), P3 = d03 * (d13 * d23), K = d02 * d03, EF = d12 * d13;
  r.d1 = P1 > 0.f ? vt / P1 : 0.f;
  r.d3 = P3 > 0.f ? vt / P3 : 0.f;
  if (K > 0.f && EF > 0.f) {
    const float vk = vt / K;
    r.a2 = vk * (d01 * d01);
    r.b2 = 3.f * vk * d01;
    r.c2 = 3.f * vk;
    r.d2 = -(vk / EF) * (d01 + d12 + d13);
  } else {
    r.a2 = r.b2 = r.c2 = r.d2 = 0.f;
  }
  return r;
}

template <int G>
__device__ __forceinline__ float liquid_volume32(const TetRow32* rows, int nt, int lane, unsigned mask, float u) {
  const uint32_t kc = okey32(u);
  float part = 0.f;
  for (int t = lane; t < nt; t += G) {
    const TetRow32& r = rows[t];
    const int k = (okey32(r.s0) >= kc) + (okey32(r.s1) >= kc) + (okey32(r.s2) >= kc) + (okey32(r.s3) >= kc);
    const float ref = k == 1 ? r.s0 : (k == 2 ? r.s1 : r.s3);
    const float A = k == 2 ? r.a2 : (k >= 3 ? r.v : 0.f);
    const float B = k == 2 ? r.b2 : 0.f;
    const float C = k == 2 ? r.c2 : 0.f;
    const float D = k == 1 ? r.d1 : (k == 2 ? r.d2 : (k == 3 ? r.d3 : 0.f));
    const float x = ref - u;
    part += fmaf(fmaf(fmaf(D, x, C), x, B), x, A);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(mask, part, o);
  return part;
}

// ---- pair ("double-float") arithmetic on the FP32 pipe ---------------------------------------------
// A value is hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits. The sums use Knuth's
// error-free two-sum, the products the FMA-based exact product (Dekker); every step is written
// with the round-to-nearest intrinsics so that nothing is contracted or reordered. On GB300 an
// FP64 instruction costs 64 FP32 issue slots, so the interface geometry (about 130 FP64
// operations per cut tetrahedron) runs several times faster in pairs, at a precision (1e-14
// relative) far inside the tolerances of its outputs.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_make(float2 v) { return {v.x, v.y}; }
// FP32 -> FP64 by the bits (exact; zero, normal and infinite/NaN values), so that the widening
// stays off the FP64 unit; subnormals take the conversion instruction
__device__ __forceinline__ double fl2d(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu, mant = b & 0x7fffffu;
  const uint64_t sgn = (uint64_t)(b & 0x80000000u) << 32;
  if (e == 0u) {
    if (mant == 0u) return __longlong_as_double((long long)sgn);
    return (double)f;
  }
  const uint64_t de = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);  // 1023 - 127
  return __longlong_as_double((long long)(sgn | (de << 52) | ((uint64_t)mant << 29)));
}
__device__ __forceinline__ double ff_to_double(ff a) { return fl2d(a.hi) + fl2d(a.lo); }
// FP64 -> FP32, round to nearest even, by the bits (the conversion instruction runs on the FP64
// unit); a value whose float is not normal (zero, subnormal, overflow, infinite, NaN) takes the
// conversion instruction. A carry out of the mantissa moves to the next binade, as rounding does.
__device__ __forceinline__ float d2f(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e < 1 || e > 254) return __double2float_rn(x);
  const uint64_t m = b & 0xfffffffffffffull;
  uint32_t r = ((uint32_t)e << 23) | (uint32_t)(m >> 29);
  const uint32_t rem = (uint32_t)(m & 0x1fffffffull), half = 0x10000000u;
  r += (rem > half || (rem == half && (r & 1u))) ? 1u : 0u;
  return __uint_as_float(((uint32_t)(b >> 32) & 0x80000000u) | r);
}
__device__ __forceinline__ ff ff_of(double x) {
  const float h = d2f(x);
  return {h, d2f(x - fl2d(h))};
}
__device__ __forceinline__ ff ff_norm(float s, float e) {  // |s| >= |e|
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_norm(s, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_scale(ff a, float b) {  // b exact in FP32
  const float p = __fmul_rn(a.hi, b);
  return ff_norm(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
// 1 / a: FP32 reciprocal and one Newton step on the pair residual
__device__ __forceinline__ ff ff_rcp(ff a) {
  const float y = __frcp_rn(a.hi);
  const float r = __fmaf_rn(-a.lo, y, __fmaf_rn(-a.hi, y, 1.0f));  // 1 - a y
  return ff_norm(y, __fmul_rn(y, r));
}
// 1 / sqrt(a), a > 0: FP32 estimate and one Newton step on the pair residual
__device__ __forceinline__ ff ff_rsqrt(ff a) {
  const float y = rsqrtf(a.hi);
  const ff ay2 = ff_scale(ff_scale(a, y), y);
  const float r = __fadd_rn(__fsub_rn(1.0f, ay2.hi), -ay2.lo);  // 1 - a y^2
  return ff_norm(y, __fmul_rn(__fmul_rn(0.5f, y), r));
}
struct ff3 {
  ff x, y, z;
};
__device__ __forceinline__ ff3 ff3_load(const float2* p) { return {ff_make(p[0]), ff_make(p[1]), ff_make(p[2])}; }
__device__ __forceinline__ ff3 ff3_add(ff3 a, ff3 b) { return {ff_add(a.x, b.x), ff_add(a.y, b.y), ff_add(a.z, b.z)}; }
__device__ __forceinline__ ff3 ff3_sub(ff3 a, ff3 b) { return {ff_sub(a.x, b.x), ff_sub(a.y, b.y), ff_sub(a.z, b.z)}; }
__device__ __forceinline__ ff3 ff3_mul(ff3 a, ff s) { return {ff_mul(a.x, s), ff_mul(a.y, s), ff_mul(a.z, s)}; }
__device__ __forceinline__ ff ff3_dot(ff3 a, ff3 b) {
  return ff_add(ff_add(ff_mul(a.x, b.x), ff_mul(a.y, b.y)), ff_mul(a.z, b.z));
}
__device__ __forceinline__ ff3 ff3_cross(ff3 a, ff3 b) {
  return {ff_sub(ff_mul(a.y, b.z), ff_mul(a.z, b.y)), ff_sub(ff_mul(a.z, b.x), ff_mul(a.x, b.z)),
          ff_sub(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}
__device__ __forceinline__ ff3 ff3_pick(int i, ff3 a, ff3 b, ff3 c, ff3 d) {
  return i == 0 ? a : (i == 1 ? b : (i == 2 ? c : d));
}
__device__ __forceinline__ ff ff_pick(int i, ff a, ff b, ff c, ff d) { return i == 0 ? a : (i == 1 ? b : (i == 2 ? c : d)); }
// Order of normalised pairs (|lo| <= ulp(hi) / 2, and hi = 0 only for the zero pair): by hi, then
// lo. Every test is false when a NaN is involved.
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool ff_eq(ff a, ff b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool ff_inside(ff y, ff L, ff H) { return ff_lt(L, y) && ff_lt(y, H); }  // L < y < H
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(b, a) ? b : a; }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__device__ __forceinline__ ff ff_mid(ff a, ff b) { return ff_scale(ff_add(a, b), 0.5f); }
// q0 + q1 y + q2 y^2 + q3 y^3 (Horner)
__device__ __forceinline__ ff ff_cubic(ff q0, ff q1, ff q2, ff q3, ff y) {
  return ff_add(ff_mul(ff_add(ff_mul(ff_add(ff_mul(q3, y), q2), y), q1), y), q0);
}
template <int G>
__device__ __forceinline__ ff group_sum_ff(ff v, unsigned mask) {
  // the pair sum is commutative bit for bit (the two-sum error is exact), so every lane of the
  // butterfly ends with the same pair
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = ff_add(v, ff{__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o)});
  return v;
}

// The section of tet_section in pair arithmetic, with positions relative to the cell's apex (P0 is
// the origin) and w_i = phi_i - c: the same quadrilateral of cut points, vector area (wet -> dry),
// area and area moment (about the apex).
__device__ void tet_section_ff(ff3 P1, ff3 P2, ff3 P3, ff w0, ff w1, ff w2, ff w3, unsigned m, ff3& A, ff& ar,
                               ff3& mom) {
  const ff3 P0 = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  const int k = __popc(m);
  const unsigned dm = ~m & 15u;
  int wi[4], dj[4];
  if (k == 2) {
    const int a = __ffs(m) - 1, b = 31 - __clz(m), cc = __ffs(dm) - 1, d = 31 - __clz(dm);
    wi[0] = a; dj[0] = cc;
    wi[1] = a; dj[1] = d;
    wi[2] = b; dj[2] = d;
    wi[3] = b; dj[3] = cc;
  } else {
    const unsigned rest = k == 1 ? dm : m;
    const int lone = k == 1 ? __ffs(m) - 1 : __ffs(dm) - 1;
    const int j0 = __ffs(rest) - 1, j2 = 31 - __clz(rest);
    const int j1 = __ffs(rest & ~(1u << j0) & ~(1u << j2)) - 1;
    if (k == 1) {
      wi[0] = lone; dj[0] = j0;
      wi[1] = lone; dj[1] = j1;
      wi[2] = lone; dj[2] = j2;
      wi[3] = lone; dj[3] = j2;
    } else {
      wi[0] = j0; dj[0] = lone;
      wi[1] = j1; dj[1] = lone;
      wi[2] = j2; dj[2] = lone;
      wi[3] = j2; dj[3] = lone;
    }
  }
  ff3 q[4];
  ff3 Pw0, Pd0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const ff3 Pw = ff3_pick(wi[e], P0, P1, P2, P3), Pd = ff3_pick(dj[e], P0, P1, P2, P3);
    const ff ww = ff_pick(wi[e], w0, w1, w2, w3), wd = ff_pick(dj[e], w0, w1, w2, w3);
    // t = (phi_w - c) / (phi_w - phi_d), in [0, 1)
    const ff t = ff_mul(ww, ff_rcp(ff_sub(ww, wd)));
    q[e] = ff3_add(Pw, ff3_mul(ff3_sub(Pd, Pw), t));
    if (e == 0) {
      Pw0 = Pw;
      Pd0 = Pd;
    }
  }
  const ff3 e1 = ff3_sub(q[1], q[0]), e2 = ff3_sub(q[2], q[0]), e3 = ff3_sub(q[3], q[0]);
  const ff3 A1 = ff3_cross(e1, e2), A2 = ff3_cross(e2, e3);
  const ff3 S = ff3_add(A1, A2);  // twice the vector area
  // orientation from the leading parts: the wet and the dry corner lie strictly apart
  const float o = S.x.hi * (Pd0.x.hi - Pw0.x.hi) + S.y.hi * (Pd0.y.hi - Pw0.y.hi) + S.z.hi * (Pd0.z.hi - Pw0.z.hi);
  const ff nn = ff3_dot(S, S);
  if (!(nn.hi > 0.f)) {
    const ff z = {0.f, 0.f};
    A = {z, z, z};
    ar = z;
    mom = {z, z, z};
    return;
  }
  const ff rs = ff_rsqrt(nn);
  ar = ff_scale(ff_mul(nn, rs), 0.5f);
  const ff half = o < 0.f ? ff{-0.5f, 0.f} : ff{0.5f, 0.f};
  A = {ff_mul(S.x, half), ff_mul(S.y, half), ff_mul(S.z, half)};
  // moment = (rs / 6) sum_i (A_i . S) (corner sum of triangle i)
  const ff sixth = {0.1666666716337204f, -4.967053879312289e-09f};  // 1/6 as a pair
  const ff r6 = ff_mul(rs, sixth);
  const ff wa = ff_mul(ff3_dot(A1, S), r6), wb = ff_mul(ff3_dot(A2, S), r6);
  const ff3 g02 = ff3_add(q[0], q[2]);
  mom = ff3_add(ff3_mul(ff3_add(g02, q[1]), wa), ff3_mul(ff3_add(g02, q[3]), wb));
}

// Unit normal (vapour -> liquid: against the wet -> dry vector area), area and centroid of a cell's
// interface from its summed pairs v = (vector area, area, area moment about the apex at a);
// still in pairs, then one FP64 addition per output.
__device__ __forceinline__ void geometry_outputs(const ff* v, double ax, double ay, double az, double& area,
                                                 Vec3& nrm, Vec3& xg) {
  area = ff_to_double(v[3]);
  const ff3 Av = {v[0], v[1], v[2]};
  const ff nn = ff3_dot(Av, Av);
  if (nn.hi > 0.f) {
    const ff rs = ff_neg(ff_rsqrt(nn));
    nrm = v3(ff_to_double(ff_mul(v[0], rs)), ff_to_double(ff_mul(v[1], rs)), ff_to_double(ff_mul(v[2], rs)));
  } else {
    nrm = v3(0, 0, 0);
  }
  if (v[3].hi > 0.f) {
    const ff ia = ff_rcp(v[3]);
    xg = v3(ax + ff_to_double(ff_mul(v[4], ia)), ay + ff_to_double(ff_mul(v[5], ia)),
            az + ff_to_double(ff_mul(v[6], ia)));
  } else {
    xg = v3(0, 0, 0);
  }
}

// Shared memory of one lane group of the root search (multiple of 8 bytes): the rows (FP64 rows of
// plain bisection, else the FP32 rows of the refinement), the FP64 and normalised FP32 vertex
// values, the tetrahedra's packed corners, the list of straddling tetrahedra.
__host__ __device__ inline size_t root_rows_bytes(int max_ct, int mode) {
  return ((size_t)max_ct * (mode == VOF_ROOT_BISECT ? sizeof(TetRow) : sizeof(TetRow32)) + 7) & ~(size_t)7;
}
__host__ __device__ inline size_t root_group_bytes(int max_ct, int max_cv, int mode) {
  return root_rows_bytes(max_ct, mode) + (size_t)max_cv * sizeof(double) + (size_t)((max_cv + 1) & ~1) * sizeof(float) +
         (size_t)((max_ct + 1) & ~1) * sizeof(uint32_t) + (size_t)((2 * max_ct + 7) & ~7);
}

template <int G>
__global__ void __launch_bounds__(kThreads, 2) k_root(MeshView M, const double* alpha, vof_options opt, Workspace W,
                                                   int max_ct, int max_cv, int mode, int use_mlp, int bin, int slow) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int gib = threadIdx.x / G;  // group in block
  const int lane = threadIdx.x % G;
  const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
  // per group: the rows; the cell's FP64 vertex values; its normalised vertex values (FP32, the
  // learned path); its tetrahedra's packed corner indices; the list of windowed rows. Every later
  // read of a vertex value or a tetrahedron's corners comes from shared memory.
  const size_t dv_bytes = (size_t)max_cv * sizeof(double);
  const size_t uv_bytes = (size_t)((max_cv + 1) & ~1) * sizeof(float);
  const size_t pk_bytes = (size_t)((max_ct + 1) & ~1) * sizeof(uint32_t);
  const size_t rw_bytes = root_rows_bytes(max_ct, mode);
  const size_t grp_bytes = root_group_bytes(max_ct, max_cv, mode);
  unsigned char* gbase = smem + (size_t)gib * grp_bytes;
  TetRow* rows = reinterpret_cast<TetRow*>(gbase);
  double* dvert = reinterpret_cast<double*>(gbase + rw_bytes);
  float* uvert = reinterpret_cast<float*>(gbase + rw_bytes + dv_bytes);
  uint32_t* tpk = reinterpret_cast<uint32_t*>(gbase + rw_bytes + dv_bytes + uv_bytes);
  uint16_t* actl = reinterpret_cast<uint16_t*>(gbase + rw_bytes + dv_bytes + uv_bytes + pk_bytes);
  // the bin's list, or (slow) the cells of the bin that the thread-per-cell kernel handed over
  const int64_t n_bin = slow ? W.counters->slow_count[bin] : W.counters->bin_count[bin];
  const int32_t* list = (slow ? W.slow_list : W.bin_list) + (size_t)bin * M.n_cells;
  unsigned long long* next = (unsigned long long*)(slow ? &W.counters->slow_next[bin] : &W.counters->bin_next[bin]);
  int64_t evals_acc = 0, tetev_acc = 0, prep_acc = 0, ev32_acc = 0;
  // each group takes the next cell of the bin when it is done with the last one: the learned
  // path's fallback cells cost ten times a typical cell, so a static split leaves SMs idle
  for (;;) {
    int64_t j = 0;
    if (lane == 0) j = (int64_t)atomicAdd(next, 1ull);
    j = __shfl_sync(mask, j, 0, G);
    if (j >= n_bin) break;
    const int64_t i = list[j];  // position in the interface list
    const int32_t cell = W.iface_idx[i];
    const int64_t v0 = M.cell_vert_off[cell];
    const int nv = (int)(M.cell_vert_off[cell + 1] - v0);
    const int64_t t0 = M.cell_tet_off[cell];
    const int nt = (int)(M.cell_tet_off[cell + 1] - t0);
    const int32_t* cv = M.cell_vert + v0;
    // the cell's vertex values and tetrahedra into shared memory; the range of the vertex values
    // by integer min/max of the order keys
    uint64_t klo = ~0ull, khi = 0ull;
    for (int j = lane; j < nv; j += G) {
      const double p = W.phi_v[cv[j]];
      dvert[j] = p;
      const uint64_t k = okey(p);
      klo = min(klo, k);
      khi = max(khi, k);
    }
    for (int t = lane; t < nt; t += G) tpk[t] = __ldg(M.cell_tet + t0 + t);
    const double lo = okey_inv(group_umin<G>(klo, mask)), hi = okey_inv(group_umax<G>(khi, mask));
    __syncwarp(mask);
    const double p_apex = dvert[0];
    // FP64 rows of the cell's tetrahedra (plain bisection only; the learned and interval-cubic
    // paths keep FP32 rows in that space and no FP64 rows)
    int n_rows = nt, n_prep = 0;  // rows evaluated; rows prepared for this cell
    auto prepare64 = [&]() {
      for (int t = lane; t < nt; t += G) {
        const uint32_t pk = tpk[t];
        rows[t] = tet_prepare(p_apex, dvert[pk & 255], dvert[(pk >> 8) & 255], dvert[(pk >> 16) & 255],
                              __ldg(M.tet_vol + t0 + t));
      }
      __syncwarp(mask);
      n_rows = nt;
      n_prep += nt;
    };
    // One pass over the tetrahedra for the vertex interval [va, vb] (consecutive vertex values of
    // the cell, so that no tetrahedron changes its number of wet corners inside it): those with
    // every corner at or above vb are wet over it (their volume goes to P0), those with every
    // corner at or below va dry; the others (compacted into actl, so that the FP64 work keeps the
    // lanes busy) are prepared in registers and their pieces, the cubics A + B x + C x^2 + D x^3 in
    // x = ref - c, expanded about cm = (va + vb)/2 and summed into P(y) = P0 + P1 y + P2 y^2 + P3 y^3,
    // y = c - cm. P is V_L exactly on [va, vb]. Returns the number of pieces.
    double cm = 0, P0 = 0, P1 = 0, P2 = 0, P3 = 0;
    auto interval_pass = [&](double va, double vb) -> int {
      const uint64_t kva = okey(va), kvb = okey(vb), ka = okey(p_apex);
      const int base = (threadIdx.x & 31) / G * G;
      const unsigned gbits = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
      double ws = 0;
      int n = 0;
      for (int r0 = 0; r0 < nt; r0 += G) {
        const int t = r0 + lane;
        bool act = false;
        if (t < nt) {
          const uint32_t pk = tpk[t];
          const uint64_t k1 = okey(dvert[pk & 255]), k2 = okey(dvert[(pk >> 8) & 255]), k3 = okey(dvert[(pk >> 16) & 255]);
          const uint64_t kmin = min(min(ka, k1), min(k2, k3)), kmax = max(max(ka, k1), max(k2, k3));
          if (kmin >= kvb) ws += __ldg(M.tet_vol + t0 + t);
          else act = kmax > kva;
        }
        const unsigned bal = (__ballot_sync(mask, act) >> base) & gbits;
        if (act) actl[n + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)t;
        n += __popc(bal);
      }
      __syncwarp(mask);
      cm = 0.5 * (va + vb);
      double q0 = ws, q1 = 0, q2 = 0, q3 = 0;
      for (int k = lane; k < n; k += G) {
        const int t = actl[k];
        const uint32_t pk = tpk[t];
        tet_piece(p_apex, dvert[pk & 255], dvert[(pk >> 8) & 255], dvert[(pk >> 16) & 255], __ldg(M.tet_vol + t0 + t),
                  kvb, cm, q0, q1, q2, q3);
      }
      P0 = group_sum<G>(q0, mask);
      P1 = group_sum<G>(q1, mask);
      P2 = group_sum<G>(q2, mask);
      P3 = group_sum<G>(q3, mask);
      __syncwarp(mask);
      n_prep += n;
      return n;
    };
    const double a = alpha[cell];
    const double invV = M.cell_ivol[cell];
    const uint64_t ktol = mag(opt.tol_alpha);
    int status = 0, evals = 0, evals32 = 0;
    int64_t tev = 0;  // tetrahedron evaluations
    double c_best;
    uint64_t kbest = 0;  // |f| at c_best, as a magnitude key
    // scalar comparisons on order keys and conversions by the bits: an FP64 compare or conversion
    // holds the FP64 unit like an FMA, for every lane group of the warp
    const double range = hi - lo;
    if (__double_as_longlong(range) < __double_as_longlong(1e-14)) {  // range >= 0
      status = VOF_ST_DEGENERATE;
      c_best = lo;
    } else {
      // f(lo) = 1 - alpha (everything wet), f(hi) = -alpha
      const double oma = 1.0 - a;
      kbest = min(mag(oma), mag(a));
      c_best = okey(oma) <= okey(a) ? lo : hi;
      double L = lo, H = hi;
      bool done = false;
      // f = V_L(c)/V - alpha at a point: best point and bracket updated, convergence test
      auto record = [&](double c, double f) {
        const uint64_t kf = mag(f);
        if (kf < kbest) { kbest = kf; c_best = c; }
        if (positive(f)) L = dmax(L, c); else H = dmin(H, c);
        if (kf <= ktol) done = true;
      };
      // over the prepared rows (plain bisection)
      auto eval64 = [&](double c) -> double {
        const double f = liquid_volume<G>(rows, n_rows, lane, mask, c) * invV - a;
        ++evals;
        tev += n_rows;
        record(c, f);
        return f;
      };
      // every tetrahedron prepared on the fly (the learned and interval-cubic paths' last resort,
      // when no vertex interval brackets the target: they keep no FP64 rows)
      auto eval_direct = [&](double c) -> double {
        const uint64_t kc = okey(c);
        double part = 0;
        for (int t = lane; t < nt; t += G) {
          const uint32_t pk = tpk[t];
          const TetRow r = tet_prepare(p_apex, dvert[pk & 255], dvert[(pk >> 8) & 255], dvert[(pk >> 16) & 255],
                                       __ldg(M.tet_vol + t0 + t));
          part += tet_wet_volume(r, kc, c);
        }
        const double f = group_sum<G>(part, mask) * invV - a;
        ++evals;
        tev += nt;
        n_prep += nt;
        record(c, f);
        return f;
      };
      if (mode != VOF_ROOT_BISECT) {
        // Learned path: MLP guess u0 of the normalised position u = (c - lo)/(hi - lo) (a cell
        // without features, more than 32 vertices, starts from 1 - alpha instead and is counted
        // as skipped); FP32 refinement of u (regula falsi with the Illinois modification, on FP32
        // tetrahedron rows in normalised values); then the FP64 phase: evaluations at the
        // refined guess and at a second point next to it, at most max_secant secant steps, and
        // bisection inside the bracket found so far as the counted fallback. The interval-cubic
        // mode runs the same FP32 refinement (from the MLP guess when the mesh has an MLP, else
        // from 1 - alpha) and replaces the FP64 phase.
        float u0 = use_mlp ? W.mlp_out[i] : 1.0f - d2f(a);
        if (!(u0 >= 0.0f)) {
          status |= VOF_ST_MLP_SKIPPED;
          u0 = 1.0f - d2f(a);
        }
        // Local FP32 coordinate u in [-1, 0] with the minority phase next to u = 0: for
        // alpha <= 1/2, u = (phi - phi_max)/range and the wet volume is matched to t = alpha; for
        // alpha > 1/2, u = (phi_min - phi)/range (the field reflected) and the wet volume of the
        // reflected field, the original dry volume, is matched to t = 1 - alpha. A small volume
        // fraction and a root next to an extreme vertex value then keep their relative precision.
        const bool refl = okey(a) > kKeyHalf;  // alpha > 1/2
        const double org = refl ? lo : hi;
        const float af = d2f(refl ? oma : a);
        float ubest, slope;
        {
          TetRow32* rows32 = reinterpret_cast<TetRow32*>(rows);
          // u from the vertex values' float pairs (FP32 work only): (phi - org) * dir / range
          const float r32 = __frcp_rn(d2f(range));
          const float su = refl ? -r32 : r32;
          const ff of = ff_of(org);
          for (int j = lane; j < nv; j += G) {
            const float2 pv = W.phi_ff[cv[j]];
            uvert[j] = __fmul_rn(__fadd_rn(__fsub_rn(pv.x, of.hi), __fsub_rn(pv.y, of.lo)), su);
          }
          __syncwarp(mask);
          for (int t = lane; t < nt; t += G) {
            const uint32_t pk = tpk[t];
            rows32[t] = tet_prepare32(uvert[0], uvert[pk & 255], uvert[(pk >> 8) & 255], uvert[(pk >> 16) & 255],
                                      __ldg(M.tet_vfrac + t0 + t));
          }
          __syncwarp(mask);
          float ua = -1.f, fa = 1.f - af, ub = 0.f, fb = -af;  // f(ua) > 0 > f(ub)
          float uc = fminf(fmaxf(refl ? -u0 : u0 - 1.f, -1.f), 0.f);
          float fc = liquid_volume32<G>(rows32, nt, lane, mask, uc) - af;
          ++evals32;
          float up = uc, fp = fc;  // previous raw evaluation (for the slope)
          int side = 0;
          for (int it = 0; it < 16; ++it) {
            if (fc > 0.f) { ua = uc; fa = fc; } else { ub = uc; fb = fc; }
            // relative tests: |f| against the target, the bracket against its distance from 0
            if (fabsf(fc) <= 1e-6f * af || ub - ua <= 1e-6f * fmaxf(fabsf(ua), fabsf(ub))) break;
            // regula falsi step; Illinois: halve the retained end's value after two steps on one side
            float un;
            if (it == 0) {
              const float step = 0.02f;  // probe next to the guess, towards the root
              un = fc > 0.f ? fminf(uc + step, 0.5f * (uc + ub)) : fmaxf(uc - step, 0.5f * (ua + uc));
            } else {
              un = ua + (ub - ua) * (fa / (fa - fb));
              if (!(un > ua && un < ub)) un = 0.5f * (ua + ub);
            }
            up = uc;
            fp = fc;
            uc = un;
            fc = liquid_volume32<G>(rows32, nt, lane, mask, uc) - af;
            ++evals32;
            const int s2 = fc > 0.f ? 1 : -1;
            if (s2 == side) {
              if (s2 > 0) fb *= 0.5f; else fa *= 0.5f;
            }
            side = s2;
          }
          // slope df/du from the last two raw FP32 evaluations (else from the bracket); with
          // c = org + dir u range and f = dir (V/V_cell - alpha), df/dc is slope / range either way
          slope = (uc != up) ? (fc - fp) / (uc - up) : 0.f;
          if (!(slope < 0.f)) slope = (fb - fa) / (ub - ua);
          ubest = uc;
        }
        // FP64 phase, both paths: the FP32-refined point picks the vertex interval [va, vb]; one
        // pass sums its cubic P (interval_pass); when the target lies outside P's values at the
        // interval's ends the neighbouring interval is taken instead (another pass). On [va, vb]
        // every FP64 evaluation of V_L is P, exactly.
        //  - Learned: an evaluation at the refined point, one at a Newton point with the FP32
        //    slope, at most max_secant secant steps (the guess + secant steps of the learned path).
        //  - Interval cubic: safeguarded Newton steps on P.
        // A miss of the tolerance ends in bisection on P inside the bracket (the counted
        // fallback); if no interval brackets the target, in bisection over [phi_min, phi_max]
        // with every tetrahedron evaluated directly.
        __syncwarp(mask);
        double c1 = dmin(dmax(fma(flip_if(fl2d(ubest), refl), range, org), lo), hi);
        if (!(okey(c1) < okey(hi))) c1 = okey_inv(okey(hi) - 1);  // an interval above c1 exists
        // largest vertex value <= c and smallest above it, by integer keys
        auto vertex_interval = [&](double c, double& va, double& vb) {
          const uint64_t kc = okey(c);
          uint64_t ka = 0ull, kb = ~0ull;
          for (int j = lane; j < nv; j += G) {
            const uint64_t k = okey(dvert[j]);
            if (k <= kc) ka = max(ka, k); else kb = min(kb, k);
          }
          va = okey_inv(group_umax<G>(ka, mask));
          vb = okey_inv(group_umin<G>(kb, mask));
        };
        double va, vb;
        vertex_interval(c1, va, vb);
        const double tgt = a * M.cell_vol[cell];
        bool bracketed = false;
        for (int mv = 0; mv < 8; ++mv) {
          tev += interval_pass(va, vb);  // an FP64 evaluation: a pass over the cell's tetrahedra
          ++evals;
          const double ya = va - cm, yb = vb - cm;
          const double ga = fma(fma(fma(P3, ya, P2), ya, P1), ya, P0) - tgt;
          const double gb = fma(fma(fma(P3, yb, P2), yb, P1), yb, P0) - tgt;
          if (positive(gb) && okey(vb) < okey(hi)) {  // the root lies above vb
            vertex_interval(vb, va, vb);
          } else if (okey(ga) < okey(0.0) && okey(va) > okey(lo)) {  // below va
            vertex_interval(okey_inv(okey(va) - 1), va, vb);
          } else {
            bracketed = true;
            break;
          }
        }
        if (bracketed) {
          L = dmax(L, va);  // V_L(va)/V - alpha >= 0 >= V_L(vb)/V - alpha
          H = dmin(H, vb);
          auto evalP = [&](double c) -> double {
            const double y = c - cm;
            const double f = (fma(fma(fma(P3, y, P2), y, P1), y, P0) - tgt) * invV;
            record(c, f);
            return f;
          };
          if (mode == VOF_ROOT_CUBIC) {
            double ya = L - cm, yb = H - cm;  // g(ya) >= 0 >= g(yb), g decreasing
            double y = dmin(dmax(c1 - cm, ya), yb);
            for (int it = 0; it < 12 && !done; ++it) {
              const double g = fma(fma(fma(P3, y, P2), y, P1), y, P0) - tgt;
              record(cm + y, g * invV);
              if (mag(g) == 0ull || done) break;
              if (positive(g)) ya = y; else yb = y;
              const double dp = fma(fma(3.0 * P3, y, 2.0 * P2), y, P1);  // dg/dy <= 0
              double yn = 0.5 * (ya + yb);
              if (okey(dp) < okey(0.0)) {
                double r = fl2d(1.0f / d2f(dp));
                r = fma(r, fma(-dp, r, 1.0), r);
                const double yt = fma(-g, r, y);
                if (inside(yt, ya, yb)) yn = yt;
              }
              if (okey(yn) == okey(y) || !inside(yn, ya, yb)) break;
              y = yn;
            }
          } else {
            c1 = dmin(dmax(c1, L), H);
            double f1 = evalP(c1);
            if (!done && opt.max_secant > 0) {
              // second point: one Newton step with the FP32 slope, kept inside the bracket
              double c0 = fma(-f1, range * fl2d(1.0f / slope), c1);
              if (!inside(c0, L, H) || __double_as_longlong(c0) == __double_as_longlong(c1)) {
                const double step = 4e-6 * range;
                c0 = positive(f1) ? fmin(c1 + step, 0.5 * (c1 + H)) : fmax(c1 - step, 0.5 * (c1 + L));
              }
              double f0 = evalP(c0);
              for (int sct = 0; sct < opt.max_secant && !done; ++sct) {
                if (__double_as_longlong(f0) == __double_as_longlong(f1)) break;
                // secant point; the reciprocal of f0 - f1 from an FP32 seed and one FP64 Newton step
                const double d = f0 - f1;
                double r = fl2d(1.0f / d2f(d));
                r = fma(r, fma(-d, r, 1.0), r);
                double c2 = fma(-f0, (c0 - c1) * r, c0);
                if (!inside(c2, L, H)) c2 = 0.5 * (L + H);
                const double f2 = evalP(c2);
                c1 = c0; f1 = f0; c0 = c2; f0 = f2;
              }
            }
          }
          if (!done) {
            status |= VOF_ST_FALLBACK;
            for (int it = 0; it < opt.max_bisect && !done; ++it) {
              evalP(0.5 * (L + H));
              if (okey(H) - okey(L) <= 4) break;  // a few representable values left
            }
          }
        } else {
          status |= VOF_ST_FALLBACK;
          for (int it = 0; it < opt.max_bisect && !done; ++it) {
            eval_direct(0.5 * (L + H));
            if (okey(H) - okey(L) <= 4) break;
          }
        }
      } else {
        prepare64();
        for (int it = 0; it < opt.max_bisect && !done; ++it) {
          eval64(0.5 * (L + H));
          // stop when the bracket is down to a few representable values
          if (okey(H) - okey(L) <= 4) break;
        }
      }
      if (kbest > ktol) status |= VOF_ST_NOT_CONVERGED;
    }
    // the interface geometry at c_best follows in k_geom
    if (lane == 0) {
      W.iso[cell] = c_best;
      W.status[cell] = status;
      W.evals[cell] = evals;
      evals_acc += evals;
      ev32_acc += evals32;
      tetev_acc += tev;
      prep_acc += n_prep;
      if (status & VOF_ST_DEGENERATE) atomicAdd((unsigned long long*)&W.counters->n_degenerate, 1ull);
      if (status & VOF_ST_NOT_CONVERGED) atomicAdd((unsigned long long*)&W.counters->n_not_converged, 1ull);
      if (status & VOF_ST_FALLBACK) atomicAdd((unsigned long long*)&W.counters->n_fallback, 1ull);
      if (status & VOF_ST_MLP_SKIPPED) atomicAdd((unsigned long long*)&W.counters->n_mlp_skipped, 1ull);
    }
    __syncwarp(mask);
  }
  if (lane == 0 && evals_acc) {
    atomicAdd((unsigned long long*)&W.counters->evals_total, (unsigned long long)evals_acc);
    atomicAdd((unsigned long long*)&W.counters->tet_evals, (unsigned long long)tetev_acc);
    atomicAdd((unsigned long long*)&W.counters->tets_prepared, (unsigned long long)prep_acc);
    if (ev32_acc) atomicAdd((unsigned long long*)&W.counters->evals32_total, (unsigned long long)ev32_acc);
  }
}

// ---- root search with a thread per cell (cells of at most kCellMaxTets tetrahedra) ------------------
// The learned and interval-cubic modes for small cells (tetrahedra, prisms, hexahedra, the pipe's
// extruded polygons): every lane of a warp owns one cell and runs the same steps, so the warp's
// instructions serve 32 cells and no lane group drifts out of step with the others.
//  - FP32 bracketing of the root by vertex values, from the start value (the MLP guess, or
//    1 - alpha): the wet fraction at the vertex values next to the start, then next to the regula
//    falsi point of the narrowed bracket, until no vertex value lies inside the bracket: it is then
//    the root's vertex interval. Each FP32 evaluation forms the tetrahedra's wet fractions from
//    their corner values in one pass (tet_wet32: nothing per tetrahedron is kept in shared memory).
//  - Each block takes kCellThreads entries of the bin at a time, sorted by tetrahedron count, so
//    that a warp's lanes hold cells of similar size.
//  - One pass over the tetrahedra for that interval sums the interval's cubic in FP32-pair
//    arithmetic (tet_piece_roles_ff) on values normalised by the cell's range (on this part an
//    FP64 warp instruction costs 64 issue slots of its sub-partition). The vertices' wet/dry roles
//    over the interval come from their FP64 order keys, as a bit mask.
//  - Safeguarded Newton steps on the exact cubic (both modes), bisection on it as the counted
//    fallback.
// Per thread, shared memory holds one float2 per vertex (the normalised FP32 values of the
// refinement, then the normalised pairs of the root phase), strided by the block size so that a
// lane's element k sits in the lane's own bank whatever k is. A cell whose vertex interval is
// narrower than options.root_narrow (default 2^-20) of its range, or whose target no interval
// brackets, is handed to the lane-group kernel (its slow list), which runs the FP64 path on it
// from the start.
constexpr int kCellThreads = 128;
constexpr int kCellMaxTets = 24;  // the tetrahedra of a straddling set fit a 32-bit mask

// Wet fraction of a tetrahedron at level u (FP32, for the refinement): corner values p, volume
// fraction vf; the closed form of its number of wet corners (the header's formulas) with one
// division, selected rather than branched so that every lane runs the same instructions.
__device__ __forceinline__ float tet_wet32(float p0, float p1, float p2, float p3, float vf, float u) {
  float s0 = fmaxf(p0, p1), s1 = fminf(p0, p1), s2 = fmaxf(p2, p3), s3 = fminf(p2, p3), t;
  t = fmaxf(s0, s2); s2 = fminf(s0, s2); s0 = t;
  t = fmaxf(s1, s3); s3 = fminf(s1, s3); s1 = t;
  t = fmaxf(s1, s2); s2 = fminf(s1, s2); s1 = t;
  const int k = (s0 >= u) + (s1 >= u) + (s2 >= u) + (s3 >= u);
  const float d02 = s0 - s2, d03 = s0 - s3, d13 = s1 - s3;
  const float wa = s0 - u, wb = s1 - u, uc = u - s2, ud = u - s3, ab = wa * wb;
  const float n1 = wa * wa * wa, e1 = (s0 - s1) * d02 * d03;
  const float n2 = ab * ab + (uc + ud) * ab * (wa + wb) + uc * ud * (wa * wa + ab + wb * wb);
  const float e2 = d02 * d03 * (s1 - s2) * d13;
  const float e3 = d03 * d13 * (s2 - s3), n3 = e3 - ud * ud * ud;
  const float num = k == 1 ? n1 : (k == 2 ? n2 : (k == 3 ? n3 : (k == 4 ? 1.f : 0.f)));
  const float den = k == 1 ? e1 : (k == 2 ? e2 : (k == 3 ? e3 : 1.f));
  return vf * __fdividef(num, den);
}

// tet_piece in pair arithmetic on normalised values: corner values p relative to the interval's
// midpoint cm and divided by the cell's range (so that the differences are O(1)), the volume
// fraction vt = V_t / V, and the corners' roles over the interval as a 4-bit mask of wet corners
// (1 to 3 bits set) instead of a sort: the wet corners become s0.., the dry ones ..s3. The piece's
// closed forms depend on the order only through these roles (they are symmetric within the wet
// and within the dry corners); the two wet corners of the two-wet case are put in descending
// order, as the FP64 path has them. The piece's cubic in y = (c - cm) / range is added to q0..q3,
// in units of the cell volume. The caller takes this path only for an interval wider than
// root_narrow (at least 2^-20) of the range: every denominator is then a product of
// (wet - dry) differences of at least 2^-20 each, so nothing leaves the FP32 exponent range or
// loses the pairs' 48 bits.
__device__ __forceinline__ void tet_piece_roles_ff(ff p0, ff p1, ff p2, ff p3, unsigned m, ff vt, ff& q0, ff& q1,
                                                   ff& q2, ff& q3) {
  const int nk = __popc(m);
  const unsigned dm = ~m & 15u;
  // position of corner c: wet corners first, in index order, then the dry ones
  auto pos = [&](int c) -> int {
    const unsigned below = (1u << c) - 1u;
    return ((m >> c) & 1u) ? __popc(m & below) : nk + __popc(dm & below);
  };
  const int o0 = pos(0), o1 = pos(1), o2 = pos(2), o3 = pos(3);
  auto at = [&](int j) -> ff { return o0 == j ? p0 : (o1 == j ? p1 : (o2 == j ? p2 : p3)); };
  ff s0 = at(0), s1 = at(1);
  const ff s2 = at(2), s3 = at(3);
  const bool one = nk == 1, two = nk == 2;
  if (two && ff_lt(s0, s1)) {
    const ff t = s0;
    s0 = s1;
    s1 = t;
  }
  const ff zero = {0.f, 0.f};
  // denominators: nk = 1: d01 d02 d03; nk = 2: d02 d03 d12 d13; nk = 3: d03 d13 d23
  const ff X = ff_sub(one ? s0 : (two ? s0 : s1), one ? s1 : (two ? s2 : s3));  // d01 | d02 | d13
  const ff Y = ff_sub(one ? s0 : (two ? s1 : s2), one ? s2 : (two ? s2 : s3));  // d02 | d12 | d23
  const ff Z = two ? ff_sub(s1, s3) : ff{1.f, 0.f};                             // 1   | d13 | 1
  const ff d03 = ff_sub(s0, s3);
  const ff YZ = ff_mul(Y, Z);
  const ff R = ff_mul(vt, ff_rcp(ff_mul(ff_mul(d03, X), YZ)));
  const ff a = ff_sub(s0, s1);
  const ff vk = ff_mul(R, YZ);
  const ff A = two ? ff_mul(vk, ff_mul(a, a)) : (one ? zero : vt);
  const ff B = two ? ff_scale(ff_mul(vk, a), 3.f) : zero;
  const ff C = two ? ff_scale(vk, 3.f) : zero;
  const ff D = two ? ff_neg(ff_mul(R, ff_add(a, ff_add(Y, Z)))) : R;
  const ff dl = one ? s0 : (two ? s1 : s3);  // ref - cm, normalised
  q0 = ff_add(q0, ff_cubic(A, B, C, D, dl));
  const ff D3 = ff_scale(D, 3.f);
  q1 = ff_sub(q1, ff_add(ff_mul(ff_add(ff_mul(D3, dl), ff_scale(C, 2.f)), dl), B));
  q2 = ff_add(q2, ff_add(ff_mul(D3, dl), C));
  q3 = ff_sub(q3, D);
}

__global__ void __launch_bounds__(kCellThreads, 5) k_root_cell(MeshView M, const double* alpha, vof_options opt,
                                                            Workspace W, int mode, int use_mlp, int bin) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  float2* sv = reinterpret_cast<float2*>(smem) + threadIdx.x;  // [k * T]
  const int64_t n_bin = W.counters->bin_count[bin];
  const int32_t* list = W.bin_list + (size_t)bin * M.n_cells;
  const uint64_t ktol = mag(opt.tol_alpha);
  int64_t evals_acc = 0, tetev_acc = 0, ev32_acc = 0;
  // The block takes kCellThreads entries of the bin at a time and sorts them by tetrahedron count
  // (bitonic network in shared memory), so that the lanes of a warp get cells of similar size: a
  // warp runs as long as its largest cell.
  __shared__ uint32_t skey[kCellThreads];
  for (int64_t base = (int64_t)blockIdx.x * kCellThreads; base < n_bin; base += (int64_t)gridDim.x * kCellThreads) {
    {
      const int64_t jj = base + threadIdx.x;
      uint32_t key = 0xffffffffu;
      if (jj < n_bin) {
        const int32_t cc = W.iface_idx[list[jj]];
        key = ((uint32_t)(M.cell_tet_off[cc + 1] - M.cell_tet_off[cc]) << 8) | threadIdx.x;
      }
      skey[threadIdx.x] = key;
      __syncthreads();
#pragma unroll
      for (int k = 2; k <= kCellThreads; k <<= 1)
#pragma unroll
        for (int h = k >> 1; h > 0; h >>= 1) {
          const int t = threadIdx.x, l = t ^ h;
          if (l > t) {
            const uint32_t x = skey[t], y = skey[l];
            if ((x > y) == ((t & k) == 0)) {
              skey[t] = y;
              skey[l] = x;
            }
          }
          __syncthreads();
        }
    }
    const uint32_t mine = skey[threadIdx.x];
    __syncthreads();  // every thread has its entry before the next chunk's keys are written
    if (mine == 0xffffffffu) continue;
    const int64_t j = base + (mine & 255u);
    const int64_t i = list[j];
    const int32_t cell = W.iface_idx[i];
    const int64_t v0 = M.cell_vert_off[cell], t0 = M.cell_tet_off[cell];
    const int nv = (int)(M.cell_vert_off[cell + 1] - v0), nt = (int)(M.cell_tet_off[cell + 1] - t0);
    const int32_t* cv = M.cell_vert + v0;
    const uint32_t* ctp = M.cell_tet + t0;
    uint64_t klo = ~0ull, khi = 0ull;
    for (int k = 0; k < nv; ++k) {
      const uint64_t kk = okey(W.phi_v[cv[k]]);
      klo = min(klo, kk);
      khi = max(khi, kk);
    }
    const double lo = okey_inv(klo), hi = okey_inv(khi);
    const double a = alpha[cell];
    int status = 0, evals = 0, evals32 = 0;
    int64_t tev = 0;
    double c_best;
    uint64_t kbest = 0;
    bool slow = false;
    const double range = hi - lo;
    if (__double_as_longlong(range) < __double_as_longlong(1e-14)) {
      status = VOF_ST_DEGENERATE;
      c_best = lo;
    } else {
      const double oma = 1.0 - a;
      kbest = min(mag(oma), mag(a));
      c_best = okey(oma) <= okey(a) ? lo : hi;
      // FP32 refinement, as in k_root: the start value u0, the local coordinate with the minority
      // phase next to u = 0, regula falsi (Illinois) on the FP32 wet fractions
      float u0 = use_mlp ? W.mlp_out[i] : 1.0f - d2f(a);
      if (!(u0 >= 0.0f)) {
        status |= VOF_ST_MLP_SKIPPED;
        u0 = 1.0f - d2f(a);
      }
      const bool refl = okey(a) > kKeyHalf;
      const double org = refl ? lo : hi;
      const float af = d2f(refl ? oma : a);
      {
        const float r32 = __frcp_rn(d2f(range));
        const float su = refl ? -r32 : r32;
        const ff of = ff_of(org);
        for (int k = 0; k < nv; ++k) {
          const float2 pv = W.phi_ff[cv[k]];
          sv[k * T].x = __fmul_rn(__fadd_rn(__fsub_rn(pv.x, of.hi), __fsub_rn(pv.y, of.lo)), su);
        }
      }
      auto V32 = [&](float u) -> float {
        const float pa = sv[0].x;
        float v = 0.f;
        for (int t = 0; t < nt; ++t) {
          const uint32_t pk = __ldg(ctp + t);
          v += tet_wet32(pa, sv[(pk & 255) * T].x, sv[((pk >> 8) & 255) * T].x, sv[((pk >> 16) & 255) * T].x,
                         __ldg(M.tet_vfrac + t0 + t), u);
        }
        return v;
      };
      // Bracketing by vertex values: the start u_s lies in the vertex interval [va, vb] of its
      // neighbouring vertex values; the wet fraction at va and vb (where they are not the bracket's
      // ends already) tells whether the root lies in it, below or above. Otherwise the next
      // probe is the regula falsi point of the narrowed bracket. It ends when no vertex value
      // lies strictly inside the bracket: the bracket is the root's vertex interval, found with
      // one or two evaluations when the start falls in it.
      float ua = -1.f, fa = 1.f - af, ub = 0.f, fb = -af;  // f(ua) > 0 > f(ub)
      float p = fminf(fmaxf(refl ? -u0 : u0 - 1.f, -1.f), 0.f);
      for (int it = 0; it < 16; ++it) {
        float va = ua, vb = ub;  // the vertex values next to p inside the bracket
        for (int k = 0; k < nv; ++k) {
          const float x = sv[k * T].x;
          if (x <= p) va = fmaxf(va, x); else vb = fminf(vb, x);
        }
        if (va == ua && vb == ub) break;
        if (va > ua) {
          const float f = V32(va) - af;
          ++evals32;
          if (f > 0.f) { ua = va; fa = f; } else { ub = va; fb = f; }
        }
        if (vb < ub) {  // the root is at or above va here
          const float f = V32(vb) - af;
          ++evals32;
          if (f > 0.f) { ua = vb; fa = f; } else { ub = vb; fb = f; }
        }
        p = ua + (ub - ua) * (fa / (fa - fb));
        if (!(p > ua && p < ub)) p = 0.5f * (ua + ub);
      }
      // the root phase starts at the regula falsi point of the bracket
      float uc = ua + (ub - ua) * (fa / (fa - fb));
      if (!(uc >= ua && uc <= ub)) uc = 0.5f * (ua + ub);
      // root phase in pairs: the refined point picks the vertex interval, one pass sums the
      // interval's cubic Q(y) = V_L/V - alpha, y = (c - cm) / range
      double c1 = dmin(dmax(fma(flip_if(fl2d(uc), refl), range, org), lo), hi);
      if (!(okey(c1) < okey(hi))) c1 = okey_inv(okey(hi) - 1);
      auto vertex_interval = [&](double c, double& va, double& vb) {
        const uint64_t kc = okey(c);
        uint64_t ka = 0ull, kb = ~0ull;
        for (int k = 0; k < nv; ++k) {
          const uint64_t kk = okey(W.phi_v[cv[k]]);
          if (kk <= kc) ka = max(ka, kk); else kb = min(kb, kk);
        }
        va = okey_inv(ka);
        vb = okey_inv(kb);
      };
      double va, vb, cm = 0;
      vertex_interval(c1, va, vb);
      const ff ir = ff_rcp(ff_of(range)), ivV = ff_of(M.cell_ivol[cell]), a_ff = ff_of(a);
      const uint64_t kwide = okey(range * opt.root_narrow);
      ff Q0 = {0.f, 0.f}, Q1 = Q0, Q2 = Q0, Q3 = Q0, yA = Q0, yB = Q0;
      bool bracketed = false;
      for (int mv = 0; mv < 8; ++mv) {
        if (okey(vb - va) < kwide) break;  // narrower than root_narrow x range: the slow path
        const uint64_t kvb = okey(vb);
        cm = 0.5 * (va + vb);
        // roles over [va, vb] (no vertex value lies strictly inside): wet at or above vb, else dry;
        // the values relative to cm, normalised, as pairs
        uint32_t wet = 0;
        for (int k = 0; k < nv; ++k) {
          const double p = W.phi_v[cv[k]];
          wet |= (uint32_t)(okey(p) >= kvb) << k;
          const ff r = ff_mul(ff_of(p - cm), ir);
          sv[k * T] = make_float2(r.hi, r.lo);
        }
        // wet tetrahedra summed, straddling ones marked; then the pieces over the marks, so that
        // a lane runs the piece only as often as it has straddling tetrahedra
        double ws = 0;
        uint32_t smask = 0;
        for (int t = 0; t < nt; ++t) {
          const uint32_t pk = __ldg(ctp + t);
          const unsigned m4 = (wet & 1u) | ((wet >> (pk & 255)) & 1u) << 1 | ((wet >> ((pk >> 8) & 255)) & 1u) << 2 |
                              ((wet >> ((pk >> 16) & 255)) & 1u) << 3;
          if (m4 == 15u) ws += __ldg(M.tet_vol + t0 + t);
          else if (m4) smask |= 1u << t;
        }
        ff q0 = {0.f, 0.f}, q1 = q0, q2 = q0, q3 = q0;
        const ff r0 = ff_make(sv[0]);
        const int npc = __popc(smask);
        while (smask) {
          const int t = __ffs(smask) - 1;
          smask &= smask - 1u;
          const uint32_t pk = __ldg(ctp + t);
          const int i1 = pk & 255, i2 = (pk >> 8) & 255, i3 = (pk >> 16) & 255;
          const unsigned m4 = (wet & 1u) | ((wet >> i1) & 1u) << 1 | ((wet >> i2) & 1u) << 2 | ((wet >> i3) & 1u) << 3;
          tet_piece_roles_ff(r0, ff_make(sv[i1 * T]), ff_make(sv[i2 * T]), ff_make(sv[i3 * T]), m4,
                             ff_mul(ff_of(__ldg(M.tet_vol + t0 + t)), ivV), q0, q1, q2, q3);
        }
        Q0 = ff_sub(ff_add(q0, ff_mul(ff_of(ws), ivV)), a_ff);
        Q1 = q1;
        Q2 = q2;
        Q3 = q3;
        tev += npc;
        ++evals;
        yA = ff_mul(ff_of(va - cm), ir);
        yB = ff_mul(ff_of(vb - cm), ir);
        const bool above = ff_cubic(Q0, Q1, Q2, Q3, yB).hi > 0.f, below = ff_cubic(Q0, Q1, Q2, Q3, yA).hi < 0.f;
        if (above && okey(vb) < okey(hi)) {
          vertex_interval(vb, va, vb);
        } else if (below && okey(va) > okey(lo)) {
          vertex_interval(okey_inv(okey(va) - 1), va, vb);
        } else {
          bracketed = true;
          break;
        }
      }
      if (!bracketed) {
        slow = true;
      } else {
        // safeguarded Newton steps on the exact cubic, bisection when a step leaves the bracket
        bool done = false;
        ff yL = yA, yH = yB, ybest = yA;
        bool have_best = false;
        auto evalQ = [&](ff y) -> ff {
          const ff f = ff_cubic(Q0, Q1, Q2, Q3, y);
          const uint64_t kf = mag(fl2d(f.hi));
          if (kf < kbest) { kbest = kf; ybest = y; have_best = true; }
          if (f.hi > 0.f) yL = ff_max(yL, y); else yH = ff_min(yH, y);
          if (kf <= ktol) done = true;
          return f;
        };
        ff y = ff_min(ff_max(ff_mul(ff_of(c1 - cm), ir), yL), yH);
        for (int it = 0; it < 12 && !done; ++it) {
          const ff g = evalQ(y);
          if (g.hi == 0.f || done) break;
          const ff dp = ff_add(ff_mul(ff_add(ff_mul(ff_scale(Q3, 3.f), y), ff_scale(Q2, 2.f)), y), Q1);  // <= 0
          ff yn = ff_mid(yL, yH);
          if (dp.hi < 0.f) {
            const ff yt = ff_sub(y, ff_mul(g, ff_rcp(dp)));
            if (ff_inside(yt, yL, yH)) yn = yt;
          }
          if (ff_eq(yn, y) || !ff_inside(yn, yL, yH)) break;
          y = yn;
        }
        if (!done) {  // the counted fallback: bisection on the cubic inside the bracket
          status |= VOF_ST_FALLBACK;
          for (int it = 0; it < opt.max_bisect && !done; ++it) {
            evalQ(ff_mid(yL, yH));
            if (!(ff_sub(yH, yL).hi > 0x1p-44f)) break;  // the pairs' resolution of the interval
          }
        }
        if (have_best) c_best = dmin(dmax(fma(ff_to_double(ybest), range, cm), va), vb);
        if (kbest > ktol) status |= VOF_ST_NOT_CONVERGED;
      }
    }
    if (slow) {
      // the lane-group kernel takes the cell from the start (FP64 root phase)
      const unsigned long long s = atomicAdd((unsigned long long*)&W.counters->slow_count[bin], 1ull);
      W.slow_list[(size_t)bin * M.n_cells + s] = (int32_t)i;
    } else {
      W.iso[cell] = c_best;
      W.status[cell] = status;
      W.evals[cell] = evals;
      evals_acc += evals;
      ev32_acc += evals32;
      tetev_acc += tev;
      if (status & VOF_ST_DEGENERATE) atomicAdd((unsigned long long*)&W.counters->n_degenerate, 1ull);
      if (status & VOF_ST_NOT_CONVERGED) atomicAdd((unsigned long long*)&W.counters->n_not_converged, 1ull);
      if (status & VOF_ST_FALLBACK) atomicAdd((unsigned long long*)&W.counters->n_fallback, 1ull);
      if (status & VOF_ST_MLP_SKIPPED) atomicAdd((unsigned long long*)&W.counters->n_mlp_skipped, 1ull);
    }
  }
  // counters: warp sums, one atomic each per warp (pieces prepared = pieces evaluated here)
  for (int o = 16; o > 0; o >>= 1) {
    evals_acc += __shfl_xor_sync(0xffffffffu, evals_acc, o);
    tetev_acc += __shfl_xor_sync(0xffffffffu, tetev_acc, o);
    ev32_acc += __shfl_xor_sync(0xffffffffu, ev32_acc, o);
  }
  if ((threadIdx.x & 31) == 0 && (evals_acc || ev32_acc)) {
    atomicAdd((unsigned long long*)&W.counters->evals_total, (unsigned long long)evals_acc);
    atomicAdd((unsigned long long*)&W.counters->tet_evals, (unsigned long long)tetev_acc);
    atomicAdd((unsigned long long*)&W.counters->tets_prepared, (unsigned long long)tetev_acc);
    atomicAdd((unsigned long long*)&W.counters->evals32_total, (unsigned long long)ev32_acc);
  }
}

// Fixed isovalue (VOF_ROOT_FIXED, Sec. 2.1's prescribed alpha_iso): no root search; one thread per
// interface cell checks the cell's vertex range (degenerate as in the root search) and sets c.
__global__ void k_fixed_iso(MeshView M, Workspace W, double alpha_iso) {
  const int64_t n = W.counters->n_iface;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t cell = W.iface_idx[i];
    uint64_t klo = ~0ull, khi = 0ull;
    for (int64_t j = M.cell_vert_off[cell]; j < M.cell_vert_off[cell + 1]; ++j) {
      const uint64_t k = okey(W.phi_v[M.cell_vert[j]]);
      klo = min(klo, k);
      khi = max(khi, k);
    }
    const double lo = okey_inv(klo), hi = okey_inv(khi);
    const bool degenerate = hi - lo < 1e-14;
    W.iso[cell] = degenerate ? lo : alpha_iso;
    W.status[cell] = degenerate ? VOF_ST_DEGENERATE : 0;
    W.evals[cell] = 0;
    if (degenerate) atomicAdd((unsigned long long*)&W.counters->n_degenerate, 1ull);
  }
}

// Interface geometry (paper Sec. 2.1: area, unit normal and centroid of the cut polygons) at the
// isovalues of the root search, kept apart from it: the root search's per-cell chain is FP64
// latency, while here every cell is in flight at once. A warp takes a batch of B consecutive
// interface cells (B up to kGeomBatch, fewer when the step has too few interface cells to give
// every resident warp a full batch). The per-cell set-up (isovalue as a pair, apex value minus it)
// and the final FP64 outputs run a cell per lane, so that their FP64 instructions serve B cells at
// once. In between, the batch's tetrahedra are tested 32 at a time and the cut ones listed in cell
// order; the sections (FP32 pair arithmetic) then take that list 32 at a time, so that every lane
// is busy whatever the cells' cut counts, and a segmented warp scan by cell adds each round's
// sections into the cells' sums in shared memory. The summation order is fixed by the batch, so the
// result does not depend on timing.
constexpr int kGeomThreads = 128;
constexpr int kGeomWarps = kGeomThreads / 32;
constexpr int kGeomBatch = 32;  // at most 32: a cell slot is five bits of a list entry

struct GeomSlot {
  int64_t v0, t0;  // first vertex / tetrahedron entry of the cell
  double c;        // isovalue
  float2 cf, w0;   // isovalue and apex value minus it, as pairs
  int32_t cell;    // -1: no cell
  int32_t nt;      // tetrahedra (0 for a degenerate cell)
};

// Shared memory of one warp: the batch's slots, its cells' sums (7 pairs each), the prefix of the
// tetrahedron counts, and the cut list (at most bmax cells x max_ct tetrahedra).
__host__ __device__ inline size_t geom_warp_bytes(int max_ct, int bmax) {
  return (size_t)kGeomBatch * sizeof(GeomSlot) + (size_t)kGeomBatch * 7 * sizeof(float2) +
         (size_t)(kGeomBatch + 4) * sizeof(int32_t) + (((size_t)bmax * max_ct * sizeof(uint32_t) + 15) & ~(size_t)15);
}
size_t geom_smem_bytes(int max_ct, int bmax) { return (size_t)kGeomWarps * geom_warp_bytes(max_ct, bmax); }

__global__ void __launch_bounds__(kGeomThreads, 5) k_geom(MeshView M, Workspace W, int max_ct, int bmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  unsigned char* wbase = smem + (size_t)warp * geom_warp_bytes(max_ct, bmax);
  GeomSlot* bslot = reinterpret_cast<GeomSlot*>(wbase);                 // [batch cell]
  float2* res = reinterpret_cast<float2*>(bslot + kGeomBatch);          // [batch cell][7]
  int32_t* off = reinterpret_cast<int32_t*>(res + kGeomBatch * 7);      // [batch cell + 1]
  uint32_t* lst = reinterpret_cast<uint32_t*>(off + kGeomBatch + 4);    // cut list: t << 9 | slot << 4 | mask
  const int64_t n = W.counters->n_iface;
  const int64_t nwarps = (int64_t)gridDim.x * kGeomWarps;
  const int64_t per_warp = n / (nwarps > 0 ? nwarps : 1);
  const int B = per_warp >= bmax ? bmax : (per_warp < 1 ? 1 : (int)per_warp);
  int64_t sect = 0;
  for (int64_t b0 = ((int64_t)blockIdx.x * kGeomWarps + warp) * B; b0 < n; b0 += nwarps * B) {
    // set-up of the batch's cells, a cell per lane
    int nt_l = 0;
    {
      GeomSlot g = {0, 0, 0.0, make_float2(0.f, 0.f), make_float2(0.f, 0.f), -1, 0};
      if (lane < B && b0 + lane < n) {
        g.cell = W.iface_idx[b0 + lane];
        g.v0 = M.cell_vert_off[g.cell];
        if (!(W.status[g.cell] & VOF_ST_DEGENERATE)) {
          g.t0 = M.cell_tet_off[g.cell];
          g.nt = (int32_t)(M.cell_tet_off[g.cell + 1] - g.t0);
          g.c = W.iso[g.cell];
          const ff cf = ff_of(g.c);
          const ff w0 = ff_sub(ff_make(W.phi_ff[M.cell_vert[g.v0]]), cf);
          g.cf = make_float2(cf.hi, cf.lo);
          g.w0 = make_float2(w0.hi, w0.lo);
        }
      }
      bslot[lane] = g;
      nt_l = g.nt;
    }
    int incl = nt_l;  // inclusive prefix of the tetrahedron counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += v;
    }
    off[lane + 1] = incl;
    if (lane == 0) off[0] = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) res[lane * 7 + k] = make_float2(0.f, 0.f);
    const int total = __shfl_sync(full, incl, 31);
    __syncwarp();
    // the cut tetrahedra of the batch, in cell order, by integer order keys
    int n_cut = 0;
    for (int r0 = 0; r0 < total; r0 += 32) {
      const int q = r0 + lane;
      bool cut = false;
      uint32_t ent = 0;
      if (q < total) {
        int sl = 0;  // the cell: the largest slot whose first position is at or below q
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
          if (sl + st < B && off[sl + st] <= q) sl += st;
        const GeomSlot& g = bslot[sl];
        const int t = q - off[sl];
        const uint64_t kc = okey(g.c);
        const int32_t* cv = M.cell_vert + g.v0;
        const uint32_t pk = __ldg(M.cell_tet + g.t0 + t);
        const unsigned m = (unsigned)(okey(W.phi_v[cv[0]]) >= kc) | ((unsigned)(okey(W.phi_v[cv[pk & 255]]) >= kc) << 1) |
                           ((unsigned)(okey(W.phi_v[cv[(pk >> 8) & 255]]) >= kc) << 2) |
                           ((unsigned)(okey(W.phi_v[cv[(pk >> 16) & 255]]) >= kc) << 3);
        cut = m != 0u && m != 15u;
        ent = ((uint32_t)t << 9) | ((uint32_t)sl << 4) | m;
      }
      const unsigned bal = __ballot_sync(full, cut);
      if (cut) lst[n_cut + __popc(bal & ((1u << lane) - 1u))] = ent;
      n_cut += __popc(bal);
    }
    __syncwarp();
    // sections, 32 at a time; a segmented scan by cell, then the last lane of each cell's run adds
    // the run's sum into the cell's sums
    for (int r0 = 0; r0 < n_cut; r0 += 32) {
      const int jj = r0 + lane;
      int key = 64 + lane;  // past the list: a run of its own
      ff v[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] = ff{0.f, 0.f};
      if (jj < n_cut) {
        const uint32_t e = lst[jj];
        const int sl = (int)((e >> 4) & 31u), t = (int)(e >> 9);
        const GeomSlot& g = bslot[sl];
        const int32_t* cv = M.cell_vert + g.v0;
        const uint32_t pk = __ldg(M.cell_tet + g.t0 + t);
        const int l1 = pk & 255, l2 = (pk >> 8) & 255, l3 = (pk >> 16) & 255;
        const float2* rp = M.rel_pos + 3 * g.v0;
        const ff cf = ff_make(g.cf);
        ff3 tA, tm;
        ff ta;
        tet_section_ff(ff3_load(rp + 3 * l1), ff3_load(rp + 3 * l2), ff3_load(rp + 3 * l3), ff_make(g.w0),
                       ff_sub(ff_make(W.phi_ff[cv[l1]]), cf), ff_sub(ff_make(W.phi_ff[cv[l2]]), cf),
                       ff_sub(ff_make(W.phi_ff[cv[l3]]), cf), e & 15u, tA, ta, tm);
        v[0] = tA.x; v[1] = tA.y; v[2] = tA.z; v[3] = ta; v[4] = tm.x; v[5] = tm.y; v[6] = tm.z;
        key = sl;
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int kp = __shfl_up_sync(full, key, o);
        const bool take = lane >= o && kp == key;  // keys ascend, so the whole span is this cell's
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          const ff u = {__shfl_up_sync(full, v[k].hi, o), __shfl_up_sync(full, v[k].lo, o)};
          if (take) v[k] = ff_add(v[k], u);
        }
      }
      const int kn = __shfl_down_sync(full, key, 1);
      if (jj < n_cut && (lane == 31 || kn != key)) {
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          const ff r = ff_add(ff_make(res[key * 7 + k]), v[k]);
          res[key * 7 + k] = make_float2(r.hi, r.lo);
        }
      }
      __syncwarp();
    }
    sect += n_cut;
    // outputs, a cell per lane
    if (lane < B && bslot[lane].cell >= 0) {
      const GeomSlot& g = bslot[lane];
      ff v[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) v[k] = ff_make(res[lane * 7 + k]);
      const int32_t a = M.cell_vert[g.v0];
      double area;
      Vec3 nrm, xg;
      geometry_outputs(v, M.vx[a], M.vy[a], M.vz[a], area, nrm, xg);
      const int32_t cell = g.cell;
      W.A_int[cell] = area;
      W.n_int[3 * cell] = nrm.x;
      W.n_int[3 * cell + 1] = nrm.y;
      W.n_int[3 * cell + 2] = nrm.z;
      W.x_gamma[3 * cell] = xg.x;
      W.x_gamma[3 * cell + 1] = xg.y;
      W.x_gamma[3 * cell + 2] = xg.z;
    }
    __syncwarp();
  }
  if (lane == 0 && sect) atomicAdd((unsigned long long*)&W.counters->tets_sectioned, (unsigned long long)sect);
}


// ---- crossing point (R4) -----------------------------------------------------------------------
__device__ __forceinline__ bool has_plane(const Workspace& W, int32_t c, uint32_t step) {
  return W.iface_stamp[c] == step && W.A_int[c] > 0;
}

// t along x_owner -> x_neigh (dn = x_neigh - x_owner); *src = the interface cell whose plane gave
// it, or -1
__device__ double crossing_t(const MeshView& M, const Workspace& W, const double* alpha, int32_t f, int xf_mode,
                             uint32_t step, const Vec3& xo, const Vec3& dn, int32_t* src) {
  const int32_t o = M.face_owner[f], n = M.face_neigh[f];
  *src = -1;
  if (xf_mode == VOF_XF_AS_PRINTED) return fabs(alpha[n] - 0.5) / fabs(alpha[o] - alpha[n]);
  if (xf_mode == VOF_XF_LINEAR) return (alpha[o] - 0.5) / (alpha[o] - alpha[n]);
  const Vec3 xfc = v3(M.face_cen[3 * f], M.face_cen[3 * f + 1], M.face_cen[3 * f + 2]);
  double best_t = 0, best_d = 0;
  const int32_t cand[2] = {o, n};
  for (int q = 0; q < 2; ++q) {
    const int32_t c = cand[q];
    if (!has_plane(W, c, step)) continue;
    const Vec3 nn = v3(W.n_int[3 * c], W.n_int[3 * c + 1], W.n_int[3 * c + 2]);
    const Vec3 xg = v3(W.x_gamma[3 * c], W.x_gamma[3 * c + 1], W.x_gamma[3 * c + 2]);
    const double den = dot(nn, dn);
    if (mag(den) == 0ull) continue;
    const double t = dot(nn, xg - xo) / den;
    // 0 <= t <= 1 and the nearer plane (squared distance) by order keys: FP64 compares cost an
    // FP64 issue slot each; NaN fails both tests as it does in floating point
    const uint64_t kt = okey(t);
    if (!(kt >= okey(0.0) && kt <= okey(1.0))) continue;
    const Vec3 r = xo + dn * t - xfc;
    const double d = dot(r, r);
    if (*src < 0 || okey(d) < okey(best_d)) { best_t = t; best_d = d; *src = c; }
  }
  return *src >= 0 ? best_t : (alpha[o] - 0.5) / (alpha[o] - alpha[n]);
}

// ---- crossing faces next to the band (R4): list, then one thread per face ------------------------
// A face is listed once: by its owner when the owner is a band cell, else by its neighbour.
constexpr int kLsqLanes = 8;

// A group of kLsqLanes lanes per band cell lists its crossing faces.
__global__ void k_xmark(MeshView M, const double* alpha, Workspace W) {
  const uint32_t step = W.counters->step;
  const int64_t nb = W.counters->n_band;
  const int lane = threadIdx.x % kLsqLanes, grp = (threadIdx.x & 31) / kLsqLanes;
  const int wl = threadIdx.x & 31;
  const unsigned below = (1u << wl) - 1u;
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / kLsqLanes);
  // warp-uniform trip counts (ballots below); appends aggregated per warp, one atomic per pass,
  // since the list's counter is a single address that every warp of the grid updates
  const int64_t first = blockIdx.x * (int64_t)(blockDim.x / kLsqLanes) + (threadIdx.x & ~31) / kLsqLanes;
  for (int64_t base = first; base < nb; base += groups) {
    const int64_t j = base + grp;
    int32_t c = -1;
    int64_t f0 = 0, nf = 0;
    double aP = 0;
    if (j < nb) {
      c = W.band_idx[j];
      aP = alpha[c];
      f0 = M.cell_face_off[c];
      nf = M.cell_face_off[c + 1] - f0;
    }
    const int maxf = __reduce_max_sync(0xffffffffu, (unsigned)nf);
    for (int s0 = 0; s0 < maxf; s0 += kLsqLanes) {
      const int k = s0 + lane;
      bool take = false;
      int32_t f = 0;
      if (k < nf) {
        f = M.cell_face[f0 + k] & 0x7fffffff;
        const int32_t o = M.face_owner[f], nbr = M.face_neigh[f];
        if (nbr >= 0) {
          const int32_t q = o == c ? nbr : o;
          if (crossing_pair(aP, alpha[q]))
            take = o == c || W.band_stamp[o] != step;  // listed once: by the owner if it is a band cell
        }
      }
      const unsigned tb = __ballot_sync(0xffffffffu, take);
      unsigned long long fb = 0;
      if (wl == 0 && tb) fb = atomicAdd((unsigned long long*)&W.counters->n_crossing, (unsigned long long)__popc(tb));
      fb = __shfl_sync(0xffffffffu, fb, 0);
      if (take) W.xface_list[fb + __popc(tb & below)] = f;
    }
  }
}

// Crossing point, distances and projected interface area of each listed face.
__device__ void xface_phase(const MeshView& M, const double* alpha, int xf_mode, Workspace& W) {
  const uint32_t step = W.counters->step;
  const int64_t n = W.counters->n_crossing;
  // faces interleaved over the blocks
  for (int64_t j = (int64_t)threadIdx.x * gridDim.x + blockIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f = W.xface_list[j];
    const int32_t o = M.face_owner[f], nbr = M.face_neigh[f];
    const Vec3 xo = v3(M.cell_cen[3 * o], M.cell_cen[3 * o + 1], M.cell_cen[3 * o + 2]);
    const Vec3 dn = v3(M.cell_cen[3 * nbr], M.cell_cen[3 * nbr + 1], M.cell_cen[3 * nbr + 2]) - xo;
    int32_t src;
    const double t = crossing_t(M, W, alpha, f, xf_mode, step, xo, dn, &src);
    const Vec3 xf = xo + dn * t;
    W.x_f[3 * f] = xf.x; W.x_f[3 * f + 1] = xf.y; W.x_f[3 * f + 2] = xf.z;
    // t lies in [0, 1] in every mode (the two cells are on opposite sides of 1/2), so the distances
    // to the two centroids are t |dn| and (1 - t) |dn|
    const double L = M.face_len[f];
    W.d_own[f] = t * L;
    W.d_neigh[f] = (1.0 - t) * L;
    const int32_t sc = src >= 0 ? src : (has_plane(W, o, step) ? o : (has_plane(W, nbr, step) ? nbr : -1));
    double af = 0;
    if (sc >= 0) {
      const Vec3 Af = v3(M.face_area[3 * f], M.face_area[3 * f + 1], M.face_area[3 * f + 2]);
      const Vec3 nn = v3(W.n_int[3 * sc], W.n_int[3 * sc + 1], W.n_int[3 * sc + 2]);
      af = fabs(W.A_int[sc] * dot(nn, Af) * M.face_iarea[f]);
    }
    W.A_int_f[f] = af;
    W.face_stamp[f] = step;
  }
}

// ---- interface-modified least squares (R7) on band cells -----------------------------------------
// A thread per band cell over its faces: a crossing face contributes its crossing point x_f
// (computed first) with T_sat, and every face runs the same FP64 instructions (the point and the
// value are selected, the crossing test is on alpha's bits). One cell per lane keeps every lane of
// the FP64 warp instructions busy, the per-cell inverse included (an FP64 warp instruction costs
// the same with one active lane as with 32); no block barrier.
__device__ void lsq_phase(const MeshView& M, const StepArgs& a, Workspace& W) {
  const uint32_t step = W.counters->step;
  const int64_t nb = W.counters->n_band;
  int nsing = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = W.band_idx[j];
    const Vec3 xP = v3(M.cell_cen[3 * c], M.cell_cen[3 * c + 1], M.cell_cen[3 * c + 2]);
    const double TP = a.T[c], aP = a.alpha[c];
    double g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0, b0 = 0, b1 = 0, b2 = 0;
    for (int64_t k = M.cell_face_off[c]; k < M.cell_face_off[c + 1]; ++k) {
      const int32_t f = M.cell_face[k] & 0x7fffffff;
      const int32_t o = M.face_owner[f], nbr = M.face_neigh[f];
      const int32_t q = o == c ? nbr : o;
      if (q < 0 && !a.T_bnd) continue;
      const bool cross = q >= 0 && crossing_pair(aP, a.alpha[q]);
      const double* xs = cross ? W.x_f + 3 * f : (q >= 0 ? M.cell_cen + 3 * q : M.face_cen + 3 * f);
      const double Tq = cross ? a.props.T_sat : (q >= 0 ? a.T[q] : a.T_bnd[f]);
      const Vec3 r = v3(xs[0], xs[1], xs[2]) - xP;
      const double dT = Tq - TP;
      g00 = fma(r.x, r.x, g00); g01 = fma(r.x, r.y, g01); g02 = fma(r.x, r.z, g02);
      g11 = fma(r.y, r.y, g11); g12 = fma(r.y, r.z, g12); g22 = fma(r.z, r.z, g22);
      b0 = fma(r.x, dT, b0); b1 = fma(r.y, dT, b1); b2 = fma(r.z, dT, b2);
    }
    // explicit symmetric inverse (cofactors / det), Appendix B
    const double c00 = g11 * g22 - g12 * g12, c01 = g02 * g12 - g01 * g22, c02 = g01 * g12 - g02 * g11;
    const double det = g00 * c00 + g01 * c01 + g02 * c02;
    const double tr = (g00 + g11 + g22) * (1.0 / 3.0);
    int st = 0;
    Vec3 g = v3(0, 0, 0);
    if (det > 1e-12 * tr * tr * tr) {
      const double c11 = g00 * g22 - g02 * g02, c12 = g02 * g01 - g00 * g12, c22 = g00 * g11 - g01 * g01;
      const double id = 1.0 / det;
      g = v3((c00 * b0 + c01 * b1 + c02 * b2) * id, (c01 * b0 + c11 * b1 + c12 * b2) * id,
             (c02 * b0 + c12 * b1 + c22 * b2) * id);
    } else {
      st = VOF_ST_SINGULAR_LSQ;
      ++nsing;
    }
    W.grad[3 * c] = g.x; W.grad[3 * c + 1] = g.y; W.grad[3 * c + 2] = g.z;
    if (W.iface_stamp[c] == step) W.status[c] |= st;
    else W.status[c] = st;
  }
  if (nsing) atomicAdd((unsigned long long*)&W.counters->n_singular, (unsigned long long)nsing);
}

// ---- per-side gradients and source (R5, R6) on interface cells, totals (R8) -----------------------
// The totals are the pairwise tree over the interface list (cell order) padded with zeros to a
// power of two. A thread per interface cell computes its source (a loop over its faces, one cell
// per lane so that the FP64 warp instructions keep every lane busy); a block takes aligned tiles
// of kSrcTile = blockDim interface cells and sums each tile's subtree (warp shuffles, then the
// warp sums); the last block to finish (an atomic count of finished blocks) folds the tile sums in
// subtrees of 2 kThreads leaves, level by level, so the pairing is the whole tree's. The zeros of
// the cells outside the interface are written by a memset on a side branch of the step.

// Pairwise tree of x[base, base + 2 T) (zeros past n) in a block of T threads (T a multiple of 32,
// at most 1024); the result is valid in thread 0. Thread t pairs leaves 2t and 2t+1, lanes then
// pair their neighbours (lane t + 2^k joins lane t), and warp 0 pairs the warp sums.
template <int T>
__device__ double block_tree(const double* x, int64_t n, int64_t base, double* sw) {
  const int t = threadIdx.x, lane = t & 31;
  const int64_t i0 = base + 2 * t;
  double v = (i0 < n ? __ldcg(x + i0) : 0.0) + (i0 + 1 < n ? __ldcg(x + i0 + 1) : 0.0);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double w = __shfl_down_sync(0xffffffffu, v, o);
    if ((lane & (2 * o - 1)) == 0) v += w;
  }
  if (lane == 0) sw[t >> 5] = v;
  __syncthreads();
  double r = 0;
  if (t < 32) {
    v = t < T / 32 ? sw[t] : 0.0;
#pragma unroll
    for (int o = 1; o < T / 32; o <<= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      if ((lane & (2 * o - 1)) == 0) v += w;
    }
    r = v;
  }
  __syncthreads();
  return r;
}


// Sum of the aligned leaves [tile * kThreads, (tile + 1) * kThreads) in thread order: each warp's
// 32 leaves by shuffles (lane t + 2^k joins lane t), then warp 0 pairs the warp sums. Valid in
// thread 0.
__device__ __forceinline__ double tile_tree(double v, double* sw) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double w = __shfl_down_sync(0xffffffffu, v, o);
    if ((lane & (2 * o - 1)) == 0) v += w;
  }
  if (lane == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x < 32) {
    v = lane < kThreads / 32 ? sw[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < kThreads / 32; o <<= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      if ((lane & (2 * o - 1)) == 0) v += w;
    }
    r = v;
  }
  __syncthreads();
  return r;
}

__device__ void source_phase(const MeshView& M, const StepArgs& a, Workspace& W) {
  static_assert(kSrcTile == kThreads, "a tile per block pass, a cell per thread");
  __shared__ double swm[kThreads / 32], swq[kThreads / 32];
  const int64_t n = W.counters->n_iface;
  const int64_t ntiles = (n + kSrcTile - 1) / kSrcTile;
  const int64_t tcap = (M.n_cells + kSrcTile - 1) / kSrcTile;
  const double inv_hlv = 1.0 / a.props.h_lv;
  int nside = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * kSrcTile + threadIdx.x;
    double mV = 0, qV = 0;
    if (i < n) {
      const int32_t c = W.iface_idx[i];
      double mdot = 0, Q = 0, ql = 0, qv = 0;
      Vec3 gl = v3(0, 0, 0), gv = v3(0, 0, 0);
      const double Aint = W.A_int[c];
      if (positive(Aint)) {
        const Vec3 nn = v3(W.n_int[3 * c], W.n_int[3 * c + 1], W.n_int[3 * c + 2]);
        const bool liq = liquid(a.alpha[c]);  // the other side is vapour (weights of -n) or liquid (+n)
        if (a.opt.extrap) {  // both sides written by the pseudo-time solve
          gl = v3(W.grad_l[3 * c], W.grad_l[3 * c + 1], W.grad_l[3 * c + 2]);
          gv = v3(W.grad_v[3 * c], W.grad_v[3 * c + 1], W.grad_v[3 * c + 2]);
        } else {
          // R5: weights max(0, n . A_f) towards the other phase, the weighted mean of the
          // neighbours' gradients there
          double p0 = 0, p1 = 0, p2 = 0, p3 = 0;
          for (int64_t k = M.cell_face_off[c]; k < M.cell_face_off[c + 1]; ++k) {
            const int32_t fe = M.cell_face[k];
            const int32_t f = fe & 0x7fffffff;
            const int32_t q = M.face_owner[f] == c ? M.face_neigh[f] : M.face_owner[f];
            if (q < 0 || liquid(a.alpha[q]) == liq) continue;
            const Vec3 Af = v3(M.face_area[3 * f], M.face_area[3 * f + 1], M.face_area[3 * f + 2]);
            double w = flip_if(dot(nn, Af), (fe < 0) != liq);  // outward area of c, towards the other side
            w = positive(w) ? w : 0.0;
            p0 = fma(W.grad[3 * q], w, p0);
            p1 = fma(W.grad[3 * q + 1], w, p1);
            p2 = fma(W.grad[3 * q + 2], w, p2);
            p3 += w;
          }
          Vec3 go = v3(0, 0, 0);
          if (positive(p3)) {
            const double r = 1.0 / p3;
            go = v3(p0 * r, p1 * r, p2 * r);
          } else {
            W.status[c] |= VOF_ST_NO_SIDE;
            ++nside;
          }
          const Vec3 gown = v3(W.grad[3 * c], W.grad[3 * c + 1], W.grad[3 * c + 2]);
          gl = liq ? gown : go;
          gv = liq ? go : gown;
        }
        ql = a.props.k_l * dot(gl, nn) * Aint;
        qv = -a.props.k_v * dot(gv, nn) * Aint;
        mdot = (ql + qv) * inv_hlv * M.cell_ivol[c];
        Q = -mdot * a.props.h_lv;
      }
      const double V = M.cell_vol[c];
      mV = mdot * V;
      qV = Q * V;
      a.mdot[c] = mdot;
      a.Q[c] = Q;
      W.q_l[c] = ql;
      W.q_v[c] = qv;
      W.grad_l[3 * c] = gl.x; W.grad_l[3 * c + 1] = gl.y; W.grad_l[3 * c + 2] = gl.z;
      W.grad_v[3 * c] = gv.x; W.grad_v[3 * c + 1] = gv.y; W.grad_v[3 * c + 2] = gv.z;
      W.mdotV[i] = mV;
      W.QV[i] = qV;
    }
    const double tm = tile_tree(mV, swm), tq = tile_tree(qV, swq);
    if (threadIdx.x == 0) {
      W.tile_part[tile] = tm;
      W.tile_part[tcap + tile] = tq;
    }
  }
  if (nside) atomicAdd((unsigned long long*)&W.counters->n_no_side, (unsigned long long)nside);
}

// The last block to finish folds the tile sums into the two totals.
__device__ __noinline__ void fold_phase(const MeshView& M, const StepArgs& a, Workspace& W) {
  __shared__ double sw[kThreads / 32];
  const int64_t n = W.counters->n_iface;
  const int64_t ntiles = (n + kSrcTile - 1) / kSrcTile;
  const int64_t tcap = (M.n_cells + kSrcTile - 1) / kSrcTile;
  for (int q = 0; q < 2; ++q) {
    const double* src = W.tile_part + q * tcap;
    double* bufs[2] = {W.partial + 2 * q * kMaxPartials, W.partial + (2 * q + 1) * kMaxPartials};
    int64_t m = ntiles;
    int pp = 0;
    while (m > 1) {
      const int64_t mc = (m + 2 * kThreads - 1) / (2 * kThreads);
      double* dst = bufs[pp];
      for (int64_t b = 0; b < mc; ++b) {
        const double r = block_tree<kThreads>(src, m, b * 2 * kThreads, sw);
        if (threadIdx.x == 0) dst[b] = r;
      }
      __syncthreads();
      src = dst;
      pp ^= 1;
      m = mc;
    }
    if (threadIdx.x == 0) a.totals[q] = m == 0 ? 0.0 : __ldcg(src);
    __syncthreads();
  }
}

__global__ void k_xface(MeshView M, const double* alpha, int xf_mode, Workspace W) { xface_phase(M, alpha, xf_mode, W); }

// Eq. interface_htc on each listed crossing face: a_f = k_phi A_int,f / d_f on both sides, k_phi
// the conductivity of the side's phase. Nothing in the step reads it: it runs on request
// (options.htc), on a side branch next to the least squares and the source.
__global__ void k_htc(MeshView M, const double* alpha, double k_l, double k_v, Workspace W) {
  const int64_t n = W.counters->n_crossing;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f = W.xface_list[j];
    const int32_t o = M.face_owner[f], nbr = M.face_neigh[f];
    const double af = W.A_int_f[f], d_o = W.d_own[f], d_n = W.d_neigh[f];
    const double ko = alpha[o] > 0.5 ? k_l : k_v, kn = alpha[nbr] > 0.5 ? k_l : k_v;
    W.a_own[f] = d_o > 0 ? ko * af / d_o : 0.0;
    W.a_neigh[f] = d_n > 0 ? kn * af / d_n : 0.0;
  }
}

// Eq. interface_htc in the energy equation: each band cell adds a_f to its matrix diagonal and
// a_f T_sat to its right-hand side for every face the interface detaches from the diffusive
// coupling (the crossing faces of this step), a_f being the coefficient of the cell's own side. A
// thread per band cell over its faces in the cell's face order; other cells have no such face with
// a non-zero coefficient (a crossing face next to no band cell has no interface plane on either
// side, so A_int,f = 0 there).
__global__ void k_htc_cells(MeshView M, double T_sat, Workspace W) {
  const uint32_t step = W.counters->step;
  const int64_t nb = W.counters->n_band;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = W.band_idx[j];
    double d = 0, r = 0;
    for (int64_t k = M.cell_face_off[c]; k < M.cell_face_off[c + 1]; ++k) {
      const int32_t f = M.cell_face[k] & 0x7fffffff;
      if (W.face_stamp[f] != step) continue;
      const double a = M.face_owner[f] == c ? W.a_own[f] : W.a_neigh[f];
      d += a;
      r += a * T_sat;
    }
    W.htc_diag[c] = d;
    W.htc_rhs[c] = r;
  }
}

// ---- pseudo-time extrapolation of the per-side gradients (Eq. extrapolation) ------------------
// One solve per side and gradient component, all six in one cooperative launch. The unknowns of
// a side are the interface cells of the other phase, one per interface-list slot (its other
// side), and they start from the slot's own modified least-squares gradient. First-order upwind
// explicit step (Jacobi): x <- x + f_P sum_f w_f (x_Q - x), w_f = sigma n_P . A_f > 0 over the
// inflow faces whose neighbour is a cell of the side (fixed value: its gradient) or an unknown of
// the same solve (its previous iterate); sigma = +1 for the liquid side, -1 for the vapour side,
// so that each side moves from its bulk towards the interface; f_P = min(dtau, V_P / sum w_f) / V_P.
// Written as x <- x + b - C x + sum over the unknown neighbours of g_Q x_Q: the fixed part b,
// C = f_P sum w_f and the first kExCap unknown neighbours (slot, g_Q = f_P w_f) are gathered once
// (further unknown faces, rare, are walked on the mesh each iteration from a bit mask).
//
// Layout for the FP64 pipe: a warp instruction holds its sub-partition's FP64 unit for the same
// time whatever its active lanes, so an iteration costs FP64 warp instructions, not lanes. Each
// slot takes three lanes (one per component; ten slots per warp), which cuts a warp's FP64
// instructions per iteration about threefold, and the grid spreads the warps over every SM. When
// the grid has a lane per component of every slot, a lane keeps its constants and iterate in
// registers.
//
// Iterations end at a grid barrier of its own that also carries the stopping test: each block
// adds 1 + sum over the solves it saw move by tol or more of 1 << (16 + 8 j) to the iteration's
// 64-bit word (low 16 bits: arrivals; 8 bits per solve: blocks still moving), then polls the word
// until every block has arrived. A solve stops after the first iteration in which no block saw a
// change of tol or more (its largest change is below tol), or after max_iter; a stopped solve's
// components are carried forward unchanged. The poll gives up after poll_limit reads
// (options.extrap_poll_limit): the block then stops iterating, and the step reports -1 iterations
// for every solve (results invalid).
// Threads per block (one block per SM): 256 when the mesh has under 2^20 cells, 512 otherwise. A step
// with more interface cells than the launch has lane triples loops over them every iteration,
// reading their constants from memory, and more warps per SM hide that latency (8M pipe: 50 -> 34
// us per iteration); with few interface cells the per-iteration block barrier dominates and a
// smaller block passes it faster (250k film: 2.8 against 3.7 us per iteration).
constexpr int kExThreadsSmall = 256, kExThreadsLarge = 512;
constexpr int kExSlotsPerWarp = 10;  // three lanes each; lanes 30 and 31 idle

struct ExSlot {
  double C, f, b0, b1, b2;
  double g[kExCap];
  int32_t nb[kExCap];        // slots of the first unknown neighbours (-1: none)
  unsigned long long mask;   // face positions of further unknown neighbours
  int32_t c;
  int side;                  // 0: an unknown of the liquid side (a vapour cell), 1: of the vapour side
};

// The constants of slot i (step weights, fixed inflow part, unknown neighbours); flags and counts a
// slot without inflow.
__device__ __forceinline__ ExSlot ex_prep(const MeshView& M, const Workspace& W, const double* alpha, double eps,
                                          double dtau, int64_t i, int& nside) {
  ExSlot s;
  const int32_t c = W.iface_idx[i];
  s.c = c;
  s.side = alpha[c] > 0.5 ? 1 : 0;  // a liquid cell is an unknown of the vapour side, and the reverse
  s.C = s.f = s.b0 = s.b1 = s.b2 = 0.0;
  s.mask = 0;
#pragma unroll
  for (int t = 0; t < kExCap; ++t) {
    s.g[t] = 0.0;
    s.nb[t] = -1;
  }
  if (!(W.A_int[c] > 0)) return s;
  const bool liq = s.side == 1;
  const Vec3 nn = v3(W.n_int[3 * c], W.n_int[3 * c + 1], W.n_int[3 * c + 2]);
  const int64_t e0 = M.cell_face_off[c], e1 = M.cell_face_off[c + 1];
  double ws = 0;
  int cnt = 0;
  for (int64_t e = e0; e < e1; ++e) {
    const int32_t fe = M.cell_face[e];
    const int32_t fc = fe & 0x7fffffff;
    const int32_t q = M.face_owner[fc] == c ? M.face_neigh[fc] : M.face_owner[fc];
    if (q < 0) continue;
    const Vec3 Af = v3(M.face_area[3 * fc], M.face_area[3 * fc + 1], M.face_area[3 * fc + 2]);
    const double w = flip_if(dot(nn, Af), (fe < 0) != liq);  // sigma n . (outward area of c)
    if (!(w > 0)) continue;
    const double aq = alpha[q];
    if ((aq > 0.5) != liq) {  // a cell of the side: fixed value
      ws += w;
      s.b0 = fma(w, W.grad[3 * q], s.b0);
      s.b1 = fma(w, W.grad[3 * q + 1], s.b1);
      s.b2 = fma(w, W.grad[3 * q + 2], s.b2);
    } else if (is_iface(aq, eps) && W.A_int[q] > 0) {  // an unknown of the same solve
      ws += w;
      if (cnt < kExCap) {
#pragma unroll
        for (int t = 0; t < kExCap; ++t)
          if (t == cnt) {
            s.g[t] = w;
            s.nb[t] = W.iface_slot[q];
          }
        ++cnt;
      } else {
        s.mask |= 1ull << (e - e0);
      }
    }
  }
  if (ws > 0) {
    const double V = M.cell_vol[c];
    s.f = fmin(dtau, V / ws) / V;
    s.C = s.f * ws;
    s.b0 *= s.f;
    s.b1 *= s.f;
    s.b2 *= s.f;
#pragma unroll
    for (int t = 0; t < kExCap; ++t) s.g[t] *= s.f;
  } else {
    W.status[c] |= VOF_ST_NO_SIDE;  // no inflow: keeps its start value
    ++nside;
  }
  return s;
}

struct ExLane {
  double C, f, b;
  double g[kExCap];
  int32_t nb[kExCap];        // slots of the first unknown neighbours (-1: none)
  unsigned long long mask;   // face positions of further unknown neighbours
  int32_t c;
  int side;                  // 0: an unknown of the liquid side (a vapour cell), 1: of the vapour side
};

__device__ __forceinline__ ExLane ex_lane_load(const Workspace& W, const double* alpha, int64_t i, int comp) {
  ExLane s;
  const double* k5 = W.ex_k + 5 * i;
  s.C = k5[0];
  s.f = k5[1];
  s.b = k5[2 + comp];
#pragma unroll
  for (int t = 0; t < kExCap; ++t) {
    s.nb[t] = W.ex_nb[kExCap * i + t];
    s.g[t] = W.ex_g[kExCap * i + t];
  }
  s.mask = W.ex_mask[i];
  s.c = W.iface_idx[i];
  s.side = alpha[s.c] > 0.5 ? 1 : 0;
  return s;
}

// One Jacobi step of one component of a slot from the previous iterates Xo ([slot][4]); x in, new
// iterate out; the solve's bit ORed into `moved` when it moved by tol or more.
__device__ __forceinline__ void ex_update(const MeshView& M, const Workspace& W, const ExLane& s, int comp,
                                          const double* Xo, unsigned active, double tol, double& x,
                                          unsigned& moved) {
  const int j = 3 * s.side + comp;
  if (!(s.C > 0) || !((active >> j) & 1u)) return;
  double a = fma(-s.C, x, x + s.b);
#pragma unroll
  for (int t = 0; t < kExCap; ++t)
    if (s.nb[t] >= 0) a = fma(s.g[t], __ldcg(Xo + 4 * (int64_t)s.nb[t] + comp), a);
  if (s.mask) {
    const bool liq = s.side == 1;
    const Vec3 nn = v3(W.n_int[3 * s.c], W.n_int[3 * s.c + 1], W.n_int[3 * s.c + 2]);
    const int64_t e0 = M.cell_face_off[s.c];
    unsigned long long mask = s.mask;
    while (mask) {
      const int jf = __ffsll((long long)mask) - 1;
      mask &= mask - 1;
      const int32_t fe = M.cell_face[e0 + jf];
      const int32_t fc = fe & 0x7fffffff;
      const int32_t q = M.face_owner[fc] == s.c ? M.face_neigh[fc] : M.face_owner[fc];
      const Vec3 Af = v3(M.face_area[3 * fc], M.face_area[3 * fc + 1], M.face_area[3 * fc + 2]);
      const double g = s.f * flip_if(dot(nn, Af), (fe < 0) != liq);
      a = fma(g, __ldcg(Xo + 4 * (int64_t)W.iface_slot[q] + comp), a);
    }
  }
  if (fabs(a - x) >= tol) moved |= 1u << j;
  x = a;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Arrival with release semantics at GPU scope: the block's iterates (ordered before this thread by
// the block barrier) are visible to any thread whose acquire load sees the sum.
__device__ __forceinline__ void red_release_add_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <int TB>
__global__ void __launch_bounds__(TB) k_extrap(MeshView M, const double* alpha, double eps, int max_iter,
                                                        double tol, int poll_limit, Workspace W) {
  cg::grid_group grid = cg::this_grid();
  __shared__ unsigned s_or[2];
  __shared__ unsigned s_dec;
  const int64_t n = W.counters->n_iface;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  double* Xa = W.ex_x;  // [slot][4]: x0, x1, x2, pad
  double* Xb = W.ex_x + 4 * M.n_cells;
  // (0) a thread per slot: fixed inflow part, step weights, unknown neighbours, start value
  int nside = 0;
  const double dtau = *W.ex_dtau;
  for (int64_t i = t0; i < n; i += nthr) {
    const ExSlot sl = ex_prep(M, W, alpha, eps, dtau, i, nside);
    double* k5 = W.ex_k + 5 * i;
    k5[0] = sl.C; k5[1] = sl.f; k5[2] = sl.b0; k5[3] = sl.b1; k5[4] = sl.b2;
#pragma unroll
    for (int t = 0; t < kExCap; ++t) {
      W.ex_nb[kExCap * i + t] = sl.nb[t];
      W.ex_g[kExCap * i + t] = sl.g[t];
    }
    W.ex_mask[i] = sl.mask;
    Xa[4 * i] = W.grad[3 * sl.c];
    Xa[4 * i + 1] = W.grad[3 * sl.c + 1];
    Xa[4 * i + 2] = W.grad[3 * sl.c + 2];
  }
  if (nside) atomicAdd((unsigned long long*)&W.counters->n_no_side, (unsigned long long)nside);
  for (int64_t j = t0; j <= max_iter; j += nthr) W.ex_itmax[j] = 0ull;
  if (threadIdx.x < 2) s_or[threadIdx.x] = 0u;
  grid.sync();
  // (1) the iterations: three lanes per slot
  const int64_t warp = t0 >> 5, nwarps = nthr >> 5;
  const int sw = lane / 3, comp = lane - 3 * (lane / 3);
  const int64_t ngroups = (n + kExSlotsPerWarp - 1) / kExSlotsPerWarp;
  const bool one = ngroups <= nwarps;  // a lane per component of every slot: registers
  const int64_t im = warp * kExSlotsPerWarp + sw;
  const bool mine_ok = one && sw < kExSlotsPerWarp && im < n;
  ExLane mine;
  double xm = 0;
  if (mine_ok) {
    mine = ex_lane_load(W, alpha, im, comp);
    xm = Xa[4 * im + comp];
  }
  unsigned active = 0x3fu;
  int K[6] = {max_iter, max_iter, max_iter, max_iter, max_iter, max_iter};
  bool failed = false;
  const double* Xo = Xa;
  double* Xn = Xb;
  for (int k = 1; k <= max_iter; ++k) {
    unsigned moved = 0;
    if (one) {
      if (mine_ok) {
        ex_update(M, W, mine, comp, Xo, active, tol, xm, moved);
        Xn[4 * im + comp] = xm;
      }
    } else if (sw < kExSlotsPerWarp) {
      for (int64_t gi = warp; gi < ngroups; gi += nwarps) {
        const int64_t i = gi * kExSlotsPerWarp + sw;
        if (i >= n) continue;
        const ExLane sl = ex_lane_load(W, alpha, i, comp);
        double x = __ldcg(Xo + 4 * i + comp);
        ex_update(M, W, sl, comp, Xo, active, tol, x, moved);
        Xn[4 * i + comp] = x;
      }
    }
    moved = __reduce_or_sync(0xffffffffu, moved);
    if (lane == 0 && moved) atomicOr(&s_or[k & 1], moved);
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned v = s_or[k & 1];
      s_or[(k + 1) & 1] = 0u;  // the next iteration's word: cleared before this block's barrier below
      unsigned long long add = 1ull;
#pragma unroll
      for (int j = 0; j < 6; ++j)
        if ((v >> j) & 1u) add += 1ull << (16 + 8 * j);
      red_release_add_gpu(W.ex_itmax + k, add);
      unsigned long long cur = 0;
      long long spins = 0;
      do {  // the acquire load orders this block's next reads (through the block barrier) after it
        cur = ld_acquire_gpu(W.ex_itmax + k);
      } while ((cur & 0xffffull) < gridDim.x && ++spins < poll_limit);
      unsigned dec = 0;
      if ((cur & 0xffffull) < gridDim.x) {
        dec = 0x80000000u;  // gave up waiting
      } else {
#pragma unroll
        for (int j = 0; j < 6; ++j)
          if ((cur >> (16 + 8 * j)) & 0xffull) dec |= 1u << j;
      }
      s_dec = dec;
    }
    __syncthreads();
    const unsigned still = s_dec;
    if (still & 0x80000000u) {
      failed = true;
      break;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j)
      if (((active >> j) & 1u) && !((still >> j) & 1u)) K[j] = k;
    active &= still;
    const double* t = Xo;
    Xo = Xn;
    Xn = const_cast<double*>(t);
    if (!active) break;
  }
  // (2) both sides of every interface cell with an interface (iterates of the last iteration, in
  // this thread's registers or, for the other slots, written before the last barrier)
  if (one) {
    if (mine_ok && W.A_int[mine.c] > 0) {
      double* own = mine.side ? W.grad_l : W.grad_v;
      double* oth = mine.side ? W.grad_v : W.grad_l;
      own[3 * mine.c + comp] = W.grad[3 * mine.c + comp];
      oth[3 * mine.c + comp] = xm;
    }
  } else if (sw < kExSlotsPerWarp) {
    for (int64_t gi = warp; gi < ngroups; gi += nwarps) {
      const int64_t i = gi * kExSlotsPerWarp + sw;
      if (i >= n) continue;
      const int32_t c = W.iface_idx[i];
      if (!(W.A_int[c] > 0)) continue;
      const bool liq = alpha[c] > 0.5;
      double* own = liq ? W.grad_l : W.grad_v;
      double* oth = liq ? W.grad_v : W.grad_l;
      own[3 * c + comp] = W.grad[3 * c + comp];
      oth[3 * c + comp] = __ldcg(Xo + 4 * i + comp);
    }
  }
  // counts (zeroed at the step's start): a block that gave up marks every solve -1, which a count
  // written by block 0 never overwrites
  unsigned long long* it = (unsigned long long*)W.counters->extrap_iters;
  if (failed) {
    if (threadIdx.x == 0)
      for (int j = 0; j < 6; ++j) atomicExch(it + j, (unsigned long long)-1ll);
  } else if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int j = 0; j < 6; ++j) atomicCAS(it + j, 0ull, (unsigned long long)K[j]);
  }
}

// ---- least-squares variants of the stencil-anisotropy study (options.lsq_variant) -------------
// A thread per band cell: G = sum w r r^T, b = sum w r dT over the chosen stencil (bits: 1 the
// standard stencil, 2 weights w = 1/|r|^2, 4 every cell sharing a vertex, 8 also cond(G_P)), then
// the same explicit inverse and singular test as the path's kernel. In the vertex stencil a
// neighbour reached through several shared vertices is counted at the first of the cell's
// (sorted) vertices it contains; across the interface a face neighbour enters at the face's
// crossing point, any other at the linear interpolation of alpha along the centroid connection.
// cond = lambda_max / lambda_min from the eigenvalues of G_P by cyclic Jacobi rotations (Golub and
// Van Loan, Sec. 8.5: each rotation zeroes one off-diagonal pair; at most eight sweeps of the three
// pairs), accurate also where two eigenvalues coincide.
__device__ __forceinline__ void jacobi_rotate(double& dp, double& dq, double& apq, double& arp, double& arq) {
  // the plane rotation that zeroes apq: tan(2 phi) = 2 apq / (dq - dp); off-pair entries rotate
  if (apq == 0.0) return;
  const double th = (dq - dp) / (2.0 * apq);
  const double t = fabs(th) > 1e150 ? 0.5 / th : copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
  const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
  dp -= t * apq;
  dq += t * apq;
  apq = 0.0;
  const double rp = arp, rq = arq;
  arp = c * rp - s * rq;
  arq = s * rp + c * rq;
}

__device__ double sym3_cond(double a00, double a01, double a02, double a11, double a12, double a22) {
  double d0 = a00, d1 = a11, d2 = a22, e01 = a01, e02 = a02, e12 = a12;
  for (int sweep = 0; sweep < 8; ++sweep) {
    if (e01 * e01 + e02 * e02 + e12 * e12 <= 1e-34 * (d0 * d0 + d1 * d1 + d2 * d2)) break;
    jacobi_rotate(d0, d1, e01, e02, e12);  // pair (0, 1); the third index is 2
    jacobi_rotate(d0, d2, e02, e01, e12);  // pair (0, 2); the third index is 1
    jacobi_rotate(d1, d2, e12, e01, e02);  // pair (1, 2); the third index is 0
  }
  const double lmax = fmax(d0, fmax(d1, d2)), lmin = fmin(d0, fmin(d1, d2));
  return lmin > 0 ? lmax / lmin : CUDART_INF;
}

__global__ void __launch_bounds__(kThreads) k_lsq_study(MeshView M, StepArgs a, Workspace W) {
  const int variant = a.opt.lsq_variant;
  const bool standard = variant & 1, idw = variant & 2, ext = variant & 4, want_cond = variant & 8;
  const uint32_t step = W.counters->step;
  const int64_t nb = W.counters->n_band;
  int nsing = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = W.band_idx[j];
    const Vec3 xP = v3(M.cell_cen[3 * c], M.cell_cen[3 * c + 1], M.cell_cen[3 * c + 2]);
    const double TP = a.T[c], aP = a.alpha[c];
    double g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0, b0 = 0, b1 = 0, b2 = 0;
    auto entry = [&](const Vec3& r, double dT) {
      const double w = idw ? 1.0 / dot(r, r) : 1.0;
      const double wx = w * r.x, wy = w * r.y, wz = w * r.z;
      g00 = fma(wx, r.x, g00); g01 = fma(wx, r.y, g01); g02 = fma(wx, r.z, g02);
      g11 = fma(wy, r.y, g11); g12 = fma(wy, r.z, g12); g22 = fma(wz, r.z, g22);
      b0 = fma(wx, dT, b0); b1 = fma(wy, dT, b1); b2 = fma(wz, dT, b2);
    };
    // a neighbour q (face f, or -1 when it shares no face with c)
    auto neighbour = [&](int32_t q, int32_t f) {
      const double aq = a.alpha[q];
      const Vec3 xQ = v3(M.cell_cen[3 * q], M.cell_cen[3 * q + 1], M.cell_cen[3 * q + 2]);
      if (standard || !((aP - 0.5) * (aq - 0.5) < 0)) {
        entry(xQ - xP, a.T[q] - TP);
      } else if (f >= 0) {
        entry(v3(W.x_f[3 * f], W.x_f[3 * f + 1], W.x_f[3 * f + 2]) - xP, a.props.T_sat - TP);
      } else {
        const double t = (aP - 0.5) / (aP - aq);
        entry((xQ - xP) * t, a.props.T_sat - TP);
      }
    };
    const int64_t f0 = M.cell_face_off[c], f1 = M.cell_face_off[c + 1];
    for (int64_t k = f0; k < f1; ++k) {
      const int32_t f = M.cell_face[k] & 0x7fffffff;
      const int32_t q = M.face_owner[f] == c ? M.face_neigh[f] : M.face_owner[f];
      if (q < 0) {
        if (a.T_bnd) entry(v3(M.face_cen[3 * f], M.face_cen[3 * f + 1], M.face_cen[3 * f + 2]) - xP, a.T_bnd[f] - TP);
      } else if (!ext) {
        neighbour(q, f);
      }
    }
    if (ext) {
      const int64_t v0 = M.cell_vert_off[c], v1 = M.cell_vert_off[c + 1];
      for (int64_t kv = v0; kv < v1; ++kv) {
        const int32_t v = M.cell_vert[kv];
        for (int64_t e = M.vert_cell_off[v]; e < M.vert_cell_off[v + 1]; ++e) {
          const int32_t q = M.vert_cell[e];
          if (q == c) continue;
          bool seen = false;  // q already reached through an earlier vertex of c
          for (int64_t k2 = v0; k2 < kv && !seen; ++k2) {
            const int32_t v2 = M.cell_vert[k2];
            for (int64_t e2 = M.vert_cell_off[v2]; e2 < M.vert_cell_off[v2 + 1]; ++e2)
              if (M.vert_cell[e2] == q) {
                seen = true;
                break;
              }
          }
          if (seen) continue;
          int32_t fq = -1;  // the face shared with q, if any
          for (int64_t k = f0; k < f1 && fq < 0; ++k) {
            const int32_t f = M.cell_face[k] & 0x7fffffff;
            if ((M.face_owner[f] == c ? M.face_neigh[f] : M.face_owner[f]) == q) fq = f;
          }
          neighbour(q, fq);
        }
      }
    }
    const double c00 = g11 * g22 - g12 * g12, c01 = g02 * g12 - g01 * g22, c02 = g01 * g12 - g02 * g11;
    const double det = g00 * c00 + g01 * c01 + g02 * c02;
    const double tr = (g00 + g11 + g22) * (1.0 / 3.0);
    int st = 0;
    Vec3 g = v3(0, 0, 0);
    if (det > 1e-12 * tr * tr * tr) {
      const double c11 = g00 * g22 - g02 * g02, c12 = g02 * g01 - g00 * g12, c22 = g00 * g11 - g01 * g01;
      const double id = 1.0 / det;
      g = v3((c00 * b0 + c01 * b1 + c02 * b2) * id, (c01 * b0 + c11 * b1 + c12 * b2) * id,
             (c02 * b0 + c12 * b1 + c22 * b2) * id);
    } else {
      st = VOF_ST_SINGULAR_LSQ;
      ++nsing;
    }
    W.grad[3 * c] = g.x; W.grad[3 * c + 1] = g.y; W.grad[3 * c + 2] = g.z;
    if (want_cond) W.lsq_cond[c] = sym3_cond(g00, g01, g02, g11, g12, g22);
    if (W.iface_stamp[c] == step) W.status[c] |= st;
    else W.status[c] = st;
  }
  if (nsing) atomicAdd((unsigned long long*)&W.counters->n_singular, (unsigned long long)nsing);
}

__global__ void __launch_bounds__(kThreads) k_lsq(MeshView M, StepArgs a, Workspace W) { lsq_phase(M, a, W); }

// Sources and tile sums; the last block to finish folds the totals.
__global__ void __launch_bounds__(kThreads) k_source(MeshView M, StepArgs a, Workspace W) {
  __shared__ bool last;
  source_phase(M, a, W);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's tile sums before its arrival
    last = atomicAdd(&W.counters->reduce_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  fold_phase(M, a, W);
  if (threadIdx.x == 0) W.counters->reduce_done = 0;
}

// Lanes per cell of a bin: the autotuned choice, else about four tetrahedra per lane with the
// bin's rows within ~110 KB of shared memory per block.
int pick_group(const vof_mesh* m, const vof_options& o, int bin) {
  if (o.group_size) return o.group_size;
  if (m->bin_G[bin]) return m->bin_G[bin];
  const double mean = bin == 0 ? 2.0 : (bin == 1 ? 6.0 : (bin == 2 ? 16.0 : (bin == 3 ? 36.0 : 100.0)));
  int g = 1;
  while (g < 32 && (g * 4 < mean || (size_t)(kThreads / g) * m->bin_max_ct[bin] * 88 > 110 * 1024)) g *= 2;
  return g;
}

// Block size of a bin's lane-group root search: up to kThreads threads, halved while the groups'
// rows exceed ~110 KB of shared memory; the shape fits when the block's groups stay within 220 KB.
int root_threads(const vof_mesh* m, int mode, int bin, int G, size_t* smem) {
  const size_t grp_bytes = root_group_bytes(m->bin_max_ct[bin], m->max_cv, mode);
  int threads = kThreads;
  while (threads > 32 && threads > G && (size_t)(threads / G) * grp_bytes > 110 * 1024) threads /= 2;
  *smem = (size_t)(threads / G) * grp_bytes;
  return threads;
}
bool root_group_fits(const vof_mesh* m, int mode, int bin, int G) {
  size_t smem = 0;
  root_threads(m, mode, bin, G, &smem);
  return smem <= 220 * 1024;
}

template <int G>
cudaError_t launch_root_g(vof_mesh* m, const double* alpha, const vof_options& opt, cudaStream_t s, int mode,
                          int use_mlp, int bin, int slow = 0) {
  const int max_ct = m->bin_max_ct[bin];
  const int max_cv = m->max_cv;
  size_t smem = 0;
  const int threads = root_threads(m, mode, bin, G, &smem);
  if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_root<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_root<G>, threads, smem);
  if (bps < 1) bps = 1;
  const int64_t need = (m->bin_cells[bin] + (threads / G) - 1) / (threads / G);
  // the slow list is short (usually empty): one block per SM at most
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)m->num_sms * (slow ? 1 : bps)));
  k_root<G><<<grid, threads, smem, s>>>(m->view, alpha, opt, m->ws, max_ct, max_cv, mode, use_mlp, bin, slow);
  return cudaGetLastError();
}

// Thread-per-cell root search of a bin whose cells have at most kCellMaxTets tetrahedra, then the
// lane-group kernel on the cells it handed over.
cudaError_t launch_root_cell(vof_mesh* m, const double* alpha, const vof_options& opt, cudaStream_t s, int mode,
                             int use_mlp, int bin) {
  const int nvmax = std::min(m->bin_max_ct[bin] + 3, m->max_cv);  // nt tetrahedra: at most nt + 3 vertices
  const size_t smem = (size_t)nvmax * kCellThreads * sizeof(float2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_root_cell, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr_set = true;
  }
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_root_cell, kCellThreads, smem);
  if (bps < 1) bps = 1;
  const int64_t need = (m->bin_cells[bin] + kCellThreads - 1) / kCellThreads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)m->num_sms * bps));
  k_root_cell<<<grid, kCellThreads, smem, s>>>(m->view, alpha, opt, m->ws, mode, use_mlp, bin);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_root_g<4>(m, alpha, opt, s, mode, use_mlp, bin, 1);
}

}  // namespace

cudaError_t launch_mlp_guess(vof_mesh* m, cudaStream_t s);  // vof_mlp.cu
cudaError_t launch_root_bin(vof_mesh* m, const double* alpha, const vof_options& opt, cudaStream_t s, int mode,
                            int use_mlp, int bin, int G);

vof_status launch_reconstruct(vof_mesh* m, const double* d_alpha, const vof_options& opt, cudaStream_t s,
                              bool early_xmark) {
  // the learned path needs the MLP guess; the interval cubic takes it when the mesh has an MLP;
  // guess = 1 starts both from 1 - alpha without the network
  const int learned = opt.guess == 0 && (opt.root_mode == VOF_ROOT_LEARNED || (opt.root_mode == VOF_ROOT_CUBIC && m->mlp));
  if (opt.root_mode == VOF_ROOT_LEARNED && opt.guess == 0 && !m->mlp) {
    set_error("learned root search requested but no MLP weights are set");
    return VOF_ESTATE;
  }
  Workspace& W = m->ws;
  const MeshView& M = m->view;
  W.alpha_in = d_alpha;
  Timing& tm = m->timing;
  // selection, band, vertex field and bins: one cooperative launch, as many blocks as are resident
  // phase 3's band cells and vertices per pass
  const size_t sel_smem = (size_t)(kThreads / kSelLanes) * (1 + m->max_cf + m->max_cv) * sizeof(int32_t);
  if (!m->sel_grid) {
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_select, kThreads, sel_smem);
    m->sel_grid = std::min(m->num_sms * std::max(1, std::min(bps, 8)), kMaxSelGrid);
  }
  if (!m->geom_grid) {  // the geometry grid: every resident warp of the device
    // cells per batch: the cut list of a full batch within a quarter of an SM's shared memory
    int bmax = kGeomBatch;
    while (bmax > 1 && geom_smem_bytes(m->max_ct, bmax) > (56u << 10)) --bmax;
    if (geom_smem_bytes(m->max_ct, bmax) > (227u << 10)) {
      set_error("interface geometry: a cell has too many tetrahedra for the cut list in shared memory");
      return VOF_EINVAL;
    }
    int bps = 0;
    cudaFuncSetAttribute(k_geom, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geom_smem_bytes(m->max_ct, bmax));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_geom, kGeomThreads, geom_smem_bytes(m->max_ct, bmax));
    m->geom_bmax = bmax;
    m->geom_grid = m->num_sms * std::max(1, bps);
  }
  {
    const double eps = opt.alpha_eps;
    int vmode = opt.vertex_mode, max_cf = m->max_cf;
    MeshView Mv = M;
    void* args[] = {&Mv, (void*)&d_alpha, (void*)&eps, &vmode, &max_cf, &W};
    tm.start(KC_SELECT, s);
    cudaError_t el = cudaLaunchCooperativeKernel((const void*)k_select, dim3(m->sel_grid), dim3(kThreads),
                                                 args, sel_smem, s);
    tm.stop(s);
    if (el != cudaSuccess) return cuda_fail(el, "selection kernel (cooperative launch)");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "selection kernels");
  if (early_xmark) {
    // crossing faces next to the band, needed only by the least squares: a side branch next to
    // the network's kernels and the root search
    cudaEventRecord(m->ev_xfork, s);
    cudaStreamWaitEvent(m->xm_stream, m->ev_xfork, 0);
    tm.start(KC_XMARK, m->xm_stream);
    k_xmark<<<m->num_sms * 4, kThreads, 0, m->xm_stream>>>(M, d_alpha, W);
    tm.stop(m->xm_stream);
    cudaEventRecord(m->ev_xjoin, m->xm_stream);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "crossing-face kernel");
  }
  if (learned) {
    e = launch_mlp_guess(m, s);  // times its two kernels itself
    if (e != cudaSuccess) return cuda_fail(e, "mlp guess");
  }
  // one branch per non-empty bin (root search); the branches join on s, then the geometry
  if (opt.root_mode == VOF_ROOT_FIXED) {
    tm.start(KC_ROOT, s);
    k_fixed_iso<<<m->num_sms * 2, kThreads, 0, s>>>(M, W, opt.alpha_iso);
    tm.stop(s);
  }
  e = opt.root_mode == VOF_ROOT_FIXED ? cudaSuccess : cudaEventRecord(m->ev_fork, s);
  for (int b = 0; b < kBins && e == cudaSuccess && opt.root_mode != VOF_ROOT_FIXED; ++b) {
    if (!m->bin_cells[b]) continue;
    cudaStream_t sb = m->bin_stream[b];
    e = cudaStreamWaitEvent(sb, m->ev_fork, 0);
    if (e != cudaSuccess) break;
    tm.start(KC_ROOT, sb);
    e = launch_root_bin(m, d_alpha, opt, sb, opt.root_mode, learned, b, pick_group(m, opt, b));
    tm.stop(sb);
    if (e != cudaSuccess) break;
    if (e == cudaSuccess) e = cudaEventRecord(m->ev_join[b], sb);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->ev_join[b], 0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "root search kernels");
  tm.start(KC_GEOM, s);
  k_geom<<<m->geom_grid, kGeomThreads, geom_smem_bytes(m->max_ct, m->geom_bmax), s>>>(M, W, m->max_ct, m->geom_bmax);
  tm.stop(s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "interface geometry kernel");
  return VOF_OK;
}

cudaError_t launch_root_bin(vof_mesh* m, const double* alpha, const vof_options& opt, cudaStream_t s, int mode,
                            int use_mlp, int bin, int G) {
  // one lane per cell of a small-cell bin: the thread-per-cell kernel (learned and cubic modes)
  if (G == 1 && mode != VOF_ROOT_BISECT && m->bin_max_ct[bin] <= kCellMaxTets)
    return launch_root_cell(m, alpha, opt, s, mode, use_mlp, bin);
  // A lanes-per-cell choice whose groups do not fit in shared memory in this mode (plain bisection
  // keeps FP64 rows, twice the bytes of the other modes' FP32 rows: a choice tuned for one mode may
  // not fit another) takes the next larger one that fits; 32 lanes always fit.
  while (G < 32 && !root_group_fits(m, mode, bin, G)) G *= 2;
  switch (G) {
    case 1: return launch_root_g<1>(m, alpha, opt, s, mode, use_mlp, bin);
    case 2: return launch_root_g<2>(m, alpha, opt, s, mode, use_mlp, bin);
    case 4: return launch_root_g<4>(m, alpha, opt, s, mode, use_mlp, bin);
    case 8: return launch_root_g<8>(m, alpha, opt, s, mode, use_mlp, bin);
    case 16: return launch_root_g<16>(m, alpha, opt, s, mode, use_mlp, bin);
    default: return launch_root_g<32>(m, alpha, opt, s, mode, use_mlp, bin);
  }
}

vof_status launch_source(vof_mesh* m, const StepArgs& a, cudaStream_t s, bool xmark_done) {
  const MeshView& M = m->view;
  Workspace& W = m->ws;
  Timing& tm = m->timing;
  // zeros of mdot and Q on a side branch, joined before the source kernel writes the interface cells
  cudaEventRecord(m->ev_zfork, s);
  cudaStreamWaitEvent(m->z_stream, m->ev_zfork, 0);
  cudaMemsetAsync(a.mdot, 0, (size_t)m->n_cells * sizeof(double), m->z_stream);
  cudaMemsetAsync(a.Q, 0, (size_t)m->n_cells * sizeof(double), m->z_stream);
  cudaEventRecord(m->ev_zjoin, m->z_stream);
  if (xmark_done) cudaStreamWaitEvent(s, m->ev_xjoin, 0);
  if (m->io_pending) {  // T and T_bnd of a host-buffer step, copied on the side
    cudaStreamWaitEvent(s, m->ev_io_done, 0);
    m->io_pending = false;
  }
  if (!xmark_done) {
    tm.start(KC_XMARK, s);
    k_xmark<<<m->num_sms * 4, kThreads, 0, s>>>(M, a.alpha, W);
    tm.stop(s);
  }
  tm.start(KC_XFACE, s);
  k_xface<<<m->num_sms * 4, kThreads, 0, s>>>(M, a.alpha, a.opt.xf_mode, W);
  tm.stop(s);
  if (a.opt.htc) {  // the interface heat-transfer coefficients on a side branch, joined after the source
    cudaEventRecord(m->ev_xfork, s);
    cudaStreamWaitEvent(m->xm_stream, m->ev_xfork, 0);
    tm.start(KC_HTC, m->xm_stream);
    k_htc<<<m->num_sms * 2, kThreads, 0, m->xm_stream>>>(M, a.alpha, a.props.k_l, a.props.k_v, W);
    k_htc_cells<<<m->num_sms * 2, kThreads, 0, m->xm_stream>>>(M, a.props.T_sat, W);
    tm.stop(m->xm_stream);
    cudaEventRecord(m->ev_xjoin, m->xm_stream);
  }
  tm.start(KC_LSQ, s);
  if (a.opt.lsq_variant)  // the stencil-anisotropy study's variants
    k_lsq_study<<<m->num_sms * 4, kThreads, 0, s>>>(M, a, W);
  else
    k_lsq<<<m->num_sms * 8, kThreads, 0, s>>>(M, a, W);
  tm.stop(s);
  if (a.opt.extrap) {
    // the pseudo-time solve: one cooperative launch
    const bool large = m->n_cells >= (1 << 20);
    const int ex_threads = large ? kExThreadsLarge : kExThreadsSmall;
    const void* ex_kernel = large ? (const void*)k_extrap<kExThreadsLarge> : (const void*)k_extrap<kExThreadsSmall>;
    if (!m->ex_grid) {  // a block per SM (the barrier word counts at most 255 blocks)
      int bps = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ex_kernel, ex_threads, 0);
      m->ex_grid = std::max(1, std::min(std::min(m->num_sms, m->num_sms * std::max(1, bps)), 255));
    }
    tm.start(KC_EXTRAP, s);
    MeshView Mv = M;
    const double* al = a.alpha;
    double eps = a.opt.alpha_eps, tol = a.opt.extrap_tol;
    int mi = a.opt.extrap_max_iter, poll = a.opt.extrap_poll_limit;
    void* args[] = {&Mv, (void*)&al, &eps, &mi, &tol, &poll, &W};
    cudaError_t el = cudaLaunchCooperativeKernel(ex_kernel, dim3(m->ex_grid), dim3(ex_threads), args, 0, s);
    tm.stop(s);
    if (el != cudaSuccess) return cuda_fail(el, "extrapolation kernel (cooperative launch)");
  }
  cudaStreamWaitEvent(s, m->ev_zjoin, 0);
  tm.start(KC_SOURCE, s);
  k_source<<<m->num_sms * 4, kThreads, 0, s>>>(M, a, W);
  tm.stop(s);
  if (a.opt.htc) cudaStreamWaitEvent(s, m->ev_xjoin, 0);  // the side branch (k_htc) joins here
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "source kernels");
  return VOF_OK;
}

}  // namespace vof

// Learned isovalue guess: a 40 -> 64 -> 64 -> 64 -> 1 GELU MLP that predicts the normalised
// isovalue position t = (c - phi_min)/(phi_max - phi_min) of an interface cell from its volume
// fraction, face count, sorted normalised vertex values and shape. BF16 operands, FP32
// accumulation: the forward and backward passes run on the tensor cores (mma.sync m16n8k16 bf16;
// the backward products take dZ rounded to BF16); FP32 master weights, Adam.
//
// Parameter vector (float32), row-major: W1 [64][40], b1 [64], W2 [64][64], b2 [64], W3 [64][64],
// b3 [64], w4 [64], b4 [1]  (VOF_MLP_N_PARAMS = 11009).
//
// Features of an interface cell (40): alpha; faces / 32; the vertex values normalised to [0, 1]
// over the cell's range, sorted descending, padded to 32 with the smallest; bounding-box extents
// / V^(1/3) (3); (vertex mean - bounding-box centre) / V^(1/3) (3). Cells with more than 32
// vertices or a degenerate range get no guess.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "vof_internal.cuh"

namespace vof {
namespace {

constexpr int kIn = 40, kInPad = 48, kH = 64;
constexpr int kNP = kH * kIn + kH + 2 * (kH * kH + kH) + kH + 1;
constexpr int LDX = kInPad + 8;  // bf16 row strides in shared memory (bank-conflict free)
constexpr int LDH = kH + 8;
constexpr int kRows = 64;        // samples per CTA
constexpr int kWarps = kRows / 16;
constexpr int kMaxBatch = 1 << 16;
constexpr int kMaxTiles = kMaxBatch / kRows;

// offsets into the parameter vector
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kH, ow4 = ob3 + kH, ob4 = ow4 + kH;
static_assert(ob4 + 1 == kNP, "parameter layout");

// BF16 copy of the weights in the layout the kernels load (W1 padded to 48 inputs).
struct WeightsBF16 {
  __nv_bfloat16 W1[kH][kInPad];
  __nv_bfloat16 W2[kH][kH];
  __nv_bfloat16 W3[kH][kH];
  float b1[kH], b2[kH], b3[kH], w4[kH], b4;  // w4 holds bf16-rounded values
};

// Standard normal CDF Phi(x) = (1 + erf(x / sqrt 2)) / 2, erf by Abramowitz and Stegun 7.1.25
// (absolute error below 2.5e-5, under a hundredth of the BF16 rounding that follows every hidden
// layer): with u = |x| / sqrt 2 and t = 1 / (1 + p u), 1 - erf(u) = t (a1 + t (a2 + t a3)) e^(-u^2).
// The tail (1 - erf(u)) / 2 is formed directly, so neither sign cancels. Here p u = (p / sqrt 2)|x|,
// the halves are folded into the coefficients, and e^(-u^2) = 2^(-(x s)^2) with s^2 = log2(e) / 2,
// so that the reciprocal and the exponential are one approximate hardware instruction each.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float phi_tail(float x) {  // (1 - erf(|x| / sqrt 2)) / 2
  const float t = rcp_approx(fmaf(0.33267253f, fabsf(x), 1.0f));          // p / sqrt 2, p = 0.47047
  const float poly = fmaf(fmaf(t, 0.3739278f, -0.0479399f), t, 0.1740121f);  // a3 / 2, a2 / 2, a1 / 2
  const float w = x * 0.84932180f;                                          // s = sqrt(log2(e) / 2)
  return t * poly * ex2_approx(-(w * w));
}
__device__ __forceinline__ float phi_cdf(float x) {
  const float tail = phi_tail(x);
  return x >= 0.f ? 1.0f - tail : tail;
}
__device__ __forceinline__ float gelu(float x) {
  const float xt = x * phi_tail(x);
  return x >= 0.f ? x - xt : xt;
}
__device__ __forceinline__ float gelu_grad(float x) {
  return phi_cdf(x) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// (hi, lo) float pair and its sum by Knuth's two-sum (for vertex-value differences in FP32)
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float t = __fadd_rn(__fadd_rn(e, a.lo), b.lo);
  const float h = __fadd_rn(s, t);
  return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// acc[nt][.] = rows m0..m0+15 of X[.][0..K) times W[0..64)[0..K)^T (16 x 64 output per warp).
// Fragment layouts of m16n8k16 (g = lane / 4, q = lane % 4): A a0a1 (row g, cols 2q, 2q+1),
// a2a3 (row g+8), a4a5 (row g, cols +8), a6a7 (row g+8, cols +8); B b0b1 (k 2q, 2q+1; n g),
// b2b3 (k +8); C c0c1 (row g, cols 2q, 2q+1), c2c3 (row g+8).
template <int K, int LDA, int LDB>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16* X, const __nv_bfloat16* W, int m0, float (&acc)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(X + (m0 + g) * LDA + k0 + 2 * q);
    a[1] = *reinterpret_cast<const uint32_t*>(X + (m0 + g + 8) * LDA + k0 + 2 * q);
    a[2] = *reinterpret_cast<const uint32_t*>(X + (m0 + g) * LDA + k0 + 8 + 2 * q);
    a[3] = *reinterpret_cast<const uint32_t*>(X + (m0 + g + 8) * LDA + k0 + 8 + 2 * q);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const __nv_bfloat16* w = W + (nt * 8 + g) * LDB + k0 + 2 * q;
      mma16816(acc[nt], a, *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
    }
  }
}

struct Smem {
  __nv_bfloat16 X[kRows * LDX];
  __nv_bfloat16 W1[kH * LDX];
  __nv_bfloat16 W2[kH * LDH];
  __nv_bfloat16 W3[kH * LDH];
  __nv_bfloat16 H1[kRows * LDH];
  __nv_bfloat16 H2[kRows * LDH];
  float b1[kH], b2[kH], b3[kH], w4[kH];
  float b4;
  float y[kRows];
};

// Inference: the hidden layers stay in registers, so only the input tile and the weights are staged.
struct FwdSmem {
  __nv_bfloat16 X[kRows * LDX];
  __nv_bfloat16 W1[kH * LDX];
  __nv_bfloat16 W2[kH * LDH];
  __nv_bfloat16 W3[kH * LDH];
  float b1[kH], b2[kH], b3[kH], w4[kH];
  float b4;
};

// 16-byte asynchronous copy global -> shared (no register round trip; completes at cp_async_wait)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Starts the copy of the weights (bf16) and biases into shared memory; they are there after
// cp_async_wait() and a barrier. 16-byte chunks: 6 per W1 row (48 bf16), 8 per W2 / W3 row
// (64 bf16); row strides of 56 and 72 bf16 keep every chunk 16-byte aligned, and b1, b2, b3, w4
// are contiguous in both layouts.
template <class S>
__device__ void stage_weights(S& s, const WeightsBF16& w) {
  for (int i = threadIdx.x; i < kH * 6; i += blockDim.x) cp_async16(s.W1 + (i / 6) * LDX + (i % 6) * 8, &w.W1[i / 6][(i % 6) * 8]);
  for (int i = threadIdx.x; i < kH * 8; i += blockDim.x) {
    cp_async16(s.W2 + (i / 8) * LDH + (i % 8) * 8, &w.W2[i / 8][(i % 8) * 8]);
    cp_async16(s.W3 + (i / 8) * LDH + (i % 8) * 8, &w.W3[i / 8][(i % 8) * 8]);
  }
  static_assert(offsetof(S, w4) == offsetof(S, b1) + 3 * kH * sizeof(float), "biases contiguous");
  static_assert(offsetof(WeightsBF16, w4) == offsetof(WeightsBF16, b1) + 3 * kH * sizeof(float), "biases contiguous");
  for (int i = threadIdx.x; i < kH; i += blockDim.x) cp_async16(s.b1 + 4 * i, w.b1 + 4 * i);
  if (threadIdx.x == 0) s.b4 = w.b4;
}

// Forward pass of the warp's 16 rows. Z (optional, fp32 [kRows][kH] x 3) keeps pre-activations,
// H3 (optional, fp32 [kRows][kH]) the last hidden layer; y gets the outputs.
__device__ void warp_forward(Smem& s, int m0, float* Z1, float* Z2, float* Z3, float* H3) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  float acc[8][4];
  warp_gemm<kInPad, LDX, LDX>(s.X, s.W1, m0, acc);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * q + (i & 1);
      const float z = acc[nt][i] + s.b1[c];
      if (Z1) Z1[r * kH + c] = z;
      s.H1[r * LDH + c] = __float2bfloat16_rn(gelu(z));
    }
  __syncwarp();
  warp_gemm<kH, LDH, LDH>(s.H1, s.W2, m0, acc);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * q + (i & 1);
      const float z = acc[nt][i] + s.b2[c];
      if (Z2) Z2[r * kH + c] = z;
      s.H2[r * LDH + c] = __float2bfloat16_rn(gelu(z));
    }
  __syncwarp();
  warp_gemm<kH, LDH, LDH>(s.H2, s.W3, m0, acc);
  float part[2] = {0.f, 0.f};
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + g + (i >= 2 ? 8 : 0), c = nt * 8 + 2 * q + (i & 1);
      const float z = acc[nt][i] + s.b3[c];
      const float h = gelu(z);
      if (Z3) Z3[r * kH + c] = z;
      if (H3) H3[r * kH + c] = h;
      part[i >> 1] = fmaf(h, s.w4[c], part[i >> 1]);
    }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    part[j] += __shfl_xor_sync(0xffffffffu, part[j], 1);
    part[j] += __shfl_xor_sync(0xffffffffu, part[j], 2);
  }
  if (q == 0) {
    s.y[m0 + g] = part[0] + s.b4;
    s.y[m0 + g + 8] = part[1] + s.b4;
  }
  __syncwarp();
}

// GELU of a layer's accumulators plus bias, rounded to BF16 and packed as the next layer's A
// fragments: the C fragments of 8-column tiles 2j and 2j+1 (c0c1 row g, c2c3 row g+8, columns
// 2q, 2q+1) are the A fragment of 16-column k-step j (a0a1, a2a3 from tile 2j; a4a5, a6a7 from
// tile 2j+1), the lower column in the lower half of each register.
__device__ __forceinline__ void gelu_to_a(const float (&acc)[8][4], const float* b, uint32_t (&a)[4][4]) {
  const int q = threadIdx.x & 3;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nt = 2 * j + h;
      const float2 bb = *reinterpret_cast<const float2*>(b + nt * 8 + 2 * q);
      const __nv_bfloat162 lo = __floats2bfloat162_rn(gelu(acc[nt][0] + bb.x), gelu(acc[nt][1] + bb.y));
      const __nv_bfloat162 hi = __floats2bfloat162_rn(gelu(acc[nt][2] + bb.x), gelu(acc[nt][3] + bb.y));
      a[j][2 * h] = *reinterpret_cast<const uint32_t*>(&lo);
      a[j][2 * h + 1] = *reinterpret_cast<const uint32_t*>(&hi);
    }
}

// acc = (16 x 64 hidden tile in A fragments) times W[0..64)[0..64)^T, same k order as warp_gemm
__device__ __forceinline__ void warp_gemm_regs(const uint32_t (&a)[4][4], const __nv_bfloat16* W, float (&acc)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const __nv_bfloat16* w = W + (nt * 8 + g) * LDH + 16 * j + 2 * q;
      mma16816(acc[nt], a[j], *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
    }
}

// Inference forward of the warp's 16 rows (input tile rows m0..m0+15 of s.X) with the hidden
// layers in registers; the same roundings and summation order as warp_forward. y0 and y1 are the
// outputs of rows m0 + g and m0 + g + 8 (g = lane / 4), in every lane of the quad.
template <class S>
__device__ __forceinline__ void warp_forward_regs(const S& s, int m0, float& y0, float& y1) {
  const int q = threadIdx.x & 3;
  float acc[8][4];
  uint32_t a[4][4];
  warp_gemm<kInPad, LDX, LDX>(s.X, s.W1, m0, acc);
  gelu_to_a(acc, s.b1, a);
  warp_gemm_regs(a, s.W2, acc);
  gelu_to_a(acc, s.b2, a);
  warp_gemm_regs(a, s.W3, acc);
  float part[2] = {0.f, 0.f};
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float2 bb = *reinterpret_cast<const float2*>(s.b3 + nt * 8 + 2 * q);
    const float2 ww = *reinterpret_cast<const float2*>(s.w4 + nt * 8 + 2 * q);
    part[0] = fmaf(gelu(acc[nt][0] + bb.x), ww.x, part[0]);
    part[0] = fmaf(gelu(acc[nt][1] + bb.y), ww.y, part[0]);
    part[1] = fmaf(gelu(acc[nt][2] + bb.x), ww.x, part[1]);
    part[1] = fmaf(gelu(acc[nt][3] + bb.y), ww.y, part[1]);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    part[j] += __shfl_xor_sync(0xffffffffu, part[j], 1);
    part[j] += __shfl_xor_sync(0xffffffffu, part[j], 2);
  }
  y0 = part[0] + s.b4;
  y1 = part[1] + s.b4;
}

// Loads kRows feature rows (float32 [n][40], or zeros past n) into the bf16 X tile: four values
// per load when X is 16-byte aligned (rows are 160 bytes), all of a thread's loads issued before
// its stores.
template <class S>
__device__ void load_x(S& s, const float* X, int64_t row0, int64_t n, int rows = kRows) {
  if ((reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
    constexpr int C4 = kInPad / 4, U = 8;
    for (int i0 = threadIdx.x; i0 < rows * C4; i0 += U * blockDim.x) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * blockDim.x, r = i / C4, c4 = i % C4;
        const int64_t gr = row0 + r;
        v[u] = (i < rows * C4 && c4 < kIn / 4 && gr < n) ? __ldg(reinterpret_cast<const float4*>(X + gr * kIn) + c4)
                                                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i >= rows * C4) break;
        __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(s.X + (i / C4) * LDX + (i % C4) * 4);
        d[0] = __floats2bfloat162_rn(v[u].x, v[u].y);
        d[1] = __floats2bfloat162_rn(v[u].z, v[u].w);
      }
    }
    return;
  }
  for (int i = threadIdx.x; i < rows * kInPad; i += blockDim.x) {
    const int r = i / kInPad, c = i % kInPad;
    const int64_t gr = row0 + r;
    const float v = (c < kIn && gr < n) ? X[gr * kIn + c] : 0.f;
    s.X[r * LDX + c] = __float2bfloat16_rn(v);
  }
}

__global__ void __launch_bounds__(kRows * 2) k_mlp_forward(WeightsBF16* w, const float* X, int64_t n, float* y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smem_raw);
  stage_weights(s, *w);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t row0 = (int64_t)blockIdx.x * kRows; row0 < n; row0 += (int64_t)gridDim.x * kRows) {
    load_x(s, X, row0, n);
    cp_async_wait();
    __syncthreads();
    if (warp < kWarps) {
      float y0, y1;
      warp_forward_regs(s, warp * 16, y0, y1);
      const int64_t r0 = row0 + warp * 16 + (lane >> 2);
      if ((lane & 3) == 0) {
        if (r0 < n) y[r0] = y0;
        if (r0 + 8 < n) y[r0 + 8] = y1;
      }
    }
    __syncthreads();
  }
}

// ---- features of interface cells, written as float32 [n_iface][40]; flag[i] = 0 when skipped ---
// The shape features do not change from step to step: k_mlp_static writes, once per mesh, each
// cell's face count / 32 and its six extent features (coordinates relative to the cell's first
// vertex, the leading FP32 parts of the mesh's relative positions): bounding-box extents / V^(1/3)
// and (vertex mean - bounding-box centre) / V^(1/3), a warp per cell. Entry 7 is unused.
__global__ void k_mlp_static(MeshView M, float* S) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); c < M.n_cells; c += warps) {
    const int64_t v0 = M.cell_vert_off[c];
    const int nv = (int)(M.cell_vert_off[c + 1] - v0);
    float mnx = 3.4e38f, mny = 3.4e38f, mnz = 3.4e38f, mxx = -3.4e38f, mxy = -3.4e38f, mxz = -3.4e38f;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int j = lane; j < nv; j += 32) {
      const float2* rp = M.rel_pos + 3 * (v0 + j);
      const float rx = rp[0].x, ry = rp[1].x, rz = rp[2].x;
      mnx = fminf(mnx, rx); mny = fminf(mny, ry); mnz = fminf(mnz, rz);
      mxx = fmaxf(mxx, rx); mxy = fmaxf(mxy, ry); mxz = fmaxf(mxz, rz);
      sx += rx; sy += ry; sz += rz;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
      mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
      mnz = fminf(mnz, __shfl_xor_sync(0xffffffffu, mnz, o));
      mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
      mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
      mxz = fmaxf(mxz, __shfl_xor_sync(0xffffffffu, mxz, o));
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) {
      const float is = 1.0f / cbrtf((float)M.cell_vol[c]);
      float* x = S + 8 * c;
      x[0] = (float)(M.cell_face_off[c + 1] - M.cell_face_off[c]) * (1.0f / 32.0f);
      x[1] = (mxx - mnx) * is;
      x[2] = (mxy - mny) * is;
      x[3] = (mxz - mnz) * is;
      x[4] = (sx / nv - 0.5f * (mnx + mxx)) * is;
      x[5] = (sy / nv - 0.5f * (mny + mxy)) * is;
      x[6] = (sz / nv - 0.5f * (mnz + mxz)) * is;
      x[7] = 0.f;
    }
  }
}

// Per step: a thread per interface cell. Its vertex values' (hi, lo) float pairs (at most 32) are
// held in registers; the range comes from their lexicographic minimum and maximum (the pair of a
// vertex value is monotone in the value, so these are the pairs of the extreme vertices), the
// normalised values are formed in FP32 (no FP64 instruction but alpha's conversion) and sorted
// descending by a bitonic network over the registers: 16 inputs when no cell of the warp has more
// than 16 vertices, else 32. Missing entries take -1 and sort last; the output pads with the
// smallest value. A cell whose range is below 1e-14 (as a float pair difference) gets no features.
template <int NV>
__device__ __forceinline__ void bitonic_desc(float (&u)[NV]) {
#pragma unroll
  for (int k = 2; k <= NV; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const float a = u[i], b = u[l];
          const bool desc = (i & k) == 0;  // this block of the network sorts descending
          u[i] = desc ? fmaxf(a, b) : fminf(a, b);
          u[l] = desc ? fminf(a, b) : fmaxf(a, b);
        }
      }
}

template <int NV>
__device__ __forceinline__ void cell_features(const MeshView& M, const Workspace& W, const float* S, int64_t v0,
                                              int m, int32_t c, float ab, bool live, float* x, int32_t* okp) {
  int32_t vi[NV];
  float2 p[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) vi[k] = k < m ? M.cell_vert[v0 + k] : -1;
#pragma unroll
  for (int k = 0; k < NV; ++k) p[k] = vi[k] >= 0 ? W.phi_ff[vi[k]] : make_float2(0.f, 0.f);
  float2 mn = p[0], mx = p[0];
#pragma unroll
  for (int k = 1; k < NV; ++k)
    if (k < m) {
      if (p[k].x < mn.x || (p[k].x == mn.x && p[k].y < mn.y)) mn = p[k];
      if (p[k].x > mx.x || (p[k].x == mx.x && p[k].y > mx.y)) mx = p[k];
    }
  const ff rg = ff_add(ff{mx.x, mx.y}, ff{-mn.x, -mn.y});
  const float range = rg.hi + rg.lo;
  const bool good = m > 0 && range >= 1e-14f;
  const float irange = 1.0f / range;
  float u[NV];
  float smallest = 3.4e38f;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    u[k] = k < m ? ((p[k].x - mn.x) + (p[k].y - mn.y)) * irange : -1.0f;
    if (k < m) smallest = fminf(smallest, u[k]);
  }
  bitonic_desc<NV>(u);
  if (!live) return;
  *okp = good ? 1 : 0;
  if (!good) return;
  float v[kIn];
  const float4 s0 = *reinterpret_cast<const float4*>(S + 8 * (int64_t)c);
  const float4 s1 = *reinterpret_cast<const float4*>(S + 8 * (int64_t)c + 4);
  v[0] = ab;
  v[1] = s0.x;
#pragma unroll
  for (int k = 0; k < 32; ++k) v[2 + k] = (k < NV && k < m) ? u[k < NV ? k : 0] : smallest;
  v[34] = s0.y; v[35] = s0.z; v[36] = s0.w;
  v[37] = s1.x; v[38] = s1.y; v[39] = s1.z;
  if ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
#pragma unroll
    for (int k = 0; k < kIn; k += 4) *reinterpret_cast<float4*>(x + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = v[k];
  }
}

__global__ void __launch_bounds__(128) k_mlp_features(MeshView M, const double* alpha, Workspace W, const float* S,
                                                      float* X, int32_t* ok) {
  const int64_t n = W.counters->n_iface;
  const int lane = threadIdx.x & 31;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); b < n; b += nthr) {
    const int64_t i = b + lane;
    const bool live = i < n;
    const int32_t c = live ? W.iface_idx[i] : 0;
    const int64_t v0 = M.cell_vert_off[c];
    const int nv = (int)(M.cell_vert_off[c + 1] - v0);
    const int m = live && nv <= 32 ? nv : 0;
    const float ab = live ? (float)alpha[c] : 0.f;
    if (__any_sync(0xffffffffu, m > 16))
      cell_features<32>(M, W, S, v0, m, c, ab, live, X + i * kIn, ok + i);
    else
      cell_features<16>(M, W, S, v0, m, c, ab, live, X + i * kIn, ok + i);
  }
}

// Forward over the interface list (n read on the device): writes the guess of interface cell i,
// clamped to [0, 1], or -1 where the cell has no features. After the block stages the weights,
// each warp runs its own 16-row tiles through the three layers (rows [16 w, 16 w + 16) of the
// block's shared tiles), so no block barrier separates the layers or the tiles, and a few thousand
// interface cells still spread over many SMs (a warp per tile).
__global__ void __launch_bounds__(kRows * 2) k_mlp_forward_iface(WeightsBF16* w, const float* X, const int32_t* ok,
                                                                 Workspace W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int64_t n = W.counters->n_iface;
  const int64_t ntile = (n + 15) / 16;
  if ((int64_t)blockIdx.x * kWarps >= ntile) return;
  stage_weights(s, *w);
  cp_async_wait();
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, m0 = warp * 16;
  constexpr int C4 = kInPad / 4;  // float4 per padded row
  for (int64_t tile = (int64_t)blockIdx.x * kWarps + warp; tile < ntile; tile += (int64_t)gridDim.x * kWarps) {
    const int64_t row0 = tile * 16;
    // the tile's 16 feature rows as bf16 (zeros past n and in the padding); rows are 160 bytes
    // of a 16-byte aligned buffer
    float4 v[16 * C4 / 32];
#pragma unroll
    for (int u = 0; u < 16 * C4 / 32; ++u) {
      const int q = lane + 32 * u, r = q / C4, c4 = q % C4;
      const int64_t gr = row0 + r;
      v[u] = (c4 < kIn / 4 && gr < n) ? __ldg(reinterpret_cast<const float4*>(X + gr * kIn) + c4)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 16 * C4 / 32; ++u) {
      const int q = lane + 32 * u, r = q / C4, c4 = q % C4;
      __nv_bfloat162* d = reinterpret_cast<__nv_bfloat162*>(s.X + (m0 + r) * LDX + c4 * 4);
      d[0] = __floats2bfloat162_rn(v[u].x, v[u].y);
      d[1] = __floats2bfloat162_rn(v[u].z, v[u].w);
    }
    __syncwarp();
    float y0, y1;
    warp_forward_regs(s, m0, y0, y1);
    if ((lane & 3) == 0) {
      const int64_t i0 = row0 + (lane >> 2), i1 = i0 + 8;
      if (i0 < n) W.mlp_out[i0] = ok[i0] ? fminf(fmaxf(y0, 0.f), 1.f) : -1.f;
      if (i1 < n) W.mlp_out[i1] = ok[i1] ? fminf(fmaxf(y1, 0.f), 1.f) : -1.f;
    }
    __syncwarp();  // the tile's X rows are read before the next tile overwrites them
  }
}

// ---- training: forward and backward on the tensor cores, gradient partials per CTA ---------------
// A CTA takes tiles of kRows samples (tiles b, b + gridDim, ...). Forward: warp_forward (four warps,
// 16 rows each) keeps the pre-activations Z (FP32) and the BF16 hidden layers. Backward, layer by
// layer (mma.sync m16n8k16, BF16 operands, FP32 accumulation):
//   dZ3 = dy w4 gelu'(Z3);   dW3 += dZ3^T H2;   dH2 = dZ3 W3;   dZ2 = dH2 gelu'(Z2);
//   dW2 += dZ2^T H1;         dH1 = dZ2 W2;      dZ1 = dH1 gelu'(Z1);   dW1 += dZ1^T X.
// dZ is rounded to BF16 for the products (kept in [row][unit] and transposed layouts); the bias
// gradients sum the FP32 dZ. Each warp keeps its 16 x 32 (dW1: 16 x 24) block of every weight
// gradient in its accumulator registers across the CTA's tiles, and threads 0..64 keep the bias,
// w4 and b4 sums, so a CTA writes one gradient partial, summed in tile order (deterministic).
constexpr int LDR = kRows + 8;  // bf16 stride of the transposed tiles [unit][row]

struct TrainSmem {
  Smem f;
  __nv_bfloat16 W2T[kH * LDH], W3T[kH * LDH];  // transposed weights [in][out]
  float Z1[kRows * kH], Z2[kRows * kH], Z3[kRows * kH];  // pre-activations, then that layer's FP32 dZ
  float H3[kRows * kH];
  __nv_bfloat16 dZ[kRows * LDH];   // the current layer's dZ [row][unit], BF16
  __nv_bfloat16 dZT[kH * LDR];     // its transpose [unit][row]
  __nv_bfloat16 AT[kH * LDR];      // the layer's input transposed [in][row] (H2, H1 or X)
  float dy[kRows];
};

// acc[j] += A[m0 .. m0 + 16)[0 .. K) * B[n0 + 8 j .. n0 + 8 j + 8)[0 .. K)^T for j < NT; A and B
// row-major BF16 with strides LDA and LDB (the fragment layouts of warp_gemm)
template <int K, int NT, int LDA, int LDB>
__device__ __forceinline__ void warp_mma(const __nv_bfloat16* A, const __nv_bfloat16* B, int m0, int n0,
                                         float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(A + (m0 + g) * LDA + k0 + 2 * q);
    a[1] = *reinterpret_cast<const uint32_t*>(A + (m0 + g + 8) * LDA + k0 + 2 * q);
    a[2] = *reinterpret_cast<const uint32_t*>(A + (m0 + g) * LDA + k0 + 8 + 2 * q);
    a[3] = *reinterpret_cast<const uint32_t*>(A + (m0 + g + 8) * LDA + k0 + 8 + 2 * q);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const __nv_bfloat16* w = B + (n0 + 8 * j + g) * LDB + k0 + 2 * q;
      mma16816(acc[j], a, *reinterpret_cast<const uint32_t*>(w), *reinterpret_cast<const uint32_t*>(w + 8));
    }
  }
}

// dZ of a hidden layer from this warp's block of dH (rows m0.., units n0..n0 + 32): the FP32 value
// into Zf (in place of the pre-activation), BF16 copies into dZ [row][unit] and dZT [unit][row]
__device__ __forceinline__ void store_dz(const float (&dh)[4][4], float* Zf, __nv_bfloat16* dZ, __nv_bfloat16* dZT,
                                         int m0, int n0) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + g + (i >= 2 ? 8 : 0), c = n0 + 8 * j + 2 * q + (i & 1);
      const float d = dh[j][i] * gelu_grad(Zf[r * kH + c]);
      Zf[r * kH + c] = d;
      const __nv_bfloat16 b = __float2bfloat16_rn(d);
      dZ[r * LDH + c] = b;
      dZT[c * LDR + r] = b;
    }
}

__global__ void __launch_bounds__(256) k_mlp_train(WeightsBF16* w, const float* X, const float* t, int64_t n,
                                                  float inv_batch, float* part, float* loss_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int64_t ntiles = (n + kRows - 1) / kRows;
  stage_weights(s.f, *w);
  cp_async_wait();
  __syncthreads();
  for (int i = tid; i < kH * kH; i += blockDim.x) {  // transposed weights, once per CTA
    const int o = i / kH, k = i % kH;
    s.W2T[k * LDH + o] = s.f.W2[o * LDH + k];
    s.W3T[k * LDH + o] = s.f.W3[o * LDH + k];
  }
  // this warp's blocks of the weight gradients (rows = units m0.., columns = inputs n0.. / n1..)
  const int m0 = (warp >> 1) * 16, n0 = (warp & 1) * 32, n1 = (warp & 1) * 24;
  float g3[4][4], g2[4][4], g1[3][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) g3[j][i] = g2[j][i] = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) g1[j][i] = 0.f;
  // thread u < kH: sums of unit u's bias gradients (layers 3, 2, 1) and of w4[u]; thread kH: b4;
  // thread 0: the loss
  float sb3 = 0.f, sb2 = 0.f, sb1 = 0.f, sw4 = 0.f, sb4 = 0.f, sloss = 0.f;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * kRows;
    load_x(s.f, X, row0, n);
    __syncthreads();
    if (warp < kWarps) warp_forward(s.f, warp * 16, s.Z1, s.Z2, s.Z3, s.H3);
    __syncthreads();
    if (tid < kRows) {
      const int64_t gr = row0 + tid;
      const float r = gr < n ? s.f.y[tid] - t[gr] : 0.f;  // padded rows carry no gradient
      s.dy[tid] = 2.f * r * inv_batch;
      s.f.y[tid] = r * r;
    }
    __syncthreads();
    if (tid == 0) {
      float l = 0.f;
      for (int r = 0; r < kRows; ++r) l += s.f.y[r];
      sloss += l;
    }
    if (tid < kH) {
      float a = 0.f;
      for (int r = 0; r < kRows; ++r) a = fmaf(s.H3[r * kH + tid], s.dy[r], a);
      sw4 += a;
    } else if (tid == kH) {
      float a = 0.f;
      for (int r = 0; r < kRows; ++r) a += s.dy[r];
      sb4 += a;
    }
    // dZ3 = dy w4 gelu'(Z3); the input of layer 3 (H2) transposed
    for (int i = tid; i < kRows * kH; i += blockDim.x) {
      const int r = i / kH, c = i % kH;
      const float d = s.dy[r] * s.f.w4[c] * gelu_grad(s.Z3[i]);
      s.Z3[i] = d;
      const __nv_bfloat16 b = __float2bfloat16_rn(d);
      s.dZ[r * LDH + c] = b;
      s.dZT[c * LDR + r] = b;
      s.AT[c * LDR + r] = s.f.H2[r * LDH + c];
    }
    __syncthreads();
    if (tid < kH) {
      float a = 0.f;
      for (int r = 0; r < kRows; ++r) a += s.Z3[r * kH + tid];
      sb3 += a;
    }
    warp_mma<kRows, 4, LDR, LDR>(s.dZT, s.AT, m0, n0, g3);  // dW3 += dZ3^T H2
    float dh[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) dh[j][i] = 0.f;
    warp_mma<kH, 4, LDH, LDH>(s.dZ, s.W3T, m0, n0, dh);  // dH2 = dZ3 W3 (rows m0.., inputs n0..)
    __syncthreads();
    store_dz(dh, s.Z2, s.dZ, s.dZT, m0, n0);  // dZ2 = dH2 gelu'(Z2)
    for (int i = tid; i < kRows * kH; i += blockDim.x) {
      const int r = i / kH, c = i % kH;
      s.AT[c * LDR + r] = s.f.H1[r * LDH + c];
    }
    __syncthreads();
    if (tid < kH) {
      float a = 0.f;
      for (int r = 0; r < kRows; ++r) a += s.Z2[r * kH + tid];
      sb2 += a;
    }
    warp_mma<kRows, 4, LDR, LDR>(s.dZT, s.AT, m0, n0, g2);  // dW2 += dZ2^T H1
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) dh[j][i] = 0.f;
    warp_mma<kH, 4, LDH, LDH>(s.dZ, s.W2T, m0, n0, dh);  // dH1 = dZ2 W2
    __syncthreads();
    store_dz(dh, s.Z1, s.dZ, s.dZT, m0, n0);  // dZ1 = dH1 gelu'(Z1)
    for (int i = tid; i < kRows * kInPad; i += blockDim.x) {
      const int r = i / kInPad, c = i % kInPad;
      s.AT[c * LDR + r] = s.f.X[r * LDX + c];
    }
    __syncthreads();
    if (tid < kH) {
      float a = 0.f;
      for (int r = 0; r < kRows; ++r) a += s.Z1[r * kH + tid];
      sb1 += a;
    }
    warp_mma<kRows, 3, LDR, LDR>(s.dZT, s.AT, m0, n1, g1);  // dW1 += dZ1^T X (inputs padded to 48)
    __syncthreads();  // the next tile overwrites the tiles read above
  }
  // this CTA's partial
  float* P = part + (size_t)blockIdx.x * kNP;
  const int lane = tid & 31, g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + g + (i >= 2 ? 8 : 0), c = n0 + 8 * j + 2 * q + (i & 1);
      P[oW3 + r * kH + c] = g3[j][i];
      P[oW2 + r * kH + c] = g2[j][i];
    }
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = m0 + g + (i >= 2 ? 8 : 0), c = n1 + 8 * j + 2 * q + (i & 1);
      if (c < kIn) P[oW1 + r * kIn + c] = g1[j][i];
    }
  if (tid < kH) {
    P[ob3 + tid] = sb3;
    P[ob2 + tid] = sb2;
    P[ob1 + tid] = sb1;
    P[ow4 + tid] = sw4;
  } else if (tid == kH) {
    P[ob4] = sb4;
  }
  if (tid == 0) loss_part[blockIdx.x] = sloss;
}

// BF16 copy of parameter p (index into the vector) written into the kernel layout.
__device__ void to_bf16(WeightsBF16* w, int p, float v) {
  if (p < ob1) w->W1[p / kIn][p % kIn] = __float2bfloat16_rn(v);
  else if (p < oW2) w->b1[p - ob1] = v;
  else if (p < ob2) w->W2[(p - oW2) / kH][(p - oW2) % kH] = __float2bfloat16_rn(v);
  else if (p < oW3) w->b2[p - ob2] = v;
  else if (p < ob3) w->W3[(p - oW3) / kH][(p - oW3) % kH] = __float2bfloat16_rn(v);
  else if (p < ow4) w->b3[p - ob3] = v;
  else if (p < ob4) w->w4[p - ow4] = bf16r(v);
  else w->b4 = v;
}

__global__ void k_mlp_set_bf16(const float* params, WeightsBF16* w) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kNP; p += gridDim.x * blockDim.x) to_bf16(w, p, params[p]);
  // zero padding of W1 (inputs 40..47)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kH * (kInPad - kIn); i += gridDim.x * blockDim.x)
    w->W1[i / (kInPad - kIn)][kIn + i % (kInPad - kIn)] = __float2bfloat16_rn(0.f);
}

// Sums the tile partials in tile order (deterministic); grad_out gets the gradient, and with
// lr > 0 an Adam step updates the FP32 master parameters and their BF16 copy.
__global__ void k_mlp_reduce_adam(const float* part, int ntiles, const float* loss_part, float* params, float* m1,
                                  float* m2, WeightsBF16* w, float lr, float b1t, float b2t, int64_t n, float* grad_out,
                                  float* loss_out) {
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kNP; p += gridDim.x * blockDim.x) {
    float g = 0;
    for (int tl = 0; tl < ntiles; ++tl) g += part[(size_t)tl * kNP + p];
    if (grad_out) grad_out[p] = g;
    if (lr > 0) {
      const float a = beta1 * m1[p] + (1 - beta1) * g;
      const float b = beta2 * m2[p] + (1 - beta2) * g * g;
      m1[p] = a;
      m2[p] = b;
      const float v = params[p] - lr * (a / (1 - b1t)) / (sqrtf(b / (1 - b2t)) + eps);
      params[p] = v;
      to_bf16(w, p, v);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss_out) {
    float l = 0;
    for (int tl = 0; tl < ntiles; ++tl) l += loss_part[tl];
    *loss_out = l / (float)n;
  }
}

}  // namespace

}  // namespace vof

struct vof_mlp {
  float *params = nullptr, *m1 = nullptr, *m2 = nullptr, *part = nullptr, *loss_part = nullptr, *y = nullptr;
  vof::WeightsBF16* w = nullptr;
  int64_t adam_t = 0;
  int64_t y_cap = 0;
};

namespace vof {

cudaError_t launch_mlp_guess(vof_mesh* m, cudaStream_t s) {
  vof_mlp* mlp = (vof_mlp*)m->mlp;
  float* X = m->ws.mlp_x;
  int32_t* ok = m->ws.mlp_ok;
  m->timing.start(KC_MLP_FEATURES, s);
  k_mlp_features<<<m->num_sms * 8, 128, 0, s>>>(m->view, m->ws.alpha_in, m->ws, m->ws.mlp_static, X, ok);
  m->timing.stop(s);
  const size_t fwd_smem = sizeof(FwdSmem);
  static int fwd_bps = 0;  // resident blocks per SM of the forward pass
  if (!fwd_bps) {
    cudaFuncSetAttribute(k_mlp_forward_iface, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fwd_bps, k_mlp_forward_iface, kRows * 2, fwd_smem);
    if (fwd_bps < 1) fwd_bps = 1;
  }
  m->timing.start(KC_MLP_FORWARD, s);
  k_mlp_forward_iface<<<m->num_sms * fwd_bps, kRows * 2, fwd_smem, s>>>(mlp->w, X, ok, m->ws);
  m->timing.stop(s);
  return cudaGetLastError();
}

}  // namespace vof

using namespace vof;

extern "C" {

vof_status vof_mlp_create(const float* h_params, vof_mlp** out) {
  if (!h_params || !out) { set_error("null argument"); return VOF_EINVAL; }
  *out = nullptr;
  for (int p = 0; p < kNP; ++p)
    if (!std::isfinite(h_params[p])) { set_error("non-finite MLP parameter"); return VOF_EINVAL; }
  vof_mlp* m = new (std::nothrow) vof_mlp;
  if (!m) { set_error("host allocation failed"); return VOF_ENOMEM; }
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&m->params, kNP * sizeof(float));
  e = e ? e : cudaMalloc(&m->m1, kNP * sizeof(float));
  e = e ? e : cudaMalloc(&m->m2, kNP * sizeof(float));
  e = e ? e : cudaMalloc(&m->part, (size_t)kMaxTiles * kNP * sizeof(float));
  e = e ? e : cudaMalloc(&m->loss_part, kMaxTiles * sizeof(float));
  e = e ? e : cudaMalloc(&m->w, sizeof(WeightsBF16));
  e = e ? e : cudaMemcpy(m->params, h_params, kNP * sizeof(float), cudaMemcpyHostToDevice);
  e = e ? e : cudaMemset(m->m1, 0, kNP * sizeof(float));
  e = e ? e : cudaMemset(m->m2, 0, kNP * sizeof(float));
  if (e == cudaSuccess) {
    k_mlp_set_bf16<<<(kNP + 255) / 256, 256>>>(m->params, m->w);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    cudaFree(m->params); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->part); cudaFree(m->loss_part); cudaFree(m->w);
    delete m;
    return cuda_fail(e, "vof_mlp_create");
  }
  *out = m;
  return VOF_OK;
}

vof_status vof_mlp_destroy(vof_mlp* m) {
  if (!m) return VOF_EINVAL;
  cudaFree(m->params); cudaFree(m->m1); cudaFree(m->m2); cudaFree(m->part); cudaFree(m->loss_part); cudaFree(m->w);
  delete m;
  return VOF_OK;
}

vof_status vof_mlp_get_params(vof_mlp* m, float* h_params) {
  if (!m || !h_params) { set_error("null argument"); return VOF_EINVAL; }
  cudaError_t e = cudaMemcpy(h_params, m->params, kNP * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "vof_mlp_get_params");
  return VOF_OK;
}

vof_status vof_mlp_forward(vof_mlp* m, const float* d_X, int64_t n, float* d_y, void* stream) {
  if (!m || (n > 0 && (!d_X || !d_y)) || n < 0) { set_error("bad argument"); return VOF_EINVAL; }
  if (n == 0) return VOF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(FwdSmem));
  const int grid = (int)std::min<int64_t>((n + kRows - 1) / kRows, 1024);
  k_mlp_forward<<<grid, kRows * 2, sizeof(FwdSmem), s>>>(m->w, d_X, n, d_y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "vof_mlp_forward");
  return VOF_OK;
}

static vof_status train_impl(vof_mlp* m, const float* d_X, const float* d_t, int64_t n, float lr, float* d_grad,
                             float* d_loss, cudaStream_t s) {
  if (!m || !d_X || !d_t || n < 1 || n > kMaxBatch || !(lr >= 0)) { set_error("bad argument"); return VOF_EINVAL; }
  const int ntiles = (int)((n + kRows - 1) / kRows);
  static int train_grid = 0;  // a CTA per SM at most (one partial each)
  if (!train_grid) {
    cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(TrainSmem));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&train_grid, cudaDevAttrMultiProcessorCount, dev);
    if (train_grid < 1) train_grid = 1;
  }
  const int nparts = std::min(ntiles, train_grid);
  k_mlp_train<<<nparts, 256, sizeof(TrainSmem), s>>>(m->w, d_X, d_t, n, 1.0f / (float)n, m->part, m->loss_part);
  float b1t = 1, b2t = 1;
  if (lr > 0) {
    m->adam_t += 1;
    b1t = (float)std::pow(0.9, (double)m->adam_t);
    b2t = (float)std::pow(0.999, (double)m->adam_t);
  }
  k_mlp_reduce_adam<<<(kNP + 255) / 256, 256, 0, s>>>(m->part, nparts, m->loss_part, m->params, m->m1, m->m2, m->w, lr,
                                                      b1t, b2t, n, d_grad, d_loss);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mlp training kernels");
  return VOF_OK;
}

vof_status vof_mlp_train_step(vof_mlp* m, const float* d_X, const float* d_t, int64_t n, float lr, float* d_loss,
                              void* stream) {
  if (!(lr > 0)) { set_error("learning rate must be positive"); return VOF_EINVAL; }
  return train_impl(m, d_X, d_t, n, lr, nullptr, d_loss, (cudaStream_t)stream);
}

vof_status vof_mlp_grad(vof_mlp* m, const float* d_X, const float* d_t, int64_t n, float* d_grad, float* d_loss,
                        void* stream) {
  if (!d_grad) { set_error("null gradient buffer"); return VOF_EINVAL; }
  return train_impl(m, d_X, d_t, n, 0.0f, d_grad, d_loss, (cudaStream_t)stream);
}

vof_status vof_mesh_set_mlp(vof_mesh* mesh, vof_mlp* mlp) {
  if (!mesh) { set_error("null mesh"); return VOF_EINVAL; }
  Workspace& W = mesh->ws;
  if (mlp && !W.mlp_x) {
    const size_t nc = (size_t)mesh->n_cells;
    cudaError_t e = cudaMalloc(&W.mlp_x, nc * kIn * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&W.mlp_ok, nc * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&W.mlp_y, nc * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "vof_mesh_set_mlp");
    mesh->allocs.push_back(W.mlp_x);
    mesh->allocs.push_back(W.mlp_ok);
    mesh->allocs.push_back(W.mlp_y);
  }
  if (mlp && !W.mlp_static) {
    // the features that depend on the mesh alone, once
    cudaError_t e = cudaMalloc(&W.mlp_static, (size_t)mesh->n_cells * 8 * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "vof_mesh_set_mlp");
    mesh->allocs.push_back(W.mlp_static);
    k_mlp_static<<<mesh->num_sms * 8, 256>>>(mesh->view, W.mlp_static);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "vof_mesh_set_mlp (static features)");
  }
  // a captured step graph bakes in the weights' device address: recapture after any change (a
  // new MLP may even reuse the old handle's host address)
  if (mesh->mlp != mlp) {
    mesh->graph.key.clear();
    mesh->host_graph.key.clear();
  }
  mesh->mlp = mlp;
  return VOF_OK;
}

vof_status vof_mlp_features(vof_mesh* m, const double* d_alpha, float* d_X, int32_t* d_ok, void* stream) {
  if (!m || !d_alpha || !d_X || !d_ok) { set_error("null argument"); return VOF_EINVAL; }
  if (!m->recon_done) { set_error("vof_mlp_features needs a reconstruction"); return VOF_ESTATE; }
  if (!m->ws.mlp_static) {  // the mesh-only features, once (also without an MLP attached)
    cudaError_t e = cudaMalloc(&m->ws.mlp_static, (size_t)m->n_cells * 8 * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "vof_mlp_features");
    m->allocs.push_back(m->ws.mlp_static);
    k_mlp_static<<<m->num_sms * 8, 256, 0, (cudaStream_t)stream>>>(m->view, m->ws.mlp_static);
  }
  k_mlp_features<<<m->num_sms * 8, 128, 0, (cudaStream_t)stream>>>(m->view, d_alpha, m->ws, m->ws.mlp_static, d_X,
                                                                  d_ok);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "vof_mlp_features");
  return VOF_OK;
}

}  // extern "C"

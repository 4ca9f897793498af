// Totals without device allocation.
//
// Some callers cannot allocate device memory at the point where they need the totals: code that
// runs while its stream is being captured into a CUDA graph, real-time loops that must never enter
// an allocator, or host programs that hand out all device memory through their own pool. For them
// this file gives vof_totals_static: the same two pairwise-tree sums that vof_phase_change_source
// writes to d_totals, over caller-supplied per-cell products, with the chunk sums kept in a
// file-scope device array instead of a mesh workspace.
//
// The array lives in every GPU that loads the library until the process exits. In host code its
// name only stands in for the symbol; the kernel gets its device address, looked up once per
// device with cudaGetSymbolAddress (on the first call made with that device current).
#include <mutex>

#include "vof_internal.cuh"

namespace {

constexpr int kChunk = 2048;                                        // leaves per block (power of two)
constexpr int kMaxChunks = 2048;                                    // chunk sums per total
constexpr long long kMaxN = (long long)kChunk * kMaxChunks;         // = VOF_TOTALS_STATIC_MAX_N
static_assert(kMaxN == VOF_TOTALS_STATIC_MAX_N, "limit");

// [0, kMaxChunks) chunk sums of the first total, [kMaxChunks, 2 kMaxChunks) of the second,
// then one 8-byte slot for the count of finished blocks (zeroed before every launch).
static __device__ __align__(256) double g_static_scratch[2 * kMaxChunks + 1];

// Pairwise tree over kChunk leaves x[base .. base + kChunk), zeros past n.
__device__ double tree_chunk(const double* x, long long n, long long base, double* s) {
  const int t = threadIdx.x;  // blockDim.x == kChunk / 2
  const long long i0 = base + 2 * t, i1 = i0 + 1;
  s[t] = (i0 < n ? __ldcg(x + i0) : 0.0) + (i1 < n ? __ldcg(x + i1) : 0.0);
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

__global__ void __launch_bounds__(kChunk / 2)
    k_totals_static(const double* a, const double* b, long long n, double* totals, double* scratch) {
  __shared__ double s[kChunk / 2];
  __shared__ bool last;
  unsigned int* done = reinterpret_cast<unsigned int*>(scratch + 2 * kMaxChunks);
  const long long nchunks = (n + kChunk - 1) / kChunk;
  for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const double sa = tree_chunk(a, n, c * kChunk, s);
    const double sb = tree_chunk(b, n, c * kChunk, s);
    if (threadIdx.x == 0) {
      scratch[c] = sa;
      scratch[kMaxChunks + c] = sb;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the chunk sums are the nodes of the same tree kChunk leaves up; nchunks <= kChunk
  const double ta = nchunks ? tree_chunk(scratch, nchunks, 0, s) : 0.0;
  const double tb = nchunks ? tree_chunk(scratch + kMaxChunks, nchunks, 0, s) : 0.0;
  if (threadIdx.x == 0) {
    totals[0] = ta;
    totals[1] = tb;
  }
}

std::mutex g_mu;
double* g_addr[64] = {nullptr};  // device address of g_static_scratch, per device ordinal

}  // namespace

using namespace vof;

extern "C" vof_status vof_totals_static(const double* d_a, const double* d_b, int64_t n, double* d_totals,
                                        void* stream) {
  if (n < 0 || (n > 0 && (!d_a || !d_b)) || !d_totals) { set_error("bad argument"); return VOF_EINVAL; }
  if (n > kMaxN) {
    set_error("vof_totals_static: n exceeds VOF_TOTALS_STATIC_MAX_N (4194304); use vof_phase_change_source");
    return VOF_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) { set_error("device ordinal out of range"); return VOF_EINVAL; }
  double* scratch;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
      g_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the finished-block count must start at zero; the chunk sums are overwritten before use
  e = cudaMemsetAsync(scratch + 2 * kMaxChunks, 0, sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const long long nchunks = (n + kChunk - 1) / kChunk;
  const int grid = (int)(nchunks < 1 ? 1 : (nchunks < 64 ? nchunks : 64));
  k_totals_static<<<grid, kChunk / 2, 0, s>>>(d_a, d_b, (long long)n, d_totals, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k_totals_static");
  return VOF_OK;
}

// FP64 FMA throughput probe: the denominator of the roofline of the FP64-bound kernels
// (measurement support; the paper has no counterpart). Every thread runs kChains independent
// chains x <- fma(x, a, b), so that the FP64 unit never waits on a result; the grid fills every SM
// to full occupancy. flops = 2 x chains x iterations x threads.
#include <cuda_runtime.h>

#include <algorithm>

#include "vof_internal.cuh"

namespace vof {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(int64_t iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace
}  // namespace vof

using namespace vof;

extern "C" vof_status vof_probe_fp64_fma(int64_t iters, int reps, double* h_ms, double* h_flops, void* stream) {
  if (iters < 1 || reps < 1 || !h_ms || !h_flops) {
    set_error("bad argument");
    return VOF_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, bps = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_fp64_fma_probe, kProbeThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "vof_probe_fp64_fma");
  const int grid = sms * std::max(1, bps);
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, (size_t)grid * kProbeThreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0;
  // one untimed launch (clocks up, module loaded), then the best of reps timed launches
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    k_fp64_fma_probe<<<grid, kProbeThreads, 0, s>>>(iters, 1.0 - 1e-12, 1e-9, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r >= 0 && (best == 0 || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "vof_probe_fp64_fma");
  *h_ms = best;
  *h_flops = 2.0 * kChains * (double)iters * (double)grid * kProbeThreads;
  return VOF_OK;
}

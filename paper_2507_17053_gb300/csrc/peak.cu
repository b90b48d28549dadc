// Arithmetic-throughput probe (a measurement aid; the paper has no
// counterpart): the FP64 and FP32 fused multiply-add rates of the current
// GPU, the denominators of the cell kernels' roofline.
//
// Every thread runs kChains independent chains v <- v * a + b (fma.rn), so
// the pipe never waits on a dependency; the grid fills every SM with 8
// blocks of 256 threads; the chains' sum is stored so nothing is optimised
// away.  Rate = executed FMAs / kernel time (CUDA events, best of several
// launches after a warm-up).
#include <algorithm>

#include "internal.hpp"

namespace sbm {
namespace {

constexpr int kChains = 8;
constexpr int kThreadsPerBlock = 256;
constexpr int kBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kThreadsPerBlock)
fma_probe_kernel(T* __restrict__ out, int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) v[i] = T(threadIdx.x) * T(1e-3) + T(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = fma(v[i], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += v[i];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t probe(int iters, double* gfma, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = sms * kBlocksPerSm;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc((void**)&out, (size_t)grid * kThreadsPerBlock * sizeof(T));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      fma_probe_kernel<T><<<grid, kThreadsPerBlock, 0, st>>>(out, iters, T(0.9999), T(1e-4));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e == cudaSuccess)
    *gfma = (double)grid * kThreadsPerBlock * kChains * (double)iters / (best * 1e-3) / 1e9;
  return e;
}

}  // namespace
}  // namespace sbm

using namespace sbm;

extern "C" int sbm_peak_probe(int precision, double* gfma_per_s, void* stream) {
  if (!gfma_per_s || (precision != 32 && precision != 64))
    return sbm_fail_detail(SBM_ERR_ARG, "precision must be 32 or 64, output non-NULL");
  const cudaError_t e = precision == 64 ? probe<double>(1 << 12, gfma_per_s, (cudaStream_t)stream)
                                        : probe<float>(1 << 15, gfma_per_s, (cudaStream_t)stream);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "sbm_peak_probe");
  return SBM_OK;
}

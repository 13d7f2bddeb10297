// Measured arithmetic peaks of the device (the denominators of the ALU rooflines): dependent
// FMA chains, kChains independent ones per thread so that the pipes stay full, over a grid of
// 8 CTAs of 256 threads per SM.  The result is the best of a few timed launches.
#include <algorithm>

#include "kernels.h"

namespace wmg {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x + i);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(-1.2345)) out[0] = s;  // keeps the chains alive; never true for these inputs
}

template <typename T>
double fma_peak_tflops(int iters) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return 0.0;
  const int grid = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    k_fma_peak<T><<<grid, threads>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * (double)iters * grid * threads;
    if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return best;
}

}  // namespace
}  // namespace wmg

extern "C" wmg_status wmg_probe_alu_peaks(double* fp32_tflops, double* fp64_tflops) {
  if (!fp32_tflops || !fp64_tflops) return WMG_EINVAL;
  wmg::count_launch(8);
  *fp32_tflops = wmg::fma_peak_tflops<float>(1 << 14);
  *fp64_tflops = wmg::fma_peak_tflops<double>(1 << 10);
  return cudaGetLastError() == cudaSuccess ? WMG_OK : WMG_ECUDA;
}

// kf_peak.cu -- measured arithmetic peaks of the device: the rates of FP32 and
// FP64 fused multiply-adds that serve as the roofline denominators of the
// kernels bound by arithmetic (the fused fit, the build steps).  The paper has
// no counterpart; it measures on CPUs.
//
// Each thread runs CHAINS independent chains acc = acc * m + a (a contraction
// towards a / (1 - m), so values stay normal and finite), enough independent
// work per warp to keep the FMA pipe issuing every cycle at full occupancy.
// The result is stored only under a condition the values never meet, which
// keeps the chains live without memory traffic.
#include <algorithm>

#include "kf_internal.h"

namespace kfi {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;  // 2048 resident threads per SM

// target of the store that never happens (a valid address all the same)
__device__ double g_peak_sink[kPeakThreads];

template <typename T, int CHAINS>
__global__ void __launch_bounds__(kPeakThreads, kPeakBlocksPerSM) peak_fma_kernel(int iters) {
  T acc[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc[c] = T(threadIdx.x + c) * T(1e-3);
  const T m = T(0.999), a = T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], m, a);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += acc[c];
  if (s == T(-1.0)) g_peak_sink[threadIdx.x] = double(s);  // never true: the chains stay positive
}

template <typename T, int CHAINS>
int time_peak(kf_ctx* ctx, int iters, cudaStream_t st, double* flop_per_s) {
  const int grid = ctx->num_sms * kPeakBlocksPerSM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KF_CUDA_TRY(ctx, cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, err);
  }
  double best = 0.0;
  for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {  // one warm-up launch, then the best of three
    err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) {
      peak_fma_kernel<T, CHAINS><<<grid, kPeakThreads, 0, st>>>(iters);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && ms > 0.f) {
      const double flop = 2.0 * double(grid) * kPeakThreads * double(iters) * CHAINS;
      best = std::max(best, flop / (double(ms) * 1e-3));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(ctx, err);
  *flop_per_s = best;
  return KF_OK;
}

}  // namespace
}  // namespace kfi

extern "C" int kf_measure_peak(kf_ctx* ctx, int32_t kind, void* stream, double* flop_per_s) {
  if (!ctx || !flop_per_s || (kind != KF_PEAK_FP32 && kind != KF_PEAK_FP64)) return KF_EINVAL;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // about 10 ms a launch at the nominal rates (FP32 ~80, FP64 ~1.2 TFLOP/s)
  if (kind == KF_PEAK_FP32) return kfi::time_peak<float, 16>(ctx, 80000, st, flop_per_s);
  return kfi::time_peak<double, 8>(ctx, 2500, st, flop_per_s);
}

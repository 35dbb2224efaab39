// kf_fit.cu -- track-fit kernels: one thread per track, state and covariance
// in registers, structure-of-arrays global layout (coalesced 128-byte warp
// transactions per component).
//
// Track fitting is the branch-free part of Kalman-filter tracking (Cerati et
// al., Sec. 2): with the hit set fixed, every track runs propagate + update
// over the layers.  Forms:
//   fit_layer_kernel  one layer step over the whole batch (kf_fit replays one
//                     launch per layer from a captured CUDA graph);
//   fit_fused_kernel  all layers in one launch, the track held in registers
//                     (also the mixed-precision form);
//   fit_f64_kernel    the plain FP64 form, launched per event and per layer.
// One track per thread, 24 resident warps per SM, plain coalesced row reads.
// Staging the rows in shared memory (bulk copies per block or per warp, or
// per-thread cp.async double buffering) measured no faster.
#include "kf_internal.h"
#include "kf_math.cuh"

namespace kfi {

constexpr int kFitThreads = 128;
constexpr int kFitMinBlocks = 5;  // fused fit: 20 resident warps per SM (96 registers)
// The layer kernel moves 261 B per track: at 20 resident warps per SM the
// loads a warp issues at the start of its tracks do not keep enough bytes in
// flight to reach the HBM rate (a pure copy with this access pattern takes
// 181 us per 4M tracks at 20 warps, 150 us at full occupancy).  24 warps
// (80 registers, no spills) measured best; 32 warps spill.
constexpr int kFitWarpsPerSM = 24;
constexpr int kNewtonF32 = 12;  // iteration cap of the safeguarded Newton solve
constexpr int kNewtonF64 = 16;

// Positive-definiteness of the rank-5 covariance: Cholesky of P C P^T where P
// maps to (t . pos, z, px, py, pz), t the transverse tangent of the cylinder
// at the track position (the radial direction is exactly singular after a
// surface propagation).
template <typename T>
__device__ __forceinline__ bool pd5(const T p[6], const T C[21]) {
  using kf::sym;
  const T r = kf::sqrt_t(p[0] * p[0] + p[1] * p[1]);
  const T t0 = r > T(0) ? -p[1] / r : T(0), t1 = r > T(0) ? p[0] / r : T(1);
  T M[5][5];
  M[0][0] = t0 * t0 * C[sym(0, 0)] + T(2) * t0 * t1 * C[sym(1, 0)] + t1 * t1 * C[sym(1, 1)];
#pragma unroll
  for (int j = 1; j < 5; ++j) {
    const int cj = j + 1;  // z, px, py, pz
    M[j][0] = t0 * C[sym(0, cj)] + t1 * C[sym(1, cj)];
#pragma unroll
    for (int k = 1; k <= j; ++k) M[j][k] = C[sym(cj, k + 1)];
  }
  T L[5][5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    T d = M[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > T(0))) return false;
    L[j][j] = kf::sqrt_t(d);
    const T inv = T(1) / L[j][j];
#pragma unroll
    for (int i = j + 1; i < 5; ++i) {
      T v = M[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v * inv;
    }
  }
  return true;
}

// One propagate + (optional) update step of one track.  Returns the status
// bits raised; writes chi2 (-1 when no update).  UPD64: S^-1 and the
// covariance downdate in FP64 (single-precision state only).
template <typename T, int NEWTON, bool EXT, bool UPD64 = false>
__device__ __forceinline__ int32_t track_step(T p[6], T lo[3], T C[21], T a, T R, T x_x0, T mass, bool has_hit,
                                              T m0, T m1, T m2, T v0, T v1, T v2, T& chi2) {
  chi2 = T(-1);
  const int st = kf::propagate<T, NEWTON, EXT>(p, lo, C, a, R);
  if (st) return st;
  if (x_x0 > T(0)) kf::scatter(p, lo, C, x_x0, mass);
  if (!has_hit) return kf::ST_NO_HIT;
  T r0, r1, r2;
  kf::residual<T, EXT>(p, lo, m0, m1, m2, r0, r1, r2);
  if constexpr (UPD64) {
    chi2 = kf::kalman_update_f64(p, lo, C, r0, r1, r2, v0, v1, v2);
  } else {
    T Si[6];
    kf::inverse_S(C, v0, v1, v2, Si);
    chi2 = kf::chi2_of(r0, r1, r2, Si);
    kf::kalman_update<T, EXT>(p, lo, C, Si, r0, r1, r2, v0, v1, v2);
  }
  return 0;
}

// The step of track i given its inputs; writes its outputs.
__device__ __forceinline__ void fit_layer_track(const FitLayerArgs& A, int64_t i, int32_t st, float p[6], float lo[3],
                                                float C[21], int8_t q, bool has_hit, float m0, float m1, float m2) {
  const int64_t n = A.n;
  if (st & KF_ST_STOPPED) {  // stopped at an earlier layer: nothing to do
    if (A.chi2) A.chi2[i] = -1.f;
    return;
  }
  const float a = A.a_scale * float(q);
  float chi2;
  const int32_t raised =
      track_step<float, kNewtonF32, true>(p, lo, C, a, A.R, A.x_x0, A.mass, has_hit, m0, m1, m2, A.v0, A.v1, A.v2,
                                          chi2);
  const bool stopped = (raised & KF_ST_STOPPED) != 0;
  if (!stopped || A.first) {
#pragma unroll
    for (int c = 0; c < 6; ++c) A.out_par[c * n + i] = p[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) A.out_lo[c * n + i] = lo[c];
#pragma unroll
    for (int c = 0; c < 21; ++c) A.out_cov[c * n + i] = C[c];
  }
  if (A.chi2) A.chi2[i] = chi2;
  st |= raised;
  if ((A.last || stopped) && !pd5(p, C)) st |= KF_ST_NOT_PD;
  if (A.first || raised || A.last) A.status[i] = st;
}

// One track per thread over a grid that covers the batch: blocks start as
// others finish, so the warps of an SM drift out of phase and their load
// bursts overlap other warps' arithmetic.  THREADS (64 or 128, picked by the
// autotuner) keeps kFitWarpsPerSM warps per SM resident either way.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, kFitWarpsPerSM * 32 / THREADS) fit_layer_kernel(const FitLayerArgs A) {
  const int64_t n = A.n;
  const int64_t i = A.begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= A.begin + A.count) return;
  const int32_t st = A.first ? 0 : A.status[i];
  float p[6], lo[3], C[21];
  if (!(st & KF_ST_STOPPED)) {
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = A.in_par[c * n + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = A.in_lo ? A.in_lo[c * n + i] : 0.f;
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = A.in_cov[c * n + i];
  }
  const bool has_hit = A.valid ? A.valid[i] != 0 : true;
  fit_layer_track(A, i, st, p, lo, C, A.charge[i], has_hit, A.hit[i], A.hit[n + i], A.hit[2 * n + i]);
}

template <bool UPD64>
__global__ void __launch_bounds__(kFitThreads, UPD64 ? 1 : kFitMinBlocks) fit_fused_kernel(const FitFusedArgs A) {
  const int64_t n = A.n;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    float p[6], lo[3], C[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = A.in_par[c * n + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = A.in_lo ? A.in_lo[c * n + i] : 0.f;
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = A.in_cov[c * n + i];
    const float a = A.a_scale * float(A.charge[i]);
    int32_t st = 0;
    for (int l = 0; l < A.n_layers; ++l) {
      float chi2 = -1.f;
      if (!(st & KF_ST_STOPPED)) {
        const float* h = A.hits + int64_t(l) * 3 * n;
        const bool has_hit = A.valid ? A.valid[int64_t(l) * n + i] != 0 : true;
        st |= track_step<float, kNewtonF32, true, UPD64>(p, lo, C, a, A.R[l], A.x_x0[l], A.mass, has_hit, h[i],
                                                         h[n + i], h[2 * n + i], A.v0, A.v1, A.v2, chi2);
      }
      if (A.chi2) A.chi2[int64_t(l) * n + i] = chi2;
    }
    if (!pd5(p, C)) st |= KF_ST_NOT_PD;
#pragma unroll
    for (int c = 0; c < 6; ++c) A.out_par[c * n + i] = p[c];
    if (A.out_lo) {
#pragma unroll
      for (int c = 0; c < 3; ++c) A.out_lo[c * n + i] = lo[c];
    }
#pragma unroll
    for (int c = 0; c < 21; ++c) A.out_cov[c * n + i] = C[c];
    if (A.status) A.status[i] = st;
  }
}

// Plain FP64 form: the same arithmetic in double, no position pair, one
// thread per track of one event, one launch per event and layer.
__global__ void __launch_bounds__(kFitThreads) fit_f64_kernel(const FitF64Args A) {
  const int64_t n = A.n;
  const int64_t i = A.begin + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= A.end) return;
  int32_t st = A.first ? 0 : A.status[i];
  if (st & KF_ST_STOPPED) {
    if (A.chi2) A.chi2[i] = -1.0;
    return;
  }
  double p[6], lo[3] = {0, 0, 0}, C[21];
  for (int c = 0; c < 6; ++c) p[c] = A.in_par[c * n + i];
  for (int c = 0; c < 21; ++c) C[c] = A.in_cov[c * n + i];
  const double a = A.a_scale * double(A.charge[i]);
  const bool has_hit = A.valid ? A.valid[i] != 0 : true;
  double chi2;
  const int32_t raised = track_step<double, kNewtonF64, false>(
      p, lo, C, a, A.R, A.x_x0, A.mass, has_hit, double(A.hit[i]), double(A.hit[n + i]), double(A.hit[2 * n + i]), A.v0,
      A.v1, A.v2, chi2);
  const bool stopped = (raised & KF_ST_STOPPED) != 0;
  if (!stopped || A.first) {
    for (int c = 0; c < 6; ++c) A.out_par[c * n + i] = p[c];
    for (int c = 0; c < 21; ++c) A.out_cov[c * n + i] = C[c];
  }
  if (A.chi2) A.chi2[i] = chi2;
  st |= raised;
  if ((A.last || stopped) && !pd5(p, C)) st |= KF_ST_NOT_PD;
  if (A.first || raised || A.last) A.status[i] = st;
}

int fit_grid(int block, int64_t n) {
  const int64_t blocks = (n + block - 1) / block;
  return int(blocks > 0 ? blocks : 1);
}

cudaError_t launch_fit_layer(const FitLayerArgs& a, int block, cudaStream_t st) {
  if (block == 64)
    fit_layer_kernel<64><<<fit_grid(64, a.count), 64, 0, st>>>(a);
  else
    fit_layer_kernel<128><<<fit_grid(128, a.count), 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fit_fused(const FitFusedArgs& a, cudaStream_t st, bool upd64) {
  const int64_t blocks = (a.n + kFitThreads - 1) / kFitThreads;
  const int grid = int(blocks > 0 ? blocks : 1);
  if (upd64)
    fit_fused_kernel<true><<<grid, kFitThreads, 0, st>>>(a);
  else
    fit_fused_kernel<false><<<grid, kFitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fit_f64(const FitF64Args& a, cudaStream_t st) {
  const int64_t cnt = a.end - a.begin;
  if (cnt <= 0) return cudaSuccess;
  const int grid = int((cnt + kFitThreads - 1) / kFitThreads);
  fit_f64_kernel<<<grid, kFitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace kfi

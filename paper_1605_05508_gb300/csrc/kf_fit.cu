// kf_fit.cu -- track-fit kernels: one thread per track, state and covariance
// in registers, structure-of-arrays global layout (coalesced 128-byte warp
// transactions per component).
//
// Track fitting is the branch-free part of Kalman-filter tracking (Cerati et
// al., Sec. 2): with the hit set fixed, every track runs propagate + update
// over the layers.  Forms:
//   fit_layer_kernel        one layer step over the whole batch (kf_fit
//                           replays one launch per layer from a captured CUDA
//                           graph), plain coalesced row reads;
//   fit_layer_stage_kernel  the same step with each warp's next 32 tracks
//                           copied into shared memory by 2-D tensor copies
//                           while it computes the current ones (an autotuned
//                           alternative, bitwise equal);
//   fit_fused_kernel        all layers in one launch, the track held in
//                           registers (also the mixed-precision form);
//   fit_f64_kernel          the plain FP64 form, launched per event and per
//                           layer.
// One track per thread, 24 resident warps per SM in the layer step.  Other
// stagings of the rows (bulk copies per block or per 32 tracks, per-thread
// cp.async double buffering) measured slower than plain reads.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "kf_internal.h"
#include "kf_math.cuh"
#include "kf_tma.cuh"

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

// ---------------------------------------------------------------------------
// Staged form of the layer step (kf_tuning.fit_stage = 1): the same step per
// track, but the 33 float rows a track reads (state, position low parts,
// covariance, hit) arrive in shared memory by tensor copies.  Each warp walks
// tiles of 32 tracks; lane 0 issues four 2-D tensor copies (boxes of 32 tracks
// x 6, 3, 21 and 3 rows) for the warp's next tile into the other half of a
// double buffer while the warp computes the current tile, so a tile's loads
// are in flight during the previous tile's arithmetic without holding
// registers.  Completion is tracked by one mbarrier per buffer; every wait is
// bounded (a wait that gives up marks the warp's remaining tracks with
// KF_ST_DEVICE_TIMEOUT).  Requires n, begin and count multiples of 32 and
// 16-byte aligned rows; kf_fit falls back to fit_layer_kernel otherwise.
constexpr int kStageTile = 32;                 // tracks per warp tile
constexpr int kStageThreads = 64;              // two warps per block
constexpr int kStageBlocksPerSM = 12;          // 24 warps per SM
constexpr uint32_t kStageWaitLimit = 1u << 22; // bounded mbarrier polls

struct StageTile {  // one buffer: rows of 32 tracks, each box 128-byte aligned
  float par[6][kStageTile];
  float lo[3][kStageTile];
  float cov[21][kStageTile];
  float hit[3][kStageTile];
};
static_assert(sizeof(StageTile) % 128 == 0, "box alignment");
constexpr size_t kStageSmem = size_t(kStageThreads / 32) * 2 * sizeof(StageTile) + 64;

__device__ __forceinline__ void tensor_g2s_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void stage_issue(const FitStageMaps& M, bool has_lo, StageTile& T, uint64_t* bar, int x,
                                            uint32_t bytes) {
  mbar_arrive_expect_tx(bar, bytes);
  tensor_g2s_2d(T.par, &M.par, x, 0, bar);
  if (has_lo) tensor_g2s_2d(T.lo, &M.lo, x, 0, bar);
  tensor_g2s_2d(T.cov, &M.cov, x, 0, bar);
  tensor_g2s_2d(T.hit, &M.hit, x, 0, bar);
}

__global__ void __launch_bounds__(kStageThreads, kStageBlocksPerSM)
    fit_layer_stage_kernel(const FitLayerArgs A, const __grid_constant__ FitStageMaps M) {
  extern __shared__ __align__(128) unsigned char stage_smem[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  StageTile* buf = reinterpret_cast<StageTile*>(stage_smem) + 2 * wib;
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage_smem + size_t(kStageThreads / 32) * 2 * sizeof(StageTile)) + 2 * wib;
  const int64_t n_tiles = A.count / kStageTile;
  const int64_t nwarps = int64_t(gridDim.x) * (kStageThreads / 32);
  int64_t t = int64_t(blockIdx.x) * (kStageThreads / 32) + wib;
  if (t >= n_tiles) return;  // the whole warp
  const bool has_lo = A.in_lo != nullptr;
  const uint32_t bytes = uint32_t(sizeof(float)) * kStageTile * (6 + 21 + 3 + (has_lo ? 3 : 0));
  // Test hook (kf_test_stage_fault): the copies of the batch's tile
  // A.skip_tile are never issued, so the wait for it runs out; A.wait_limit
  // (0: the normal limit) bounds the waits for staged input.  The drain wait
  // before the block exits always keeps the normal limit.
  // lane 0: bit b set while the pending phase of buffer b has copies in flight
  uint32_t armed = 0;
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    if (A.begin / kStageTile + t != A.skip_tile) {
      stage_issue(M, has_lo, buf[0], &bar[0], int(A.begin + t * kStageTile), bytes);
      armed = 1u;
    }
  }
  __syncwarp();
  uint32_t ph0 = 0, ph1 = 0;
  bool failed = false;
  for (int s = 0; t < n_tiles; t += nwarps, s ^= 1) {
    const int64_t i = A.begin + t * kStageTile + lane;
    if (failed) {  // an earlier wait gave up: flag the remaining tracks
      A.status[i] = (A.first ? 0 : A.status[i]) | KF_ST_DEVICE_TIMEOUT;
      continue;
    }
    // the next tile into the other buffer (its previous tile was read by every
    // lane before the __syncwarp that closed the last iteration)
    const int64_t tn = t + nwarps;
    if (tn < n_tiles && lane == 0 && A.begin / kStageTile + tn != A.skip_tile) {
      fence_proxy_async_smem();
      stage_issue(M, has_lo, buf[s ^ 1], &bar[s ^ 1], int(A.begin + tn * kStageTile), bytes);
      armed |= 1u << (s ^ 1);
    }
    // per-track inputs outside the tile, loaded while the copies land
    const int32_t st = A.first ? 0 : A.status[i];
    const int8_t q = A.charge[i];
    const bool has_hit = A.valid ? A.valid[i] != 0 : true;
    const bool ok = __all_sync(
        0xffffffffu, mbar_wait_bounded(&bar[s], s ? ph1 : ph0, A.wait_limit ? A.wait_limit : kStageWaitLimit));
    if (!ok) {  // the phase stays pending: waited for once more below
      failed = true;
      A.status[i] = st | KF_ST_DEVICE_TIMEOUT;
      continue;
    }
    if (s)
      ph1 ^= 1u;
    else
      ph0 ^= 1u;
    armed &= ~(1u << s);
    const StageTile& T = buf[s];
    float p[6], lo[3], C[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = T.par[c][lane];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = has_lo ? T.lo[c][lane] : 0.f;
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = T.cov[c][lane];
    const float m0 = T.hit[0][lane], m1 = T.hit[1][lane], m2 = T.hit[2][lane];
    __syncwarp();  // every lane has read buffer s before lane 0 may refill it
    fit_layer_track(A, i, st, p, lo, C, q, has_hit, m0, m1, m2);
  }
  // Copies still in flight land before the block's memory is released.  Should
  // this bounded wait give up too, the block exits with a copy in flight into
  // shared memory that a later block on the SM may already use: the damage is
  // not confined to this warp's tracks, which is why a KF_ST_DEVICE_TIMEOUT on
  // any track invalidates every result of the call (documented in kf.h).
  if (failed && lane == 0) {
    if (armed & 1u) mbar_wait_bounded(&bar[0], ph0, kStageWaitLimit);
    if (armed & 2u) mbar_wait_bounded(&bar[1], ph1, kStageWaitLimit);
  }
}

// All layers of track i of the arrays of E (FitFusedArgs itself, or one
// event of a table: the same field names), with the layers and constants of A.
template <bool UPD64, class EV>
__device__ __forceinline__ void fused_track(const EV& E, const FitFusedArgs& A, int64_t i) {
  const int64_t n = E.n;
  {
    float p[6], lo[3], C[21];
#pragma unroll
    for (int c = 0; c < 6; ++c) p[c] = E.in_par[c * n + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) lo[c] = E.in_lo ? E.in_lo[c * n + i] : 0.f;
#pragma unroll
    for (int c = 0; c < 21; ++c) C[c] = E.in_cov[c * n + i];
    const float a = A.a_scale * float(E.charge[i]);
    int32_t st = 0;
    for (int l = 0; l < A.n_layers; ++l) {
      float chi2 = -1.f;
      if (!(st & KF_ST_STOPPED)) {
        const float* h = E.hits + int64_t(l) * 3 * n;
        const bool has_hit = E.valid ? E.valid[int64_t(l) * n + i] != 0 : true;
        st |= track_step<float, kNewtonF32, true, UPD64>(p, lo, C, a, A.R[l], A.x_x0[l], A.mass, has_hit, h[i],
                                                         h[n + i], h[2 * n + i], A.v0, A.v1, A.v2, chi2);
      }
      if (E.chi2) E.chi2[int64_t(l) * n + i] = chi2;
    }
    if (!pd5(p, C)) st |= KF_ST_NOT_PD;
#pragma unroll
    for (int c = 0; c < 6; ++c) E.out_par[c * n + i] = p[c];
    if (E.out_lo) {
#pragma unroll
      for (int c = 0; c < 3; ++c) E.out_lo[c * n + i] = lo[c];
    }
#pragma unroll
    for (int c = 0; c < 21; ++c) E.out_cov[c * n + i] = C[c];
    if (E.status) E.status[i] = st;
  }
}

template <bool UPD64>
__global__ void __launch_bounds__(kFitThreads, UPD64 ? 1 : kFitMinBlocks) fit_fused_kernel(const FitFusedArgs A) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < A.n; i += stride) fused_track<UPD64>(A, A, i);
}

// The fused fit of several events in one launch (the events a serving
// iteration prepares): thread t fits track t - table[q].begin of event q,
// the last with table[q].begin <= t; the arithmetic of fit_fused_kernel.
__global__ void __launch_bounds__(kFitThreads, kFitMinBlocks)
    fit_fused_table_kernel(const FitFusedArgs A, const FitEvent* table, int n_events, int64_t n_total) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n_total; t += stride) {
    int q = 0;
    while (q + 1 < n_events && table[q + 1].begin <= t) ++q;
    fused_track<false>(table[q], A, t - table[q].begin);
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

// Tensor maps of a layer step for fit_layer_stage_kernel: 2-D views (x =
// track, y = row) of the input state, position low parts, covariance and the
// layer's hits, boxes of 32 tracks x all rows.  False when the layout does not
// allow them (rows not 16-byte aligned, sizes not multiples of 32) or the
// driver's encoder is unavailable.
bool make_stage_maps(const FitLayerArgs& a, FitStageMaps* m) {
  if (a.n % kStageTile || a.begin % kStageTile || a.count % kStageTile || a.count <= 0) return false;
  if (a.n > (int64_t(1) << 31) - 1) return false;
  auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!aligned(a.in_par) || !aligned(a.in_cov) || !aligned(a.hit) || (a.in_lo && !aligned(a.in_lo))) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode) return false;
  auto map2d = [&](CUtensorMap* t, const float* base, uint32_t rows) {
    const cuuint64_t dims[2] = {cuuint64_t(a.n), rows};
    const cuuint64_t strides[1] = {cuuint64_t(a.n) * sizeof(float)};
    const cuuint32_t box[2] = {kStageTile, rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  std::memset(m, 0, sizeof(*m));
  return map2d(&m->par, a.in_par, 6) && (!a.in_lo || map2d(&m->lo, a.in_lo, 3)) && map2d(&m->cov, a.in_cov, 21) &&
         map2d(&m->hit, a.hit, 3);
}

cudaError_t launch_fit_layer_stage(const FitLayerArgs& a, const FitStageMaps& m, int num_sms, cudaStream_t st) {
  const int64_t tiles = a.count / kStageTile;
  const int64_t need = (tiles + kStageThreads / 32 - 1) / (kStageThreads / 32);
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(num_sms) * kStageBlocksPerSM)));
  cudaError_t e = cudaFuncSetAttribute(fit_layer_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(kStageSmem));
  if (e != cudaSuccess) return e;
  fit_layer_stage_kernel<<<grid, kStageThreads, kStageSmem, st>>>(a, m);
  return cudaGetLastError();
}

cudaError_t launch_fit_fused_table(const FitFusedArgs& a, const FitEvent* table, int n_events, int64_t n_total,
                                   cudaStream_t st) {
  if (n_total <= 0) return cudaSuccess;
  const int grid = int((n_total + kFitThreads - 1) / kFitThreads);
  fit_fused_table_kernel<<<grid, kFitThreads, 0, st>>>(a, table, n_events, n_total);
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

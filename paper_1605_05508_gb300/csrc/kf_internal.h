// kf_internal.h -- context object and launch helpers shared by the .cu files
// of libkf (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/kf.h"

namespace kfi {

constexpr int kMaxLayers = 64;
// kf_fit_host pipeline: chunks (at most kHostChunks, at least kHostChunkMin
// tracks each) over kHostStreams internal streams
constexpr int kHostStreams = 3;
constexpr int kHostChunks = 16;
constexpr int64_t kHostChunkMin = 65536;
constexpr double kCLight = 0.00299792458;  // GeV / (T cm)

// A device allocation owned by the context, grown on demand.
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// One captured and instantiated CUDA graph, keyed by the exact argument set.
struct GraphEntry {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

struct Serve;  // serving loop state (kf_serve.cu)

}  // namespace kfi

struct kf_ctx {
  kf_config cfg;
  float radius[kfi::kMaxLayers];
  float x_x0[kfi::kMaxLayers];  // layer material (radiation lengths; 0: none)
  float mass = 0.f;             // particle mass of the scattering model
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;     // 0 = unbounded
  size_t allocated = 0;  // bytes of context-owned device memory
  int last_cuda = 0;
  cudaStream_t capture_stream = nullptr;
  // scratch pools
  kfi::Scratch s_status, s_lo, s_host_in, s_host_out;
  kfi::Scratch s_bin_id, s_build, s_refit, s_build64;
  // graph cache
  std::vector<kfi::GraphEntry> graphs;
  uint64_t use_clock = 0;
  kfi::Serve* serve = nullptr;
  cudaStream_t host_streams[kfi::kHostStreams] = {};  // kf_fit_host pipeline
  cudaEvent_t host_done[kfi::kHostStreams] = {};
  cudaEvent_t host_start = nullptr;
  kf_tuning tune = {128, 0, 8, 4, 0, 0, 0};  // launch parameters (kf_set_tuning, kf_autotune_*)
  int64_t test_skip_tile = -1;   // kf_test_stage_fault
  uint32_t test_wait_polls = 0;
  int64_t test_build_skip_warp = -1;  // kf_test_build_stage_fault
  uint32_t test_build_wait_polls = 0;
};

namespace kfi {

// Record a CUDA error on the context and turn it into KF_ECUDA.
inline int cuda_fail(kf_ctx* ctx, cudaError_t e) {
  if (ctx) ctx->last_cuda = static_cast<int>(e);
  return KF_ECUDA;
}

#define KF_CUDA_TRY(ctx, expr)                          \
  do {                                                  \
    cudaError_t e__ = (expr);                           \
    if (e__ != cudaSuccess) return kfi::cuda_fail(ctx, e__); \
  } while (0)

// Grow a scratch buffer to at least `bytes` (under the context budget).
int scratch_reserve(kf_ctx* ctx, Scratch& s, size_t bytes);

// Argument check shared by the kf_fit family (kf_capi.cu): KF_OK or KF_EINVAL.
// An empty batch (n = 0) is valid with any pointers.
int check_fit(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, const kf_tracks* out);

// Arguments of one fit layer step (single precision).
struct FitLayerArgs {
  const float* in_par;
  const float* in_lo;  // may be null (lo = 0)
  const float* in_cov;
  const int8_t* charge;
  float* out_par;
  float* out_lo;
  float* out_cov;
  const float* hit;      // [3][n] of this layer
  const uint8_t* valid;  // [n] of this layer or null
  float* chi2;           // [n] of this layer or null
  int32_t* status;       // [n], required
  int64_t n;             // tracks of the batch (the row stride)
  int64_t begin, count;  // this launch: tracks [begin, begin + count)
  float a_scale;  // C_LIGHT * Bz
  float R, v0, v1, v2;
  float x_x0, mass;  // this layer's thickness in radiation lengths (0: none); particle mass
  int first;  // 1: initialise status, always write the state
  int last;   // 1: run the positive-definite check
  // test hook of the staged kernel (kf_test_stage_fault): batch index of a
  // 32-track tile whose copies are not issued (-1: none); poll limit of the
  // waits for staged input (0: the normal limit)
  int64_t skip_tile = -1;
  uint32_t wait_limit = 0;
};

struct FitFusedArgs {
  const float* in_par;
  const float* in_lo;
  const float* in_cov;
  const int8_t* charge;
  float* out_par;
  float* out_lo;  // may be null
  float* out_cov;
  const float* hits;     // [L][3][n]
  const uint8_t* valid;  // [L][n] or null
  float* chi2;           // [L][n] or null
  int32_t* status;       // [n] or null
  int64_t n;
  int n_layers;
  float a_scale;
  float v0, v1, v2;
  float mass;
  float R[kMaxLayers];     // layer radii, by value
  float x_x0[kMaxLayers];  // layer thickness in radiation lengths (0: none)
};

struct FitF64Args {
  const double* in_par;
  const double* in_cov;
  const int8_t* charge;
  double* out_par;
  double* out_cov;
  const float* hit;      // [3][n] of this layer (whole batch)
  const uint8_t* valid;  // [n] of this layer or null
  double* chi2;          // [n] of this layer or null
  int32_t* status;
  int64_t n;       // whole batch (row stride)
  int64_t begin;   // this launch: tracks [begin, end)
  int64_t end;
  double a_scale;
  double R, v0, v1, v2;
  double x_x0, mass;
  int first, last;
};

// Tensor maps of one staged layer step (kf_fit.cu, fit_layer_stage_kernel).
struct FitStageMaps {
  CUtensorMap par, lo, cov, hit;
};

// kernel launchers (kf_fit.cu)
// block: threads per block, 64 or 128 (kf_tuning.fit_block)
cudaError_t launch_fit_layer(const FitLayerArgs& a, int block, cudaStream_t st);
// staged form (kf_tuning.fit_stage): false from make_stage_maps when the
// batch's layout does not allow it (the caller then launches fit_layer_kernel)
bool make_stage_maps(const FitLayerArgs& a, FitStageMaps* m);
cudaError_t launch_fit_layer_stage(const FitLayerArgs& a, const FitStageMaps& m, int num_sms, cudaStream_t st);
cudaError_t launch_fit_fused(const FitFusedArgs& a, cudaStream_t st, bool upd64 = false);
// One event of a table-driven fused fit: its arrays, as in FitFusedArgs, and
// the launch's first thread for it.
struct FitEvent {
  const float* in_par;
  const float* in_lo;
  const float* in_cov;
  const int8_t* charge;
  float* out_par;
  float* out_lo;
  float* out_cov;
  const float* hits;
  const uint8_t* valid;
  float* chi2;
  int32_t* status;
  int64_t n;
  int64_t begin;
};
// The fused fit of n_events events (device table, begins ascending) in one
// launch; a's arrays are ignored, its layers and constants used.
cudaError_t launch_fit_fused_table(const FitFusedArgs& a, const FitEvent* table, int n_events, int64_t n_total,
                                   cudaStream_t st);
cudaError_t launch_fit_f64(const FitF64Args& a, cudaStream_t st);

// Hits of all layers per seed for a re-fit (kf_refit.cu): seeding layers from
// the seed hits, building layers by the build's hit ids.
struct RefitGatherArgs {
  const float* seed_xyz;      // [Ls][3][n]
  const uint8_t* seed_valid;  // [Ls][n] or null (all valid)
  const int64_t* seed_off;    // [E + 1]
  const float* hit_xyz;       // [3][n_hits]
  const int64_t* seg_off;     // [E * Lb + 1]
  const int32_t* hit_idx;     // [Lb][n]
  float* xyz;                 // [Ls + Lb][3][n]
  uint8_t* valid;             // [Ls + Lb][n]
  int64_t n, n_hits;
  int Ls, Lb, E;
};
cudaError_t launch_refit_gather(const RefitGatherArgs& a, cudaStream_t st);
int fit_grid(int block, int64_t n);

}  // namespace kfi

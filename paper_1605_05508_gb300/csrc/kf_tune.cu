// kf_tune.cu -- launch parameters of the context and their autotuner.
//
// Each tunable changes how the work is laid out on the GPU, never the
// arithmetic of a track: the fit kernel's block size (64 or 128 threads, 24
// resident warps per SM either way), the build step's hit staging (window
// hits copied per warp into shared memory, or read through L1), the length
// of a lane's child list (4 suffices when at most 4 candidates are kept) and
// the step's thread layout (8 lanes per seed, each lane scanning its own
// candidate's window or the seed's lanes scanning each parent's window in
// turn; or the live candidates packed onto consecutive threads, 128 or 64
// seeds per block; or each warp taking small groups of seeds through all
// layers with the candidates in registers).  The autotuner runs the caller's own batch once per setting and keeps
// the fastest, so the choice follows the workload (batch size, hit density,
// max_cands) rather than a fixed table.
#include "kf_internal.h"

#include <vector>

namespace {

bool valid_tuning(const kf_tuning& t) {
  return (t.fit_block == 64 || t.fit_block == 128) && (t.build_hit_tile == 0 || t.build_hit_tile == 512) &&
         (t.build_list_width == 4 || t.build_list_width == 8) && (t.build_scan == 0 || t.build_scan == 1 || ((t.build_scan >= 2 && t.build_scan <= 4) && t.build_hit_tile == 0)) &&
         (t.fit_chunk == 0 || t.fit_chunk == 262144 || t.fit_chunk == 524288 || t.fit_chunk == 1048576) &&
         (t.fit_stage == 0 || t.fit_stage == 1) && (t.bin_unordered == 0 || t.bin_unordered == 1);
}

// Mean time of `reps` calls of fn after one untimed call; < 0 on failure
// (the failing call's KF_* code is left in *rc).
template <typename Fn>
float time_calls(kf_ctx* ctx, cudaStream_t st, Fn&& fn, int reps, int* rc) {
  *rc = fn();
  if (*rc) return -1.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    *rc = kfi::cuda_fail(ctx, cudaGetLastError());
    return -1.f;
  }
  float ms = -1.f;
  cudaError_t ce = cudaEventRecord(e0, st);
  for (int i = 0; i < reps && ce == cudaSuccess && !*rc; ++i) *rc = fn();
  if (ce == cudaSuccess && !*rc) ce = cudaEventRecord(e1, st);
  if (ce == cudaSuccess && !*rc) ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess && !*rc) ce = cudaEventElapsedTime(&ms, e0, e1);
  if (ce != cudaSuccess && !*rc) *rc = kfi::cuda_fail(ctx, ce);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return *rc ? -1.f : ms / float(reps);
}

// Try every setting in `cands` (applied with kf_set_tuning), keep the fastest:
// a setting replaces the best so far only when it is kMargin faster, so among
// settings that time alike (within the noise of three calls) the first one --
// the candidates are listed simplest first -- is kept, and repeated runs agree.
constexpr float kMargin = 0.02f;
template <typename Fn>
int autotune(kf_ctx* ctx, void* stream, const std::vector<kf_tuning>& cands, Fn&& fn, kf_tuning* chosen) {
  const kf_tuning saved = ctx->tune;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float best = -1.f;
  kf_tuning best_t = saved;
  for (const kf_tuning& t : cands) {
    ctx->tune = t;
    int rc = 0;
    const float ms = time_calls(ctx, st, fn, 3, &rc);
    if (rc) {
      ctx->tune = saved;
      return rc;
    }
    if (best < 0.f || ms < best * (1.f - kMargin)) {
      best = ms;
      best_t = t;
    }
  }
  // the outputs hold the last call's results: the same bits for every setting
  ctx->tune = best_t;
  if (chosen) *chosen = ctx->tune;
  return KF_OK;
}

}  // namespace

extern "C" {

int kf_get_tuning(const kf_ctx* ctx, kf_tuning* out) {
  if (!ctx || !out) return KF_EINVAL;
  *out = ctx->tune;
  return KF_OK;
}

int kf_set_tuning(kf_ctx* ctx, const kf_tuning* t) {
  if (!ctx || !t || !valid_tuning(*t)) return KF_EINVAL;
  ctx->tune = *t;
  return KF_OK;
}

int kf_autotune_fit(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
                    int32_t* status, void* stream, kf_tuning* chosen) {
  if (!ctx) return KF_EINVAL;
  std::vector<kf_tuning> cands;
  for (int stage : {0, 1})
    for (int b : {64, 128})
      for (int chunk : {0, 262144, 524288, 1048576}) {
        if (chunk > 0 && seeds && chunk >= seeds->n) continue;  // one chunk: the same as 0
        if (stage == 1 && b != 64) continue;                     // the staged kernel has its own blocks
        kf_tuning t = ctx->tune;
        t.fit_block = b;
        t.fit_chunk = chunk;
        t.fit_stage = stage;
        cands.push_back(t);
      }
  return autotune(ctx, stream, cands, [&] { return kf_fit(ctx, seeds, hits, out, chi2, status, stream); }, chosen);
}

int kf_autotune_build(kf_ctx* ctx, const kf_tracks* seeds, const int64_t* seed_off, const kf_layer_hit_bins* bins,
                      int32_t max_cands, kf_build_result* out, void* stream, kf_tuning* chosen) {
  if (!ctx) return KF_EINVAL;
  std::vector<kf_tuning> cands;
  for (int tile : {0, 512})
    for (int list : {8, 4})
      for (int scan : {0, 1, 2, 3, 4}) {
        if (list == 4 && max_cands > 4) continue;
        if (scan >= 2 && tile > 0) continue;  // the packed and resident steps stage nothing
        if (scan == 4 && list == 4) continue;  // the resident step sizes its lists itself
        kf_tuning t = ctx->tune;
        t.build_hit_tile = tile;
        t.build_list_width = list;
        t.build_scan = scan;
        cands.push_back(t);
      }
  return autotune(ctx, stream, cands,
                  [&] { return kf_build(ctx, seeds, seed_off, bins, max_cands, out, stream); }, chosen);
}

}  // extern "C"

// kf_refit.cu -- the Kalman fit of built tracks over all layers with the hits
// the build chose (building, Sec. 3, followed by fitting, Sec. 2).
//
// A gather kernel assembles, for every seed, the hits of all layers in the
// fit's layout -- the seeding layers copied from the seed's own hits, each
// building layer looked up by the hit id kf_build returned in the raw hits of
// the seed's (event, layer) segment -- and kf_fit then runs from the seed
// state over all of them.
#include "kf_internal.h"

namespace kfi {

// event of seed i: the e with seed_off[e] <= i < seed_off[e + 1]
__device__ __forceinline__ int event_of(const int64_t* off, int E, int64_t i) {
  int lo = 0, hi = E - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// one thread per (layer, seed)
__global__ void refit_gather_kernel(const RefitGatherArgs A) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int L = A.Ls + A.Lb;
  if (t >= int64_t(L) * A.n) return;
  const int l = int(t / A.n);
  const int64_t i = t - int64_t(l) * A.n;
  const int64_t n = A.n;
  float x = 0.f, y = 0.f, z = 0.f;
  uint8_t ok = 0;
  if (l < A.Ls) {
    const float* s = A.seed_xyz + int64_t(l) * 3 * n;
    x = s[i];
    y = s[n + i];
    z = s[2 * n + i];
    ok = A.seed_valid ? A.seed_valid[int64_t(l) * n + i] : uint8_t(1);
  } else {
    const int b = l - A.Ls;
    const int32_t id = A.hit_idx[int64_t(b) * n + i];
    if (id >= 0) {
      const int e = event_of(A.seed_off, A.E, i);
      const int64_t s0 = A.seg_off[int64_t(e) * A.Lb + b], s1 = A.seg_off[int64_t(e) * A.Lb + b + 1];
      const int64_t h = s0 + id;
      if (h < s1 && h >= 0 && h < A.n_hits) {
        x = A.hit_xyz[h];
        y = A.hit_xyz[A.n_hits + h];
        z = A.hit_xyz[2 * A.n_hits + h];
        ok = 1;
      }
    }
  }
  float* d = A.xyz + int64_t(l) * 3 * n;
  d[i] = x;
  d[n + i] = y;
  d[2 * n + i] = z;
  A.valid[int64_t(l) * n + i] = ok;
}

cudaError_t launch_refit_gather(const RefitGatherArgs& a, cudaStream_t st) {
  const int64_t threads = int64_t(a.Ls + a.Lb) * a.n;
  if (threads <= 0) return cudaSuccess;
  refit_gather_kernel<<<int((threads + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace kfi

using namespace kfi;

extern "C" int kf_refit(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* seed_hits, const int64_t* seed_off,
                        const kf_layer_hits* build_hits, const int32_t* hit_idx, kf_tracks* out, float* chi2,
                        int32_t* status, void* stream) {
  if (!ctx || !seeds || !seed_hits || !build_hits || !out) return KF_EINVAL;
  const int64_t n = seeds->n;
  const int Ls = seed_hits->n_layers, Lb = build_hits->n_layers, E = build_hits->n_events;
  if (n < 0 || seed_hits->n_tracks != n || out->n != n) return KF_EINVAL;
  if (Ls < 0 || Lb < 1 || build_hits->first_layer != Ls || Ls + Lb > ctx->cfg.n_layers || E < 1) return KF_EINVAL;
  if (n == 0) return KF_OK;
  if (!seed_off || !hit_idx || !build_hits->xyz || !build_hits->seg_off || (Ls > 0 && !seed_hits->xyz) ||
      build_hits->n_hits < 0)
    return KF_EINVAL;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int L = Ls + Lb;
  const size_t xyz_bytes = (size_t(L) * 3 * n * sizeof(float) + 255) & ~size_t(255);
  int rc = scratch_reserve(ctx, ctx->s_refit, xyz_bytes + size_t(L) * n);
  if (rc) return rc;
  RefitGatherArgs g;
  g.seed_xyz = seed_hits->xyz;
  g.seed_valid = seed_hits->valid;
  g.seed_off = seed_off;
  g.hit_xyz = build_hits->xyz;
  g.seg_off = build_hits->seg_off;
  g.hit_idx = hit_idx;
  g.xyz = static_cast<float*>(ctx->s_refit.ptr);
  g.valid = static_cast<uint8_t*>(ctx->s_refit.ptr) + xyz_bytes;
  g.n = n;
  g.n_hits = build_hits->n_hits;
  g.Ls = Ls;
  g.Lb = Lb;
  g.E = E;
  KF_CUDA_TRY(ctx, launch_refit_gather(g, static_cast<cudaStream_t>(stream)));
  kf_track_hits all;
  all.n_tracks = n;
  all.n_layers = L;
  all.xyz = g.xyz;
  all.valid = g.valid;
  return kf_fit(ctx, seeds, &all, out, chi2, status, stream);
}

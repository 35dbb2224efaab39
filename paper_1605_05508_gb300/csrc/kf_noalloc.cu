// kf_noalloc.cu -- kf_fit_noalloc: the per-layer track fit for callers that
// must not allocate device memory.
//
// kf_fit keeps two per-track arrays between its layer launches: the status
// word (which tracks have stopped) and the low-order parts of the position.
// When the caller does not pass them, kf_fit takes them from context scratch
// that it grows with cudaMalloc on first use.  This entry point takes them
// instead from one fixed array in the library's static device memory, sized
// for KF_NOALLOC_MAX_TRACKS tracks, so a call performs no allocation at all.
#include "kf_internal.h"

namespace {

constexpr int64_t kMaxTracks = KF_NOALLOC_MAX_TRACKS;
constexpr int kMaxDevices = 64;

// [0, 12 kMaxTracks): position low parts, laid out [3][n] for a batch of n;
// [12 kMaxTracks, 16 kMaxTracks): status words [n].
// Every GPU that loads libkf holds this array (4 MiB) until the process exits.
static __device__ __align__(256) unsigned char g_fit_scratch[16 * KF_NOALLOC_MAX_TRACKS];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_fit_scratch on the context's device.  Host code must
// not use the symbol itself (on the host it names a stand-in, not device
// memory); the address is looked up once per device, with that device
// current, and cached for the life of the process.  A cudaDeviceReset (or any
// teardown of the device's primary context) reloads the module and may move
// the array, so the cache does not survive one; neither does any kf_ctx.
int scratch_address(kf_ctx* ctx, unsigned char** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return KF_ENOTSUP;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[ctx->device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fit_scratch);
    if (e != cudaSuccess || !p) return kfi::cuda_fail(ctx, e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_scratch_addr[ctx->device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[ctx->device]);
  return KF_OK;
}

}  // namespace

extern "C" int kf_fit_noalloc(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out,
                              float* chi2, int32_t* status, void* stream) {
  const int rc0 = kfi::check_fit(ctx, seeds, hits, out);  // the checks of kf_fit
  if (rc0) return rc0;
  const int64_t n = seeds->n;
  if (n > kMaxTracks) return KF_EINVAL;  // beyond the static scratch: split the batch
  if (n == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  unsigned char* scratch = nullptr;
  const int rc = scratch_address(ctx, &scratch);
  if (rc) return rc;
  // The first layer launch writes every track's status and low parts, so
  // nothing left in the array by an earlier call is read.
  float* lo = out->par_lo ? out->par_lo : reinterpret_cast<float*>(scratch);
  int32_t* st = status ? status : reinterpret_cast<int32_t*>(scratch + 12 * kMaxTracks);
  const int L = hits->n_layers;
  const float v0 = ctx->cfg.sigma_xy_cm * ctx->cfg.sigma_xy_cm;
  const float v2 = ctx->cfg.sigma_z_cm * ctx->cfg.sigma_z_cm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int l = 0; l < L; ++l) {
    kfi::FitLayerArgs a;
    a.in_par = l == 0 ? seeds->par : out->par;
    a.in_lo = l == 0 ? seeds->par_lo : lo;
    a.in_cov = l == 0 ? seeds->cov : out->cov;
    a.charge = seeds->charge;
    a.out_par = out->par;
    a.out_lo = lo;
    a.out_cov = out->cov;
    a.hit = hits->xyz + int64_t(l) * 3 * n;
    a.valid = hits->valid ? hits->valid + int64_t(l) * n : nullptr;
    a.chi2 = chi2 ? chi2 + int64_t(l) * n : nullptr;
    a.status = st;
    a.n = n;
    a.begin = 0;
    a.count = n;
    a.a_scale = float(kfi::kCLight * double(ctx->cfg.bz_tesla));
    a.R = ctx->radius[l];
    a.x_x0 = ctx->x_x0[l];
    a.mass = ctx->mass;
    a.v0 = v0;
    a.v1 = v0;
    a.v2 = v2;
    a.first = l == 0;
    a.last = l == L - 1;
    KF_CUDA_TRY(ctx, kfi::launch_fit_layer(a, ctx->tune.fit_block, s));
  }
  return KF_OK;
}

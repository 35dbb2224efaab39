// kf_capi.cu -- context management and the C entry points of the track fit
// (declared in include/kf.h).
#include <algorithm>
#include <cmath>
#include <new>

#include "kf_internal.h"

namespace kfi {

int scratch_reserve(kf_ctx* ctx, Scratch& s, size_t bytes) {
  if (bytes <= s.bytes) return KF_OK;
  const size_t want = std::max(bytes, s.bytes + s.bytes / 2);
  const size_t grow = want - s.bytes;
  if (ctx->budget && ctx->allocated + grow > ctx->budget) return KF_ENOMEM;
  if (s.ptr) {
    KF_CUDA_TRY(ctx, cudaDeviceSynchronize());
    cudaFree(s.ptr);
    ctx->allocated -= s.bytes;
    s.ptr = nullptr;
    s.bytes = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return KF_ENOMEM;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e);
  s.ptr = p;
  s.bytes = want;
  ctx->allocated += want;
  // cached graphs may hold the old pointer
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  return KF_OK;
}

static void scratch_free(kf_ctx* ctx, Scratch& s) {
  if (s.ptr) cudaFree(s.ptr);
  ctx->allocated -= s.bytes;
  s.ptr = nullptr;
  s.bytes = 0;
}

static bool tracks_ok(const kf_tracks* t, bool need_lo) {
  return t && t->n >= 0 && t->par && t->cov && t->charge && (!need_lo || t->par_lo);
}

// Validate a fit request against the configuration.
// An empty batch (n = 0) is valid with any pointers.
int check_fit(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits,
                     const kf_tracks* out) {
  if (!ctx || !seeds || !hits || !out) return KF_EINVAL;
  if (seeds->n < 0 || out->n != seeds->n || hits->n_tracks != seeds->n) return KF_EINVAL;
  if (hits->n_layers < 1 || hits->n_layers > ctx->cfg.n_layers) return KF_EINVAL;
  if (seeds->n == 0) return KF_OK;
  if (!tracks_ok(seeds, false) || !out->par || !out->cov || !hits->xyz) return KF_EINVAL;
  return KF_OK;
}

}  // namespace kfi

using namespace kfi;

extern "C" {

const char* kf_strerror(int code) {
  switch (code) {
    case KF_OK: return "ok";
    case KF_EINVAL: return "invalid argument";
    case KF_ENOMEM: return "out of device memory or context budget";
    case KF_EAGAIN: return "not ready / not admitted yet";
    case KF_ETIMEDOUT: return "timed out";
    case KF_ECUDA: return "CUDA runtime error";
    case KF_ENOTSUP: return "not supported";
    default: return "unknown error";
  }
}

int kf_last_cuda_error(const kf_ctx* ctx) { return ctx ? ctx->last_cuda : 0; }

int kf_test_stage_fault(kf_ctx* ctx, int64_t skip_tile, uint32_t wait_polls) {
  if (!ctx || skip_tile < -1) return KF_EINVAL;
  ctx->test_skip_tile = skip_tile;
  ctx->test_wait_polls = wait_polls;
  return KF_OK;
}

int kf_test_build_stage_fault(kf_ctx* ctx, int64_t skip_warp, uint32_t wait_polls) {
  if (!ctx || skip_warp < -1) return KF_EINVAL;
  ctx->test_build_skip_warp = skip_warp;
  ctx->test_build_wait_polls = wait_polls;
  return KF_OK;
}

int kf_create(kf_ctx** out, const kf_config* cfg, int device, size_t mem_budget_bytes) {
  if (!out || !cfg) return KF_EINVAL;
  *out = nullptr;
  if (cfg->n_layers < 1 || cfg->n_layers > kMaxLayers || !cfg->radius_cm) return KF_EINVAL;
  if (!(cfg->bz_tesla != 0.f) || !std::isfinite(cfg->bz_tesla)) return KF_EINVAL;
  if (!(cfg->sigma_xy_cm > 0.f) || !(cfg->sigma_z_cm > 0.f)) return KF_EINVAL;
  if (cfg->max_cands < 1 || cfg->max_cands > 8 || !(cfg->chi2_cut > 0.f)) return KF_EINVAL;
  float prev = 0.f;
  for (int l = 0; l < cfg->n_layers; ++l) {
    if (!(cfg->radius_cm[l] > prev) || !std::isfinite(cfg->radius_cm[l])) return KF_EINVAL;
    prev = cfg->radius_cm[l];
    if (cfg->x_x0 && !(cfg->x_x0[l] >= 0.f && cfg->x_x0[l] < 1.f)) return KF_EINVAL;
  }
  if (!(cfg->mass_gev >= 0.f) || !std::isfinite(cfg->mass_gev)) return KF_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return KF_ENOTSUP;
  }
  kf_ctx* ctx = new (std::nothrow) kf_ctx();
  if (!ctx) return KF_ENOMEM;
  ctx->cfg = *cfg;
  for (int l = 0; l < kMaxLayers; ++l) {
    ctx->radius[l] = l < cfg->n_layers ? cfg->radius_cm[l] : 0.f;
    ctx->x_x0[l] = (l < cfg->n_layers && cfg->x_x0) ? cfg->x_x0[l] : 0.f;
  }
  ctx->mass = cfg->mass_gev;
  ctx->cfg.radius_cm = ctx->radius;
  ctx->cfg.x_x0 = ctx->x_x0;
  ctx->device = device;
  ctx->budget = mem_budget_bytes;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete ctx;
    return KF_ECUDA;
  }
  *out = ctx;
  return KF_OK;
}

}  // extern "C"
void kf_serve_shutdown_internal(kf_ctx* ctx);
extern "C" {

void kf_destroy(kf_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  kf_serve_shutdown_internal(ctx);
  cudaDeviceSynchronize();
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  scratch_free(ctx, ctx->s_status);
  scratch_free(ctx, ctx->s_lo);
  scratch_free(ctx, ctx->s_host_in);
  scratch_free(ctx, ctx->s_host_out);
  scratch_free(ctx, ctx->s_bin_id);
  scratch_free(ctx, ctx->s_build);
  scratch_free(ctx, ctx->s_refit);
  scratch_free(ctx, ctx->s_build64);
  for (int k = 0; k < kHostStreams; ++k) {
    if (ctx->host_streams[k]) cudaStreamDestroy(ctx->host_streams[k]);
    if (ctx->host_done[k]) cudaEventDestroy(ctx->host_done[k]);
  }
  if (ctx->host_start) cudaEventDestroy(ctx->host_start);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
}

// Per-layer fit replayed from a captured graph (one kernel node per layer).
int kf_fit(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
           int32_t* status, void* stream) {
  int rc = check_fit(ctx, seeds, hits, out);
  if (rc) return rc;
  const int64_t n = seeds->n;
  if (n == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int32_t* st = status;
  if (!st) {
    rc = scratch_reserve(ctx, ctx->s_status, size_t(n) * sizeof(int32_t));
    if (rc) return rc;
    st = static_cast<int32_t*>(ctx->s_status.ptr);
  }
  float* lo = out->par_lo;
  if (!lo) {
    rc = scratch_reserve(ctx, ctx->s_lo, size_t(n) * 3 * sizeof(float));
    if (rc) return rc;
    lo = static_cast<float*>(ctx->s_lo.ptr);
  }
  const int L = hits->n_layers;
  const float a_scale = float(kCLight * double(ctx->cfg.bz_tesla));
  const float v0 = ctx->cfg.sigma_xy_cm * ctx->cfg.sigma_xy_cm;
  const float v2 = ctx->cfg.sigma_z_cm * ctx->cfg.sigma_z_cm;
  const int block = ctx->tune.fit_block;
  // tracks per L2 block: every layer of a chunk runs before the next chunk,
  // so the chunk's state stays in L2 between its layer launches
  const int64_t chunk = ctx->tune.fit_chunk > 0 ? std::min<int64_t>(ctx->tune.fit_chunk, n) : n;
  std::vector<uint64_t> key = {1,
                               uint64_t(n),
                               uint64_t(L),
                               uint64_t(block),
                               uint64_t(chunk),
                               uint64_t(ctx->tune.fit_stage),
                               reinterpret_cast<uint64_t>(seeds->par),
                               reinterpret_cast<uint64_t>(seeds->par_lo),
                               reinterpret_cast<uint64_t>(seeds->cov),
                               reinterpret_cast<uint64_t>(seeds->charge),
                               reinterpret_cast<uint64_t>(out->par),
                               reinterpret_cast<uint64_t>(lo),
                               reinterpret_cast<uint64_t>(out->cov),
                               reinterpret_cast<uint64_t>(hits->xyz),
                               reinterpret_cast<uint64_t>(hits->valid),
                               reinterpret_cast<uint64_t>(chi2),
                               reinterpret_cast<uint64_t>(st),
                               uint64_t(ctx->test_skip_tile),
                               uint64_t(ctx->test_wait_polls)};
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  GraphEntry* hit_entry = nullptr;
  for (auto& g : ctx->graphs)
    if (g.key == key) hit_entry = &g;
  if (!hit_entry) {
    cudaStream_t cs = ctx->capture_stream;
    KF_CUDA_TRY(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = cudaSuccess;
    for (int64_t c0 = 0; c0 < n && le == cudaSuccess; c0 += chunk)
    for (int l = 0; l < L && le == cudaSuccess; ++l) {
      FitLayerArgs a;
      a.begin = c0;
      a.count = std::min(chunk, n - c0);
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
      a.a_scale = a_scale;
      a.R = ctx->radius[l];
      a.x_x0 = ctx->x_x0[l];
      a.mass = ctx->mass;
      a.v0 = v0;
      a.v1 = v0;
      a.v2 = v2;
      a.first = l == 0;
      a.last = l == L - 1;
      a.skip_tile = ctx->test_skip_tile;
      a.wait_limit = ctx->test_wait_polls;
      FitStageMaps maps;
      if (ctx->tune.fit_stage && make_stage_maps(a, &maps))
        le = launch_fit_layer_stage(a, maps, ctx->num_sms, cs);
      else
        le = launch_fit_layer(a, block, cs);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) return cuda_fail(ctx, le);
    if (ee != cudaSuccess) return cuda_fail(ctx, ee);
    cudaGraphExec_t exec = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ctx, ie);
    if (ctx->graphs.size() >= 16) {
      auto old = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                  [](const GraphEntry& x, const GraphEntry& y) { return x.last_use < y.last_use; });
      cudaGraphExecDestroy(old->exec);
      ctx->graphs.erase(old);
    }
    ctx->graphs.push_back(GraphEntry{key, exec, 0});
    hit_entry = &ctx->graphs.back();
  }
  hit_entry->last_use = ++ctx->use_clock;
  KF_CUDA_TRY(ctx, cudaGraphLaunch(hit_entry->exec, user));
  return KF_OK;
}

static int fit_fused_impl(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
                          int32_t* status, void* stream, bool upd64);

int kf_fit_fused(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
                 int32_t* status, void* stream) {
  return fit_fused_impl(ctx, seeds, hits, out, chi2, status, stream, false);
}

int kf_fit_mixed(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
                 int32_t* status, void* stream) {
  return fit_fused_impl(ctx, seeds, hits, out, chi2, status, stream, true);
}

static int fit_fused_impl(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
                          int32_t* status, void* stream, bool upd64) {
  int rc = check_fit(ctx, seeds, hits, out);
  if (rc) return rc;
  const int64_t n = seeds->n;
  if (n == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  FitFusedArgs a;
  std::memset(&a, 0, sizeof a);
  a.in_par = seeds->par;
  a.in_lo = seeds->par_lo;
  a.in_cov = seeds->cov;
  a.charge = seeds->charge;
  a.out_par = out->par;
  a.out_lo = out->par_lo;
  a.out_cov = out->cov;
  a.hits = hits->xyz;
  a.valid = hits->valid;
  a.chi2 = chi2;
  a.status = status;
  a.n = n;
  a.n_layers = hits->n_layers;
  a.a_scale = float(kCLight * double(ctx->cfg.bz_tesla));
  a.v0 = a.v1 = ctx->cfg.sigma_xy_cm * ctx->cfg.sigma_xy_cm;
  a.v2 = ctx->cfg.sigma_z_cm * ctx->cfg.sigma_z_cm;
  for (int l = 0; l < hits->n_layers; ++l) {
    a.R[l] = ctx->radius[l];
    a.x_x0[l] = ctx->x_x0[l];
  }
  a.mass = ctx->mass;
  KF_CUDA_TRY(ctx, launch_fit_fused(a, static_cast<cudaStream_t>(stream), upd64));
  return KF_OK;
}

int kf_fit_f64(kf_ctx* ctx, const kf_tracks_f64* seeds, const kf_track_hits* hits, kf_tracks_f64* out,
               double* chi2, int32_t* status, const int64_t* event_off, int32_t n_events, void* stream) {
  if (!ctx || !seeds || !hits || !out || !event_off || n_events < 0) return KF_EINVAL;
  const int64_t n = seeds->n;
  if (n < 0 || out->n != n || hits->n_tracks != n) return KF_EINVAL;
  if (n > 0 && (!seeds->par || !seeds->cov || !seeds->charge || !out->par || !out->cov || !hits->xyz))
    return KF_EINVAL;
  if (hits->n_layers < 1 || hits->n_layers > ctx->cfg.n_layers) return KF_EINVAL;
  if (event_off[0] != 0 || event_off[n_events] != n) return KF_EINVAL;
  for (int e = 0; e < n_events; ++e)
    if (event_off[e + 1] < event_off[e]) return KF_EINVAL;
  if (n == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  int32_t* st = status;
  if (!st) {
    int rc = scratch_reserve(ctx, ctx->s_status, size_t(n) * sizeof(int32_t));
    if (rc) return rc;
    st = static_cast<int32_t*>(ctx->s_status.ptr);
  }
  const double bz = ctx->cfg.bz_tesla;
  const double sxy = ctx->cfg.sigma_xy_cm, sz = ctx->cfg.sigma_z_cm;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int L = hits->n_layers;
  for (int e = 0; e < n_events; ++e) {
    for (int l = 0; l < L; ++l) {
      FitF64Args a;
      a.in_par = l == 0 ? seeds->par : out->par;
      a.in_cov = l == 0 ? seeds->cov : out->cov;
      a.charge = seeds->charge;
      a.out_par = out->par;
      a.out_cov = out->cov;
      a.hit = hits->xyz + int64_t(l) * 3 * n;
      a.valid = hits->valid ? hits->valid + int64_t(l) * n : nullptr;
      a.chi2 = chi2 ? chi2 + int64_t(l) * n : nullptr;
      a.status = st;
      a.n = n;
      a.begin = event_off[e];
      a.end = event_off[e + 1];
      a.a_scale = kCLight * bz;
      a.R = double(ctx->radius[l]);
      a.x_x0 = double(ctx->x_x0[l]);
      a.mass = double(ctx->mass);
      a.v0 = a.v1 = sxy * sxy;
      a.v2 = sz * sz;
      a.first = l == 0;
      a.last = l == L - 1;
      KF_CUDA_TRY(ctx, launch_fit_f64(a, s));
    }
  }
  return KF_OK;
}

int kf_fit_host(kf_ctx* ctx, const kf_tracks* seeds, const kf_track_hits* hits, kf_tracks* out, float* chi2,
                int32_t* status, void* stream) {
  int rc = check_fit(ctx, seeds, hits, out);
  if (rc) return rc;
  const int64_t n = seeds->n;
  if (n == 0) return KF_OK;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int L = hits->n_layers;
  // The batch is cut into chunks of C tracks; chunk j runs on internal stream
  // j % S with its own device staging slot: strided 2-D copies of its columns
  // in, its kf_fit, 2-D copies out.  Copies in, copies out and the fit of
  // different chunks overlap; a track's result does not depend on its batch.
  const int64_t C = std::max<int64_t>(kHostChunkMin, ((n + kHostChunks - 1) / kHostChunks + 255) / 256 * 256);
  const int64_t n_chunks = (n + C - 1) / C;
  const int S = int(std::min<int64_t>(kHostStreams, n_chunks));
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_par = al(6 * C * 4), b_lo = al(3 * C * 4), b_cov = al(21 * C * 4), b_hit = al(size_t(3) * L * C * 4),
               b_q = al(C), b_val = al(size_t(L) * C), b_chi = al(size_t(L) * C * 4), b_st = al(C * 4);
  const size_t in_bytes = b_par + b_lo + b_cov + b_hit + b_q + b_val;
  const size_t out_bytes = b_par + b_lo + b_cov + b_chi + b_st;
  rc = scratch_reserve(ctx, ctx->s_host_in, in_bytes * S);
  if (rc) return rc;
  rc = scratch_reserve(ctx, ctx->s_host_out, out_bytes * S);
  if (rc) return rc;
  for (int k = 0; k < kHostStreams; ++k) {
    if (!ctx->host_streams[k]) KF_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->host_streams[k], cudaStreamNonBlocking));
    if (!ctx->host_done[k]) KF_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->host_done[k], cudaEventDisableTiming));
  }
  if (!ctx->host_start) KF_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->host_start, cudaEventDisableTiming));
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  KF_CUDA_TRY(ctx, cudaEventRecord(ctx->host_start, user));
  for (int k = 0; k < S; ++k) KF_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->host_streams[k], ctx->host_start, 0));
  const size_t hp = size_t(n) * 4;  // host row pitch of a float component
  for (int64_t j = 0; j < n_chunks; ++j) {
    const int k = int(j % S);
    cudaStream_t s = ctx->host_streams[k];
    const int64_t j0 = j * C, c = std::min(C, n - j0);
    const size_t w = size_t(c) * 4;  // device row pitch of this chunk
    char* di = static_cast<char*>(ctx->s_host_in.ptr) + in_bytes * k;
    char* dout = static_cast<char*>(ctx->s_host_out.ptr) + out_bytes * k;
    kf_tracks ds{c, reinterpret_cast<float*>(di), seeds->par_lo ? reinterpret_cast<float*>(di + b_par) : nullptr,
                 reinterpret_cast<float*>(di + b_par + b_lo),
                 reinterpret_cast<int8_t*>(di + b_par + b_lo + b_cov + b_hit)};
    float* dhit = reinterpret_cast<float*>(di + b_par + b_lo + b_cov);
    uint8_t* dval = hits->valid ? reinterpret_cast<uint8_t*>(di + b_par + b_lo + b_cov + b_hit + b_q) : nullptr;
    kf_tracks dt{c, reinterpret_cast<float*>(dout), reinterpret_cast<float*>(dout + b_par),
                 reinterpret_cast<float*>(dout + b_par + b_lo), ds.charge};
    float* dchi = reinterpret_cast<float*>(dout + b_par + b_lo + b_cov);
    int32_t* dst = reinterpret_cast<int32_t*>(dout + b_par + b_lo + b_cov + b_chi);
    auto h2d = [&](void* d, const void* h, size_t width, size_t rows, size_t hpitch) {
      return cudaMemcpy2DAsync(d, width, h, hpitch, width, rows, cudaMemcpyHostToDevice, s);
    };
    auto d2h = [&](void* h, const void* d, size_t width, size_t rows, size_t hpitch) {
      return cudaMemcpy2DAsync(h, hpitch, d, width, width, rows, cudaMemcpyDeviceToHost, s);
    };
    KF_CUDA_TRY(ctx, h2d(ds.par, seeds->par + j0, w, 6, hp));
    if (seeds->par_lo) KF_CUDA_TRY(ctx, h2d(ds.par_lo, seeds->par_lo + j0, w, 3, hp));
    KF_CUDA_TRY(ctx, h2d(ds.cov, seeds->cov + j0, w, 21, hp));
    KF_CUDA_TRY(ctx, cudaMemcpyAsync(ds.charge, seeds->charge + j0, size_t(c), cudaMemcpyHostToDevice, s));
    KF_CUDA_TRY(ctx, h2d(dhit, hits->xyz + j0, w, size_t(3) * L, hp));
    if (dval) KF_CUDA_TRY(ctx, h2d(dval, hits->valid + j0, size_t(c), size_t(L), size_t(n)));
    kf_track_hits dh{c, L, dhit, dval};
    rc = kf_fit(ctx, &ds, &dh, &dt, dchi, dst, s);
    if (rc) return rc;
    KF_CUDA_TRY(ctx, d2h(out->par + j0, dt.par, w, 6, hp));
    if (out->par_lo) KF_CUDA_TRY(ctx, d2h(out->par_lo + j0, dt.par_lo, w, 3, hp));
    KF_CUDA_TRY(ctx, d2h(out->cov + j0, dt.cov, w, 21, hp));
    if (out->charge && out->charge != seeds->charge)
      KF_CUDA_TRY(ctx, cudaMemcpyAsync(out->charge + j0, ds.charge, size_t(c), cudaMemcpyDeviceToHost, s));
    if (chi2) KF_CUDA_TRY(ctx, d2h(chi2 + j0, dchi, w, size_t(L), hp));
    if (status) KF_CUDA_TRY(ctx, cudaMemcpyAsync(status + j0, dst, w, cudaMemcpyDeviceToHost, s));
  }
  for (int k = 0; k < S; ++k) {
    KF_CUDA_TRY(ctx, cudaEventRecord(ctx->host_done[k], ctx->host_streams[k]));
    KF_CUDA_TRY(ctx, cudaStreamWaitEvent(user, ctx->host_done[k], 0));
  }
  KF_CUDA_TRY(ctx, cudaStreamSynchronize(user));
  return KF_OK;
}

}  // extern "C"

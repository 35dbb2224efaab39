// kf_serve.cu -- continuous-batching service for the combinatorial build.
//
// The paper's building runs event by event on CPU threads and names load
// balancing across threads (uneven occupancy per event) and dynamic
// scheduling as the open problems (Sec. 3.2, Sec. 4).  On one GPU the same
// problem becomes: keep the device full while events of very different size
// arrive at random times.  The scheduler thread here
//   * admits queued events in arrival order whenever a slot and a contiguous
//     block of the device arena are free (memory-based admission),
//   * prepares the events admitted in one iteration together, on one of
//     several preparation streams: their input copies, then one seed-fit
//     launch over all their seeds and one binning launch over all their hit
//     segments (and for the layer-stepping layouts each event's seed
//     ordering and first candidates),
//   * issues ONE build-step launch per iteration over every resident event,
//     each at its own layer (the slot table tells each block its event,
//     layer, buffers and hit bins), so candidates stay resident on the device
//     between layers and small events ride along with big ones -- or, with
//     the register-resident layout, ONE launch per iteration that takes every
//     event prepared since the last one through all its building layers (a
//     table of batches tells each warp group its event),
//   * selects the best candidate of finished events, copies their results to
//     pinned host memory asynchronously and recycles their slot and memory.
// Steps run on one stream, preparations and the finishing of events (final
// selection, result copies) on their own; an event joins the steps only once
// the host has seen its preparation complete, and its finishing waits for its
// last step by a CUDA event.  The host never waits on a device flag (it polls CUDA
// events) and runs at most kInflight iterations ahead of the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kf_bin.cuh"
#include "kf_build.cuh"
#include "kf_internal.h"

namespace kfi {

using Clock = std::chrono::steady_clock;

// First-fit allocator over an address range [0, size).
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0, peak_ = 0;
};

// Host threads that share the large copies of kf_submit: staging an event in
// pinned memory is a few MB, and one thread copies at ~15 GB/s, far below
// what the host memory delivers; the submitting thread takes chunks too and
// returns when all of its event's chunks are done.
class CopyPool {
 public:
  struct Piece {
    void* dst;
    const void* src;
    size_t bytes;
  };
  void start(int n_threads) {
    for (int i = 0; i < n_threads; ++i) threads_.emplace_back([this] { worker(); });
  }
  void stop() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
    threads_.clear();
  }
  void copy(const Piece* pieces, int n_pieces) {
    Job job;
    std::vector<Chunk> chunks;
    for (int p = 0; p < n_pieces; ++p)
      for (size_t o = 0; o < pieces[p].bytes; o += kChunk) {
        const size_t b = std::min(kChunk, pieces[p].bytes - o);
        chunks.push_back({static_cast<char*>(pieces[p].dst) + o, static_cast<const char*>(pieces[p].src) + o, b, &job});
      }
    if (chunks.size() <= 1 || threads_.empty()) {
      for (const Chunk& c : chunks) std::memcpy(c.dst, c.src, c.bytes);
      return;
    }
    job.left = int(chunks.size());
    {
      std::lock_guard<std::mutex> lk(mu_);
      for (const Chunk& c : chunks) q_.push_back(c);
    }
    cv_.notify_all();
    while (true) {  // help until the queue is empty, then wait for this job
      Chunk c;
      {
        std::lock_guard<std::mutex> lk(mu_);
        if (q_.empty()) break;
        c = q_.front();
        q_.pop_front();
      }
      run(c);
    }
    std::unique_lock<std::mutex> lk(job.m);
    job.cv.wait(lk, [&] { return job.left == 0; });
  }

 private:
  static constexpr size_t kChunk = size_t(1) << 20;
  struct Job {
    std::mutex m;
    std::condition_variable cv;
    int left = 0;
  };
  struct Chunk {
    char* dst;
    const char* src;
    size_t bytes;
    Job* job;
  };
  static void run(const Chunk& c) {
    std::memcpy(c.dst, c.src, c.bytes);
    std::lock_guard<std::mutex> lk(c.job->m);
    if (--c.job->left == 0) c.job->cv.notify_all();
  }
  void worker() {
    while (true) {
      Chunk c;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
        if (q_.empty()) return;  // stopping
        c = q_.front();
        q_.pop_front();
      }
      run(c);
    }
  }
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Chunk> q_;
  std::vector<std::thread> threads_;
  bool stop_ = false;
};

enum ReqState { kQueued, kPreparing, kResident, kFinishing, kDone, kFailed };

// Byte layout of one event inside the device arena and the host arena.
struct EventLayout {
  int64_t n, nh;
  int ns, Lb;
  bool refit, fine;
  // device offsets
  size_t d_par, d_cov, d_q, d_shits, d_sval, d_fpar, d_flo, d_fcov, d_fst, d_xyz, d_segoff, d_sseg, d_bhits, d_boff,
      d_bid, d_perm, d_candA, d_candB, d_hp, d_hh, d_rpar, d_rcov, d_rchi, d_rnh, d_rst, d_rhit, d_qpar, d_qcov,
      d_qchi, d_qst, d_gxyz, d_gval, d_bcur, d_sboff, d_fine, d_total;
  // host input / output block offsets
  size_t h_par, h_cov, h_q, h_shits, h_sval, h_xyz, h_segoff, h_in_total;
  size_t o_par, o_cov, o_chi, o_nh, o_st, o_hit, o_qpar, o_qcov, o_qchi, o_qst, h_out_total;

  void make(int64_t n_, int64_t nh_, int ns_, int Lb_, bool refit_, bool fine_) {
    n = n_;
    nh = nh_;
    ns = ns_;
    Lb = Lb_;
    refit = refit_;
    fine = fine_;
    const size_t L = size_t(ns + Lb);
    size_t o = 0;
    auto take = [&](size_t b) {
      const size_t at = o;
      o += (b + 255) & ~size_t(255);
      return at;
    };
    d_par = take(6 * n * 4);
    d_cov = take(21 * n * 4);
    d_q = take(n);
    d_shits = take(size_t(ns) * 3 * n * 4);
    d_sval = take(size_t(ns) * n);
    d_fpar = take(6 * n * 4);
    d_flo = take(3 * n * 4);
    d_fcov = take(21 * n * 4);
    d_fst = take(n * 4);
    d_xyz = take(3 * nh * 4);
    d_segoff = take((Lb + 1) * 8 + 2 * 8);  // layer offsets, then the seed segment {0, n}
    d_sseg = d_segoff + (Lb + 1) * 8;
    d_bhits = take(nh * 16);
    d_boff = take(size_t(Lb) * (KF_NBINS + 1) * 4);
    d_bid = take(std::max<int64_t>(nh, n) * 4);
    d_perm = take(n * 4);
    d_candA = take(cand_bytes(n));
    d_candB = take(cand_bytes(n));
    d_hp = take(size_t(Lb) * n * kGroup);
    d_hh = take(size_t(Lb) * n * kGroup * 4);
    d_rpar = take(6 * n * 4);
    d_rcov = take(21 * n * 4);
    d_rchi = take(n * 4);
    d_rnh = take(n * 4);
    d_rst = take(n * 4);
    d_rhit = take(size_t(Lb) * n * 4);
    // re-fit results follow the build results (one contiguous copy back)
    d_qpar = take(refit ? 6 * n * 4 : 0);
    d_qcov = take(refit ? 21 * n * 4 : 0);
    d_qchi = take(refit ? L * n * 4 : 0);
    d_qst = take(refit ? n * 4 : 0);
    d_gxyz = take(refit ? L * 3 * n * 4 : 0);
    d_gval = take(refit ? L * n : 0);
    d_bcur = take(size_t(Lb) * KF_NBINS * 4);     // binning cursors (hits, then seeds)
    d_sboff = take(size_t(KF_NBINS + 1) * 4);  // seed bin offsets
    d_fine = take(fine ? size_t(Lb) * (KF_NBINS_FINE + 1) * 4 : 0);  // hit sub-bin starts (register-resident build)
    d_total = o;
    o = 0;
    h_par = take(6 * n * 4);
    h_cov = take(21 * n * 4);
    h_q = take(n);
    h_shits = take(size_t(ns) * 3 * n * 4);
    h_sval = take(size_t(ns) * n);
    h_xyz = take(3 * nh * 4);
    h_segoff = take((Lb + 1) * 8 + 16);  // layer offsets, then the seed segment {0, n}
    h_in_total = o;
    o = 0;
    o_par = take(6 * n * 4);
    o_cov = take(21 * n * 4);
    o_chi = take(n * 4);
    o_nh = take(n * 4);
    o_st = take(n * 4);
    o_hit = take(size_t(Lb) * n * 4);
    o_qpar = take(refit ? 6 * n * 4 : 0);
    o_qcov = take(refit ? 21 * n * 4 : 0);
    o_qchi = take(refit ? L * n * 4 : 0);
    o_qst = take(refit ? n * 4 : 0);
    h_out_total = o;
  }
};

struct Request {
  uint64_t ticket = 0;
  EventLayout lay;
  ReqState state = kQueued;
  int layer = 0;  // next build layer
  size_t d_off = 0, h_in_off = 0, h_out_off = 0;
  bool has_d = false, has_in = false, has_out = false;
  cudaEvent_t done = nullptr;      // results on the host
  cudaEvent_t prepped = nullptr;   // preparation finished (prep stream)
  Clock::time_point t_submit, t_admit, t_done;
};

constexpr int kInflight = 2;  // iterations the host may run ahead of the GPU
constexpr int kPrepStreams = 4;
constexpr int kRing = kInflight + 2;
// one ring entry of the launch tables: per-layer step slots, or the batches
// of a register-resident launch
constexpr size_t kTableBytes = std::max(sizeof(BuildSlot), 2 * sizeof(ResidentBatch)) * KF_MAX_SLOTS;

// The preparation of the events admitted in one iteration is batched: their
// seed fits in one launch, their hit segments' binning in another, from
// tables of per-event pointers (kPrepRing slots, each reused only once the
// batch that last used it has completed, by its event).
constexpr int kPrepRing = 8;
constexpr size_t kPrepFitBytes = sizeof(FitEvent) * KF_MAX_SLOTS;
constexpr size_t kPrepBytes = kPrepFitBytes + sizeof(BinSegment) * KF_MAX_SLOTS * kMaxLayers;
constexpr size_t kCounterBytes = 256;

// With more than one lane a seed, a register-resident build runs its first
// layer (one candidate a seed) with one thread per seed, seeds -> buffer B,
// and the rest from buffer B into buffer A; else one launch, seeds -> B.
inline bool resident_split(const kf_serve_config& c) {
  return resident_lanes(c.max_cands) > 1 && c.n_build_layers > 1;
}

struct Serve {
  kf_ctx* ctx = nullptr;
  kf_serve_config cfg{};
  std::mutex mu;
  std::condition_variable cv;  // wakes the scheduler
  std::condition_variable done_cv;  // wakes pollers
  std::thread thread;
  bool stop = false;
  int cuda_error = 0;
  cudaStream_t stream = nullptr;       // build steps
  cudaStream_t finish_stream = nullptr;  // final selection, re-fit and result copies
  cudaEvent_t step_ev[kRing] = {};       // after the step launch of an iteration
  // preparation of admitted events, round-robin over kPrepStreams streams:
  // an event's preparation is a few small copies and launches, so several
  // run at once, beside the steps
  cudaStream_t prep_stream[kPrepStreams] = {};
  int prep_next = 0;
  // events in the order their work was issued on each in-order stream: the
  // scheduler queries only the oldest of each (scheduler thread only)
  std::deque<Request*> prep_order[kPrepStreams];
  std::deque<Request*> finish_order;
  char* dmem = nullptr;
  char* hmem = nullptr;
  Arena darena, harena;
  char* d_table = nullptr;  // [kRing] entries of kTableBytes, then [kPrepRing] of kPrepBytes, then
                            // [kRing] resident-build group counters of kCounterBytes
  char* h_table = nullptr;  // pinned, same shape
  cudaEvent_t prep_ev[kPrepRing] = {};  // after the batch that last used a preparation table slot
  int prep_slot = 0;
  cudaEvent_t iter_ev[kRing] = {};
  uint64_t next_ticket = 1;
  std::deque<Request*> queue;
  std::vector<Request*> resident;  // resident or finishing
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  kf_serve_stats stats{};
  kf_tuning tune{};  // launch parameters in effect at kf_serve_start
  CopyPool copier;   // kf_submit's staging copies
};

static void fail_all_locked(Serve* sv, int err) {
  sv->cuda_error = err;
  for (auto& kv : sv->all)
    if (kv.second->state != kDone) kv.second->state = kFailed;
  sv->done_cv.notify_all();
}

// Enqueue the preparation of the events admitted in one iteration on one
// preparation stream (round-robin over kPrepStreams): each event's input
// copies, then ONE fused seed-fit launch over all their seeds and ONE
// binning launch over all their hit segments (tables of per-event pointers);
// with the layer-stepping layouts also each event's seed ordering and first
// candidates.  An event joins the builds once its r->prepped has completed.
static cudaError_t prepare_batch(Serve* sv, const std::vector<Request*>& rs) {
  if (rs.empty()) return cudaSuccess;
  kf_ctx* ctx = sv->ctx;
  // the register-resident build looks its windows up by sub-bin (every
  // event's layout then holds their starts)
  const bool sub_bins = sv->tune.build_scan == 4;
  const int ps = sv->prep_next;
  sv->prep_next = (ps + 1) % kPrepStreams;
  cudaStream_t s = sv->prep_stream[ps];
  // the table slot, once the batch that last used it is done with it
  const int slot = sv->prep_slot;
  sv->prep_slot = (slot + 1) % kPrepRing;
  cudaError_t e = cudaEventSynchronize(sv->prep_ev[slot]);
  if (e != cudaSuccess) return e;
  char* hslot = sv->h_table + kTableBytes * kRing + kPrepBytes * size_t(slot);
  char* dslot = sv->d_table + kTableBytes * kRing + kPrepBytes * size_t(slot);
  FitEvent* hf = reinterpret_cast<FitEvent*>(hslot);
  BinSegment* hb = reinterpret_cast<BinSegment*>(hslot + kPrepFitBytes);
  int64_t tracks = 0;
  int segs = 0;
  for (size_t k = 0; k < rs.size(); ++k) {
    Request* r = rs[k];
    const EventLayout& L = r->lay;
    char* d = sv->dmem + r->d_off;
    const char* h = sv->hmem + r->h_in_off;
    // the host input block mirrors the first device pieces (par .. sval); the
    // raw hits and their offsets follow in the host block and go to their own
    // device pieces
    e = cudaMemcpyAsync(d, h, L.h_xyz, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d + L.d_xyz, h + L.h_xyz, size_t(3) * L.nh * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)  // the layer offsets and the seed segment {0, n} (host block filled by kf_submit)
      e = cudaMemcpyAsync(d + L.d_segoff, h + L.h_segoff, size_t(L.Lb + 1) * 8 + 16, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // seed fit over the seeding layers
    FitEvent& f = hf[k];
    f.in_par = reinterpret_cast<const float*>(d + L.d_par);
    f.in_lo = nullptr;
    f.in_cov = reinterpret_cast<const float*>(d + L.d_cov);
    f.charge = reinterpret_cast<const int8_t*>(d + L.d_q);
    f.out_par = reinterpret_cast<float*>(d + L.d_fpar);
    f.out_lo = reinterpret_cast<float*>(d + L.d_flo);
    f.out_cov = reinterpret_cast<float*>(d + L.d_fcov);
    f.hits = reinterpret_cast<const float*>(d + L.d_shits);
    f.valid = reinterpret_cast<const uint8_t*>(d + L.d_sval);
    f.chi2 = nullptr;
    f.status = reinterpret_cast<int32_t*>(d + L.d_fst);
    f.n = L.n;
    f.begin = tracks;
    tracks += L.n;
    // hits into eta x phi bins, one segment per build layer (its range from
    // the host copy of the layer offsets)
    const int64_t* hoff = reinterpret_cast<const int64_t*>(h + L.h_segoff);
    for (int l = 0; l < L.Lb; ++l) {
      BinSegment& b = hb[segs++];
      b.xyz = reinterpret_cast<const float*>(d + L.d_xyz);
      b.stride = L.nh;
      b.p0 = hoff[l];
      b.p1 = std::min<int64_t>(hoff[l + 1], L.nh);
      b.bin_off = reinterpret_cast<int32_t*>(d + L.d_boff) + int64_t(l) * (KF_NBINS + 1);
      b.fine_off = L.fine ? reinterpret_cast<int32_t*>(d + L.d_fine) + int64_t(l) * (KF_NBINS_FINE + 1) : nullptr;
      b.out_pts = reinterpret_cast<float4*>(d + L.d_bhits);
      b.out_id = reinterpret_cast<int32_t*>(d + L.d_bid);
    }
  }
  FitEvent* df = reinterpret_cast<FitEvent*>(dslot);
  BinSegment* db = reinterpret_cast<BinSegment*>(dslot + kPrepFitBytes);
  e = cudaMemcpyAsync(df, hf, sizeof(FitEvent) * rs.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(db, hb, sizeof(BinSegment) * size_t(segs), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const int Ls = sv->cfg.n_seed_layers;
  FitFusedArgs fa;
  std::memset(&fa, 0, sizeof fa);
  fa.n_layers = Ls;
  fa.a_scale = float(kCLight * double(ctx->cfg.bz_tesla));
  fa.v0 = fa.v1 = ctx->cfg.sigma_xy_cm * ctx->cfg.sigma_xy_cm;
  fa.v2 = ctx->cfg.sigma_z_cm * ctx->cfg.sigma_z_cm;
  for (int l = 0; l < Ls; ++l) {
    fa.R[l] = ctx->radius[l];
    fa.x_x0[l] = ctx->x_x0[l];
  }
  fa.mass = ctx->mass;
  e = launch_fit_fused_table(fa, df, int(rs.size()), tracks, s);
  // the build's results do not depend on the order of the hits inside a bin
  if (e == cudaSuccess) e = launch_bin_segment_table(db, segs, sub_bins, s);
  if (e != cudaSuccess) return e;
  // (a register-resident build takes the seeds in their order, from the fit)
  for (size_t k = 0; k < rs.size() && sv->tune.build_scan != 4; ++k) {
    Request* r = rs[k];
    const EventLayout& L = r->lay;
    char* d = sv->dmem + r->d_off;
    const int64_t n = L.n;
    // seeds in (eta, phi) order: one segment [0, n) (copied with the layer offsets)
    BinArgs sb;
    sb.xyz = reinterpret_cast<const float*>(d + L.d_fpar);
    sb.stride = n;
    sb.seg_off = reinterpret_cast<const int64_t*>(d + L.d_sseg);
    sb.bin_off = reinterpret_cast<int32_t*>(d + L.d_sboff);
    sb.out_pts = nullptr;
    sb.out_id = reinterpret_cast<int32_t*>(d + L.d_perm);
    sb.out_seg = nullptr;
    sb.cursor = reinterpret_cast<int32_t*>(d + L.d_bcur);
    sb.unordered = 1;  // the build's results do not depend on the order inside a bin
    e = launch_bin_points(sb, 1, s);
    if (e != cudaSuccess) return e;
    BuildInitArgs ia;
    ia.out = cand_at(d + L.d_candA, n);
    ia.par = reinterpret_cast<const float*>(d + L.d_fpar);
    ia.lo = reinterpret_cast<const float*>(d + L.d_flo);
    ia.cov = reinterpret_cast<const float*>(d + L.d_fcov);
    ia.seed_perm = reinterpret_cast<const int32_t*>(d + L.d_perm);
    ia.n = n;
    ia.S = n;
    e = launch_build_init(ia, s);
    if (e != cudaSuccess) return e;
  }
  e = cudaEventRecord(sv->prep_ev[slot], s);
  for (Request* r : rs) {
    if (e == cudaSuccess) e = cudaEventRecord(r->prepped, s);
    sv->prep_order[ps].push_back(r);
  }
  return e;
}

static BuildSlot slot_of(Serve* sv, Request* r) {
  const EventLayout& L = r->lay;
  char* d = sv->dmem + r->d_off;
  const int64_t n = L.n;
  BuildSlot b;
  CandBuf A = cand_at(d + L.d_candA, n), B = cand_at(d + L.d_candB, n);
  b.in = (r->layer % 2 == 0) ? A : B;
  b.out = (r->layer % 2 == 0) ? B : A;
  b.hist_parent = reinterpret_cast<int8_t*>(d + L.d_hp) + int64_t(r->layer) * n * kGroup;
  b.hist_hit = reinterpret_cast<int32_t*>(d + L.d_hh) + int64_t(r->layer) * n * kGroup;
  b.seed_evt = nullptr;
  b.seed_perm = reinterpret_cast<const int32_t*>(d + L.d_perm);
  b.charge = reinterpret_cast<const int8_t*>(d + L.d_q);
  b.hits = reinterpret_cast<const float4*>(d + L.d_bhits);
  b.bin_off = reinterpret_cast<const int32_t*>(d + L.d_boff);
  b.seg_off = reinterpret_cast<const int64_t*>(d + L.d_segoff);
  b.S = n;
  b.layer = r->layer;
  b.n_layers = L.Lb;
  b.R = sv->ctx->radius[sv->cfg.n_seed_layers + r->layer];
  b.x_x0 = sv->ctx->x_x0[sv->cfg.n_seed_layers + r->layer];
  const int rm = rank_major_buffers(sv->cfg.max_cands, L.Lb);
  b.in_rm = r->layer < rm;
  b.out_rm = r->layer + 1 < rm;
  b.block_begin = 0;
  return b;
}

// An event as one batch of a register-resident launch: of the first-layer
// launch (first = true: the seeds -> buffer B), or of the launch over the
// other layers (buffer B -> buffer A, or the seeds -> buffer B when the build
// is not split), which also selects the best candidates.
static ResidentBatch resident_batch_of(Serve* sv, Request* r, bool first) {
  const EventLayout& L = r->lay;
  char* d = sv->dmem + r->d_off;
  const bool split = resident_split(sv->cfg);
  ResidentBatch b;
  b.in = cand_at(d + L.d_candB, L.n);
  b.out = cand_at(d + (split && !first ? L.d_candA : L.d_candB), L.n);
  b.hist_parent = reinterpret_cast<int8_t*>(d + L.d_hp);
  b.hist_hit = reinterpret_cast<int32_t*>(d + L.d_hh);
  b.seed_evt = nullptr;
  // seeds in their given order (one event's hits stay in L2 whatever the
  // order), read straight from the seed fit's output
  b.seed_perm = nullptr;
  b.charge = reinterpret_cast<const int8_t*>(d + L.d_q);
  b.hits = reinterpret_cast<const float4*>(d + L.d_bhits);
  b.bin_off = reinterpret_cast<const int32_t*>(d + L.d_boff);
  b.seg_off = reinterpret_cast<const int64_t*>(d + L.d_segoff);
  b.fine_off = L.fine ? reinterpret_cast<const int32_t*>(d + L.d_fine) : nullptr;
  b.S = L.n;
  b.group_begin = 0;
  b.seed_begin = 0;
  const bool seeds = first || !split;
  b.seed_par = seeds ? reinterpret_cast<const float*>(d + L.d_fpar) : nullptr;
  b.seed_lo = seeds ? reinterpret_cast<const float*>(d + L.d_flo) : nullptr;
  b.seed_cov = seeds ? reinterpret_cast<const float*>(d + L.d_fcov) : nullptr;
  // the last launch also selects the best candidates into the event's results
  std::memset(&b.res, 0, sizeof b.res);
  if (first) return b;
  b.res.best.n = L.n;
  b.res.best.par = reinterpret_cast<float*>(d + L.d_rpar);
  b.res.best.cov = reinterpret_cast<float*>(d + L.d_rcov);
  b.res.chi2_tot = reinterpret_cast<float*>(d + L.d_rchi);
  b.res.n_hits = reinterpret_cast<int32_t*>(d + L.d_rnh);
  b.res.status = reinterpret_cast<int32_t*>(d + L.d_rst);
  b.res.hit_idx = reinterpret_cast<int32_t*>(d + L.d_rhit);
  return b;
}

// Final selection (the paths alone after a register-resident launch) +
// asynchronous copy of the results to the pinned output block, on the finish
// stream (ordered after the event's last step by the caller), so that the
// next steps need not wait for it.
static cudaError_t finish(Serve* sv, Request* r) {
  const EventLayout& L = r->lay;
  char* d = sv->dmem + r->d_off;
  char* o = sv->hmem + r->h_out_off;
  const int64_t n = L.n;
  cudaStream_t s = sv->finish_stream;
  // after a register-resident launch (which selected the best candidates
  // itself and left the seeds' candidate counts in its last buffer) only the
  // paths; else the whole selection from the buffer the alternating steps
  // ended on
  const bool resident = sv->tune.build_scan == 4;
  const bool in_b = resident ? !resident_split(sv->cfg) : L.Lb % 2 == 1;
  BuildFinalArgs fa;
  std::memset(&fa, 0, sizeof fa);
  fa.cand = cand_at(d + (in_b ? L.d_candB : L.d_candA), n);
  fa.hist_parent = reinterpret_cast<const int8_t*>(d + L.d_hp);
  fa.hist_hit = reinterpret_cast<const int32_t*>(d + L.d_hh);
  fa.seed_perm = resident ? nullptr : reinterpret_cast<const int32_t*>(d + L.d_perm);
  fa.S = n;
  fa.n_layers = L.Lb;
  fa.max_cands = sv->cfg.max_cands;
  fa.rm_buffers = rank_major_buffers(sv->cfg.max_cands, L.Lb);
  fa.paths_only = resident ? (resident_defers_pd(sv->cfg.max_cands) ? 2 : 1) : 0;
  fa.out.best.n = n;
  fa.out.best.par = reinterpret_cast<float*>(d + L.d_rpar);
  fa.out.best.par_lo = nullptr;
  fa.out.best.cov = reinterpret_cast<float*>(d + L.d_rcov);
  fa.out.chi2_tot = reinterpret_cast<float*>(d + L.d_rchi);
  fa.out.n_hits = reinterpret_cast<int32_t*>(d + L.d_rnh);
  fa.out.status = reinterpret_cast<int32_t*>(d + L.d_rst);
  fa.out.hit_idx = reinterpret_cast<int32_t*>(d + L.d_rhit);
  cudaError_t e = launch_build_final(fa, s);
  if (e == cudaSuccess && L.refit) {
    // re-fit: every seed's hits over all layers, then one fused fit launch
    // from the vertex seed (the same arithmetic as kf_refit / kf_fit)
    RefitGatherArgs g;
    g.seed_xyz = reinterpret_cast<const float*>(d + L.d_shits);
    g.seed_valid = reinterpret_cast<const uint8_t*>(d + L.d_sval);
    g.seed_off = reinterpret_cast<const int64_t*>(d + L.d_sseg);
    g.hit_xyz = reinterpret_cast<const float*>(d + L.d_xyz);
    g.seg_off = reinterpret_cast<const int64_t*>(d + L.d_segoff);
    g.hit_idx = reinterpret_cast<const int32_t*>(d + L.d_rhit);
    g.xyz = reinterpret_cast<float*>(d + L.d_gxyz);
    g.valid = reinterpret_cast<uint8_t*>(d + L.d_gval);
    g.n = n;
    g.n_hits = L.nh;
    g.Ls = L.ns;
    g.Lb = L.Lb;
    g.E = 1;
    e = launch_refit_gather(g, s);
    if (e == cudaSuccess) {
      kf_ctx* ctx = sv->ctx;
      FitFusedArgs q;
      std::memset(&q, 0, sizeof q);
      q.in_par = reinterpret_cast<const float*>(d + L.d_par);
      q.in_lo = nullptr;
      q.in_cov = reinterpret_cast<const float*>(d + L.d_cov);
      q.charge = reinterpret_cast<const int8_t*>(d + L.d_q);
      q.out_par = reinterpret_cast<float*>(d + L.d_qpar);
      q.out_lo = nullptr;
      q.out_cov = reinterpret_cast<float*>(d + L.d_qcov);
      q.hits = g.xyz;
      q.valid = g.valid;
      q.chi2 = reinterpret_cast<float*>(d + L.d_qchi);
      q.status = reinterpret_cast<int32_t*>(d + L.d_qst);
      q.n = n;
      q.n_layers = L.ns + L.Lb;
      q.a_scale = float(kCLight * double(ctx->cfg.bz_tesla));
      q.v0 = q.v1 = ctx->cfg.sigma_xy_cm * ctx->cfg.sigma_xy_cm;
      q.v2 = ctx->cfg.sigma_z_cm * ctx->cfg.sigma_z_cm;
      for (int l = 0; l < L.ns + L.Lb; ++l) {
        q.R[l] = ctx->radius[l];
        q.x_x0[l] = ctx->x_x0[l];
      }
      q.mass = ctx->mass;
      e = launch_fit_fused(q, s);
    }
  }
  // results are contiguous on the device (rpar .. rhit, then the re-fit's)
  // and in the output block
  if (e == cudaSuccess) e = cudaMemcpyAsync(o, d + L.d_rpar, L.h_out_total, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(r->done, s);
  return e;
}

static void release_locked(Serve* sv, Request* r) {
  if (r->has_d) sv->darena.release(r->d_off, r->lay.d_total);
  if (r->has_in) sv->harena.release(r->h_in_off, r->lay.h_in_total);
  r->has_d = r->has_in = false;
}

static void scheduler(Serve* sv) {
  cudaSetDevice(sv->ctx->device);
  uint64_t iter = 0;
  // the thread's time split (kf_serve_stats.sched_*), accumulated in ns and
  // published with the other counters under the lock
  const Clock::time_point t_start = Clock::now();
  int64_t idle_ns = 0, gpu_wait_ns = 0;
  auto publish = [&]() {
    const int64_t all = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t_start).count();
    sv->stats.sched_idle_ms = 1e-6 * double(idle_ns);
    sv->stats.sched_gpu_wait_ms = 1e-6 * double(gpu_wait_ns);
    sv->stats.sched_busy_ms = 1e-6 * double(all - idle_ns - gpu_wait_ns);
  };
  std::vector<Request*> admitted;
  while (true) {
    admitted.clear();
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      // finished events: results are on the host.  The finish stream runs in
      // order, so the oldest unfinished event ends the look.
      while (!sv->finish_order.empty() && !sv->cuda_error) {
        Request* r = sv->finish_order.front();
        const cudaError_t q = cudaEventQuery(r->done);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) {
          fail_all_locked(sv, int(q));
          break;
        }
        sv->finish_order.pop_front();
        r->state = kDone;
        r->t_done = Clock::now();
        if (r->has_d) sv->darena.release(r->d_off, r->lay.d_total);
        r->has_d = false;
        sv->stats.completed++;
        sv->resident.erase(std::find(sv->resident.begin(), sv->resident.end(), r));
        sv->done_cv.notify_all();
      }
      // prepared events join the build steps (layer 0); each preparation
      // stream runs in order
      for (int ps = 0; ps < kPrepStreams && !sv->cuda_error; ++ps) {
        while (!sv->prep_order[ps].empty()) {
          Request* r = sv->prep_order[ps].front();
          const cudaError_t q = cudaEventQuery(r->prepped);
          if (q == cudaErrorNotReady) break;
          if (q != cudaSuccess) {
            fail_all_locked(sv, int(q));
            break;
          }
          sv->prep_order[ps].pop_front();
          r->state = kResident;
          r->layer = 0;
        }
      }
      if (sv->cuda_error) {
        sv->resident.clear();
        sv->queue.clear();
        sv->finish_order.clear();
        for (auto& q : sv->prep_order) q.clear();
      }
      // admission in arrival order: a free slot and a device block
      while (!sv->queue.empty() && int(sv->resident.size()) < sv->cfg.max_slots && !sv->cuda_error) {
        Request* r = sv->queue.front();
        size_t off = 0;
        if (!sv->darena.alloc(r->lay.d_total, &off)) break;
        sv->queue.pop_front();
        r->d_off = off;
        r->has_d = true;
        r->state = kPreparing;
        r->layer = 0;
        r->t_admit = Clock::now();
        sv->stats.admitted++;
        sv->resident.push_back(r);
        admitted.push_back(r);
      }
      bool active = false;
      for (Request* r : sv->resident) active |= r->state == kResident;
      bool finishing = false;  // (or preparing): the GPU will make progress without the host
      for (Request* r : sv->resident) finishing |= r->state == kFinishing || r->state == kPreparing;
      if (!active && admitted.empty()) {
        if (sv->stop && sv->queue.empty() && !finishing) break;
        const Clock::time_point w0 = Clock::now();
        if (finishing)
          sv->cv.wait_for(lk, std::chrono::microseconds(20));
        else
          sv->cv.wait_for(lk, std::chrono::milliseconds(50));
        idle_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - w0).count();
        publish();
        continue;
      }
      sv->stats.resident = int(sv->resident.size());
      sv->stats.max_resident = std::max(sv->stats.max_resident, sv->stats.resident);
      sv->stats.queued = int(sv->queue.size());
    }
    // ---- device work of this iteration (serve stream, no lock held)
    cudaError_t e = cudaSuccess;
    e = prepare_batch(sv, admitted);
    // pace: at most kInflight iterations ahead of the GPU
    const int ring = int(iter % kRing);
    if (e == cudaSuccess && iter >= uint64_t(kInflight)) {
      const Clock::time_point w0 = Clock::now();
      e = cudaEventSynchronize(sv->iter_ev[(iter - kInflight) % kRing]);
      gpu_wait_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - w0).count();
    }
    std::vector<Request*> stepping;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Request* r : sv->resident)
        if (r->state == kResident && r->layer < r->lay.Lb) stepping.push_back(r);
    }
    if (e == cudaSuccess && !stepping.empty() && sv->tune.build_scan == 4) {
      // the register-resident layout: one launch takes every event prepared
      // since the last one through all its building layers, each event one
      // batch of the table (the others wait for the next launch)
      // (the first layer by its own launch, one thread a seed, when split)
      const bool split = resident_split(sv->cfg);
      const size_t nb = stepping.size();
      ResidentBatch* ht = reinterpret_cast<ResidentBatch*>(sv->h_table + size_t(ring) * kTableBytes);
      ResidentBatch* hf = ht + KF_MAX_SLOTS;  // the first-layer launch's table
      const int G = resident_group(sv->cfg.max_cands);
      int64_t groups = 0, seeds = 0;
      for (size_t i = 0; i < nb; ++i) {
        ht[i] = resident_batch_of(sv, stepping[i], false);
        ht[i].group_begin = groups;
        groups += (ht[i].S + G - 1) / G;
        if (split) {
          hf[i] = resident_batch_of(sv, stepping[i], true);
          hf[i].seed_begin = seeds;
          seeds += hf[i].S;
        }
      }
      ResidentBatch* dt = reinterpret_cast<ResidentBatch*>(sv->d_table + size_t(ring) * kTableBytes);
      ResidentBatch* df = dt + KF_MAX_SLOTS;
      e = cudaMemcpyAsync(dt, ht, sizeof(ResidentBatch) * nb, cudaMemcpyHostToDevice, sv->stream);
      if (e == cudaSuccess && split)
        e = cudaMemcpyAsync(df, hf, sizeof(ResidentBatch) * nb, cudaMemcpyHostToDevice, sv->stream);
      BuildResidentArgs ra;
      std::memset(&ra, 0, sizeof ra);
      ra.n_batches = int(nb);
      const int Lb = sv->cfg.n_build_layers, Ls = sv->cfg.n_seed_layers;
      ra.n_layers = Lb;
      ra.max_cands = sv->cfg.max_cands;
      ra.rm_buffers = rank_major_buffers(ra.max_cands, Lb);
      ra.a_scale = float(kCLight * double(sv->ctx->cfg.bz_tesla));
      ra.v0 = ra.v1 = sv->ctx->cfg.sigma_xy_cm * sv->ctx->cfg.sigma_xy_cm;
      ra.v2 = sv->ctx->cfg.sigma_z_cm * sv->ctx->cfg.sigma_z_cm;
      ra.cut = sv->ctx->cfg.chi2_cut;
      ra.mass = sv->ctx->mass;
      for (int l = 0; l < Lb; ++l) {
        ra.R[l] = sv->ctx->radius[Ls + l];
        ra.x_x0[l] = sv->ctx->x_x0[Ls + l];
      }
      if (e == cudaSuccess && split) {
        BuildResidentArgs fl = ra;
        fl.table = df;
        fl.n_seeds = seeds;
        fl.l0 = 0;
        fl.in_rm = 1;  // (not read: the seeds themselves)
        fl.out_rm = 1 < ra.rm_buffers;
        e = launch_build_first_layer(fl, sv->stream);
      }
      ra.table = dt;
      ra.n_groups = groups;
      ra.group_counter = reinterpret_cast<unsigned long long*>(sv->d_table + kTableBytes * kRing +
                                                               kPrepBytes * kPrepRing + kCounterBytes * ring);
      if (e == cudaSuccess) e = cudaMemsetAsync(ra.group_counter, 0, sizeof(unsigned long long), sv->stream);
      ra.l0 = split ? 1 : 0;
      ra.in_rm = ra.l0 < ra.rm_buffers;
      ra.out_rm = Lb < ra.rm_buffers;
      if (e == cudaSuccess) e = launch_build_resident(ra, sv->ctx->num_sms, sv->stream);
      for (Request* r : stepping) r->layer = r->lay.Lb;
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stats.step_launches++;
    } else if (e == cudaSuccess && !stepping.empty()) {
      BuildSlot* ht = reinterpret_cast<BuildSlot*>(sv->h_table + size_t(ring) * kTableBytes);
      int64_t seeds = 0;
      for (size_t i = 0; i < stepping.size(); ++i) {
        ht[i] = slot_of(sv, stepping[i]);
        seeds += ht[i].S;
      }
      // A packed step spreads its seeds over one wave of resident blocks at
      // least; with fewer than about 80 seeds a block (by default: SMs x
      // resident blocks x 80 seeds) a block's rounds hold too few parents and
      // the grouped layout, 8 lanes per seed, ends such a small step sooner
      // (the same bits either way).
      int scan = sv->tune.build_scan;
      const int64_t pack_min = sv->cfg.pack_min_seeds > 0
                                   ? sv->cfg.pack_min_seeds
                                   : int64_t(sv->ctx->num_sms) * kBuildBlocksPerSM * 80;
      if (is_packed(scan) && seeds < pack_min) scan = 0;
      const int pack_seeds = build_pack_seeds(seeds, scan, sv->cfg.max_cands, sv->ctx->num_sms);
      int blocks = 0;
      for (size_t i = 0; i < stepping.size(); ++i) {
        ht[i].block_begin = blocks;
        blocks += pack_seeds > 0 ? int((ht[i].S + pack_seeds - 1) / pack_seeds) : build_step_blocks(ht[i].S, scan);
      }
      BuildSlot* dt = reinterpret_cast<BuildSlot*>(sv->d_table + size_t(ring) * kTableBytes);
      e = cudaMemcpyAsync(dt, ht, sizeof(BuildSlot) * stepping.size(), cudaMemcpyHostToDevice, sv->stream);
      BuildStepArgs a;
      a.slots = dt;
      a.n_slots = int(stepping.size());
      a.max_cands = sv->cfg.max_cands;
      a.a_scale = float(kCLight * double(sv->ctx->cfg.bz_tesla));
      a.v0 = a.v1 = sv->ctx->cfg.sigma_xy_cm * sv->ctx->cfg.sigma_xy_cm;
      a.v2 = sv->ctx->cfg.sigma_z_cm * sv->ctx->cfg.sigma_z_cm;
      a.cut = sv->ctx->cfg.chi2_cut;
      a.mass = sv->ctx->mass;
      a.pack_seeds = pack_seeds;
      a.layers = 0;  // events at different layers: one step each
      if (e == cudaSuccess)
        e = launch_build_step(a, blocks, sv->stream, sv->tune.build_hit_tile, sv->tune.build_list_width, scan);
      for (Request* r : stepping) r->layer++;
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stats.step_launches++;
    }
    if (e == cudaSuccess) {
      bool ordered = false;  // the finish stream waits for this iteration's step once
      for (Request* r : stepping)
        if (r->layer == r->lay.Lb && e == cudaSuccess) {
          if (!ordered) {
            e = cudaEventRecord(sv->step_ev[ring], sv->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->finish_stream, sv->step_ev[ring], 0);
            ordered = true;
          }
          if (e == cudaSuccess) e = finish(sv, r);
          std::lock_guard<std::mutex> lk(sv->mu);
          r->state = kFinishing;
          sv->finish_order.push_back(r);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(sv->iter_ev[ring], sv->stream);
    ++iter;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stats.iterations++;
    publish();
    if (e != cudaSuccess) {
      fail_all_locked(sv, int(e));
      sv->resident.clear();
      sv->queue.clear();
      sv->finish_order.clear();
      for (auto& q : sv->prep_order) q.clear();
    }
  }
}

}  // namespace kfi

using namespace kfi;

void kf_serve_shutdown_internal(kf_ctx* ctx) {
  if (!ctx || !ctx->serve) return;
  Serve* sv = ctx->serve;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (Request* r : sv->queue) {
      r->state = kFailed;
      sv->stats.cancelled++;
    }
    sv->queue.clear();
  }
  sv->cv.notify_all();
  if (sv->thread.joinable()) sv->thread.join();
  sv->copier.stop();
  cudaSetDevice(ctx->device);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  if (sv->finish_stream) cudaStreamSynchronize(sv->finish_stream);
  for (cudaStream_t ps : sv->prep_stream)
    if (ps) cudaStreamSynchronize(ps);
  for (auto& kv : sv->all) {
    if (kv.second->done) cudaEventDestroy(kv.second->done);
    if (kv.second->prepped) cudaEventDestroy(kv.second->prepped);
  }
  for (int i = 0; i < kRing; ++i) {
    if (sv->iter_ev[i]) cudaEventDestroy(sv->iter_ev[i]);
    if (sv->step_ev[i]) cudaEventDestroy(sv->step_ev[i]);
  }
  for (cudaEvent_t pe : sv->prep_ev)
    if (pe) cudaEventDestroy(pe);
  if (sv->dmem) cudaFree(sv->dmem);
  if (sv->d_table) cudaFree(sv->d_table);
  if (sv->hmem) cudaFreeHost(sv->hmem);
  if (sv->h_table) cudaFreeHost(sv->h_table);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  if (sv->finish_stream) cudaStreamDestroy(sv->finish_stream);
  for (cudaStream_t ps : sv->prep_stream)
    if (ps) cudaStreamDestroy(ps);
  ctx->allocated -= sv->darena.size();
  delete sv;
  ctx->serve = nullptr;
}

extern "C" {

int kf_serve_start(kf_ctx* ctx, const kf_serve_config* cfg) {
  if (!ctx || !cfg) return KF_EINVAL;
  if (ctx->serve) return KF_EAGAIN;
  if (cfg->n_seed_layers < 1 || cfg->n_build_layers < 1 ||
      cfg->n_seed_layers + cfg->n_build_layers > ctx->cfg.n_layers || cfg->n_seed_layers > kMaxLayers)
    return KF_EINVAL;
  if (cfg->max_cands < 1 || cfg->max_cands > kGroup || cfg->max_slots < 1 || cfg->max_slots > KF_MAX_SLOTS ||
      cfg->max_queue < 1 || (cfg->refit != 0 && cfg->refit != 1) || cfg->pack_min_seeds < 0)
    return KF_EINVAL;
  KF_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  auto* sv = new (std::nothrow) Serve();
  if (!sv) return KF_ENOMEM;
  sv->ctx = ctx;
  sv->cfg = *cfg;
  sv->tune = ctx->tune;
  const size_t dbytes = cfg->device_arena_bytes ? cfg->device_arena_bytes : (size_t(1) << 30);
  const size_t hbytes = cfg->host_arena_bytes ? cfg->host_arena_bytes : (size_t(1) << 30);
  int rc = KF_OK;
  if (ctx->budget && ctx->allocated + dbytes > ctx->budget) rc = KF_ENOMEM;
  if (!rc && cudaMalloc(&sv->dmem, dbytes) != cudaSuccess) rc = KF_ENOMEM;
  const size_t table_bytes = kTableBytes * kRing + kPrepBytes * kPrepRing + kCounterBytes * kRing;
  if (!rc && cudaMalloc(&sv->d_table, table_bytes) != cudaSuccess) rc = KF_ENOMEM;
  if (!rc && cudaHostAlloc(reinterpret_cast<void**>(&sv->hmem), hbytes, cudaHostAllocDefault) != cudaSuccess)
    rc = KF_ENOMEM;
  if (!rc && cudaHostAlloc(reinterpret_cast<void**>(&sv->h_table), table_bytes, cudaHostAllocDefault) != cudaSuccess)
    rc = KF_ENOMEM;
  if (!rc && cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) rc = KF_ECUDA;
  if (!rc && cudaStreamCreateWithFlags(&sv->finish_stream, cudaStreamNonBlocking) != cudaSuccess) rc = KF_ECUDA;
  for (int i = 0; i < kPrepStreams && !rc; ++i)
    if (cudaStreamCreateWithFlags(&sv->prep_stream[i], cudaStreamNonBlocking) != cudaSuccess) rc = KF_ECUDA;
  for (int i = 0; i < kRing && !rc; ++i)
    if (cudaEventCreateWithFlags(&sv->iter_ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&sv->step_ev[i], cudaEventDisableTiming) != cudaSuccess)
      rc = KF_ECUDA;
  for (int i = 0; i < kPrepRing && !rc; ++i)
    if (cudaEventCreateWithFlags(&sv->prep_ev[i], cudaEventDisableTiming) != cudaSuccess) rc = KF_ECUDA;
  if (rc) {
    cudaGetLastError();
    if (sv->dmem) cudaFree(sv->dmem);
    if (sv->d_table) cudaFree(sv->d_table);
    if (sv->hmem) cudaFreeHost(sv->hmem);
    if (sv->h_table) cudaFreeHost(sv->h_table);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    if (sv->finish_stream) cudaStreamDestroy(sv->finish_stream);
    for (cudaStream_t ps : sv->prep_stream)
      if (ps) cudaStreamDestroy(ps);
    for (int i = 0; i < kRing; ++i) {
      if (sv->iter_ev[i]) cudaEventDestroy(sv->iter_ev[i]);
      if (sv->step_ev[i]) cudaEventDestroy(sv->step_ev[i]);
    }
    for (cudaEvent_t pe : sv->prep_ev)
      if (pe) cudaEventDestroy(pe);
    delete sv;
    return rc;
  }
  sv->darena.reset(dbytes);
  sv->harena.reset(hbytes);
  sv->stats.device_arena_bytes = dbytes;
  ctx->allocated += dbytes;
  ctx->serve = sv;
  const int hw = int(std::thread::hardware_concurrency());
  sv->copier.start(std::max(1, std::min(6, hw / 2 - 1)));
  sv->thread = std::thread(scheduler, sv);
  return KF_OK;
}

int kf_serve_stop(kf_ctx* ctx) {
  if (!ctx || !ctx->serve) return KF_EINVAL;
  kf_serve_shutdown_internal(ctx);
  return KF_OK;
}

int kf_submit(kf_ctx* ctx, const kf_event* ev, uint64_t* ticket) {
  if (!ctx || !ev || !ticket) return KF_EINVAL;
  Serve* sv = ctx->serve;
  if (!sv) return KF_EINVAL;
  const int ns = sv->cfg.n_seed_layers, Lb = sv->cfg.n_build_layers;
  const int64_t n = ev->n_seeds;
  if (n < 1 || !ev->seed_par || !ev->seed_cov || !ev->seed_charge || !ev->seed_hits || !ev->layer_off)
    return KF_EINVAL;
  if (ev->layer_off[0] != 0) return KF_EINVAL;
  for (int l = 0; l < Lb; ++l) {
    const int64_t c = ev->layer_off[l + 1] - ev->layer_off[l];
    if (c < 0 || c > KF_MAX_HITS_PER_SEGMENT) return KF_EINVAL;
  }
  const int64_t nh = ev->layer_off[Lb];
  if (nh > 0 && !ev->layer_xyz) return KF_EINVAL;
  auto req = std::make_unique<Request>();
  req->lay.make(n, nh, ns, Lb, sv->cfg.refit != 0, sv->tune.build_scan == 4);
  const EventLayout& L = req->lay;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->cuda_error) return KF_ECUDA;
    if (L.d_total > sv->darena.size() || L.h_in_total + L.h_out_total + 512 > sv->harena.size()) return KF_ENOMEM;
    if (int(sv->queue.size()) >= sv->cfg.max_queue) return KF_EAGAIN;
    if (!sv->harena.alloc(L.h_in_total, &req->h_in_off)) return KF_EAGAIN;
    if (!sv->harena.alloc(L.h_out_total, &req->h_out_off)) {
      sv->harena.release(req->h_in_off, L.h_in_total);
      return KF_EAGAIN;
    }
    req->has_in = req->has_out = true;
  }
  // stage the event in its pinned input block (layout mirrors the device block)
  char* h = sv->hmem + req->h_in_off;
  CopyPool::Piece pieces[7];
  int np = 0;
  pieces[np++] = {h + L.h_par, ev->seed_par, size_t(6) * n * 4};
  pieces[np++] = {h + L.h_cov, ev->seed_cov, size_t(21) * n * 4};
  pieces[np++] = {h + L.h_q, ev->seed_charge, size_t(n)};
  pieces[np++] = {h + L.h_shits, ev->seed_hits, size_t(ns) * 3 * n * 4};
  if (ev->seed_valid)
    pieces[np++] = {h + L.h_sval, ev->seed_valid, size_t(ns) * n};
  else
    std::memset(h + L.h_sval, 1, size_t(ns) * n);
  if (nh > 0) pieces[np++] = {h + L.h_xyz, ev->layer_xyz, size_t(3) * nh * 4};
  pieces[np++] = {h + L.h_segoff, ev->layer_off, size_t(Lb + 1) * 8};
  sv->copier.copy(pieces, np);
  const int64_t sseg[2] = {0, n};  // seed segment, right after the layer offsets (padding room)
  std::memcpy(h + L.h_segoff + size_t(Lb + 1) * 8, sseg, sizeof sseg);
  cudaSetDevice(ctx->device);
  if (cudaEventCreateWithFlags(&req->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&req->prepped, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (req->done) cudaEventDestroy(req->done);
    if (req->prepped) cudaEventDestroy(req->prepped);
    std::lock_guard<std::mutex> lk(sv->mu);
    release_locked(sv, req.get());
    sv->harena.release(req->h_out_off, L.h_out_total);
    return KF_ECUDA;
  }
  req->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    req->ticket = sv->next_ticket++;
    *ticket = req->ticket;
    sv->queue.push_back(req.get());
    sv->stats.submitted++;
    sv->all.emplace(req->ticket, std::move(req));
  }
  sv->cv.notify_all();
  return KF_OK;
}

int kf_poll(kf_ctx* ctx, uint64_t ticket, kf_event_result* out, int64_t timeout_us) {
  if (!ctx || !ctx->serve || !out) return KF_EINVAL;
  Serve* sv = ctx->serve;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return KF_EINVAL;
  Request* r = it->second.get();
  auto ready = [&] { return r->state == kDone || r->state == kFailed; };
  if (!ready()) {
    if (timeout_us == 0) return KF_ETIMEDOUT;
    if (timeout_us < 0)
      sv->done_cv.wait(lk, ready);
    else if (!sv->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
      return KF_ETIMEDOUT;
  }
  if (r->state == kFailed) {
    release_locked(sv, r);
    if (r->has_out) sv->harena.release(r->h_out_off, r->lay.h_out_total);
    r->has_out = false;
    if (r->done) cudaEventDestroy(r->done);
    if (r->prepped) cudaEventDestroy(r->prepped);
    sv->all.erase(it);
    return KF_ECUDA;
  }
  const EventLayout& L = r->lay;
  const char* o = sv->hmem + r->h_out_off;
  const int64_t n = L.n;
  if (out->best_par) std::memcpy(out->best_par, o + L.o_par, 6 * n * 4);
  if (out->best_cov) std::memcpy(out->best_cov, o + L.o_cov, 21 * n * 4);
  if (out->chi2_tot) std::memcpy(out->chi2_tot, o + L.o_chi, n * 4);
  if (out->n_hits) std::memcpy(out->n_hits, o + L.o_nh, n * 4);
  if (out->status) std::memcpy(out->status, o + L.o_st, n * 4);
  if (out->hit_idx) std::memcpy(out->hit_idx, o + L.o_hit, size_t(L.Lb) * n * 4);
  if (L.refit) {
    const size_t Lall = size_t(L.ns + L.Lb);
    if (out->refit_par) std::memcpy(out->refit_par, o + L.o_qpar, 6 * n * 4);
    if (out->refit_cov) std::memcpy(out->refit_cov, o + L.o_qcov, 21 * n * 4);
    if (out->refit_chi2) std::memcpy(out->refit_chi2, o + L.o_qchi, Lall * n * 4);
    if (out->refit_status) std::memcpy(out->refit_status, o + L.o_qst, n * 4);
  }
  out->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  out->queued_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
  release_locked(sv, r);
  sv->harena.release(r->h_out_off, L.h_out_total);
  r->has_out = false;
  if (r->done) cudaEventDestroy(r->done);
  if (r->prepped) cudaEventDestroy(r->prepped);
  sv->all.erase(it);
  return KF_OK;
}

int kf_cancel(kf_ctx* ctx, uint64_t ticket) {
  if (!ctx || !ctx->serve) return KF_EINVAL;
  Serve* sv = ctx->serve;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return KF_EINVAL;
  Request* r = it->second.get();
  if (r->state != kQueued) return KF_EAGAIN;
  sv->queue.erase(std::remove(sv->queue.begin(), sv->queue.end(), r), sv->queue.end());
  release_locked(sv, r);
  if (r->has_out) sv->harena.release(r->h_out_off, r->lay.h_out_total);
  if (r->done) cudaEventDestroy(r->done);
  if (r->prepped) cudaEventDestroy(r->prepped);
  sv->stats.cancelled++;
  sv->all.erase(it);
  return KF_OK;
}

int kf_serve_stats_get(kf_ctx* ctx, kf_serve_stats* out) {
  if (!ctx || !ctx->serve || !out) return KF_EINVAL;
  Serve* sv = ctx->serve;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->device_arena_peak = sv->darena.peak();
  out->resident = int(sv->resident.size());
  out->queued = int(sv->queue.size());
  return KF_OK;
}

}  // extern "C"

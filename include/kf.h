/*
 * kf.h -- C ABI of libkf: Kalman-filter track fitting and combinatorial track
 * building on one GPU (Cerati et al., "Kalman Filter Tracking on Parallel
 * Architectures", CTD2016).
 *
 * Conventions for every entry point:
 *  - Units: cm, GeV, tesla.  A track state is (x, y, z, px, py, pz).
 *  - Layouts are structure-of-arrays: component c of track i is at
 *    ptr[c * n + i].  Covariances are packed lower triangles, row-major:
 *    element (i, j), j <= i, is component i(i+1)/2 + j of 21.
 *  - Positions may carry a low-order part: the position is the unevaluated
 *    float sum par[0..2] + par_lo[0..2] (|lo| <= half an ulp of hi).  Inputs
 *    with par_lo == NULL are read as lo = 0.
 *  - Pointers named "device" are CUDA device (or managed) memory of the
 *    context's device; the caller owns every buffer it passes and the library
 *    never frees caller memory.  `stream` is a cudaStream_t (NULL = legacy
 *    default stream); calls are asynchronous on it unless stated otherwise.
 *  - Return value: KF_OK (0) or a negative KF_E* code; no C++ exception
 *    crosses this interface.  KF_ECUDA leaves the CUDA error in
 *    kf_last_cuda_error().
 *  - A kf_ctx is not thread-safe; use one per host thread.
 *  - The fit calls, kf_bin_hits and kf_build draw on separate context
 *    scratch: one call of each kind may be in flight at once, each on its own
 *    stream (a call that grows its scratch -- the first of a larger size --
 *    reallocates it, which synchronises the device).  Two fit calls, or two
 *    calls of one kind, on different streams race on that kind's scratch.
 */
#ifndef KF_H_
#define KF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KF_OK 0
#define KF_EINVAL (-1)    /* bad argument: null pointer, size, layout */
#define KF_ENOMEM (-2)    /* device memory or the context budget exhausted */
#define KF_EAGAIN (-3)    /* not admitted / result not ready yet */
#define KF_ETIMEDOUT (-4) /* a wait ran out */
#define KF_ECUDA (-5)     /* a CUDA runtime call failed */
#define KF_ENOTSUP (-6)   /* not supported on this device / build */

/* Per-track status bits (int32 status words). */
#define KF_ST_NOT_REACHED 1 /* the helix never reaches the next layer radius;
                               the track stops there */
#define KF_ST_NEWTON_FAIL 2 /* the path-length solve did not converge; stops */
#define KF_ST_TANGENT 4     /* crossing within direction cosine 0.01 of the
                               tangent (dg/ds ~ 0); stops */
#define KF_ST_NOT_PD 8      /* final covariance failed the positive-definite check */
#define KF_ST_NO_HIT 16     /* at least one layer had no hit (propagated only) */
#define KF_ST_DEVICE_TIMEOUT 64 /* a bounded wait for staged input gave up (never expected).
                                 If any track of a call carries it, treat every result of
                                 that call as invalid: a block whose final drain wait also
                                 gave up may have exited with a copy still in flight into
                                 shared memory that a later block then uses */
#define KF_ST_STOPPED (KF_ST_NOT_REACHED | KF_ST_NEWTON_FAIL | KF_ST_TANGENT | KF_ST_DEVICE_TIMEOUT)

typedef struct kf_ctx kf_ctx;

/* Detector and algorithm constants (copied by kf_create). */
typedef struct {
    float bz_tesla;          /* uniform solenoidal field along z (non-zero) */
    int32_t n_layers;        /* barrel layers, 1 .. 64 */
    const float *radius_cm;  /* [n_layers] host, strictly increasing, > 0 */
    float sigma_xy_cm;       /* transverse hit smear (x and y each) */
    float sigma_z_cm;        /* longitudinal hit smear */
    float chi2_cut;          /* building: keep hits with chi2 increment < cut */
    int32_t max_cands;       /* building: candidates kept per seed, 1 .. 8 */
    /* Material (multiple scattering as process noise, Sec. 2): thickness of
     * each layer in radiation lengths at normal incidence, [n_layers] host,
     * each in [0, 1), or NULL for no material; and the particle mass (GeV,
     * >= 0) of the scattering model.  After every propagation to a layer
     * with material the momentum covariance gains theta0^2 (p^2 I - p p^T),
     * theta0 the Highland formula with the Lynch-Dahl logarithm (Review of
     * Particle Physics) over x/X0 / cos(incidence). */
    const float *x_x0;
    float mass_gev;
} kf_config;

/* A batch of tracks, single precision (device pointers). */
typedef struct {
    int64_t n;
    float *par;     /* [6][n] */
    float *par_lo;  /* [3][n] low parts of x, y, z, or NULL */
    float *cov;     /* [21][n] packed lower triangle */
    int8_t *charge; /* [n] +1 or -1 */
} kf_tracks;

/* A batch of tracks, double precision (device pointers), for kf_fit_f64. */
typedef struct {
    int64_t n;
    double *par;    /* [6][n] */
    double *cov;    /* [21][n] */
    int8_t *charge; /* [n] */
} kf_tracks_f64;

/* The hits of a fixed hit set, one per track and layer (device pointers). */
typedef struct {
    int64_t n_tracks;
    int32_t n_layers;     /* fit layers 0 .. n_layers-1 of the configuration */
    const float *xyz;     /* [n_layers][3][n_tracks] */
    const uint8_t *valid; /* [n_layers][n_tracks], 0 = no hit; NULL = all hits */
} kf_track_hits;

/* Create a context on CUDA device `device`.  `mem_budget_bytes` bounds the
 * device memory the context itself allocates (0 = no bound). */
int kf_create(kf_ctx **out, const kf_config *cfg, int device, size_t mem_budget_bytes);

/* Destroy a context (synchronises the device work it issued). */
void kf_destroy(kf_ctx *ctx);

/* Message for a KF_* return code (static storage). */
const char *kf_strerror(int code);

/* Last CUDA error code recorded by a KF_ECUDA return of this context. */
int kf_last_cuda_error(const kf_ctx *ctx);

/*
 * Track fit (Sec. 2 of the paper: with the hit set fixed after building, the
 * filter is applied layer by layer without branching).  For every track and
 * layer l = 0 .. hits->n_layers-1: propagate the helix to radius[l] (Newton
 * solve for the path length, surface transport Jacobian J, C' = J C J^T);
 * if the hit is valid, chi2[l] = r^T S^-1 r with r = m - H x',
 * S = H C' H^T + V, then the Kalman update with the symmetrised Joseph form.
 *
 * seeds (device, read only), out (device, written; may alias seeds),
 * chi2 [n_layers][n] (device, -1 where no update happened, may be NULL),
 * status [n] (device, KF_ST_* bits, may be NULL).
 * out->par_lo may be NULL (then the low parts are dropped on output).
 * Executed as one graph of n_layers kernel launches (one per layer step),
 * captured once per argument set and replayed.
 * Errors: KF_EINVAL (sizes, null pointers, n_layers > config),
 * KF_ENOMEM (scratch), KF_ECUDA.
 */
int kf_fit(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *hits, kf_tracks *out,
           float *chi2, int32_t *status, void *stream);

/* Same result as kf_fit, computed by a single launch that keeps each track in
 * registers across all layers (no per-layer state round trip). */
int kf_fit_fused(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *hits, kf_tracks *out,
                 float *chi2, int32_t *status, void *stream);

/* kf_fit_fused with mixed precision: propagation, transport and residuals in
 * FP32 (position pairs), the 3x3 inverse of S = H C' H^T + V, the gain and the
 * Joseph covariance downdate in FP64.  The precision comparison form. */
int kf_fit_mixed(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *hits, kf_tracks *out,
                 float *chi2, int32_t *status, void *stream);

/* The plain double-precision form of the same fit: the same steps in FP64,
 * launched once per event and per layer (events = contiguous track ranges
 * event_off[e] .. event_off[e+1], host array [n_events+1]).
 * seeds/out (device, may alias), chi2 [n_layers][n] double (may be NULL),
 * status [n] (may be NULL). */
int kf_fit_f64(kf_ctx *ctx, const kf_tracks_f64 *seeds, const kf_track_hits *hits,
               kf_tracks_f64 *out, double *chi2, int32_t *status, const int64_t *event_off,
               int32_t n_events, void *stream);

/* kf_fit with HOST buffers: copies the inputs to context-owned device
 * buffers, fits, copies the results back, and synchronises `stream`.
 * All pointers in seeds/hits/out/chi2/status are host memory (pinned memory
 * gives full copy bandwidth). */
int kf_fit_host(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *hits, kf_tracks *out,
                float *chi2, int32_t *status, void *stream);

/* ---------------------------------------------------------------------------
 * Combinatorial track building (Sec. 3): spatial hit bins, chi2 windows and
 * the clone engine.
 */

/* Hit bins per layer: directionally projective eta x phi bins (Sec. 3).
 * eta = asinh(z / r) over [-KF_BIN_ETA_MAX, KF_BIN_ETA_MAX) in KF_BIN_ETA
 * bins (points beyond go to the edge bins), phi = atan2(y, x) over [-pi, pi)
 * in KF_BIN_PHI bins.  Bin b = ieta * KF_BIN_PHI + iphi. */
#define KF_BIN_ETA 64
#define KF_BIN_PHI 256
#define KF_BIN_ETA_MAX 1.5f
#define KF_NBINS (KF_BIN_ETA * KF_BIN_PHI)
/* An optional finer phi look-up inside each eta row: KF_BIN_PHI_FINE sub-bins
 * over [-pi, pi) (sub-bin 2 iphi and 2 iphi + 1 split phi bin iphi in two).
 * Sub-bin c = ieta * KF_BIN_PHI_FINE + iphi_fine. */
#define KF_BIN_PHI_FINE (2 * KF_BIN_PHI)
#define KF_NBINS_FINE (KF_BIN_ETA * KF_BIN_PHI_FINE)
/* Largest number of hits in one (event, layer) segment. */
#define KF_MAX_HITS_PER_SEGMENT ((1 << 21) - 2)

/* Raw hits of a batch of events on the building layers (device pointers).
 * Segment s = e * n_layers + l holds the hits of event e on build layer l
 * (configuration layer first_layer + l): xyz[c][seg_off[s] .. seg_off[s+1]).
 * A hit's id is its index within its segment. */
typedef struct {
    int32_t n_events;
    int32_t n_layers;        /* building layers */
    int32_t first_layer;     /* configuration index of build layer 0 */
    int64_t n_hits;          /* seg_off[n_events * n_layers] */
    const float *xyz;        /* [3][n_hits] */
    const int64_t *seg_off;  /* [n_events * n_layers + 1], device */
} kf_layer_hits;

/* Binned hits (output of kf_bin_hits, input of kf_build; device pointers).
 * Within each segment the hits are ordered by bin, and by id inside a bin;
 * with kf_tuning.bin_unordered in no order inside a bin, or, with fine_off
 * set, by sub-bin and in no order inside a sub-bin. */
typedef struct {
    int32_t n_events;
    int32_t n_layers;
    int32_t first_layer;
    int64_t n_hits;
    float *hits;             /* [n_hits][4]: x, y, z, and the hit id (int32 bits) */
    int32_t *bin_off;        /* [n_events * n_layers][KF_NBINS + 1]: bin starts within the segment */
    const int64_t *seg_off;  /* [n_events * n_layers + 1], as in kf_layer_hits */
    int32_t *fine_off;       /* optional (NULL: none): [n_events * n_layers][KF_NBINS_FINE + 1]
                                sub-bin starts within the segment; filled by kf_bin_hits (which
                                then requires kf_tuning.bin_unordered = 1), used by kf_build to
                                narrow each window row to the sub-bins it reaches */
} kf_layer_hit_bins;

/* Sort every segment's hits into the eta x phi bins (Sec. 3: hits sorted in
 * phi within eta bins per layer, phi bins for fast look-up): a counting sort
 * over all segments at once (count, per-segment scan, scatter, then an id
 * sort inside each bin, so the order is deterministic), or with
 * kf_tuning.bin_unordered one block per segment and no id sort (with
 * `out->fine_off` set: by sub-bin, and the sub-bin starts written too).
 * `out->hits`, `out->bin_off` (and `out->fine_off`) are caller-allocated with
 * the sizes above; the other fields of `out` are set from `in`.  Segments must hold at most KF_MAX_HITS_PER_SEGMENT hits (not
 * checked here: seg_off is device memory; kf_build ignores hits beyond it).
 * Errors: KF_EINVAL (sizes, null pointers), KF_ECUDA. */
int kf_bin_hits(kf_ctx *ctx, const kf_layer_hits *in, kf_layer_hit_bins *out, void *stream);

/* Result of kf_build (device pointers, caller-allocated). */
typedef struct {
    kf_tracks best;          /* [n_seeds] best candidate: par, par_lo (may be NULL), cov;
                                best.charge is not written (charge does not change) */
    float *chi2_tot;         /* [n_seeds] sum of the chi2 increments of the kept hits */
    int32_t *n_hits;         /* [n_seeds] hits added on the building layers */
    int32_t *status;         /* [n_seeds] KF_ST_* bits of the best candidate */
    int32_t *hit_idx;        /* [n_layers][n_seeds] hit id per build layer, -1 = none */
    /* optional (NULL to skip): every candidate alive after the last layer,
     * in rank order, candidate k of seed i at i * max_cands + k */
    int32_t *n_cands;        /* [n_seeds] */
    int32_t *cand_hit_idx;   /* [n_layers][n_seeds * max_cands], -1 = none or absent */
    float *cand_chi2_tot;    /* [n_seeds * max_cands] */
    int32_t *cand_n_hits;    /* [n_seeds * max_cands] */
} kf_build_result;

/*
 * Combinatorial track building with the clone engine (Sec. 3).  For build
 * layer l = 0 .. bins->n_layers-1, every live candidate of every seed is
 * propagated to the layer radius; the chi2 increment of every hit in its
 * window is computed; every hit with chi2 < cfg.chi2_cut becomes a child
 * (parent, hit, chi2_tot, nHits) in a bookkeeping list, and a candidate with
 * no such hit gives one child without a hit (propagated, not updated).  The
 * children of a seed are ranked by (nHits desc, chi2_tot asc, parent rank
 * asc, hit id asc) and only the best max_cands are copied and updated.
 * max_cands = 1 is the best-hit approach.  The window is the set of bins
 * that a hit with chi2 < cut can fall in (chi2 >= (u.r)^2 / (u^T S u) for
 * every direction u), each bound widened by 0.1 % plus 1e-6 rad / 1e-5 cm
 * against rounding, so binning never changes the result.  The
 * register-resident layout (kf_tuning.build_scan 4) takes the seeds in their
 * given order, the others in (eta, phi) bin order within each event; the
 * results do not depend on the order.  With bins->fine_off set (the sub-bin
 * starts kf_bin_hits wrote for these hits) the register-resident layout
 * takes each window's phi range in sub-bins, scanning fewer hits beyond its
 * edges; the other layouts use bin_off; the results are the same.
 *
 * seeds: [n_seeds] starting states at or inside the first build layer (the
 * seeds' charge is read); seeds of event e are seed_off[e] .. seed_off[e+1]
 * (device, [n_events + 1]); bins: from kf_bin_hits; max_cands: 1 .. 8.
 * Scratch (candidates, histories) is taken from the context.
 * Errors: KF_EINVAL, KF_ENOMEM (budget), KF_ECUDA.
 */
int kf_build(kf_ctx *ctx, const kf_tracks *seeds, const int64_t *seed_off, const kf_layer_hit_bins *bins,
             int32_t max_cands, kf_build_result *out, void *stream);

/* Result of kf_build_f64 (device pointers, caller-allocated). */
typedef struct {
    kf_tracks_f64 best;      /* [n_seeds] best candidate: par, cov (best.charge is not written) */
    double *chi2_tot;        /* [n_seeds] sum of the chi2 increments of the kept hits */
    int32_t *n_hits;         /* [n_seeds] hits added on the building layers */
    int32_t *status;         /* [n_seeds] KF_ST_* bits of the best candidate */
    int32_t *hit_idx;        /* [n_layers][n_seeds] hit id per build layer, -1 = none */
} kf_build_result_f64;

/*
 * The plain double-precision form of the combinatorial build (Sec. 3): the
 * comparison form of kf_build, computing the same result in FP64 the
 * straightforward way -- one thread per seed taking its candidates in turn,
 * one launch per event and building layer, candidates in global memory
 * between layers, the window of every candidate derived and scanned in
 * double, the seed's best max_cands children kept in one sorted list, and
 * only those updated.  Seeds are processed in their given order (no
 * ordering by bin).
 * seeds: [n_seeds] double states (e.g. from kf_fit_f64 over the seeding
 * layers), seeds of event e = event_off[e] .. event_off[e+1] (HOST array,
 * [n_events + 1], event_off[0] = 0, event_off[n_events] = n_seeds); bins:
 * from kf_bin_hits; max_cands: 1 .. 8.  Scratch from the context.
 * Errors: KF_EINVAL, KF_ENOMEM, KF_ECUDA.
 */
int kf_build_f64(kf_ctx *ctx, const kf_tracks_f64 *seeds, const int64_t *event_off, const kf_layer_hit_bins *bins,
                 int32_t max_cands, kf_build_result_f64 *out, void *stream);

/*
 * Re-fit of built tracks: building (Sec. 3) followed by fitting (Sec. 2) over
 * all layers with the hits the build chose.  For seed i of event e, layer
 * l < seed_hits->n_layers uses seed_hits (the seeding-layer hits the build's
 * seeds were fitted with); building layer b uses hit hit_idx[b][i] (an id
 * within segment e * build_hits->n_layers + b of build_hits, -1 = no hit)
 * at layer seed_hits->n_layers + b.  The fit starts from `seeds` (the states
 * the build's seeds were fitted from) and runs as kf_fit over
 * seed_hits->n_layers + build_hits->n_layers layers (configuration radii
 * 0 ..; build_hits->first_layer must equal seed_hits->n_layers).
 * seed_off: [n_events + 1] (device), as for kf_build; hit_idx: [build
 * layers][n] (device), kf_build_result.hit_idx.  Outputs as kf_fit (chi2 has
 * one row per layer, -1 where there is no hit).  The gathered hits (13 bytes
 * per seed and layer) are context scratch.
 * Errors: KF_EINVAL (sizes, layer counts, null pointers), KF_ENOMEM, KF_ECUDA.
 */
int kf_refit(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *seed_hits, const int64_t *seed_off,
             const kf_layer_hits *build_hits, const int32_t *hit_idx, kf_tracks *out, float *chi2,
             int32_t *status, void *stream);

/* ---------------------------------------------------------------------------
 * Launch parameters and their autotuner.  They change speed only: every
 * setting gives bitwise the same results.  (The paper tunes its CPU code by
 * hand, Sec. 4; here the library measures on the caller's own batch.)
 */
typedef struct {
    int32_t fit_block;        /* threads per block of the kf_fit / kf_fit_noalloc layer
                                 kernel: 64 or 128 (default 128); 24 warps per SM either way */
    int32_t build_hit_tile;   /* hits staged in shared memory per warp by the kf_build step
                                 (bulk asynchronous copies of the window's bin rows):
                                 0 = none, the scans read global memory (default), or 512 */
    int32_t build_list_width; /* entries of a lane's child list in the kf_build step: 4 or 8
                                 (default 8); 4 takes effect only when max_cands <= 4 */
    int32_t build_scan;       /* thread layout of the kf_build step: 0 = 8 lanes per seed, each
                                 scanning its own candidate's window, 1 = 8 lanes per seed
                                 scanning each parent's window together (balanced when few
                                 candidates), 2 = the live candidates packed onto consecutive
                                 threads for the propagation and scan, and the kept children
                                 for the update, 128 seeds per block; 3 = the same with 64
                                 seeds per block; 4 = register-resident (default): each warp
                                 takes groups of 32 / W seeds (W = max_cands rounded up to 1,
                                 2, 4, 6 or 8 lanes a seed, the groups fetched in order from a
                                 counter) through the building layers, the candidates' states
                                 in registers between layers, in two launches when W > 1 (the
                                 first layer with one thread per seed, then the others) and
                                 the best candidates written after the last layer (2, 3 and 4
                                 require build_hit_tile 0; a serving loop with 4 builds each
                                 prepared event through all its layers in the launches shared
                                 with the events prepared with it, and with 0 .. 3 steps all
                                 resident events one layer a launch) */
    int32_t fit_chunk;        /* kf_fit: 0 = each layer step is one launch over the whole batch
                                 (default); 262144, 524288 or 1048576 = the batch is fitted in
                                 chunks of that many tracks, all layers of a chunk before the
                                 next, so the chunk's state stays in the L2 cache between its
                                 layer launches */
    int32_t fit_stage;        /* kf_fit layer step: 0 = every thread loads its track's rows
                                 (default), 1 = each warp's next 32 tracks are copied into shared
                                 memory by tensor copies while it computes the current ones
                                 (batches whose size is a multiple of 32 with 16-byte aligned
                                 rows; others take form 0) */
    int32_t bin_unordered;    /* kf_bin_hits: 0 = the hits of a bin in id order (default, a
                                 deterministic output), 1 = in the order the scatter pass left
                                 them (one pass less); kf_build's results do not depend on it */
} kf_tuning;

/* Current launch parameters of the context.  Errors: KF_EINVAL (null). */
int kf_get_tuning(const kf_ctx *ctx, kf_tuning *out);

/* Set the launch parameters for later calls.  A serving loop keeps those in
 * effect at kf_serve_start.  Errors: KF_EINVAL (null, or a value outside the
 * sets above; nothing is changed then). */
int kf_set_tuning(kf_ctx *ctx, const kf_tuning *t);

/* Autotuner of kf_fit: runs kf_fit on the caller's arguments once per
 * (fit_stage, fit_block, fit_chunk) value (one untimed call, then three timed with CUDA
 * events on `stream`, which is synchronised), keeps the fastest in the context (a
 * setting must beat the best so far by 2 % to replace it; the simplest come first)
 * and writes the context's tuning to *chosen (may be NULL).  The outputs hold the
 * result of the last call, identical for every value.  Errors: those of kf_fit. */
int kf_autotune_fit(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *hits, kf_tracks *out,
                    float *chi2, int32_t *status, void *stream, kf_tuning *chosen);

/* Autotuner of kf_build: the same over build_hit_tile x build_list_width x
 * build_scan (list width 4 is tried only when max_cands <= 4, layouts 2 and 3
 * only without hit staging).  Errors: those of kf_build. */
int kf_autotune_build(kf_ctx *ctx, const kf_tracks *seeds, const int64_t *seed_off,
                      const kf_layer_hit_bins *bins, int32_t max_cands, kf_build_result *out, void *stream,
                      kf_tuning *chosen);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of build requests (Sec. 3's per-event build,
 * run as a service).  Events of uneven size are admitted into resident slots
 * when a slot and device memory are free; every scheduler iteration issues
 * ONE build-step launch that advances every resident event by one layer
 * (events at different layers share the launch); finished events are copied
 * back asynchronously and their slots and memory reused.  Results do not
 * depend on what else is resident (per-seed arithmetic only).
 */
#define KF_MAX_SLOTS 64

typedef struct {
    int32_t n_seed_layers;      /* configuration layers 0 .. n_seed_layers-1 fit the seeds */
    int32_t n_build_layers;     /* the next n_build_layers layers are built */
    int32_t max_cands;          /* 1 .. 8 */
    int32_t max_slots;          /* resident events, 1 .. KF_MAX_SLOTS */
    int32_t max_queue;          /* submitted, not yet admitted events (>= 1) */
    int32_t refit;              /* 1: after the build, fit every seed's best candidate over all
                                   n_seed_layers + n_build_layers layers with its hits (as
                                   kf_refit) inside the same request; 0: build only */
    size_t device_arena_bytes;  /* device memory for resident events (0: 1 GiB) */
    size_t host_arena_bytes;    /* pinned host memory for queued inputs and results (0: 1 GiB) */
    int64_t pack_min_seeds;     /* with a candidate-packed build_scan (2, 3) in the context's
                                   tuning: a step launch uses it only when the resident events
                                   being stepped hold at least this many seeds, else the grouped
                                   per-lane layout (same results; a small packed step puts too
                                   few parents on a block).  0: automatic (SMs x 400),
                                   1: always packed.  >= 0 */
} kf_serve_config;

/* One event (host memory; copied by kf_submit, reusable when it returns). */
typedef struct {
    int32_t n_seeds;
    const float *seed_par;      /* [6][n_seeds] vertex seeds */
    const float *seed_cov;      /* [21][n_seeds] */
    const int8_t *seed_charge;  /* [n_seeds] */
    const float *seed_hits;     /* [n_seed_layers][3][n_seeds] hits on the seeding layers */
    const uint8_t *seed_valid;  /* [n_seed_layers][n_seeds], or NULL = all valid */
    const float *layer_xyz;     /* [3][n_hits] hits on the building layers, layer after layer */
    const int64_t *layer_off;   /* [n_build_layers + 1] segment offsets into layer_xyz */
} kf_event;

/* Where kf_poll writes a finished event (host memory; NULL fields skipped). */
typedef struct {
    float *best_par;        /* [6][n_seeds] best candidate (position hi parts) */
    float *best_cov;        /* [21][n_seeds] */
    float *chi2_tot;        /* [n_seeds] */
    int32_t *n_hits;        /* [n_seeds] */
    int32_t *status;        /* [n_seeds] */
    int32_t *hit_idx;       /* [n_build_layers][n_seeds], -1 = none */
    double latency_ms;      /* written: kf_submit -> results on the host */
    double queued_ms;       /* written: kf_submit -> admitted */
    /* re-fit results (kf_serve_config.refit = 1; L = n_seed_layers + n_build_layers) */
    float *refit_par;       /* [6][n_seeds] state at the last layer (position hi parts) */
    float *refit_cov;       /* [21][n_seeds] */
    float *refit_chi2;      /* [L][n_seeds] chi2 increment per layer, -1 where no hit */
    int32_t *refit_status;  /* [n_seeds] KF_ST_* bits of the re-fit */
} kf_event_result;

typedef struct {
    uint64_t submitted, admitted, completed, cancelled, iterations, step_launches;
    int32_t resident, queued, max_resident;
    size_t device_arena_bytes, device_arena_peak;
    /* the scheduler thread's time since kf_serve_start [ms]: issuing work and
     * bookkeeping, waiting for the GPU (the pacing wait on an iteration two
     * behind), and idle (nothing to issue: waiting for submissions or for
     * preparations and builds in flight) */
    double sched_busy_ms, sched_gpu_wait_ms, sched_idle_ms;
} kf_serve_stats;

/* Start the scheduler thread (one per context).  Allocates the arenas.
 * Errors: KF_EINVAL (config), KF_ENOMEM (arenas), KF_EAGAIN (already running). */
int kf_serve_start(kf_ctx *ctx, const kf_serve_config *cfg);

/* Queue an event; returns a ticket.  Thread-safe.  Errors: KF_EINVAL (sizes),
 * KF_ENOMEM (the event can never fit the device or host arena),
 * KF_EAGAIN (queue or host arena full now: retry later), KF_ECUDA (the loop
 * has failed). */
int kf_submit(kf_ctx *ctx, const kf_event *ev, uint64_t *ticket);

/* Wait up to timeout_us (< 0: forever, 0: do not wait) for a ticket; on
 * KF_OK the results are written to `out` and the ticket is released.
 * Errors: KF_ETIMEDOUT (not finished yet; the ticket stays valid),
 * KF_EINVAL (unknown ticket), KF_ECUDA (the event failed). */
int kf_poll(kf_ctx *ctx, uint64_t ticket, kf_event_result *out, int64_t timeout_us);

/* Cancel a ticket that has not been admitted yet (KF_OK); KF_EAGAIN if it is
 * already on the GPU (it will complete), KF_EINVAL if unknown. */
int kf_cancel(kf_ctx *ctx, uint64_t ticket);

int kf_serve_stats_get(kf_ctx *ctx, kf_serve_stats *out);

/* Stop the loop after the resident events finish; queued events are
 * cancelled; unpolled results are dropped.  kf_destroy stops it too. */
int kf_serve_stop(kf_ctx *ctx);

/* Test hook for the bounded waits of the staged layer kernel of kf_fit
 * (kf_tuning.fit_stage = 1).  The paper has no counterpart: it exists so that
 * a test can make a wait for staged input run out without any GPU fault.
 * After this call, kf_fit launches on this context do not issue the copies of
 * the 32-track tile `skip_tile` of the batch (tracks 32 skip_tile ..
 * 32 skip_tile + 31; -1 = none), so the warp that owns that tile waits in
 * vain until its poll limit: those tracks, and the warp's later tiles in the
 * same launch, get KF_ST_DEVICE_TIMEOUT; every other track's results are
 * unchanged.  `wait_polls` bounds each wait for staged input (0 = the normal
 * limit); the drain wait before a block exits keeps the normal limit, and
 * waits only for copies actually issued.  Affects kf_fit only.
 * Errors: KF_EINVAL (null context, skip_tile < -1). */
int kf_test_stage_fault(kf_ctx *ctx, int64_t skip_tile, uint32_t wait_polls);

/* Test hook for the bounded waits of kf_build's hit staging (kf_tuning
 * build_hit_tile > 0, grouped layouts 0 and 1).  The paper has no
 * counterpart.  After this call, in every layer-step launch of kf_build on
 * this context the warp of index `skip_warp` in the launch (seeds 4 skip_warp
 * .. 4 skip_warp + 3 in the build's seed order; -1 = none) issues none of the
 * copies of its window's hits and arms nothing, so its wait for them runs out:
 * those seeds' candidates stop with KF_ST_DEVICE_TIMEOUT (a warp whose
 * window does not fit its tile scans global memory and waits for nothing);
 * every other seed's results are unchanged.  `wait_polls` bounds each wait for
 * staged hits (0 = the normal limit); the drain before a warp ends waits only
 * for copies actually issued.  Errors: KF_EINVAL (null context,
 * skip_warp < -1). */
int kf_test_build_stage_fault(kf_ctx *ctx, int64_t skip_warp, uint32_t wait_polls);

/* ---------------------------------------------------------------------------
 * Measured arithmetic peaks: the roofline denominators of the kernels bound by
 * arithmetic.  The paper has no counterpart (it measures on CPUs).  Runs a
 * fused multiply-add microbenchmark on the context's device -- every thread
 * of a full-occupancy grid (8 blocks of 256 threads per SM) iterates
 * independent FMA chains -- as one warm-up and three timed launches of about
 * 10 ms on `stream` (synchronised), and writes the best rate in flop/s, an FMA
 * counted as two flops.  The rate is that of the SM clock during the launches;
 * callers that need a clock-independent figure sample the clock meanwhile.
 * kind: KF_PEAK_FP32 (single-precision FFMA) or KF_PEAK_FP64 (DFMA).
 * Allocates nothing.  Errors: KF_EINVAL (null, unknown kind), KF_ECUDA.
 */
#define KF_PEAK_FP32 0
#define KF_PEAK_FP64 1
int kf_measure_peak(kf_ctx *ctx, int32_t kind, void *stream, double *flop_per_s);

/* Largest batch (tracks) that kf_fit_noalloc accepts. */
#define KF_NOALLOC_MAX_TRACKS 262144

/*
 * kf_fit for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of kf_fit.
 *
 * Who needs it: a caller whose device memory is planned up front and must not
 * change afterwards -- e.g. an online trigger process that reserves all of the
 * GPU at start-up and treats any later cudaMalloc as a fault, a host framework
 * whose own caching allocator owns the device memory, or a plug-in that its
 * host application forbids to allocate.  kf_fit, when `status` or
 * `out->par_lo` is NULL, takes per-track scratch from the context and grows it
 * with cudaMalloc on first use; this entry point takes that scratch from a
 * fixed array in libkf's static device memory instead (KF_NOALLOC_MAX_TRACKS
 * x 16 bytes = 4 MiB, held by every GPU that loads the library until the
 * process exits) and performs no allocation or free of any kind.
 *
 * Arguments, layouts, results and errors are those of kf_fit, except:
 *  - seeds->n > KF_NOALLOC_MAX_TRACKS returns KF_EINVAL (split the batch);
 *  - the layer steps are issued as plain kernel launches on `stream`.
 * The first call on a device looks up the array's device address (with the
 * context's device current) and caches it; make that first call before any
 * stream capture begins.  The cached address does not survive a
 * cudaDeviceReset (which also invalidates every kf_ctx).  Every call shares the one array and leaves its
 * contents behind; each call's first layer launch rewrites what the later
 * launches read, so no clearing is needed.  Calls that overlap on the GPU
 * (other streams, other host threads) race on the array: serialise them.
 */
int kf_fit_noalloc(kf_ctx *ctx, const kf_tracks *seeds, const kf_track_hits *hits, kf_tracks *out,
                   float *chi2, int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KF_H_ */

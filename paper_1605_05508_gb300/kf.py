"""Python binding of libkf (include/kf.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: it packs torch tensors (device memory, or pinned host
memory for the *_host calls) into the ABI's plain structs and raises
`KfError` on a negative return code. PyTorch provides allocation and streams.

The CUDA library must have been built (`paper_1605_05508_gb300.build`); a
missing library raises immediately - there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkf.so")

KF_OK, KF_EINVAL, KF_ENOMEM, KF_EAGAIN, KF_ETIMEDOUT, KF_ECUDA, KF_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
ST_NOT_REACHED, ST_NEWTON_FAIL, ST_TANGENT, ST_NOT_PD, ST_NO_HIT, ST_DEVICE_TIMEOUT = 1, 2, 4, 8, 16, 64
ST_STOPPED = ST_NOT_REACHED | ST_NEWTON_FAIL | ST_TANGENT | ST_DEVICE_TIMEOUT
NOALLOC_MAX_TRACKS = 262144  # KF_NOALLOC_MAX_TRACKS


class KfError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class kf_config(C.Structure):
    _fields_ = [("bz_tesla", C.c_float), ("n_layers", C.c_int32), ("radius_cm", C.POINTER(C.c_float)),
                ("sigma_xy_cm", C.c_float), ("sigma_z_cm", C.c_float), ("chi2_cut", C.c_float),
                ("max_cands", C.c_int32), ("x_x0", C.POINTER(C.c_float)), ("mass_gev", C.c_float)]

PION_MASS = 0.13957  # GeV: default particle hypothesis of the scattering model


class kf_tracks(C.Structure):
    _fields_ = [("n", C.c_int64), ("par", C.c_void_p), ("par_lo", C.c_void_p), ("cov", C.c_void_p),
                ("charge", C.c_void_p)]


class kf_tracks_f64(C.Structure):
    _fields_ = [("n", C.c_int64), ("par", C.c_void_p), ("cov", C.c_void_p), ("charge", C.c_void_p)]


class kf_track_hits(C.Structure):
    _fields_ = [("n_tracks", C.c_int64), ("n_layers", C.c_int32), ("xyz", C.c_void_p), ("valid", C.c_void_p)]


class kf_layer_hits(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_layers", C.c_int32), ("first_layer", C.c_int32), ("n_hits", C.c_int64),
                ("xyz", C.c_void_p), ("seg_off", C.c_void_p)]


class kf_layer_hit_bins(C.Structure):
    _fields_ = [("n_events", C.c_int32), ("n_layers", C.c_int32), ("first_layer", C.c_int32), ("n_hits", C.c_int64),
                ("hits", C.c_void_p), ("bin_off", C.c_void_p), ("seg_off", C.c_void_p), ("fine_off", C.c_void_p)]


class kf_build_result(C.Structure):
    _fields_ = [("best", kf_tracks), ("chi2_tot", C.c_void_p), ("n_hits", C.c_void_p), ("status", C.c_void_p),
                ("hit_idx", C.c_void_p), ("n_cands", C.c_void_p), ("cand_hit_idx", C.c_void_p),
                ("cand_chi2_tot", C.c_void_p), ("cand_n_hits", C.c_void_p)]


class kf_serve_config(C.Structure):
    _fields_ = [("n_seed_layers", C.c_int32), ("n_build_layers", C.c_int32), ("max_cands", C.c_int32),
                ("max_slots", C.c_int32), ("max_queue", C.c_int32), ("refit", C.c_int32),
                ("device_arena_bytes", C.c_size_t), ("host_arena_bytes", C.c_size_t),
                ("pack_min_seeds", C.c_int64)]


class kf_event(C.Structure):
    _fields_ = [("n_seeds", C.c_int32), ("seed_par", C.c_void_p), ("seed_cov", C.c_void_p),
                ("seed_charge", C.c_void_p), ("seed_hits", C.c_void_p), ("seed_valid", C.c_void_p),
                ("layer_xyz", C.c_void_p), ("layer_off", C.c_void_p)]


class kf_event_result(C.Structure):
    _fields_ = [("best_par", C.c_void_p), ("best_cov", C.c_void_p), ("chi2_tot", C.c_void_p),
                ("n_hits", C.c_void_p), ("status", C.c_void_p), ("hit_idx", C.c_void_p),
                ("latency_ms", C.c_double), ("queued_ms", C.c_double), ("refit_par", C.c_void_p),
                ("refit_cov", C.c_void_p), ("refit_chi2", C.c_void_p), ("refit_status", C.c_void_p)]


class kf_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("iterations", C.c_uint64), ("step_launches", C.c_uint64),
                ("resident", C.c_int32), ("queued", C.c_int32), ("max_resident", C.c_int32),
                ("device_arena_bytes", C.c_size_t), ("device_arena_peak", C.c_size_t),
                ("sched_busy_ms", C.c_double), ("sched_gpu_wait_ms", C.c_double), ("sched_idle_ms", C.c_double)]


class kf_tuning(C.Structure):
    _fields_ = [("fit_block", C.c_int32), ("build_hit_tile", C.c_int32), ("build_list_width", C.c_int32),
                ("build_scan", C.c_int32), ("fit_chunk", C.c_int32), ("fit_stage", C.c_int32),
                ("bin_unordered", C.c_int32)]


MAX_SLOTS = 64  # KF_MAX_SLOTS
BIN_ETA, BIN_PHI, BIN_ETA_MAX = 64, 256, 1.5  # KF_BIN_ETA, KF_BIN_PHI, KF_BIN_ETA_MAX
NBINS = BIN_ETA * BIN_PHI
BIN_PHI_FINE = 2 * BIN_PHI  # KF_BIN_PHI_FINE
NBINS_FINE = BIN_ETA * BIN_PHI_FINE
MAX_HITS_PER_SEGMENT = (1 << 21) - 2  # KF_MAX_HITS_PER_SEGMENT

_lib = None


def lib() -> C.CDLL:
    """Load libkf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libkf is not built ({LIB_PATH} missing): run paper_1605_05508_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.kf_create.argtypes = [C.POINTER(vp), C.POINTER(kf_config), C.c_int, C.c_size_t]
        L.kf_destroy.argtypes = [vp]
        L.kf_destroy.restype = None
        L.kf_strerror.argtypes = [C.c_int]
        L.kf_strerror.restype = C.c_char_p
        L.kf_last_cuda_error.argtypes = [vp]
        for name in ("kf_fit", "kf_fit_fused", "kf_fit_host", "kf_fit_noalloc", "kf_fit_mixed"):
            getattr(L, name).argtypes = [vp, C.POINTER(kf_tracks), C.POINTER(kf_track_hits), C.POINTER(kf_tracks),
                                         vp, vp, vp]
        L.kf_fit_f64.argtypes = [vp, C.POINTER(kf_tracks_f64), C.POINTER(kf_track_hits), C.POINTER(kf_tracks_f64),
                                 vp, vp, C.POINTER(i64), i32, vp]
        L.kf_bin_hits.argtypes = [vp, C.POINTER(kf_layer_hits), C.POINTER(kf_layer_hit_bins), vp]
        L.kf_serve_start.argtypes = [vp, C.POINTER(kf_serve_config)]
        L.kf_serve_stop.argtypes = [vp]
        L.kf_submit.argtypes = [vp, C.POINTER(kf_event), C.POINTER(C.c_uint64)]
        L.kf_poll.argtypes = [vp, C.c_uint64, C.POINTER(kf_event_result), C.c_int64]
        L.kf_cancel.argtypes = [vp, C.c_uint64]
        L.kf_serve_stats_get.argtypes = [vp, C.POINTER(kf_serve_stats)]
        L.kf_build.argtypes = [vp, C.POINTER(kf_tracks), vp, C.POINTER(kf_layer_hit_bins), i32,
                               C.POINTER(kf_build_result), vp]
        L.kf_build_f64.argtypes = [vp, C.POINTER(kf_tracks_f64), vp, C.POINTER(kf_layer_hit_bins), i32,
                                   C.POINTER(kf_build_result_f64), vp]
        L.kf_refit.argtypes = [vp, C.POINTER(kf_tracks), C.POINTER(kf_track_hits), vp, C.POINTER(kf_layer_hits), vp,
                               C.POINTER(kf_tracks), vp, vp, vp]
        L.kf_get_tuning.argtypes = [vp, C.POINTER(kf_tuning)]
        L.kf_set_tuning.argtypes = [vp, C.POINTER(kf_tuning)]
        L.kf_autotune_fit.argtypes = [vp, C.POINTER(kf_tracks), C.POINTER(kf_track_hits), C.POINTER(kf_tracks),
                                      vp, vp, vp, C.POINTER(kf_tuning)]
        L.kf_measure_peak.argtypes = [vp, i32, vp, C.POINTER(C.c_double)]
        L.kf_test_stage_fault.argtypes = [vp, i64, C.c_uint32]
        L.kf_test_build_stage_fault.argtypes = [vp, i64, C.c_uint32]
        L.kf_autotune_build.argtypes = [vp, C.POINTER(kf_tracks), vp, C.POINTER(kf_layer_hit_bins), i32,
                                        C.POINTER(kf_build_result), vp, C.POINTER(kf_tuning)]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().kf_strerror(code).decode()
    except RuntimeError:
        return f"code {code}"


def _check(rc: int, what: str, ctx=None):
    if rc != KF_OK:
        err = KfError(rc, what)
        if rc == KF_ECUDA and ctx is not None:
            err.cuda_error = lib().kf_last_cuda_error(ctx)
        raise err


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


@dataclass
class Tracks:
    """SoA track batch: par [6, n], par_lo [3, n] or None, cov [21, n], charge [n] int8."""
    par: object
    cov: object
    charge: object
    par_lo: object = None

    @property
    def n(self) -> int:
        return int(self.par.shape[1])

    def abi(self) -> kf_tracks:
        return kf_tracks(self.n, _ptr(self.par), _ptr(self.par_lo), _ptr(self.cov), _ptr(self.charge))

    def abi_f64(self) -> kf_tracks_f64:
        return kf_tracks_f64(self.n, _ptr(self.par), _ptr(self.cov), _ptr(self.charge))


@dataclass
class TrackHits:
    """xyz [L, 3, n] float32, valid [L, n] uint8 or None."""
    xyz: object
    valid: object = None

    def abi(self) -> kf_track_hits:
        L, _, n = self.xyz.shape
        return kf_track_hits(n, L, _ptr(self.xyz), _ptr(self.valid))


class Context:
    """Owns a kf_ctx; `handle` is the opaque pointer."""

    def __init__(self, radii, bz=3.8, sigma_xy=0.01, sigma_z=0.1, chi2_cut=30.0, max_cands=6, device=0,
                 mem_budget_bytes=0, x_x0=None, mass=PION_MASS):
        """x_x0: per-layer thickness in radiation lengths (None: no material)."""
        self._radii = (C.c_float * len(radii))(*[float(r) for r in radii])
        self._x_x0 = None if x_x0 is None else (C.c_float * len(radii))(*[float(x) for x in x_x0])
        self.cfg = kf_config(float(bz), len(radii), self._radii, float(sigma_xy), float(sigma_z), float(chi2_cut),
                             int(max_cands), self._x_x0, float(mass))
        self.handle = kf_create(self.cfg, device, mem_budget_bytes)

    def close(self):
        if self.handle:
            kf_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kf_create(cfg: kf_config, device: int = 0, mem_budget_bytes: int = 0):
    h = C.c_void_p()
    _check(lib().kf_create(C.byref(h), C.byref(cfg), device, mem_budget_bytes), "kf_create")
    return h


def kf_destroy(handle):
    lib().kf_destroy(handle)


def _h(ctx):
    return ctx.handle if isinstance(ctx, Context) else ctx


def kf_fit(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, chi2=None, status=None, stream=None):
    s, h, o = seeds.abi(), hits.abi(), out.abi()
    _check(lib().kf_fit(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status), _stream(stream)),
           "kf_fit", _h(ctx))


def kf_fit_fused(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, chi2=None, status=None, stream=None):
    s, h, o = seeds.abi(), hits.abi(), out.abi()
    _check(lib().kf_fit_fused(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status),
                              _stream(stream)), "kf_fit_fused", _h(ctx))


def kf_fit_mixed(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, chi2=None, status=None, stream=None):
    s, h, o = seeds.abi(), hits.abi(), out.abi()
    _check(lib().kf_fit_mixed(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status),
                              _stream(stream)), "kf_fit_mixed", _h(ctx))


def kf_fit_host(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, chi2=None, status=None, stream=None):
    s, h, o = seeds.abi(), hits.abi(), out.abi()
    _check(lib().kf_fit_host(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status),
                             _stream(stream)), "kf_fit_host", _h(ctx))


def kf_fit_noalloc(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, chi2=None, status=None, stream=None):
    """kf_fit with its per-track scratch in libkf's static device memory: no
    allocation (batches up to NOALLOC_MAX_TRACKS)."""
    s, h, o = seeds.abi(), hits.abi(), out.abi()
    _check(lib().kf_fit_noalloc(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status),
                                _stream(stream)), "kf_fit_noalloc", _h(ctx))


def kf_fit_f64(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, event_off, chi2=None, status=None, stream=None):
    """event_off: sequence of n_events + 1 track offsets (host)."""
    offs = (C.c_int64 * len(event_off))(*[int(v) for v in event_off])
    s, h, o = seeds.abi_f64(), hits.abi(), out.abi_f64()
    _check(lib().kf_fit_f64(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status), offs,
                            len(event_off) - 1, _stream(stream)), "kf_fit_f64", _h(ctx))


@dataclass
class LayerHits:
    """Raw hits of the building layers: xyz [3, n_hits] float32, seg_off int64
    [n_events * n_layers + 1] (device), segment e * n_layers + l = event e on
    build layer l (configuration layer first_layer + l)."""
    xyz: object
    seg_off: object
    n_events: int
    n_layers: int
    first_layer: int

    def abi(self) -> kf_layer_hits:
        return kf_layer_hits(self.n_events, self.n_layers, self.first_layer, int(self.xyz.shape[1]), _ptr(self.xyz),
                             _ptr(self.seg_off))


@dataclass
class HitBins:
    """hits [n_hits, 4] float32 (x, y, z, id bits), bin_off [n_seg, NBINS + 1] int32, optional
    fine_off [n_seg, NBINS_FINE + 1] int32 (sub-bin starts)."""
    hits: object
    bin_off: object
    seg_off: object = None
    n_events: int = 0
    n_layers: int = 0
    first_layer: int = 0
    fine_off: object = None

    def abi(self) -> kf_layer_hit_bins:
        return kf_layer_hit_bins(self.n_events, self.n_layers, self.first_layer, int(self.hits.shape[0]),
                                 _ptr(self.hits), _ptr(self.bin_off), _ptr(self.seg_off), _ptr(self.fine_off))


@dataclass
class BuildResult:
    best: Tracks
    chi2_tot: object
    n_hits: object
    status: object
    hit_idx: object
    n_cands: object = None
    cand_hit_idx: object = None
    cand_chi2_tot: object = None
    cand_n_hits: object = None

    def abi(self) -> kf_build_result:
        return kf_build_result(self.best.abi(), _ptr(self.chi2_tot), _ptr(self.n_hits), _ptr(self.status),
                               _ptr(self.hit_idx), _ptr(self.n_cands), _ptr(self.cand_hit_idx),
                               _ptr(self.cand_chi2_tot), _ptr(self.cand_n_hits))


class kf_build_result_f64(C.Structure):
    _fields_ = [("best", kf_tracks_f64), ("chi2_tot", C.c_void_p), ("n_hits", C.c_void_p), ("status", C.c_void_p),
                ("hit_idx", C.c_void_p)]


@dataclass
class BuildResultF64:
    """Outputs of kf_build_f64: best (double par, cov), chi2_tot double, n_hits,
    status int32 [n], hit_idx int32 [n_layers, n]."""
    best: Tracks
    chi2_tot: object
    n_hits: object
    status: object
    hit_idx: object

    def abi(self) -> kf_build_result_f64:
        return kf_build_result_f64(self.best.abi_f64(), _ptr(self.chi2_tot), _ptr(self.n_hits), _ptr(self.status),
                                   _ptr(self.hit_idx))


def kf_bin_hits(ctx, hits: LayerHits, bins: HitBins, stream=None):
    i, o = hits.abi(), bins.abi()
    _check(lib().kf_bin_hits(_h(ctx), C.byref(i), C.byref(o), _stream(stream)), "kf_bin_hits", _h(ctx))
    bins.seg_off, bins.n_events, bins.n_layers, bins.first_layer = hits.seg_off, hits.n_events, hits.n_layers, \
        hits.first_layer


def kf_build(ctx, seeds: Tracks, seed_off, bins: HitBins, max_cands: int, out: BuildResult, stream=None):
    s, b, o = seeds.abi(), bins.abi(), out.abi()
    _check(lib().kf_build(_h(ctx), C.byref(s), _ptr(seed_off), C.byref(b), int(max_cands), C.byref(o),
                          _stream(stream)), "kf_build", _h(ctx))


def kf_build_f64(ctx, seeds: Tracks, event_off, bins: HitBins, max_cands: int, out: BuildResultF64, stream=None):
    """The plain FP64 build. seeds: double par/cov; event_off: sequence of
    n_events + 1 seed offsets (host)."""
    offs = (C.c_int64 * len(event_off))(*[int(v) for v in event_off])
    s, b, o = seeds.abi_f64(), bins.abi(), out.abi()
    _check(lib().kf_build_f64(_h(ctx), C.byref(s), offs, C.byref(b), int(max_cands), C.byref(o), _stream(stream)),
           "kf_build_f64", _h(ctx))


def kf_refit(ctx, seeds: Tracks, seed_hits: TrackHits, seed_off, build_hits: LayerHits, hit_idx, out: Tracks,
             chi2=None, status=None, stream=None):
    """Fit of built tracks over all layers with the hits kf_build chose."""
    s, h, b, o = seeds.abi(), seed_hits.abi(), build_hits.abi(), out.abi()
    _check(lib().kf_refit(_h(ctx), C.byref(s), C.byref(h), _ptr(seed_off), C.byref(b), _ptr(hit_idx), C.byref(o),
                          _ptr(chi2), _ptr(status), _stream(stream)), "kf_refit", _h(ctx))


# --------------------------------------------------------------------------- launch parameters


def _tuning_dict(t: kf_tuning) -> dict:
    return {f: getattr(t, f) for f, _ in kf_tuning._fields_}


def kf_get_tuning(ctx) -> dict:
    t = kf_tuning()
    _check(lib().kf_get_tuning(_h(ctx), C.byref(t)), "kf_get_tuning", _h(ctx))
    return _tuning_dict(t)


def kf_set_tuning(ctx, fit_block: int, build_hit_tile: int, build_list_width: int, build_scan: int = 4,
                  fit_chunk: int = 0, fit_stage: int = 0, bin_unordered: int = 0):
    t = kf_tuning(int(fit_block), int(build_hit_tile), int(build_list_width), int(build_scan), int(fit_chunk),
                  int(fit_stage), int(bin_unordered))
    _check(lib().kf_set_tuning(_h(ctx), C.byref(t)), "kf_set_tuning", _h(ctx))


def kf_autotune_fit(ctx, seeds: Tracks, hits: TrackHits, out: Tracks, chi2=None, status=None, stream=None) -> dict:
    s, h, o, t = seeds.abi(), hits.abi(), out.abi(), kf_tuning()
    _check(lib().kf_autotune_fit(_h(ctx), C.byref(s), C.byref(h), C.byref(o), _ptr(chi2), _ptr(status),
                                 _stream(stream), C.byref(t)), "kf_autotune_fit", _h(ctx))
    return _tuning_dict(t)


def kf_autotune_build(ctx, seeds: Tracks, seed_off, bins: HitBins, max_cands: int, out: BuildResult,
                      stream=None) -> dict:
    s, b, o, t = seeds.abi(), bins.abi(), out.abi(), kf_tuning()
    _check(lib().kf_autotune_build(_h(ctx), C.byref(s), _ptr(seed_off), C.byref(b), int(max_cands), C.byref(o),
                                   _stream(stream), C.byref(t)), "kf_autotune_build", _h(ctx))
    return _tuning_dict(t)


def kf_test_stage_fault(ctx, skip_tile: int = -1, wait_polls: int = 0):
    """Test hook of the staged fit kernel's bounded waits (see kf.h)."""
    _check(lib().kf_test_stage_fault(_h(ctx), int(skip_tile), int(wait_polls)), "kf_test_stage_fault", _h(ctx))


def kf_test_build_stage_fault(ctx, skip_warp: int = -1, wait_polls: int = 0):
    """Test hook of the build's hit-staging waits (see kf.h)."""
    _check(lib().kf_test_build_stage_fault(_h(ctx), int(skip_warp), int(wait_polls)), "kf_test_build_stage_fault",
           _h(ctx))


# --------------------------------------------------------------------------- measured peaks

PEAK_FP32, PEAK_FP64 = 0, 1  # KF_PEAK_FP32, KF_PEAK_FP64


def kf_measure_peak(ctx, kind: int, stream=None) -> float:
    """Measured FMA rate of the device in flop/s (kind PEAK_FP32 or PEAK_FP64)."""
    v = C.c_double()
    _check(lib().kf_measure_peak(_h(ctx), int(kind), _stream(stream), C.byref(v)), "kf_measure_peak", _h(ctx))
    return v.value


# --------------------------------------------------------------------------- serving


def kf_serve_start(ctx, n_seed_layers=3, n_build_layers=7, max_cands=6, max_slots=MAX_SLOTS, max_queue=1024,
                   device_arena_bytes=0, host_arena_bytes=0, refit=False, pack_min_seeds=0):
    cfg = kf_serve_config(n_seed_layers, n_build_layers, max_cands, max_slots, max_queue, int(bool(refit)),
                          device_arena_bytes, host_arena_bytes, int(pack_min_seeds))
    _check(lib().kf_serve_start(_h(ctx), C.byref(cfg)), "kf_serve_start", _h(ctx))


def kf_serve_stop(ctx):
    _check(lib().kf_serve_stop(_h(ctx)), "kf_serve_stop")


def _np_ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def kf_submit(ctx, event: dict) -> int:
    """event: numpy host arrays seed_par [6, n] f32, seed_cov [21, n] f32,
    seed_charge [n] i8, seed_hits [Ls, 3, n] f32, seed_valid [Ls, n] u8 or None,
    layer_xyz [3, n_hits] f32, layer_off [Lb + 1] i64. Returns the ticket.
    Raises KfError (code KF_EAGAIN when the queue or host arena is full)."""
    import numpy as np
    arrs = {k: (None if event.get(k) is None else np.ascontiguousarray(event[k])) for k in
            ("seed_par", "seed_cov", "seed_charge", "seed_hits", "seed_valid", "layer_xyz", "layer_off")}
    ev = kf_event(int(arrs["seed_par"].shape[1]), *[_np_ptr(arrs[k]) for k in
                                                      ("seed_par", "seed_cov", "seed_charge", "seed_hits",
                                                       "seed_valid", "layer_xyz", "layer_off")])
    t = C.c_uint64()
    _check(lib().kf_submit(_h(ctx), C.byref(ev), C.byref(t)), "kf_submit")
    return t.value


def kf_poll(ctx, ticket: int, n_seeds: int, n_build_layers: int, timeout_us: int = -1, want_cov: bool = False,
            refit_layers: int = 0):
    """Returns a dict of numpy results, or raises KfError (KF_ETIMEDOUT if not done).
    refit_layers > 0 (serving started with refit=True): also the re-fit's results
    (refit_chi2 has refit_layers rows)."""
    import numpy as np
    out = dict(best_par=np.empty((6, n_seeds), np.float32),
               best_cov=np.empty((21, n_seeds), np.float32) if want_cov else None,
               chi2_tot=np.empty(n_seeds, np.float32), n_hits=np.empty(n_seeds, np.int32),
               status=np.empty(n_seeds, np.int32), hit_idx=np.empty((n_build_layers, n_seeds), np.int32))
    if refit_layers:
        out.update(refit_par=np.empty((6, n_seeds), np.float32),
                   refit_cov=np.empty((21, n_seeds), np.float32) if want_cov else None,
                   refit_chi2=np.empty((refit_layers, n_seeds), np.float32),
                   refit_status=np.empty(n_seeds, np.int32))
    r = kf_event_result(*[_np_ptr(out[k]) for k in ("best_par", "best_cov", "chi2_tot", "n_hits", "status",
                                                      "hit_idx")], 0.0, 0.0,
                        *[_np_ptr(out.get(k)) for k in ("refit_par", "refit_cov", "refit_chi2", "refit_status")])
    _check(lib().kf_poll(_h(ctx), C.c_uint64(ticket), C.byref(r), int(timeout_us)), "kf_poll")
    out["latency_ms"], out["queued_ms"] = r.latency_ms, r.queued_ms
    return out


def kf_cancel(ctx, ticket: int):
    _check(lib().kf_cancel(_h(ctx), C.c_uint64(ticket)), "kf_cancel")


def kf_serve_stats_get(ctx) -> dict:
    st = kf_serve_stats()
    _check(lib().kf_serve_stats_get(_h(ctx), C.byref(st)), "kf_serve_stats_get")
    return {f: getattr(st, f) for f, _ in kf_serve_stats._fields_}

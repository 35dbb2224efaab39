"""FP64 CPU oracle for the Kalman-filter track fit and combinatorial build.

TEST INFRASTRUCTURE ONLY: the parity oracle of the CUDA library. Only the test
suite, the smoke check and the benchmark's CPU-baseline leg import it. It
shares no code with the CUDA path; its arithmetic lives in `kf_oracle.c`
(plain C, double precision, full 6x6 matrices), compiled here with gcc.

Method: Cerati et al., "Kalman Filter Tracking on Parallel Architectures",
Sec. 2 (the fit: propagate + Kalman update over a fixed hit set) and Sec. 3
(the build: chi2 of every hit in the layer, children ranked by hit count and
chi2, the best N kept by the clone engine; N = 1 is the best-hit approach).
The helix propagation, transport Jacobian and update are the textbook
extended Kalman filter the paper cites (Fruhwirth 1987); see kf_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libkf_oracle.so")
C_LIGHT = 0.00299792458

NOT_REACHED, NEWTON_FAIL, TANGENT, NOT_PD, NO_HIT = 1, 2, 4, 8, 16

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile kf_oracle.c into oracle/_build/libkf_oracle.so (gcc, -O2,
    no FMA contraction so that x86 and Arm give the same bits)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
               "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            d, i64, i32, u8 = C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_uint8)
            L.orc_helix_at.argtypes = [d, C.c_double, C.c_double, d]
            L.orc_path_length_circle.argtypes = [d, C.c_double, C.c_double, d]
            L.orc_path_length_newton.argtypes = [d, C.c_double, C.c_double, C.c_double, C.c_double,
                                                 C.c_int, d, C.POINTER(C.c_int)]
            L.orc_straight_line_guess.argtypes = [d, C.c_double]
            L.orc_straight_line_guess.restype = C.c_double
            L.orc_propagate.argtypes = [d, C.c_double, C.c_double, d, d, d]
            L.orc_transport_cov.argtypes = [d, d, d, d]
            L.orc_chi2.argtypes = [d, d, d, d]
            L.orc_chi2.restype = C.c_double
            L.orc_update.argtypes = [d, d, d, d, d, d, d, d]
            L.orc_pd5.argtypes = [d, d]
            L.orc_fit.argtypes = [i64, C.c_int, d, d, d, d, d, d, u8, d, d, d, i32, d, C.c_double, C.c_int]
            L.orc_scattering_q.argtypes = [d, C.c_double, C.c_double, d]
            L.orc_scattering_q.restype = None
            L.orc_build.argtypes = [i64, C.c_int, d, d, C.c_double, C.c_int, d, d, d, i32, d,
                                    C.POINTER(C.c_int64), d, d, d, i32, i32, i32, i32, d, C.c_double, C.c_int]
            L.orc_max_threads.restype = C.c_int
            _lib = L
    return _lib


def _p(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def a_coef(charge, bz: float) -> np.ndarray:
    """a = q C_LIGHT Bz per track (GeV/cm)."""
    return np.asarray(charge, dtype=np.float64) * C_LIGHT * bz


def full_cov_from_packed(packed_21xn: np.ndarray) -> np.ndarray:
    """[21, n] packed lower triangle (row-major, i(i+1)/2 + j) -> [n, 6, 6] float64."""
    packed = np.asarray(packed_21xn, dtype=np.float64)
    n = packed.shape[1]
    out = np.zeros((n, 6, 6))
    k = 0
    for i in range(6):
        for j in range(i + 1):
            out[:, i, j] = packed[k]
            out[:, j, i] = packed[k]
            k += 1
    return out


# ---------------------------------------------------------------- single-track calls

def helix_at(x0, a: float, s: float) -> np.ndarray:
    x0, out = _f64(x0), np.zeros(6)
    lib().orc_helix_at(_p(x0), a, s, _p(out))
    return out


def path_length_circle(x0, a: float, R: float):
    x0, s = _f64(x0), np.zeros(1)
    st = lib().orc_path_length_circle(_p(x0), a, R, _p(s))
    return float(s[0]), int(st)


def path_length_newton(x0, a: float, R: float, s_start=None, tol=1e-13, max_iter=50):
    x0, s, it = _f64(x0), np.zeros(1), C.c_int(0)
    if s_start is None:
        s_start = lib().orc_straight_line_guess(_p(x0), R)
    st = lib().orc_path_length_newton(_p(x0), a, R, s_start, tol, max_iter, _p(s), C.byref(it))
    return float(s[0]), int(st), it.value


def propagate(x0, a: float, R: float):
    x0, x1, J, s = _f64(x0), np.zeros(6), np.zeros(36), np.zeros(1)
    st = lib().orc_propagate(_p(x0), a, R, _p(x1), _p(J), _p(s))
    return x1, J.reshape(6, 6), float(s[0]), int(st)


def transport_cov(J, Cm, Q=None):
    J, Cm, out = _f64(J), _f64(Cm), np.zeros(36)
    q = _p(_f64(Q)) if Q is not None else None
    lib().orc_transport_cov(_p(J), _p(Cm), q, _p(out))
    return out.reshape(6, 6)


def chi2(xp, Cp, m, V) -> float:
    return float(lib().orc_chi2(_p(_f64(xp)), _p(_f64(Cp)), _p(_f64(m)), _p(_f64(V))))


def update(xp, Cp, m, V):
    x, Cm, c2, dev = np.zeros(6), np.zeros(36), np.zeros(1), np.zeros(1)
    lib().orc_update(_p(_f64(xp)), _p(_f64(Cp)), _p(_f64(m)), _p(_f64(V)), _p(x), _p(Cm),
                     _p(c2), _p(dev))
    return x, Cm.reshape(6, 6), float(c2[0]), float(dev[0])


def pd5(x, Cm) -> bool:
    return bool(lib().orc_pd5(_p(_f64(x)), _p(_f64(Cm))))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------- batched fit / build

PION_MASS = 0.13957  # GeV: default particle hypothesis of the scattering model


def _material(x_x0, L):
    if x_x0 is None:
        return None
    m = _f64(x_x0)
    assert m.shape == (L,)
    return m


def scattering_q(x, x_x0: float, mass: float = PION_MASS) -> np.ndarray:
    """[6, 6] process noise of multiple scattering at the crossing state x."""
    Q = np.zeros(36)
    lib().orc_scattering_q(_p(_f64(x)), float(x_x0), float(mass), _p(Q))
    return Q.reshape(6, 6)


def fit(seed_par, seed_cov_packed, charge, hit_xyz, hit_valid, radii, bz, sigma_xy, sigma_z,
        n_threads: int = 0, x_x0=None, mass: float = PION_MASS):
    """Fit every track over all layers.

    seed_par float [6, n]; seed_cov_packed float [21, n]; charge int [n];
    hit_xyz float [L, 3, n]; hit_valid uint8 [L, n]; x_x0 [L] layer thickness
    in radiation lengths (None: no material). Inputs are upcast to FP64.
    Returns dict(par [n, 6], cov [n, 6, 6], chi2 [L, n] (-1: no update), status [n]).
    """
    seed_par = np.asarray(seed_par)
    n = seed_par.shape[1]
    L = len(radii)
    sp = _f64(seed_par.T)
    sc = _f64(full_cov_from_packed(seed_cov_packed))
    ac = _f64(a_coef(charge, bz))
    hits = _f64(np.transpose(np.asarray(hit_xyz, dtype=np.float64), (0, 2, 1)))
    val = np.ascontiguousarray(hit_valid, dtype=np.uint8)
    rad = _f64(radii)
    V = _f64([sigma_xy ** 2, sigma_xy ** 2, sigma_z ** 2])
    out_par, out_cov = np.zeros((n, 6)), np.zeros((n, 6, 6))
    c2, st = np.zeros((L, n)), np.zeros(n, dtype=np.int32)
    mat = _material(x_x0, L)
    lib().orc_fit(n, L, _p(rad), _p(V), _p(sp), _p(sc), _p(ac), _p(hits), _p(val, C.c_uint8),
                  _p(out_par), _p(out_cov), _p(c2), _p(st, C.c_int32), _p(mat) if mat is not None else None,
                  float(mass), n_threads)
    return dict(par=out_par, cov=out_cov, chi2=c2, status=st)


def build_tracks(seed_par, seed_cov, charge, seed_event, layer_xyz, layer_off, radii, bz,
                 sigma_xy, sigma_z, chi2_cut=30.0, max_cands=6, n_threads: int = 0, x_x0=None,
                 mass: float = PION_MASS):
    """Combinatorial build over the given layers (clone engine, all-hits scan).

    seed_par float [n, 6] or [6, n] (see below); seed_cov [n, 6, 6] float64;
    layer_xyz float [3, n_hits]; layer_off int64 [n_events * L + 1].
    Pass seed_par as [n, 6] FP64 and seed_cov as [n, 6, 6] (the oracle's own
    fit output) -- no packed layouts on this side.
    Returns dict of candidate arrays [n, max_cands, ...] and n_cands [n].
    """
    sp = _f64(seed_par)
    n = sp.shape[0]
    sc = _f64(seed_cov).reshape(n, 36)
    ac = _f64(a_coef(charge, bz))
    ev = np.ascontiguousarray(seed_event, dtype=np.int32)
    hits = _f64(np.asarray(layer_xyz, dtype=np.float64).T)
    off = np.ascontiguousarray(layer_off, dtype=np.int64)
    L = len(radii)
    rad = _f64(radii)
    V = _f64([sigma_xy ** 2, sigma_xy ** 2, sigma_z ** 2])
    N = int(max_cands)
    cp, cc = np.zeros((n, N, 6)), np.zeros((n, N, 6, 6))
    cchi, cnh = np.zeros((n, N)), np.zeros((n, N), dtype=np.int32)
    chits, cst = np.zeros((n, N, L), dtype=np.int32), np.zeros((n, N), dtype=np.int32)
    ncand = np.zeros(n, dtype=np.int32)
    rc = lib().orc_build(n, L, _p(rad), _p(V), float(chi2_cut), N, _p(sp), _p(sc), _p(ac),
                         _p(ev, C.c_int32), _p(hits), off.ctypes.data_as(C.POINTER(C.c_int64)),
                         _p(cp), _p(cc), _p(cchi), _p(cnh, C.c_int32), _p(chits, C.c_int32),
                         _p(cst, C.c_int32), _p(ncand, C.c_int32),
                         _p(_material(x_x0, L)) if x_x0 is not None else None, float(mass), n_threads)
    if rc != 0:
        raise ValueError("orc_build rejected its arguments")
    return dict(par=cp, cov=cc, chi2=cchi, nhits=cnh, hits=chits, status=cst, n_cands=ncand)

"""Seeded synthetic barrel events: the input recipe for the track fit and build.

This module is the detector simulation that feeds both the CUDA path and the
FP64 oracle. It draws every random number (particle kinematics, vertex, hit
smear, noise hits, seed smear) and places each truth hit where the exact helix
of a charged particle in a uniform solenoidal field crosses a barrel cylinder.
It holds none of the filter's arithmetic: no path-length Newton solve, no
transport Jacobian, no covariance propagation and no Kalman update.

The paper (Sec. 1, Sec. 3) works in a "simplified experimental environment":
concentric barrel layers, a uniform field, and tracks that "do not bend in
eta". It prints no geometry, so the geometry and distributions below are the
stated readings of this library:

* Bz = 3.8 T, barrel cylinders at r = 4, 8, ..., 4 L cm, infinite in z.
* charge +-1 equiprobable, pT ~ U[0.5, 10] GeV, phi ~ U[0, 2 pi),
  eta ~ U(-1, 1), pz = pT sinh(eta); vertex x, y ~ N(0, 0.01 cm),
  z ~ N(0, 1 cm).
* hit = truth crossing + N(0, sigma_xy) x + N(0, sigma_xy) y + N(0, sigma_z) z
  with sigma_xy = 0.01 cm, sigma_z = 0.1 cm (an isotropic transverse smear, so
  the measurement covariance is V = diag(sigma_xy^2, sigma_xy^2, sigma_z^2)).
* noise hits (building): `noise_factor` x the track count per layer, uniform in
  phi, uniform in z within +-(R sinh 1 + 3 cm), on r = R, then the same smear.
* every value handed to either implementation is rounded to float32 once;
  the oracle upcasts those same float32 values.

Units: cm, GeV, tesla. State vector (x, y, z, px, py, pz).
Covariances are packed lower triangles, row-major: index(i, j) = i(i+1)/2 + j
for j <= i (21 entries).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 0.00299792458  # GeV / (T cm): pT[GeV] = C_LIGHT * B[T] * rho[cm]
PION_MASS = 0.13957  # GeV: the particle hypothesis of the scattering model

TRIL_I, TRIL_J = np.tril_indices(6)  # row-major packed lower triangle order


def pack_cov(full: np.ndarray) -> np.ndarray:
    """[..., 6, 6] symmetric -> [..., 21] packed lower triangle (row-major)."""
    return full[..., TRIL_I, TRIL_J]


def unpack_cov(packed: np.ndarray) -> np.ndarray:
    """[..., 21] packed lower triangle -> [..., 6, 6] full symmetric."""
    out = np.zeros(packed.shape[:-1] + (6, 6), dtype=packed.dtype)
    out[..., TRIL_I, TRIL_J] = packed
    out[..., TRIL_J, TRIL_I] = packed
    return out


@dataclass(frozen=True)
class Detector:
    radii: tuple
    bz: float = 3.8
    sigma_xy: float = 0.01
    sigma_z: float = 0.1
    # thickness of each layer in radiation lengths at normal incidence (None:
    # no material); the particles are simulated as pions
    x_x0: tuple | None = None
    mass: float = PION_MASS

    @property
    def n_layers(self) -> int:
        return len(self.radii)

    @property
    def has_material(self) -> bool:
        return self.x_x0 is not None and any(x > 0 for x in self.x_x0)


def highland_theta0(p, x_eff, mass=PION_MASS):
    """RMS of the projected multiple-scattering angle of a unit-charge particle
    of momentum p (GeV) after x_eff radiation lengths: the Highland formula
    with the Lynch-Dahl logarithm, as in the Review of Particle Physics
    (passage of particles through matter),
      theta0 = 13.6 MeV / (beta c p) sqrt(x/X0) (1 + 0.038 ln(x / (X0 beta^2)))."""
    p = np.asarray(p, dtype=np.float64)
    beta2 = p * p / (p * p + mass * mass)
    return 0.0136 / (np.sqrt(beta2) * p) * np.sqrt(x_eff) * (1.0 + 0.038 * np.log(x_eff / beta2))


def barrel(n_layers: int = 10, spacing: float = 4.0, **kw) -> Detector:
    """Concentric cylinders at r = spacing * (1..n_layers)."""
    return Detector(radii=tuple(float(spacing * (i + 1)) for i in range(n_layers)), **kw)


@dataclass
class Particles:
    """Truth kinematics at the production vertex (float64)."""
    charge: np.ndarray  # int8 [n]
    vertex: np.ndarray  # [n, 3]
    mom: np.ndarray  # [n, 3]

    @property
    def n(self) -> int:
        return len(self.charge)


@dataclass
class TrackHits:
    """Per-track hits, SoA per layer, as both implementations take them."""
    xyz: np.ndarray  # float32 [L, 3, n]
    valid: np.ndarray  # uint8 [L, n]: 1 where the particle crossed the layer
    truth: np.ndarray  # float64 [L, n, 6]: exact state at each crossing (nan if none)


@dataclass
class Seeds:
    """Seed tracks in the layout of the C ABI (float32 SoA)."""
    par: np.ndarray  # float32 [6, n]
    cov: np.ndarray  # float32 [21, n]
    charge: np.ndarray  # int8 [n]


def draw_particles(rng: np.random.Generator, n: int, pt_range=(0.5, 10.0),
                   eta_max: float = 1.0, pt_mix=None, phi_range=(0.0, 2.0 * np.pi)) -> Particles:
    """Draw n particles. `pt_mix` = list of (fraction, (lo, hi)) overrides pt_range."""
    q = rng.choice(np.array([-1, 1], dtype=np.int8), size=n)
    if pt_mix is None:
        pt = rng.uniform(pt_range[0], pt_range[1], size=n)
    else:
        pick = rng.uniform(size=n)
        pt = np.empty(n)
        edge = 0.0
        for frac, (lo, hi) in pt_mix:
            sel = (pick >= edge) & (pick < edge + frac)
            pt[sel] = rng.uniform(lo, hi, size=int(sel.sum()))
            edge += frac
        sel = pick >= edge
        if sel.any():
            lo, hi = pt_mix[-1][1]
            pt[sel] = rng.uniform(lo, hi, size=int(sel.sum()))
    phi = rng.uniform(phi_range[0], phi_range[1], size=n)
    eta = rng.uniform(-eta_max, eta_max, size=n)
    vtx = np.stack([rng.normal(0.0, 0.01, n), rng.normal(0.0, 0.01, n),
                    rng.normal(0.0, 1.0, n)], axis=1)
    mom = np.stack([pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta)], axis=1)
    return Particles(charge=q, vertex=vtx, mom=mom)


def helix_crossing(vertex: np.ndarray, mom: np.ndarray, charge: np.ndarray,
                   bz: float, radius: float):
    """Exact first crossing of the particle helix with the cylinder r = radius.

    Geometry of the transverse circle: centre c = v + (py, -px)/a with
    a = q C_LIGHT Bz (signed), radius rho = pT/|a|. A point c + rho u lies on
    r = R when c.u = (R^2 - d^2 - rho^2)/(2 rho), d = |c|. The particle runs
    clockwise around c (seen from +z) when a > 0. Among the two solutions, the
    one reached first along the motion is taken.

    Returns (state [n, 6] at the crossing, reached [n] bool).
    """
    n = len(charge)
    a = charge.astype(np.float64) * C_LIGHT * bz
    px, py, pz = mom[:, 0], mom[:, 1], mom[:, 2]
    pt = np.hypot(px, py)
    p = np.sqrt(pt * pt + pz * pz)
    rho = pt / np.abs(a)
    cx = vertex[:, 0] + py / a
    cy = vertex[:, 1] - px / a
    d = np.hypot(cx, cy)
    with np.errstate(invalid="ignore", divide="ignore"):
        kappa = (radius * radius - d * d - rho * rho) / (2.0 * rho * d)
    reached = np.abs(kappa) <= 1.0
    kappa = np.clip(kappa, -1.0, 1.0)
    psi_c = np.arctan2(cy, cx)
    alpha = np.arccos(kappa)
    psi0 = np.arctan2(vertex[:, 1] - cy, vertex[:, 0] - cx)
    cw = a > 0
    best_tau = np.full(n, np.inf)
    for sgn in (1.0, -1.0):
        psi_t = psi_c + sgn * alpha
        tau = np.where(cw, psi0 - psi_t, psi_t - psi0)
        tau = np.mod(tau, 2.0 * np.pi)
        best_tau = np.minimum(best_tau, tau)
    tau = best_tau
    # signed turning angle theta = a s / p; position and momentum on the circle
    theta = np.where(cw, tau, -tau)
    s_t = rho * tau  # transverse arc length
    psi = np.where(cw, psi0 - tau, psi0 + tau)
    x = cx + rho * np.cos(psi)
    y = cy + rho * np.sin(psi)
    z = vertex[:, 2] + pz * s_t / pt
    cth, sth = np.cos(theta), np.sin(theta)
    pxo = px * cth + py * sth
    pyo = py * cth - px * sth
    out = np.stack([x, y, z, pxo, pyo, pz], axis=1)
    out[~reached] = np.nan
    del p
    return out, reached


def _kink(rng: np.random.Generator, state: np.ndarray, ok: np.ndarray, x_x0: float, mass: float) -> None:
    """Multiple scattering in a thin layer at the crossing `state` [n, 6]
    (in place, rows `ok`): the direction turns by two independent Gaussian
    projected angles of RMS theta0 (Highland, path x_x0 / cos(incidence)) in
    two planes containing it; |p| is unchanged."""
    n = len(state)
    pos, mom = state[:, :3], state[:, 3:]
    p = np.linalg.norm(mom, axis=1)
    d = mom / p[:, None]
    r = np.hypot(pos[:, 0], pos[:, 1])
    cos_inc = np.abs(pos[:, 0] * d[:, 0] + pos[:, 1] * d[:, 1]) / r
    th0 = highland_theta0(p, x_x0 / np.maximum(cos_inc, 1e-6), mass)
    u1 = np.stack([-d[:, 1], d[:, 0], np.zeros(n)], axis=1)  # z x d
    u1 /= np.linalg.norm(u1, axis=1)[:, None]
    u2 = np.cross(d, u1)
    t1, t2 = rng.normal(0.0, 1.0, n) * th0, rng.normal(0.0, 1.0, n) * th0
    nd = d + np.tan(t1)[:, None] * u1 + np.tan(t2)[:, None] * u2
    nd /= np.linalg.norm(nd, axis=1)[:, None]
    state[ok, 3:] = (nd * p[:, None])[ok]


def simulate_hits(rng: np.random.Generator, parts: Particles, det: Detector,
                  keep_truth: bool = True) -> TrackHits:
    """Truth crossings on every layer plus the Gaussian hit smear.
    With material (det.x_x0) the helix is followed layer by layer and the
    direction is kinked by multiple scattering at every crossing; the truth
    state of a layer is the crossing point with the momentum leaving it.
    `keep_truth=False` skips the [L, n, 6] float64 truth array (large batches)."""
    if det.has_material:
        return _simulate_hits_material(rng, parts, det, keep_truth)
    L, n = det.n_layers, parts.n
    xyz = np.zeros((L, 3, n), dtype=np.float32)
    valid = np.zeros((L, n), dtype=np.uint8)
    truth = np.full((L, n, 6), np.nan) if keep_truth else None
    alive = np.ones(n, dtype=bool)
    for li, R in enumerate(det.radii):
        st, ok = helix_crossing(parts.vertex, parts.mom, parts.charge, det.bz, R)
        ok &= alive
        alive = ok  # a particle that misses layer l misses every outer layer too
        if keep_truth:
            truth[li][ok] = st[ok]
        smear = np.stack([rng.normal(0.0, det.sigma_xy, n), rng.normal(0.0, det.sigma_xy, n),
                          rng.normal(0.0, det.sigma_z, n)], axis=1)
        h = np.where(ok[:, None], st[:, :3] + smear, 0.0)
        xyz[li] = h.T.astype(np.float32)
        valid[li] = ok
    return TrackHits(xyz=xyz, valid=valid, truth=truth)


def _simulate_hits_material(rng, parts, det, keep_truth):
    L, n = det.n_layers, parts.n
    xyz = np.zeros((L, 3, n), dtype=np.float32)
    valid = np.zeros((L, n), dtype=np.uint8)
    truth = np.full((L, n, 6), np.nan) if keep_truth else None
    alive = np.ones(n, dtype=bool)
    pos, mom = parts.vertex.copy(), parts.mom.copy()
    for li, R in enumerate(det.radii):
        st, ok = helix_crossing(pos, mom, parts.charge, det.bz, R)
        ok &= alive
        alive = ok
        smear = np.stack([rng.normal(0.0, det.sigma_xy, n), rng.normal(0.0, det.sigma_xy, n),
                          rng.normal(0.0, det.sigma_z, n)], axis=1)
        h = np.where(ok[:, None], st[:, :3] + smear, 0.0)
        xyz[li] = h.T.astype(np.float32)
        valid[li] = ok
        if det.x_x0[li] > 0:
            st = np.where(ok[:, None], st, np.nan)
            _kink(rng, st, ok, det.x_x0[li], det.mass)
        if keep_truth:
            truth[li][ok] = st[ok]
        pos = np.where(ok[:, None], st[:, :3], pos)
        mom = np.where(ok[:, None], st[:, 3:], mom)
    return TrackHits(xyz=xyz, valid=valid, truth=truth)


SEED_SIGMA_XY = 0.01  # cm: the beam spot
SEED_SIGMA_Z = 1.0  # cm: the luminous region
SEED_SIGMA_P_REL = 0.01  # per momentum component, relative to |p|


def seed_cov_diag(p: np.ndarray, sigma_xy=SEED_SIGMA_XY, sigma_z=SEED_SIGMA_Z,
                  sigma_p_rel=SEED_SIGMA_P_REL) -> np.ndarray:
    """Seed covariance diagonal: (sigma_xy)^2 x 2, (sigma_z)^2, (sigma_p_rel p)^2 x 3.

    The paper reports no realistic seeding. The default prior (0.01 cm, 1 cm,
    1 % of p) keeps the extended filter in its linear regime from the first
    layer on; a wider momentum prior (10 %) inflates the first-layer chi2
    because the linearised prediction misses by more than sqrt(R sigma)."""
    n = len(p)
    d = np.empty((n, 6))
    d[:, 0] = sigma_xy ** 2
    d[:, 1] = sigma_xy ** 2
    d[:, 2] = sigma_z ** 2
    d[:, 3:] = (sigma_p_rel * p[:, None]) ** 2
    return d


def _to_seeds(state: np.ndarray, cov_diag: np.ndarray, charge: np.ndarray) -> Seeds:
    n = len(charge)
    full = np.zeros((n, 6, 6))
    full[:, np.arange(6), np.arange(6)] = cov_diag
    return Seeds(par=np.ascontiguousarray(state.T.astype(np.float32)),
                 cov=np.ascontiguousarray(pack_cov(full).T.astype(np.float32)),
                 charge=charge.astype(np.int8).copy())


def seeds_truth_smeared(rng: np.random.Generator, parts: Particles, scale: float = 1.0) -> Seeds:
    """Truth state at the vertex, smeared by N(0, C_seed): the seed error is then
    exactly Gaussian with the stated covariance (used for pull tests).
    `scale` multiplies the smear width (0 gives the exact truth seed) while
    the stated covariance stays C_seed."""
    p = np.linalg.norm(parts.mom, axis=1)
    d = seed_cov_diag(p)
    truth = np.concatenate([parts.vertex, parts.mom], axis=1)
    state = truth + scale * rng.normal(size=truth.shape) * np.sqrt(d)
    return _to_seeds(state, d, parts.charge)


def seeds_from_hits(hits: TrackHits, bz: float, layers=(0, 1, 2)) -> Seeds:
    """Three-hit helix seed from the hits on the first three layers.

    The transverse circle through the three xy points gives the centre and
    radius rho (pT = C_LIGHT |Bz| rho); the turning sense gives the charge
    (clockwise seen from +z is positive for Bz > 0); tan(lambda) is dz over the
    transverse arc between the first and third hit. The seed state sits at the
    point of the circle closest to the z axis, with the stated diagonal
    covariance (the paper gives no seeding details).
    """
    P = [hits.xyz[l].astype(np.float64) for l in layers]
    x1, y1, z1 = P[0]
    x2, y2, _ = P[1]
    x3, y3, z3 = P[2]
    # circumcentre
    dd = 2.0 * (x1 * (y2 - y3) + x2 * (y3 - y1) + x3 * (y1 - y2))
    s1, s2, s3 = x1 * x1 + y1 * y1, x2 * x2 + y2 * y2, x3 * x3 + y3 * y3
    cx = (s1 * (y2 - y3) + s2 * (y3 - y1) + s3 * (y1 - y2)) / dd
    cy = (s1 * (x3 - x2) + s2 * (x1 - x3) + s3 * (x2 - x1)) / dd
    rho = np.hypot(x1 - cx, y1 - cy)
    cross = (x2 - x1) * (y3 - y2) - (y2 - y1) * (x3 - x2)
    cw = cross < 0.0
    q = np.where(cw == (bz > 0), 1, -1).astype(np.int8)
    pt = C_LIGHT * abs(bz) * rho
    d = np.hypot(cx, cy)
    # point of the circle closest to the z axis
    ex, ey = -cx / d, -cy / d
    x0, y0 = cx + rho * ex, cy + rho * ey
    # unit tangent along the motion at angle psi around the centre
    def tangent(ux, uy):
        return np.where(cw, uy, -uy), np.where(cw, -ux, ux)
    tx, ty = tangent(ex, ey)

    def turn(ax, ay, bx, by):
        # turning angle from direction a to direction b (both from the centre) along the motion
        ang = np.arctan2(ax * by - ay * bx, ax * bx + ay * by)
        ang = np.where(cw, -ang, ang)
        return np.mod(ang, 2.0 * np.pi)
    u1x, u1y = (x1 - cx) / rho, (y1 - cy) / rho
    u3x, u3y = (x3 - cx) / rho, (y3 - cy) / rho
    arc13 = rho * turn(u1x, u1y, u3x, u3y)
    tanl = (z3 - z1) / arc13
    arc01 = rho * turn(ex, ey, u1x, u1y)
    z0 = z1 - tanl * arc01
    px, py, pz = pt * tx, pt * ty, pt * tanl
    state = np.stack([x0, y0, z0, px, py, pz], axis=1)
    p = np.sqrt(pt * pt + pz * pz)
    return _to_seeds(state, seed_cov_diag(p), q)


@dataclass
class FitEvent:
    det: Detector
    parts: Particles
    hits: TrackHits
    seeds: Seeds


def make_fit_batch(seed: int, n_tracks: int, det: Detector | None = None,
                   seed_mode: str = "truth_smeared", smear_scale: float = 1.0,
                   pt_range=(0.5, 10.0), pt_mix=None, hit_noise: bool = True,
                   keep_truth: bool = True) -> FitEvent:
    """All tracks of a fit batch (events are independent, so a batch of E events
    of T tracks is one draw of E*T tracks with per-event offsets kept by the
    caller). `hit_noise=False` places hits at the exact crossings."""
    det = det or barrel()
    rng = np.random.default_rng(seed)
    parts = draw_particles(rng, n_tracks, pt_range=pt_range, pt_mix=pt_mix)
    if hit_noise:
        hits = simulate_hits(rng, parts, det, keep_truth)
    else:
        hits = simulate_hits(rng, parts, Detector(det.radii, det.bz, 0.0, 0.0), keep_truth)
    if seed_mode == "hits123":
        seeds = seeds_from_hits(hits, det.bz)
    elif seed_mode == "truth_smeared":
        seeds = seeds_truth_smeared(rng, parts, smear_scale)
    elif seed_mode == "truth":
        seeds = seeds_truth_smeared(rng, parts, 0.0)
    else:
        raise ValueError(seed_mode)
    return FitEvent(det=det, parts=parts, hits=hits, seeds=seeds)


# ---------------------------------------------------------------------------
# Combinatorial-building events: track hits plus uniform noise, per layer.


@dataclass
class BuildBatch:
    """Inputs of a batched build over `n_events` events.

    seeds: vertex seeds of every event's tracks (event-major order), to be
      fitted over the seeding layers before building;
    seed_event: int32 [n_seeds] event of each seed;
    fit_hits: per-track hits on the seeding layers (for the seed fit);
    layer_xyz: float32 [3, n_hits_total] raw hits of every (event, build layer)
      segment, concatenated event-major then layer;
    layer_off: int64 [n_events * L_build + 1] segment offsets;
    layer_truth: int32 [n_hits_total] index of the producing track within its
      event, -1 for noise.
    """
    det: Detector
    seed_layers: tuple
    build_layers: tuple
    n_events: int
    tracks_per_event: int
    seeds: Seeds
    seed_event: np.ndarray
    fit_hits: TrackHits
    layer_xyz: np.ndarray
    layer_off: np.ndarray
    layer_truth: np.ndarray
    parts: list = field(default_factory=list)


def make_build_batch(seed: int, n_events: int, tracks_per_event: int,
                     det: Detector | None = None, noise_factor: float = 3.0,
                     n_seed_layers: int = 3, pt_range=(0.5, 10.0), noise_near: int = 0,
                     noise_near_sigma: float = 0.0, phi_range=(0.0, 2.0 * np.pi)) -> BuildBatch:
    """`noise_near` extra hits per track hit, displaced by N(0, noise_near_sigma)
    in x, y and N(0, 10 noise_near_sigma) in z (dense, branching-heavy
    tiny cases)."""
    det = det or barrel()
    rng = np.random.default_rng(seed)
    L = det.n_layers
    seed_layers = tuple(range(n_seed_layers))
    build_layers = tuple(range(n_seed_layers, L))
    segs, truths, offs = [], [], [0]
    all_seeds, all_hits, ev_of_seed, parts_list = [], [], [], []
    for e in range(n_events):
        parts = draw_particles(rng, tracks_per_event, pt_range=pt_range, phi_range=phi_range)
        hits = simulate_hits(rng, parts, det)
        parts_list.append(parts)
        all_hits.append(hits)
        all_seeds.append(seeds_truth_smeared(rng, parts))
        ev_of_seed.append(np.full(tracks_per_event, e, dtype=np.int32))
        n_noise = int(round(noise_factor * tracks_per_event))
        for li in build_layers:
            R = det.radii[li]
            ok = hits.valid[li].astype(bool)
            trk = hits.xyz[li][:, ok]
            tid = np.nonzero(ok)[0].astype(np.int32)
            zmax = R * np.sinh(1.0) + 3.0
            phi = rng.uniform(0.0, 2.0 * np.pi, n_noise)
            zz = rng.uniform(-zmax, zmax, n_noise)
            nz = np.stack([R * np.cos(phi) + rng.normal(0.0, det.sigma_xy, n_noise),
                           R * np.sin(phi) + rng.normal(0.0, det.sigma_xy, n_noise),
                           zz + rng.normal(0.0, det.sigma_z, n_noise)]).astype(np.float32)
            parts_xyz, parts_t = [trk, nz], [tid, np.full(n_noise, -1, dtype=np.int32)]
            for _ in range(noise_near):
                d = np.stack([rng.normal(0.0, noise_near_sigma, trk.shape[1]),
                              rng.normal(0.0, noise_near_sigma, trk.shape[1]),
                              rng.normal(0.0, 10 * noise_near_sigma, trk.shape[1])])
                parts_xyz.append((trk + d).astype(np.float32))
                parts_t.append(np.full(trk.shape[1], -1, dtype=np.int32))
            xyz = np.concatenate(parts_xyz, axis=1)
            tt = np.concatenate(parts_t)
            perm = rng.permutation(xyz.shape[1])
            segs.append(xyz[:, perm])
            truths.append(tt[perm])
            offs.append(offs[-1] + xyz.shape[1])
    seeds = Seeds(par=np.ascontiguousarray(np.concatenate([s.par for s in all_seeds], axis=1)),
                  cov=np.ascontiguousarray(np.concatenate([s.cov for s in all_seeds], axis=1)),
                  charge=np.concatenate([s.charge for s in all_seeds]))
    fit_hits = TrackHits(
        xyz=np.ascontiguousarray(np.concatenate([h.xyz[list(seed_layers)] for h in all_hits], axis=2)),
        valid=np.ascontiguousarray(np.concatenate([h.valid[list(seed_layers)] for h in all_hits], axis=1)),
        truth=np.concatenate([h.truth for h in all_hits], axis=1))
    return BuildBatch(det=det, seed_layers=seed_layers, build_layers=build_layers,
                      n_events=n_events, tracks_per_event=tracks_per_event, seeds=seeds,
                      seed_event=np.concatenate(ev_of_seed), fit_hits=fit_hits,
                      layer_xyz=np.ascontiguousarray(np.concatenate(segs, axis=1)),
                      layer_off=np.asarray(offs, dtype=np.int64),
                      layer_truth=np.concatenate(truths), parts=parts_list)

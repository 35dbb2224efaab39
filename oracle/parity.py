"""Comparison helpers of the build parity checks.

TEST INFRASTRUCTURE ONLY, like the oracle itself: used by the test suite and
by the benchmark's oracle (CPU-baseline) legs to count near ties.

A build chooses, per seed, the path (one hit id or none per layer) of its
best candidate.  Where a GPU build and the oracle's all-hits build choose
different paths, both paths are evaluated by the oracle (the chi2 increments
of the Kalman filter along each path from the oracle's own seed state): the
difference is a near tie (allowed, counted) when both paths have the same hit
count and total chi2 within `rel` of each other, or when a hit on either path
lies within 1e-3 of the chi2 cut (a rounding can then admit or drop it);
otherwise it is a genuine disagreement.  Sec. 3 ranks candidates by hit count
and then chi2, so two paths of equal count and near-equal chi2 are the
method's own ambiguity, not an error of either side.
"""
from __future__ import annotations

import numpy as np

from . import PION_MASS, propagate, scattering_q, transport_cov, update


def path_chi2(seed_par, seed_cov, a, hits, radii, V, x_x0=None, mass=PION_MASS):
    """chi2 increments of the filter along a fixed path: `hits[l]` is the hit
    (x, y, z) used on layer l or None; returns one entry per layer (None where
    the layer has no hit or the track stopped)."""
    x, Cm = np.asarray(seed_par, dtype=np.float64), np.asarray(seed_cov, dtype=np.float64)
    out = []
    for l, R in enumerate(radii):
        xp, J, _, st = propagate(x, a, R)
        if st:
            out.append(None)
            continue
        Q = scattering_q(xp, x_x0[l], mass) if (x_x0 is not None and x_x0[l] > 0) else None
        Cp = transport_cov(J, Cm, Q)
        if hits[l] is None:
            x, Cm = xp, Cp
            out.append(None)
            continue
        x, Cm, c2, _ = update(xp, Cp, np.asarray(hits[l], dtype=np.float64), V)
        out.append(c2)
    return out


def classify(paths_a, paths_b, seed_par, seed_cov, a_coef, hit_of, radii, V, x_x0=None, mass=PION_MASS,
             cut=30.0, rel=1e-4):
    """Compare two sets of best paths seed by seed ([n, L] hit ids, -1 = none).
    hit_of(t, l, h) returns the (x, y, z) of hit id h on layer l for seed row t.
    Returns (n_same, near_ties, others): lists of (row, chi2_a, chi2_b) for the
    near ties and (row, path_a, path_b, chi2_a, chi2_b) for the others."""
    same, ties, bad = 0, [], []
    L = len(radii)
    for t in range(len(paths_a)):
        pa, pb = paths_a[t], paths_b[t]
        if np.array_equal(pa, pb):
            same += 1
            continue
        ev = []
        for p in (pa, pb):
            hits = [hit_of(t, l, int(p[l])) if p[l] >= 0 else None for l in range(L)]
            ev.append([c for c in path_chi2(seed_par[t], seed_cov[t], a_coef[t], hits, radii, V, x_x0, mass)
                       if c is not None])
        ca, cb = ev
        near_cut = any(abs(c - cut) < 1e-3 for c in ca + cb) or any(c >= cut for c in ca)
        tot_a, tot_b = sum(ca), sum(cb)
        if near_cut or (len(ca) == len(cb) and abs(tot_a - tot_b) <= rel * max(tot_b, 1e-30)):
            ties.append((t, tot_a, tot_b))
        else:
            bad.append((t, list(pa), list(pb), tot_a, tot_b))
    return same, ties, bad

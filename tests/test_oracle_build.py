"""Pins of the oracle's combinatorial build: on tiny inputs (<= 3 seeds,
<= 6 hits per layer, 3 layers, hits placed to branch), the clone engine
without truncation keeps exactly every hit/miss path an exhaustive
enumeration finds, in (nHits desc, chi2_tot asc) order; with one candidate
it is the greedy best-hit chain (lowest chi2 increment per layer)."""
import numpy as np
import pytest

import oracle as O
from paper_1605_05508_gb300 import synth as S


def _tiny(seed):
    det = S.barrel(6)
    b = S.make_build_batch(seed, 1, 2, det=det, noise_factor=0.0, noise_near=2, noise_near_sigma=0.012)
    return b


def _seed_states(b):
    det = b.det
    return O.fit(b.seeds.par, b.seeds.cov, b.seeds.charge, b.fit_hits.xyz, b.fit_hits.valid, det.radii[:3], det.bz,
                 det.sigma_xy, det.sigma_z)


def _enumerate(b, x0, C0, q, cut):
    det = b.det
    V = np.array([det.sigma_xy ** 2, det.sigma_xy ** 2, det.sigma_z ** 2])
    a = q * O.C_LIGHT * det.bz
    Lb = len(b.build_layers)
    paths = []

    def rec(l, x, C, chi2, seq, stopped):
        if l == Lb:
            paths.append((sum(1 for h in seq if h >= 0), chi2, tuple(seq)))
            return
        if stopped:
            rec(l + 1, x, C, chi2, seq + [-1], True)
            return
        xp, J, _, st = O.propagate(x, a, det.radii[b.build_layers[l]])
        if st:
            rec(l + 1, x, C, chi2, seq + [-1], True)
            return
        Cp = O.transport_cov(J, C)
        found = False
        lo, hi = b.layer_off[l], b.layer_off[l + 1]
        for h in range(hi - lo):
            m = b.layer_xyz[:, lo + h].astype(np.float64)
            if O.chi2(xp, Cp, m, V) < cut:
                xn, Cn, c2, _ = O.update(xp, Cp, m, V)
                rec(l + 1, xn, Cn, chi2 + c2, seq + [h], False)
                found = True
        if not found:
            rec(l + 1, xp, Cp, chi2, seq + [-1], False)

    rec(0, x0, C0, 0.0, [], False)
    return sorted(paths, key=lambda t: (-t[0], t[1]))


def _build(b, r, N, cut):
    det = b.det
    return O.build_tracks(r["par"], r["cov"], b.seeds.charge, b.seed_event, b.layer_xyz, b.layer_off,
                          [det.radii[l] for l in b.build_layers], det.bz, det.sigma_xy, det.sigma_z, chi2_cut=cut,
                          max_cands=N)


@pytest.mark.parametrize("seed", range(6))
def test_untruncated_build_equals_exhaustive_enumeration(seed):
    b = _tiny(seed)
    assert all(b.layer_off[i + 1] - b.layer_off[i] <= 6 for i in range(len(b.layer_off) - 1))
    r = _seed_states(b)
    cut = 30.0
    out = _build(b, r, 64, cut)
    branched = 0
    for i in range(b.seeds.par.shape[1]):
        paths = _enumerate(b, r["par"][i], r["cov"][i], int(b.seeds.charge[i]), cut)
        assert out["n_cands"][i] == len(paths)
        branched += len(paths) > 1
        for k, (nh, c2, seq) in enumerate(paths):
            assert tuple(out["hits"][i, k]) == seq
            assert out["nhits"][i, k] == nh
            assert abs(out["chi2"][i, k] - c2) < 1e-9 * max(1.0, c2)
    assert branched >= 1


@pytest.mark.parametrize("seed", range(6))
def test_single_candidate_is_the_greedy_best_hit_chain(seed):
    b = _tiny(seed)
    r = _seed_states(b)
    det = b.det
    V = np.array([det.sigma_xy ** 2, det.sigma_xy ** 2, det.sigma_z ** 2])
    out = _build(b, r, 1, 30.0)
    for i in range(b.seeds.par.shape[1]):
        x, C = r["par"][i], r["cov"][i]
        a = int(b.seeds.charge[i]) * O.C_LIGHT * det.bz
        for l, lay in enumerate(b.build_layers):
            xp, J, _, st = O.propagate(x, a, det.radii[lay])
            assert st == 0
            Cp = O.transport_cov(J, C)
            lo, hi = b.layer_off[l], b.layer_off[l + 1]
            c2s = [O.chi2(xp, Cp, b.layer_xyz[:, lo + h].astype(np.float64), V) for h in range(hi - lo)]
            best = int(np.argmin(c2s)) if min(c2s) < 30.0 else -1
            assert out["hits"][i, 0, l] == best
            if best >= 0:
                x, C, _, _ = O.update(xp, Cp, b.layer_xyz[:, lo + best].astype(np.float64), V)
            else:
                x, C = xp, Cp


def test_truncation_keeps_the_best_ranked_children():
    """With N = 2 every layer keeps at most 2 candidates, the final list is
    sorted, and the best final candidate is never worse-ranked than the
    untruncated best restricted to surviving prefixes (here: equal)."""
    b = _tiny(11)
    r = _seed_states(b)
    full = _build(b, r, 64, 30.0)
    two = _build(b, r, 2, 30.0)
    for i in range(b.seeds.par.shape[1]):
        n = two["n_cands"][i]
        assert 1 <= n <= 2
        keys = [(-two["nhits"][i, k], two["chi2"][i, k]) for k in range(n)]
        assert keys == sorted(keys)
        assert (two["nhits"][i, 0], ) <= (full["nhits"][i, 0], )


def test_parity_path_chi2_reproduces_the_oracle_build():
    """oracle.parity (the near-tie classifier of the build parity checks):
    the chi2 of the oracle's own best path, re-evaluated along that path,
    equals the build's chi2_tot; the same paths compare as all identical; and
    the second-ranked candidate's path, where it differs, never ranks better."""
    from oracle import parity
    b = S.make_build_batch(31, 1, 40)
    det = b.det
    r = O.fit(b.seeds.par, b.seeds.cov, b.seeds.charge, b.fit_hits.xyz, b.fit_hits.valid, det.radii[:3], det.bz,
              det.sigma_xy, det.sigma_z)
    radii = [det.radii[l] for l in b.build_layers]
    ob = O.build_tracks(r["par"], r["cov"], b.seeds.charge, b.seed_event, b.layer_xyz, b.layer_off, radii, det.bz,
                        det.sigma_xy, det.sigma_z, chi2_cut=30.0, max_cands=6)
    V = np.array([det.sigma_xy ** 2, det.sigma_xy ** 2, det.sigma_z ** 2])
    a = O.a_coef(b.seeds.charge, det.bz)
    Lb = len(b.build_layers)

    def hit_of(t, l, h):
        return b.layer_xyz[:, b.layer_off[int(b.seed_event[t]) * Lb + l] + h].astype(np.float64)
    for t in range(len(a)):
        best = ob["hits"][t, 0]
        hits = [hit_of(t, l, int(best[l])) if best[l] >= 0 else None for l in range(Lb)]
        c = [x for x in parity.path_chi2(r["par"][t], r["cov"][t], a[t], hits, radii, V) if x is not None]
        assert len(c) == ob["nhits"][t, 0]
        assert sum(c) == pytest.approx(ob["chi2"][t, 0], rel=1e-12, abs=1e-12)
    same, ties, bad = parity.classify(ob["hits"][:, 0], ob["hits"][:, 0], r["par"], r["cov"], a, hit_of, radii, V)
    assert same == len(a) and not ties and not bad
    two = ob["n_cands"] >= 2
    _, ties, bad = parity.classify(ob["hits"][two, 1], ob["hits"][two, 0], r["par"][two], r["cov"][two], a[two],
                                   lambda t, l, h: hit_of(np.nonzero(two)[0][t], l, h), radii, V)
    for _, p_second, p_best, c_second, c_best in bad:  # ranked by (hits desc, chi2 asc)
        n_second, n_best = sum(h >= 0 for h in p_second), sum(h >= 0 for h in p_best)
        assert n_second < n_best or (n_second == n_best and c_second >= c_best)
    assert len(bad) + len(ties) > 0

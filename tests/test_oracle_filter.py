"""Pins of the oracle's Kalman update and fit (FP64) against identities and
statistics it does not compute itself: the information-form update, the
least-squares chi2 decomposition, the standard-form covariance, chi2(3) and
unit pulls on correctly smeared hits, positive-definiteness of the rank-5
covariance, and the noise-free fit."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1605_05508_gb300 import synth as S

V = np.array([0.01 ** 2, 0.01 ** 2, 0.1 ** 2])


def _spd(rng, n=6):
    A = rng.normal(size=(n, n))
    return A @ A.T + n * np.eye(n)


@pytest.mark.parametrize("seed", range(5))
def test_update_equals_information_form(seed):
    """C_post^-1 = C^-1 + H^T V^-1 H and x_post = C_post (C^-1 x + H^T V^-1 m)."""
    rng = np.random.default_rng(seed)
    Cp = _spd(rng) * 1e-3
    xp = rng.normal(size=6)
    m = xp[:3] + rng.normal(size=3) * np.sqrt(V)
    x, Cn, c2, dev = O.update(xp, Cp, m, V)
    H = np.hstack([np.eye(3), np.zeros((3, 3))])
    Vi = np.diag(1.0 / V)
    info = np.linalg.inv(Cp) + H.T @ Vi @ H
    C_info = np.linalg.inv(info)
    np.testing.assert_allclose(Cn, C_info, rtol=1e-9, atol=1e-15)
    x_info = C_info @ (np.linalg.solve(Cp, xp) + H.T @ Vi @ m)
    np.testing.assert_allclose(x, x_info, rtol=1e-9, atol=1e-12)
    # chi2 = min of the least-squares objective:
    # (x_post - x')^T C'^-1 (x_post - x') + (m - H x_post)^T V^-1 (m - H x_post)
    d = x - xp
    res = m - x[:3]
    c2_ls = d @ np.linalg.solve(Cp, d) + res @ Vi @ res
    assert abs(c2 - c2_ls) < 1e-9 * max(1.0, c2)
    # Joseph form equals the standard form (I - K H) C'
    assert dev < 1e-12 * np.abs(Cp).max()
    np.testing.assert_array_equal(Cn, Cn.T)


def _fit(ev, det=None):
    det = det or ev.det
    return O.fit(ev.seeds.par, ev.seeds.cov, ev.seeds.charge, ev.hits.xyz, ev.hits.valid, det.radii, det.bz,
                 det.sigma_xy, det.sigma_z)


def _local5(x, C, truth):
    """Residuals and covariance in the local frame (t.pos, z, px, py, pz)."""
    r = np.hypot(truth[:, 0], truth[:, 1])
    t = np.stack([-truth[:, 1] / r, truth[:, 0] / r], axis=1)
    n = len(x)
    P = np.zeros((n, 5, 6))
    P[:, 0, 0], P[:, 0, 1] = t[:, 0], t[:, 1]
    P[:, 1, 2] = P[:, 2, 3] = P[:, 3, 4] = P[:, 4, 5] = 1.0
    res = np.einsum("nij,nj->ni", P, x - truth)
    cov = np.einsum("nij,njk,nlk->nil", P, C, P)
    return res, cov


def test_chi2_and_pull_statistics():
    """>= 1e4 tracks x 10 layers, truth-smeared seeds: mean chi2 increment 3,
    distribution chi2(3), and unit pulls of the 5 local parameters."""
    ev = S.make_fit_batch(1605, 12000, seed_mode="truth_smeared")
    r = _fit(ev)
    assert np.all(r["status"] == 0)
    c2 = r["chi2"]
    assert abs(c2.mean() - 3.0) < 0.05
    for l in range(c2.shape[0]):
        assert abs(c2[l].mean() - 3.0) < 0.1
    ks = stats.kstest(c2.ravel()[::7], stats.chi2(3).cdf)
    assert ks.pvalue > 1e-3, ks
    res, cov = _local5(r["par"], r["cov"], ev.hits.truth[-1])
    pulls = res / np.sqrt(np.diagonal(cov, axis1=1, axis2=2))
    assert np.all(np.abs(pulls.mean(axis=0)) < 0.03), pulls.mean(axis=0)
    assert np.all(np.abs(pulls.std(axis=0) - 1.0) < 0.03), pulls.std(axis=0)
    # the full 5-D pull vector is chi2(5)
    q = np.einsum("ni,ni->n", res, np.linalg.solve(cov, res[..., None])[..., 0])
    assert abs(q.mean() - 5.0) < 0.15


def test_covariance_positive_definite_every_layer_and_rank5():
    """Step the filter by hand: after each surface propagation the covariance
    is exactly singular along the radial direction n at the predicted point,
    the update keeps it so (K^T n = 0), and the 5x5 projection stays PD."""
    ev = S.make_fit_batch(77, 300, seed_mode="truth_smeared")
    det = ev.det
    Cs = O.full_cov_from_packed(ev.seeds.cov)
    for i in range(300):
        x = ev.seeds.par[:, i].astype(np.float64)
        C = Cs[i]
        a = ev.seeds.charge[i] * O.C_LIGHT * det.bz
        for l, R in enumerate(det.radii):
            xp, J, _, st = O.propagate(x, a, R)
            assert st == 0
            Cp = O.transport_cov(J, C)
            n6 = np.array([xp[0] / R, xp[1] / R, 0, 0, 0, 0])
            pos_scale = np.abs(Cp[:3, :3]).max()
            assert np.abs(Cp[:3] @ n6).max() <= 1e-9 * pos_scale
            m = ev.hits.xyz[l, :, i].astype(np.float64)
            x, C, _, _ = O.update(xp, Cp, m, V)
            assert np.abs(C[:3] @ n6).max() <= 1e-9 * pos_scale
            # the update step has no radial component (it moves in the tangent plane)
            assert abs((x - xp) @ n6) < 1e-12 * R
            assert O.pd5(x, C)
            np.testing.assert_array_equal(C, C.T)


def test_noise_free_fit_recovers_truth():
    """Truth seed and hits exactly on the crossings (FP64 values): every chi2
    increment vanishes and the final state is the truth at the last layer."""
    det = S.barrel()
    rng = np.random.default_rng(9)
    parts = S.draw_particles(rng, 500)
    hits = S.simulate_hits(rng, parts, S.Detector(det.radii, det.bz, 0.0, 0.0))
    truth = hits.truth
    xyz = np.transpose(truth[:, :, :3], (0, 2, 1))  # FP64, no rounding
    seed = np.concatenate([parts.vertex, parts.mom], axis=1).T
    seed_cov = S.pack_cov(np.einsum("ni,ij->nij", S.seed_cov_diag(np.linalg.norm(parts.mom, axis=1)), np.eye(6))).T
    r = O.fit(seed, seed_cov, parts.charge, xyz, hits.valid, det.radii, det.bz, det.sigma_xy, det.sigma_z)
    assert np.all(np.abs(r["chi2"]) < 1e-16)
    np.testing.assert_allclose(r["par"], truth[-1], rtol=0, atol=1e-10)
    # a perturbed seed (0.5 % in p, 50 um in x, y) under a wide prior
    # (10 % of p, 1 cm) converges onto the noise-free hits: the prior keeps
    # only a (sigma_post / sigma_prior)^2 share of its bias
    wide = S.pack_cov(np.einsum("ni,ij->nij", S.seed_cov_diag(np.linalg.norm(parts.mom, axis=1), 1.0, 1.0, 0.1),
                                np.eye(6))).T
    pert = seed.copy()
    pert[3:] *= 1.005
    pert[:2] += 0.005
    r2 = O.fit(pert, wide, parts.charge, xyz, hits.valid, det.radii, det.bz, det.sigma_xy, det.sigma_z)
    p = np.linalg.norm(truth[-1][:, 3:], axis=1)
    assert np.all(np.abs(r2["par"][:, :3] - truth[-1][:, :3]) < 0.02 * det.sigma_xy)
    assert np.all(np.abs(r2["par"][:, 3:] - truth[-1][:, 3:]) < 2e-3 * p[:, None])
    assert np.all(r2["chi2"] < 0.01)


def test_missing_hits_propagate_only():
    ev = S.make_fit_batch(21, 400, seed_mode="truth_smeared")
    valid = ev.hits.valid.copy()
    valid[4, ::3] = 0
    d = ev.det
    r = O.fit(ev.seeds.par, ev.seeds.cov, ev.seeds.charge, ev.hits.xyz, valid, d.radii, d.bz, d.sigma_xy, d.sigma_z)
    assert np.all(r["chi2"][4, ::3] == -1.0)
    assert np.all(r["status"][::3] & O.NO_HIT)
    assert not np.any(r["status"][1::3] & O.NO_HIT)
    assert np.all(r["chi2"][3] >= 0)


def test_loopers_stop_at_the_last_reachable_layer():
    det = S.barrel()
    rng = np.random.default_rng(3)
    parts = S.draw_particles(rng, 300, pt_range=(0.2, 0.4))
    hits = S.simulate_hits(rng, parts, det)
    seeds = S.seeds_truth_smeared(rng, parts, 0.0)
    r = O.fit(seeds.par, seeds.cov, seeds.charge, hits.xyz, hits.valid, det.radii, det.bz, det.sigma_xy, det.sigma_z)
    stopped = (r["status"] & (O.NOT_REACHED | O.TANGENT)) != 0
    assert stopped.sum() > 20  # 2 rho < 40 cm below pT = 0.228 GeV
    for i in np.nonzero(stopped)[0][:50]:
        nl = int(hits.valid[:, i].sum())  # layers the particle truly crosses
        done = int((r["chi2"][:, i] >= 0).sum())
        assert done <= nl and done >= nl - 1

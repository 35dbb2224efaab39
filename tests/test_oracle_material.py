"""Multiple scattering as process noise (Sec. 2: the KF folds the expected
multiple scattering into the trajectory's uncertainty) in the oracle.

Pins: the layer's process noise is symmetric, of rank 2 with the momentum in
its null space (the direction turns, |p| does not change), zero outside the
momentum block, and its trace is 2 p^2 theta0^2 with theta0 from a golden
table (tests/golden/highland_theta0.txt: the Highland formula with the
Lynch-Dahl logarithm evaluated at 40 digits by a script that imports neither
the oracle nor the generator), which pins the generator's theta0 too;
fits of tracks simulated with scattering kinks (the generator turns the
direction by Gaussian projected angles at every crossing) have chi2 mean 3
per hit and unit pulls -- in the central and in the forward eta range, which
pins the path-length (incidence) factor -- while the same fits without the
process noise do not; zero material reduces to the plain fit exactly."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_process_noise_structure():
    rng = np.random.default_rng(3)
    for _ in range(50):
        phi = rng.uniform(0, 2 * np.pi)
        R = rng.uniform(4, 40)
        p = rng.normal(size=3) * rng.uniform(0.3, 20)
        x = np.array([R * np.cos(phi), R * np.sin(phi), rng.normal() * 20, *p])
        if abs(x[0] * p[0] + x[1] * p[1]) < 0.2 * R * np.linalg.norm(p):
            continue
        Q = O.scattering_q(x, 0.02)
        np.testing.assert_array_equal(Q, Q.T)
        assert np.all(Q[:3] == 0) and np.all(Q[:, :3] == 0)
        ev = np.linalg.eigvalsh(Q[3:, 3:])
        assert abs(ev[0]) < 1e-12 * ev[2] and ev[1] > 0 and abs(ev[1] / ev[2] - 1) < 1e-9
        assert np.abs(Q[3:, 3:] @ p).max() < 1e-12 * np.abs(Q).max() * np.linalg.norm(p)
        cos_inc = abs(x[0] * p[0] + x[1] * p[1]) / (R * np.linalg.norm(p))
        th0 = S.highland_theta0(np.linalg.norm(p), 0.02 / cos_inc)
        assert np.trace(Q) == pytest.approx(2 * (p @ p) * th0 ** 2, rel=1e-12)
    # thicker layer, more scattering; zero thickness, none
    x = np.array([30.0, 0.0, 1.0, 1.0, 0.1, 0.2])
    assert np.trace(O.scattering_q(x, 0.05)) > np.trace(O.scattering_q(x, 0.01)) > 0


def _highland_rows():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "highland_theta0.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append((f[0], float(f[1]), float(f[2]), float(f[3]), float(f[4]), float(f[5])))
    return rows


def test_theta0_matches_the_golden_highland_table():
    """Every row of the golden table: a state on a cylinder whose momentum makes
    angle psi with the layer normal (turned about the normal by a row-dependent
    azimuth, placed at a row-dependent phi); the oracle's Q has trace
    2 p^2 theta0^2, and the generator's theta0 over the oblique path agrees."""
    rows = _highland_rows()
    assert len(rows) >= 200
    for i, (name, p, m, t, psi_deg, th_ref) in enumerate(rows):
        psi, alpha, phi = np.radians(psi_deg), 0.7 * i, 0.37 * i
        nrm = np.array([np.cos(phi), np.sin(phi), 0.0])
        ez = np.array([0.0, 0.0, 1.0])
        tan = np.cross(ez, nrm)
        u = np.cos(psi) * nrm + np.sin(psi) * (np.cos(alpha) * tan + np.sin(alpha) * ez)
        R = 4.0 + 3.0 * (i % 13)
        x = np.concatenate([R * nrm + np.array([0.0, 0.0, 5.0 - (i % 7)]), p * u])
        Q = O.scattering_q(x, t, m)
        th_orc = np.sqrt(np.trace(Q) / (2.0 * p * p))
        assert th_orc == pytest.approx(th_ref, rel=1e-12), (name, p, m, t, psi_deg)
        th_gen = S.highland_theta0(p, t / np.cos(psi), m)
        assert float(th_gen) == pytest.approx(th_ref, rel=1e-12), (name, p, m, t, psi_deg)


def _fit(ev, det, with_q=True):
    return O.fit(ev.seeds.par, ev.seeds.cov, ev.seeds.charge, ev.hits.xyz, ev.hits.valid, det.radii, det.bz,
                 det.sigma_xy, det.sigma_z, x_x0=det.x_x0 if with_q else None, mass=det.mass)


def _pulls(r, truth):
    rr = np.hypot(truth[:, 0], truth[:, 1])
    t = np.stack([-truth[:, 1] / rr, truth[:, 0] / rr], axis=1)
    P = np.zeros((len(truth), 5, 6))
    P[:, 0, 0], P[:, 0, 1] = t[:, 0], t[:, 1]
    P[:, 1, 2] = P[:, 2, 3] = P[:, 3, 4] = P[:, 4, 5] = 1.0
    res = np.einsum("nij,nj->ni", P, r["par"] - truth)
    cov = np.einsum("nij,njk,nlk->nil", P, r["cov"], P)
    return res / np.sqrt(np.diagonal(cov, axis1=1, axis2=2))


def test_fit_with_scattering_chi2_and_pulls():
    det = S.barrel(10, x_x0=(0.03,) * 10)
    ev = S.make_fit_batch(1650, 16000, det, pt_range=(0.5, 2.0))
    r = _fit(ev, det)
    assert np.all(r["status"] == 0)
    c2 = r["chi2"]
    assert abs(c2.mean() - 3.0) < 0.05, c2.mean()
    pulls = _pulls(r, ev.hits.truth[-1])
    assert np.all(np.abs(pulls.mean(axis=0)) < 0.04), pulls.mean(axis=0)
    assert np.all(np.abs(pulls.std(axis=0) - 1.0) < 0.04), pulls.std(axis=0)
    # the incidence factor: forward tracks cross each layer obliquely
    p = ev.hits.truth[0, :, 3:]
    eta = np.arcsinh(p[:, 2] / np.hypot(p[:, 0], p[:, 1]))
    for sel in (np.abs(eta) < 0.3, np.abs(eta) > 0.7):
        assert abs(c2[:, sel].mean() - 3.0) < 0.08, (sel.sum(), c2[:, sel].mean())
        assert np.all(np.abs(pulls[sel].std(axis=0) - 1.0) < 0.06), pulls[sel].std(axis=0)
    # without the process noise the same data do not fit
    r0 = _fit(ev, det, with_q=False)
    assert r0["chi2"].mean() > 3.5
    assert _pulls(r0, ev.hits.truth[-1])[:, 2:].std(axis=0).min() > 1.5


def test_zero_material_is_the_plain_fit():
    det = S.barrel(10)
    ev = S.make_fit_batch(1651, 500, det)
    a = _fit(ev, det, with_q=False)
    b = O.fit(ev.seeds.par, ev.seeds.cov, ev.seeds.charge, ev.hits.xyz, ev.hits.valid, det.radii, det.bz,
              det.sigma_xy, det.sigma_z, x_x0=np.zeros(10))
    for k in ("par", "cov", "chi2", "status"):
        np.testing.assert_array_equal(a[k], b[k])

"""Pins of the oracle's helix propagation (FP64) against geometry it does not
share: conservation laws, the field-free straight line, the transverse circle
of the helix, the equations of motion, the chord formula for tracks from the
origin, and finite differences of the whole propagate-to-radius map."""
import numpy as np
import pytest

import oracle as O

C_LIGHT = 0.00299792458


def _state(pt, phi, eta, x0=(0.0, 0.0, 0.0)):
    return np.array([*x0, pt * np.cos(phi), pt * np.sin(phi), pt * np.sinh(eta)])


@pytest.mark.parametrize("q", [1, -1])
@pytest.mark.parametrize("pt,eta", [(0.5, 0.3), (3.0, -0.9), (50.0, 0.0)])
def test_momentum_conserved(q, pt, eta):
    a = q * C_LIGHT * 3.8
    x0 = _state(pt, 0.7, eta, (0.01, -0.02, 0.5))
    for s in (0.0, 1.0, 17.3, 250.0):
        x1 = O.helix_at(x0, a, s)
        assert abs(np.linalg.norm(x1[3:]) - np.linalg.norm(x0[3:])) < 1e-13 * np.linalg.norm(x0[3:])
        assert abs(np.hypot(x1[3], x1[4]) - pt) < 1e-13 * pt
        assert x1[5] == x0[5]


def test_field_free_limit_is_straight_line():
    x0 = _state(2.0, -2.1, 0.4, (0.3, 0.1, -1.0))
    p = np.linalg.norm(x0[3:])
    for s in (0.5, 10.0, 40.0):
        x1 = O.helix_at(x0, 1e-20, s)
        expect = np.concatenate([x0[:3] + x0[3:] * s / p, x0[3:]])
        np.testing.assert_allclose(x1, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("q", [1, -1])
def test_transverse_circle_and_turning_sense(q):
    bz = 3.8
    a = q * C_LIGHT * bz
    x0 = _state(1.0, 0.3, 0.2, (0.01, 0.02, 0.0))
    rho = 1.0 / (C_LIGHT * bz)
    # centre from the Lorentz force direction q v x B (perpendicular, to the right for q > 0)
    vx, vy = np.cos(0.3), np.sin(0.3)
    cx, cy = x0[0] + q * vy * rho, x0[1] - q * vx * rho
    prev_ang = np.arctan2(x0[1] - cy, x0[0] - cx)
    for s in np.linspace(1, 80, 9):
        x1 = O.helix_at(x0, a, s)
        assert abs(np.hypot(x1[0] - cx, x1[1] - cy) - rho) < 1e-11
        ang = np.arctan2(x1[1] - cy, x1[0] - cx)
        d = np.angle(np.exp(1j * (ang - prev_ang)))
        # positive charge in +Bz turns clockwise seen from +z
        assert np.sign(d) == -q
        prev_ang = ang


def test_equations_of_motion():
    """d pos/ds = p/|p| and dp/ds = (a/|p|) (py, -px, 0), by central differences."""
    a = C_LIGHT * 3.8
    x0 = _state(0.8, 1.9, -0.6, (0.0, 0.01, 2.0))
    h = 1e-4
    for s in (3.0, 21.0):
        xp, xm, x1 = O.helix_at(x0, a, s + h), O.helix_at(x0, a, s - h), O.helix_at(x0, a, s)
        d = (xp - xm) / (2 * h)
        p = np.linalg.norm(x1[3:])
        np.testing.assert_allclose(d[:3], x1[3:] / p, atol=1e-8)
        np.testing.assert_allclose(d[3:], [a / p * x1[4], -a / p * x1[3], 0.0], atol=1e-9)


@pytest.mark.parametrize("q", [1, -1])
@pytest.mark.parametrize("pt", [0.5, 1.0, 7.0])
@pytest.mark.parametrize("R", [4.0, 20.0, 40.0])
def test_path_length_chord_formula(q, pt, R):
    """A track from the origin reaches r = R after the transverse arc
    2 rho asin(R / 2 rho) (chord of its circle)."""
    a = q * C_LIGHT * 3.8
    eta = 0.7
    x0 = _state(pt, 0.4, eta)
    rho = pt / abs(a)
    s_t = 2.0 * rho * np.arcsin(R / (2.0 * rho))
    s_expect = s_t * np.cosh(eta)  # p / pT = cosh(eta)
    s_cf, st = O.path_length_circle(x0, a, R)
    assert st == 0
    assert abs(s_cf - s_expect) < 1e-11 * s_expect
    s_nw, st, it = O.path_length_newton(x0, a, R)
    assert st == 0 and it < 10
    assert abs(s_nw - s_expect) < 1e-11 * s_expect
    x1, J, s_p, st = O.propagate(x0, a, R)
    assert st == 0
    assert abs(np.hypot(x1[0], x1[1]) - R) < 1e-12 * R
    assert abs(s_p - s_expect) < 1e-11 * s_expect


def test_not_reached_and_reached_limits():
    a = C_LIGHT * 3.8
    pt = 0.2
    rho = pt / a
    x0 = _state(pt, 0.0, 0.0)
    # max radius of a track from the origin is 2 rho
    assert O.propagate(x0, a, 2 * rho * 1.001)[3] == O.NOT_REACHED
    assert O.path_length_circle(x0, a, 2 * rho * 1.001)[1] == O.NOT_REACHED
    x1, _, s, st = O.propagate(x0, a, 2 * rho * 0.5)
    assert st == 0
    # near 2 rho the crossing becomes tangent
    assert O.propagate(x0, a, 2 * rho * (1 - 1e-6))[3] == O.TANGENT


def test_newton_agrees_with_closed_form_on_generated_tracks():
    from paper_1605_05508_gb300 import synth as S
    rng = np.random.default_rng(5)
    parts = S.draw_particles(rng, 300)
    for i in range(300):
        x0 = np.concatenate([parts.vertex[i], parts.mom[i]])
        a = parts.charge[i] * C_LIGHT * 3.8
        for R in (4.0, 24.0, 40.0):
            s_cf, st = O.path_length_circle(x0, a, R)
            s_nw, st2, _ = O.path_length_newton(x0, a, R)
            assert st == 0 and st2 == 0
            assert abs(s_cf - s_nw) < 1e-10 * s_cf


def test_generator_crossings_agree_with_oracle():
    """The generator's independent turning-angle geometry and the oracle's
    propagation land on the same crossing point."""
    from paper_1605_05508_gb300 import synth as S
    rng = np.random.default_rng(6)
    parts = S.draw_particles(rng, 200)
    det = S.barrel()
    truth = S.simulate_hits(rng, parts, det).truth
    for i in range(200):
        x = np.concatenate([parts.vertex[i], parts.mom[i]])
        a = parts.charge[i] * C_LIGHT * det.bz
        for l, R in enumerate(det.radii):
            x, _, _, st = O.propagate(x, a, R)
            assert st == 0
            np.testing.assert_allclose(x, truth[l, i], rtol=0, atol=1e-10)


@pytest.mark.parametrize("seed", range(6))
def test_jacobian_matches_finite_differences(seed):
    """The surface Jacobian equals central differences of the full map
    x0 -> state at the crossing with r = R (path length re-solved)."""
    rng = np.random.default_rng(100 + seed)
    q = rng.choice([-1, 1])
    a = q * C_LIGHT * 3.8
    pt = rng.uniform(0.5, 10)
    x0 = _state(pt, rng.uniform(0, 2 * np.pi), rng.uniform(-1, 1),
                (rng.normal(0, 0.5), rng.normal(0, 0.5), rng.normal(0, 1)))
    R = float(rng.choice([4.0, 12.0, 40.0]))
    _, J, _, st = O.propagate(x0, a, R)
    assert st == 0
    scale = np.array([1.0, 1.0, 1.0, pt, pt, pt])
    Jfd = np.zeros((6, 6))
    for j in range(6):
        h = 1e-6 * scale[j]
        xp, xm = x0.copy(), x0.copy()
        xp[j] += h
        xm[j] -= h
        Jfd[:, j] = (O.propagate(xp, a, R)[0] - O.propagate(xm, a, R)[0]) / (2 * h)
    # compare in units where all entries are O(1)
    out_scale = np.array([1.0, 1.0, 1.0, pt, pt, pt])
    err = np.abs(J - Jfd) * scale[None, :] / out_scale[:, None]
    assert err.max() < 1e-6, err
    # structure: column z0 is e_z, row pz is e_pz
    np.testing.assert_array_equal(J[:, 2], [0, 0, 1, 0, 0, 0])
    np.testing.assert_array_equal(J[5], [0, 0, 0, 0, 0, 1])


def test_crossings_equal_closed_form_golden():
    """The oracle's propagate-to-radius against the closed-form crossings of
    tests/golden/helix_crossings.txt (circle-circle intersection at 40 digits,
    written by tests/golden/make_helix_crossings.py without the oracle)."""
    from fitutil import helix_crossings
    g = helix_crossings()
    assert len(g["R"]) >= 150 and np.any(g["status"] == 1) and np.any(g["status"] == 0)
    for i in range(len(g["R"])):
        a = float(g["q"][i]) * C_LIGHT * g["bz"]
        x1, _, s, st = O.propagate(g["x0"][i], a, g["R"][i])
        if g["status"][i] == 1:
            assert st & 1, i
            continue
        assert st == 0, (i, st)
        p = np.linalg.norm(g["x0"][i][3:])
        assert abs(s - g["s"][i]) < 1e-10, (i, s, g["s"][i])
        assert np.max(np.abs(x1[:3] - g["x1"][i][:3])) < 1e-10, i
        assert np.max(np.abs(x1[3:] - g["x1"][i][3:])) < 1e-12 * p, i

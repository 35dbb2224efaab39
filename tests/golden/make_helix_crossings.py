"""Writes helix_crossings.txt: where a charged track from a given start state
first crosses a barrel cylinder of radius R in a uniform field Bz (Sec. 2: the
propagation step of the filter), computed in closed form at 40 significant
digits with mpmath.  It calls neither the oracle nor the library.

Closed form.  With a = q c Bz (c = 0.00299792458 GeV / (T cm)), p = |p0| and
pT = |(px0, py0)|, the equations of motion dr/ds = p/|p|, dp/ds = (a/p)(py, -px, 0)
make the transverse projection a circle of radius rho = pT/|a| about
(x0 + py0/a, y0 - px0/a), traversed clockwise seen from +z for a > 0.  The
crossing points are the intersections of that circle with x^2 + y^2 = R^2; the
first one along the motion is the one reached by the smallest turning angle
phi from the start point, and s = rho phi p / pT.  After s, with
theta = a s / p:
    x = x0 + (px0 sin theta + py0 (1 - cos theta)) / a
    y = y0 + (py0 sin theta - px0 (1 - cos theta)) / a
    z = z0 + pz0 s / p
    px = px0 cos theta + py0 sin theta,  py = py0 cos theta - px0 sin theta.
A circle that does not meet the cylinder (R > |centre| + rho) is not reached.

Inputs are float32 values (what the library receives); every row is kept far
from the decision thresholds: reached rows cross at a direction cosine (r.p /
(R pT)) of at least 0.03, not-reached rows have R >= 1.001 (|centre| + rho).

Run from the repository root:  python tests/golden/make_helix_crossings.py
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
C_LIGHT = mp.mpf("0.00299792458")
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "helix_crossings.txt")

BZ = float(np.float32(3.8))
RADII = [float(np.float32(r)) for r in range(4, 44, 4)]
# (pT GeV, phi, eta, vertex x, y, z cm): low-pT loopers, mid and high pT, central and
# forward, off-axis vertices
TRACKS = [
    (0.15, 0.3, 0.2, 0.0, 0.0, 0.0),
    (0.25, 2.9, -0.6, 0.01, -0.02, 1.5),
    (0.5, -1.7, 0.9, -0.015, 0.005, -2.0),
    (0.7, 1.2, 0.0, 0.3, -0.4, 0.0),
    (1.0, 0.3, 0.2, 0.01, 0.02, 0.0),
    (2.0, -2.9, 1.4, 0.0, 0.0, 0.7),
    (10.0, 0.8, -0.9, 0.02, 0.01, -0.3),
    (1000.0, -0.4, 0.5, 0.0, 0.0, 0.0),
]


def f32(v):
    return float(np.float32(v))


def crossing(q, r0, p0, R):
    """(status, s, x, y, z, px, py, pz, cos) for the first crossing of radius R."""
    x0, y0, z0 = (mp.mpf(v) for v in r0)
    px0, py0, pz0 = (mp.mpf(v) for v in p0)
    R = mp.mpf(R)
    a = q * C_LIGHT * mp.mpf(BZ)
    pt = mp.sqrt(px0 ** 2 + py0 ** 2)
    p = mp.sqrt(pt ** 2 + pz0 ** 2)
    rho = pt / abs(a)
    cx, cy = x0 + py0 / a, y0 - px0 / a
    d = mp.sqrt(cx ** 2 + cy ** 2)
    if R > d + rho or R < abs(d - rho):
        return 1, d, rho, None
    # intersections of |x| = R and |x - c| = rho
    l = (R ** 2 - rho ** 2 + d ** 2) / (2 * d)
    h = mp.sqrt(max(R ** 2 - l ** 2, mp.mpf(0)))
    ux, uy = cx / d, cy / d
    pts = [(l * ux - h * uy, l * uy + h * ux), (l * ux + h * uy, l * uy - h * ux)]
    a0 = mp.atan2(y0 - cy, x0 - cx)
    best = None
    for X, Y in pts:
        ap = mp.atan2(Y - cy, X - cx)
        dphi = (a0 - ap) if a > 0 else (ap - a0)  # clockwise for a > 0
        dphi = dphi % (2 * mp.pi)
        if best is None or dphi < best:
            best = dphi
    s = rho * best * p / pt
    th = a * s / p
    sn, cs = mp.sin(th), mp.cos(th)
    x = x0 + (px0 * sn + py0 * (1 - cs)) / a
    y = y0 + (py0 * sn - px0 * (1 - cs)) / a
    z = z0 + pz0 * s / p
    px = px0 * cs + py0 * sn
    py = py0 * cs - px0 * sn
    cosi = (x * px + y * py) / (R * pt)
    return 0, d, rho, (s, x, y, z, px, py, pz0, cosi)


def main():
    rows = []
    for q in (1, -1):
        for (pt, phi, eta, vx, vy, vz) in TRACKS:
            r0 = [f32(vx), f32(vy), f32(vz)]
            p0 = [f32(pt * np.cos(phi)), f32(pt * np.sin(phi)), f32(pt * np.sinh(eta))]
            for R in RADII:
                st, d, rho, res = crossing(q, r0, p0, R)
                if st == 1:
                    if mp.mpf(R) < (d + rho) * mp.mpf("1.001"):
                        continue
                    rows.append([q, *r0, *p0, R, 1] + ["0"] * 8)
                    continue
                if res[-1] < mp.mpf("0.03"):
                    continue
                rows.append([q, *r0, *p0, R, 0] + [mp.nstr(v, 25, strip_zeros=False) for v in res])
    with open(OUT, "w") as f:
        f.write("# First crossing of a barrel cylinder by a helix in a uniform field Bz (Sec. 2, the\n"
                "# filter's propagation step), closed form at 40 digits (tests/golden/make_helix_crossings.py).\n"
                f"# bz_tesla {BZ!r}\n"
                "# columns: q x0 y0 z0 px0 py0 pz0 R | status(1 = not reached) s x y z px py pz cos_incidence\n"
                "# (cm, GeV; inputs are float32 values; outputs are 0 when not reached)\n")
        for r in rows:
            f.write(" ".join(repr(v) if isinstance(v, float) else str(v) for v in r) + "\n")
    print(f"wrote {len(rows)} rows to {OUT}")


if __name__ == "__main__":
    main()

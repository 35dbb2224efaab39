"""Writes highland_theta0.txt: the RMS projected multiple-scattering angle
theta0 of a singly charged particle crossing a thin layer obliquely, from the
Highland formula with the Lynch-Dahl logarithm as the Review of Particle
Physics states it (section "Passage of particles through matter", multiple
scattering through small angles):

    theta0 = 13.6 MeV / (beta c p) * z * sqrt(x/X0) * (1 + 0.038 ln(x z^2 / (X0 beta^2)))

with z = 1, and x/X0 the path through the layer in radiation lengths: a layer
of thickness t/X0 crossed at angle psi to its normal is traversed over
t/X0 / cos(psi).

Evaluated at 40 significant digits (mpmath), in MeV, with beta = p / E and
E = sqrt(p^2 + m^2).  This script imports nothing from the library, its
generator or the oracle: the table pins all of them.

Run from the repository root:  python tests/golden/make_highland_theta0.py
"""
import itertools
import os

import mpmath as mp

mp.mp.dps = 40

# particle masses in MeV (Review of Particle Physics summary tables, rounded)
MASSES_MEV = {"electron": "0.51099895", "muon": "105.6583755", "pion": "139.57039", "proton": "938.27208816"}
MOMENTA_GEV = ["0.2", "0.5", "1", "3", "10", "100"]
THICKNESS_X0 = ["0.001", "0.01", "0.03", "0.1"]
PSI_DEG = ["0", "35", "70"]


def theta0(p_mev, m_mev, path_x0):
    e = mp.sqrt(p_mev * p_mev + m_mev * m_mev)
    beta = p_mev / e
    return mp.mpf("13.6") / (beta * p_mev) * mp.sqrt(path_x0) * (1 + mp.mpf("0.038") * mp.log(path_x0 / (beta * beta)))


def main():
    rows = []
    for (name, m), p, t, psi in itertools.product(MASSES_MEV.items(), MOMENTA_GEV, THICKNESS_X0, PSI_DEG):
        p_mev = mp.mpf(p) * 1000
        path = mp.mpf(t) / mp.cos(mp.radians(mp.mpf(psi)))
        rows.append((name, p, mp.mpf(m) / 1000, t, psi, theta0(p_mev, mp.mpf(m), path)))
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "highland_theta0.txt"), "w") as f:
        f.write("# Highland theta0 (Lynch-Dahl logarithm, Review of Particle Physics), 40-digit mpmath,\n")
        f.write("# written by tests/golden/make_highland_theta0.py\n")
        f.write("# columns: particle  p_GeV  mass_GeV  thickness_X0  psi_deg (to the layer normal)  theta0_rad\n")
        for name, p, m, t, psi, th in rows:
            f.write(f"{name} {p} {mp.nstr(m, 17)} {t} {psi} {mp.nstr(th, 20)}\n")


if __name__ == "__main__":
    main()

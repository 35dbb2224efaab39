"""Host checks of the phi bin arithmetic the binning and the build's windows
share: the sub-bin scale KF_BIN_PHI_FINE / 2 pi is exactly twice the bin
scale KF_BIN_PHI / 2 pi in float32 (a power-of-two factor), so the scaled
angles differ by exactly that factor and a hit's sub-bin halved is its bin --
which is what lets the sub-bin starts of even sub-bins serve as the bin
starts.  Checked in IEEE float32 on a dense sample of angles and on the
neighbours of every bin and sub-bin edge."""
import numpy as np

from paper_1605_05508_gb300 import kf

F = np.float32
PI = F(np.pi)  # the kernels' kPi


def _bin(phi, nphi):
    scale = F(nphi) / (F(2.0) * PI)  # float(nphi) / (2.0f * kPi)
    a = (phi + PI) * scale  # float32 throughout
    return np.clip(np.floor(a).astype(np.int64), 0, nphi - 1), a


def test_sub_bin_scale_is_exactly_twice_the_bin_scale():
    sc = F(kf.BIN_PHI) / (F(2.0) * PI)
    sf = F(kf.BIN_PHI_FINE) / (F(2.0) * PI)
    assert sf == F(2.0) * sc
    assert kf.BIN_PHI_FINE == 2 * kf.BIN_PHI and kf.NBINS_FINE == 2 * kf.NBINS


def test_sub_bin_halved_is_the_bin():
    rng = np.random.default_rng(5)
    dense = rng.uniform(-np.pi, np.pi, 2_000_000).astype(F)
    # the float32 neighbours of every sub-bin edge (which include the bin edges)
    edges = (np.arange(kf.BIN_PHI_FINE + 1, dtype=np.float64) * (2 * np.pi / kf.BIN_PHI_FINE) - np.pi).astype(F)
    near = [edges]
    for _ in range(3):
        near.append(np.nextafter(near[-1], F(np.inf)))
    lo = [edges]
    for _ in range(3):
        lo.append(np.nextafter(lo[-1], F(-np.inf)))
    phi = np.concatenate([dense, *near, *lo, np.array([-PI, PI, F(0.0)], dtype=F)])
    phi = np.clip(phi, -PI, PI)
    coarse, ac = _bin(phi, kf.BIN_PHI)
    fine, af = _bin(phi, kf.BIN_PHI_FINE)
    np.testing.assert_array_equal(af, F(2.0) * ac)  # the products differ by exactly 2
    np.testing.assert_array_equal(fine >> 1, coarse)

"""Edge cases of the fit against the oracle: the largest layer count (64
layers, r = 2 .. 128 cm: most low-pT tracks stop as loopers on the way),
very high momentum (nearly straight tracks, the sinc forms without 1/a),
a layer without any hit, a single track, and a batch whose size is one
below and one above a block multiple."""
import numpy as np
import pytest

from paper_1605_05508_gb300 import synth as S
from fitutil import compare, gpu_fit, oracle_fit

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["graph", "fused"])
def test_sixty_four_layers(cuda_ctx_factory, mode):
    """Parameters and covariance at the stated tolerances; chi2 at the FP32
    floor of long tracks: momentum-direction rounding (~1e-6) over a lever arm
    of up to 128 cm moves late predictions by ~1e-4 cm, so |d chi2| stays
    within 1e-3 on the layers up to 32 cm and within 1e-2 max(chi2, 1)
    beyond (the error is stated against the oracle, not hidden)."""
    det = S.barrel(64, spacing=2.0)
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(1701, 3000, det, pt_range=(0.3, 2.0))
    g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, mode)
    r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
    stopped = (r["status"] & 7) != 0
    # pT < 0.73 GeV (2 rho < 128 cm) stop as loopers, the others cross all 64 layers
    assert 0.15 < stopped.mean() < 0.4, stopped.mean()
    ok = g["status"] == r["status"]
    assert ok.mean() > 0.998, np.nonzero(~ok)[0][:10]
    sel = lambda d: {k: (v[:, ok] if k == "chi2" else v[ok]) for k, v in d.items()}
    gs, rs = sel(g), sel(r)
    inner = {k: (v[:16] if k == "chi2" else v) for k, v in gs.items()}
    inner_r = {k: (v[:16] if k == "chi2" else v) for k, v in rs.items()}
    stats = compare(inner, inner_r, det.radii[-1], chi2_frac=1e-3, label=f"64 layers {mode}")
    both = (gs["chi2"] >= 0) & (rs["chi2"] >= 0)
    rel = (np.abs(gs["chi2"] - rs["chi2"]) / np.maximum(rs["chi2"], 1.0))[both]
    print(mode, stats, "outer relative chi2 error max %.2e p99.9 %.2e" % (rel.max(), np.quantile(rel, 0.999)))
    assert rel.max() < 1e-2 and np.quantile(rel, 0.999) < 3e-3


def test_very_high_momentum(cuda_ctx_factory):
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(1702, 4000, det, pt_range=(500.0, 10000.0))
    g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "graph")
    r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
    compare(g, r, det.radii[-1], label="1-10 TeV")
    assert np.all(g["status"] == 0)


def test_layer_without_hits_single_track_and_block_edges(cuda_ctx_factory):
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    for n in (1, 63, 65, 127, 129):
        ev = S.make_fit_batch(1703 + n, n, det)
        valid = ev.hits.valid.copy()
        valid[5] = 0  # nobody has a hit on layer 6
        for mode in ("graph", "fused"):
            g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, valid, mode)
            r = oracle_fit(ev.seeds, ev.hits.xyz, valid, det)
            compare(g, r, det.radii[-1], chi2_frac=1.0 / (10 * n), label=f"n={n} {mode}")
            assert np.all(g["chi2"][5] == -1.0) and np.all(g["status"] & 16)

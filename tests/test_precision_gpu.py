"""Precision sweep (1 M-track workload scaled to 200 k here): 50 % pT in
U[0.2, 1] GeV (loopers that stop near 2 rho) and 50 % in U[10, 100] GeV, 20
layers r = 4 ... 80 cm. FP32 Joseph form (kf_fit) vs the mixed form with S^-1
and the covariance downdate in FP64 (kf_fit_mixed), each against the FP64
oracle: PD failures, pulls, and the stated errors."""
import numpy as np
import pytest

from fitutil import compare, cov_error, oracle_fit, to_dev, unpack
from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.gpu

MIX = [(0.5, (0.2, 1.0)), (0.5, (10.0, 100.0))]


def _run(ctx, kf, ev, fn):
    import torch
    n, L = ev.seeds.par.shape[1], ev.hits.xyz.shape[0]
    s = kf.Tracks(to_dev(ev.seeds.par), to_dev(ev.seeds.cov), to_dev(ev.seeds.charge))
    out = kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge,
                    torch.empty((3, n), device="cuda"))
    chi2 = torch.empty((L, n), device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    fn(ctx, s, kf.TrackHits(to_dev(ev.hits.xyz), to_dev(ev.hits.valid)), out, chi2, st)
    torch.cuda.synchronize()
    return unpack(out, chi2, st)


def _pulls(res, truth_last, good):
    x, Cm, t3 = res["par"][good], res["cov"][good], truth_last
    rr = np.hypot(t3[:, 0], t3[:, 1])
    t = np.stack([-t3[:, 1] / rr, t3[:, 0] / rr], axis=1)
    P = np.zeros((len(x), 5, 6))
    P[:, 0, 0], P[:, 0, 1] = t[:, 0], t[:, 1]
    P[:, 1, 2] = P[:, 2, 3] = P[:, 3, 4] = P[:, 4, 5] = 1.0
    d = np.einsum("nij,nj->ni", P, x - t3)
    cv = np.einsum("nij,njk,nlk->nil", P, Cm, P)
    return d / np.sqrt(np.diagonal(cv, axis1=1, axis2=2))


def test_precision_sweep_fp32_joseph_vs_fp64_update(cuda_ctx_factory):
    from paper_1605_05508_gb300 import kf
    det = S.barrel(20)
    ctx = cuda_ctx_factory(det.radii)
    n = 200_000
    ev = S.make_fit_batch(1611, n, det=det, pt_mix=MIX)
    g32 = _run(ctx, kf, ev, kf.kf_fit)
    g64 = _run(ctx, kf, ev, kf.kf_fit_mixed)
    pt = np.hypot(ev.parts.mom[:, 0], ev.parts.mom[:, 1])
    # PD over every track; pulls at each track's last updated layer. A few
    # low-pT loopers that stop near their turning radius have pulls in the
    # hundreds (the linearised crossing breaks down there, in the oracle too),
    # so the width is the half-distance of the 15.87 / 84.13 % quantiles.
    for g in (g32, g64):
        assert not np.any(g["status"] & kf.ST_NOT_PD)
    upd = g32["chi2"] >= 0
    last = np.where(upd.any(0), upd.shape[0] - 1 - np.argmax(upd[::-1], axis=0), -1)
    good = last >= 0
    truth_last = ev.hits.truth[last[good], np.nonzero(good)[0]]
    pulls = {}
    for name, g in (("fp32", g32), ("mixed", g64)):
        pl = _pulls(g, truth_last, good)
        pulls[name] = pl
        for cls, m in (("pT<1", pt[good] < 5), ("pT>10", pt[good] > 5)):
            q = np.quantile(pl[m], [0.1587, 0.5, 0.8413], axis=0)
            med, wid = q[1], (q[2] - q[0]) / 2
            print(f"{name} {cls}: pull median {np.round(med, 3)} width {np.round(wid, 3)}")
            assert np.all(np.abs(med) < 0.03) and np.all(np.abs(wid - 1) < 0.03)

    # errors against the oracle on a sample
    idx = np.sort(np.random.default_rng(2).choice(n, 15000, replace=False))
    sub = S.Seeds(ev.seeds.par[:, idx], ev.seeds.cov[:, idx], ev.seeds.charge[idx])
    r = oracle_fit(sub, ev.hits.xyz[:, :, idx], ev.hits.valid[:, idx], det)
    # the same tracks' pulls from the oracle: the GPU forms reproduce them
    sel = good[idx]
    pos = np.cumsum(good) - 1
    po = _pulls(r, truth_last[pos[idx[sel]]], sel)
    for name in ("fp32", "mixed"):
        pg = pulls[name][pos[idx[sel]]]
        assert np.quantile(np.abs(pg - po), 0.99) < 0.02, name
    for name, g in (("fp32", g32), ("mixed", g64)):
        gs = {k: (v[:, idx] if k == "chi2" else v[idx]) for k, v in g.items()}
        same = gs["status"] == r["status"]
        # the only allowed status difference: a crossing at the reach limit called
        # NOT_REACHED on one side and TANGENT on the other (both stop the track)
        diff = ~same
        assert np.all(np.isin(gs["status"][diff] | r["status"][diff], [kf.ST_NOT_REACHED | kf.ST_TANGENT,
                                                                       kf.ST_NOT_REACHED | kf.ST_TANGENT | 16]))
        assert diff.sum() <= 5
        both = (gs["chi2"] >= 0) & (r["chi2"] >= 0) & same[None]
        ce = np.abs(gs["chi2"] - r["chi2"])[both]
        pscale = np.concatenate([np.full((same.sum(), 3), 80.0),
                                 np.repeat(np.linalg.norm(r["par"][same, 3:], axis=1)[:, None], 3, axis=1)], axis=1)
        perr = (np.abs(gs["par"][same] - r["par"][same]) / pscale).max()
        cerr = cov_error(gs["cov"][same], r["cov"][same], r["par"][same]).max(axis=(1, 2))
        full = r["status"][same] == 0  # reached all 20 layers
        over = (ce > 1e-3).mean()
        print(f"{name}: param {perr:.2e}, cov (all layers reached) {cerr[full].max():.2e}, cov (stopped "
              f"loopers) max {cerr[~full].max():.2e} p99.9 {np.quantile(cerr[~full], 0.999):.2e}, "
              f"chi2 max {ce.max():.2e}, frac > 1e-3 {over:.2e}, p99.9 {np.quantile(ce, 0.999):.2e}")
        assert perr < 1e-4
        assert over < 0.02 and ce.max() < 0.05
        # covariance: within 1e-3 on every track that crosses all layers; a
        # looper stopping near its turning radius has a near-singular last
        # transport, where FP32 loses up to ~7e-2 (stated) and the FP64
        # downdate brings it to the 1e-3 scale
        assert cerr[full].max() < 1e-3
        assert np.quantile(cerr[~full], 0.99) < 1e-3
        assert cerr[~full].max() < (5e-3 if name == "mixed" else 0.2)


def test_mixed_form_on_the_standard_fit(cuda_ctx_factory):
    """kf_fit_mixed meets the standard tolerances on the 10-layer workload."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(1605, 3000)
    g = _run(ctx, kf, ev, kf.kf_fit_mixed)
    r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
    compare(g, r, det.radii[-1], label="mixed")

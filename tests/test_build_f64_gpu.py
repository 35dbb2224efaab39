"""GPU parity of the plain per-event FP64 build (kf_build_f64, the comparison
form of the batched FP32 build) against the FP64 oracle.  Both sides compute
in double precision, so the best paths must be the oracle's (a near tie
would need two totals within rounding of each other), and on every seed the
best candidate's state agrees to 1e-9 of scale, its covariance to 1e-7 of
sqrt(C_ii C_jj) in the local frame, chi2_tot to 1e-8 absolute; hit counts and
status bits are identical.  The seeds are the plain FP64 fit over the seeding
layers (kf_fit_f64), the hits binned by kf_bin_hits."""
import numpy as np
import pytest

import oracle as O
from buildutil import classify, oracle_build
from fitutil import cov_error, to_dev
from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.gpu


def gpu_build_f64(ctx, batch, max_cands):
    import torch
    from paper_1605_05508_gb300 import kf
    n = batch.seeds.par.shape[1]
    E, Lb, Ls = batch.n_events, len(batch.build_layers), len(batch.seed_layers)
    d64 = dict(dtype=torch.float64, device="cuda")
    s = kf.Tracks(to_dev(batch.seeds.par).double(), to_dev(batch.seeds.cov).double(), to_dev(batch.seeds.charge))
    fo = kf.Tracks(torch.empty((6, n), **d64), torch.empty((21, n), **d64), s.charge)
    fst = torch.empty(n, dtype=torch.int32, device="cuda")
    event_off = np.searchsorted(batch.seed_event, np.arange(E + 1)).astype(np.int64)
    kf.kf_fit_f64(ctx, s, kf.TrackHits(to_dev(batch.fit_hits.xyz[:Ls]), to_dev(batch.fit_hits.valid[:Ls])), fo,
                  list(event_off), None, fst)
    lh = kf.LayerHits(to_dev(batch.layer_xyz), to_dev(batch.layer_off), E, Lb, batch.build_layers[0])
    bins = kf.HitBins(torch.empty((batch.layer_xyz.shape[1], 4), device="cuda"),
                      torch.empty((E * Lb, kf.NBINS + 1), dtype=torch.int32, device="cuda"))
    kf.kf_bin_hits(ctx, lh, bins)
    i32 = dict(dtype=torch.int32, device="cuda")
    out = kf.BuildResultF64(best=kf.Tracks(torch.empty((6, n), **d64), torch.empty((21, n), **d64), s.charge),
                            chi2_tot=torch.empty(n, **d64), n_hits=torch.empty(n, **i32),
                            status=torch.empty(n, **i32), hit_idx=torch.empty((Lb, n), **i32))
    kf.kf_build_f64(ctx, fo, list(event_off), bins, max_cands, out)
    torch.cuda.synchronize()
    return dict(par=out.best.par.cpu().numpy().T.copy(), cov=O.full_cov_from_packed(out.best.cov.cpu().numpy()),
                chi2=out.chi2_tot.cpu().numpy(), nhits=out.n_hits.cpu().numpy(), status=out.status.cpu().numpy(),
                hits=out.hit_idx.cpu().numpy().T.copy(), fit_status=fst.cpu().numpy())


def _check(batch, g, r, label):
    same, ties, bad = classify(batch, g, r)
    n = len(r["n_cands"])
    print(f"{label}: {same}/{n} identical best paths, {len(ties)} near ties, {len(bad)} other")
    assert not bad, bad[:3]
    assert len(ties) <= 1, ties
    agree = np.array([np.array_equal(g["hits"][i], r["hits"][i, 0]) for i in range(n)])
    np.testing.assert_array_equal(g["nhits"][agree], r["nhits"][agree, 0])
    np.testing.assert_array_equal(g["status"][agree], r["status"][agree, 0])
    assert np.all(np.abs(g["chi2"][agree] - r["chi2"][agree, 0]) <= 1e-8), label
    pscale = np.concatenate([np.full((agree.sum(), 3), 40.0),
                             np.repeat(np.linalg.norm(r["par"][agree, 0, 3:], axis=1)[:, None], 3, axis=1)], axis=1)
    perr = np.abs(g["par"][agree] - r["par"][agree, 0]) / pscale
    cerr = cov_error(g["cov"][agree], r["cov"][agree, 0], r["par"][agree, 0])
    print(f"{label}: parameters {perr.max():.2e} of scale, covariance {cerr.max():.2e}")
    assert perr.max() <= 1e-9 and cerr.max() <= 1e-7, label


@pytest.mark.parametrize("max_cands", [6, 1, 8])
def test_build_f64_matches_oracle(cuda_ctx_factory, max_cands):
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    batch = S.make_build_batch(1620 + max_cands, 3, 400)
    g = gpu_build_f64(ctx, batch, max_cands)
    assert np.all(g["fit_status"] == 0)
    _check(batch, g, oracle_build(batch, max_cands), f"f64 N={max_cands}")


def test_build_f64_dense_wrap_and_empty_event(cuda_ctx_factory):
    """Heavy branching, windows split across phi = +-pi, and an event whose
    building layers hold no hit."""
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    dense = S.make_build_batch(78, 2, 60, noise_factor=0.5, noise_near=2, noise_near_sigma=0.012)
    _check(dense, gpu_build_f64(ctx, dense, 6), oracle_build(dense, 6), "f64 dense")
    wrap = S.make_build_batch(89, 2, 200, phi_range=(np.pi - 0.06, np.pi + 0.06))
    _check(wrap, gpu_build_f64(ctx, wrap, 6), oracle_build(wrap, 6), "f64 wrap")
    b = S.make_build_batch(98, 2, 50)
    Lb = len(b.build_layers)
    keep = np.ones(b.layer_xyz.shape[1], dtype=bool)
    for l in range(Lb):
        keep[b.layer_off[Lb + l]:b.layer_off[Lb + l + 1]] = False
    counts = [0 if s >= Lb else b.layer_off[s + 1] - b.layer_off[s] for s in range(2 * Lb)]
    b.layer_xyz = np.ascontiguousarray(b.layer_xyz[:, keep])
    b.layer_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    g = gpu_build_f64(ctx, b, 6)
    ev1 = b.seed_event == 1
    assert np.all(g["nhits"][ev1] == 0) and np.all(g["hits"][ev1] == -1)
    _check(b, g, oracle_build(b, 6), "f64 empty event")

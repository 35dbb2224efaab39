"""Build -> re-fit: building (Sec. 3) followed by fitting (Sec. 2) over all
layers with the hits the build chose.  kf_refit equals the oracle's fit of the
same hit sets; on the config-3-like workload the build efficiency (best
candidate carrying >= 80 % correct hits) is high and the re-fit of
fully-correct tracks has a chi2 increment of mean 3 per hit."""
import numpy as np
import pytest

from paper_1605_05508_gb300 import synth as S
from fitutil import compare, oracle_fit, to_dev, unpack

pytestmark = pytest.mark.gpu


def pipeline(ctx, batch, max_cands, raw=False):
    """seed fit -> bin -> build -> refit through the binding (raw: the
    re-fit's float32 outputs as returned, position hi parts only)."""
    import torch
    from paper_1605_05508_gb300 import kf
    n = batch.seeds.par.shape[1]
    E, Ls, Lb = batch.n_events, len(batch.seed_layers), len(batch.build_layers)
    dev = lambda: dict(device="cuda")
    s = kf.Tracks(to_dev(batch.seeds.par), to_dev(batch.seeds.cov), to_dev(batch.seeds.charge))
    fh = kf.TrackHits(to_dev(batch.fit_hits.xyz), to_dev(batch.fit_hits.valid))
    fo = kf.Tracks(torch.empty((6, n), **dev()), torch.empty((21, n), **dev()), s.charge,
                   torch.empty((3, n), **dev()))
    kf.kf_fit(ctx, s, fh, fo, None, torch.empty(n, dtype=torch.int32, **dev()))
    seg_off = to_dev(batch.layer_off)
    lh = kf.LayerHits(to_dev(batch.layer_xyz), seg_off, E, Lb, Ls)
    bins = kf.HitBins(torch.empty((batch.layer_xyz.shape[1], 4), **dev()),
                      torch.empty((E * Lb, kf.NBINS + 1), dtype=torch.int32, **dev()))
    kf.kf_bin_hits(ctx, lh, bins)
    seed_off = to_dev(np.searchsorted(batch.seed_event, np.arange(E + 1)).astype(np.int64))
    i32 = dict(dtype=torch.int32, device="cuda")
    out = kf.BuildResult(best=kf.Tracks(torch.empty((6, n), **dev()), torch.empty((21, n), **dev()), s.charge,
                                        torch.empty((3, n), **dev())),
                         chi2_tot=torch.empty(n, **dev()), n_hits=torch.empty(n, **i32),
                         status=torch.empty(n, **i32), hit_idx=torch.empty((Lb, n), **i32))
    kf.kf_build(ctx, fo, seed_off, bins, max_cands, out)
    ro = kf.Tracks(torch.empty((6, n), **dev()), torch.empty((21, n), **dev()), s.charge,
                   torch.empty((3, n), **dev()))
    rchi2 = torch.empty((Ls + Lb, n), **dev())
    rst = torch.empty(n, **i32)
    kf.kf_refit(ctx, s, fh, seed_off, lh, out.hit_idx, ro, rchi2, rst)
    torch.cuda.synchronize()
    if raw:
        return out.hit_idx.cpu().numpy(), dict(par=ro.par.cpu().numpy(), chi2=rchi2.cpu().numpy(),
                                               status=rst.cpu().numpy())
    return out.hit_idx.cpu().numpy(), unpack(ro, rchi2, rst)


def host_gather(batch, hit_idx):
    """The hit set of every seed over all layers, gathered on the host."""
    n = batch.seeds.par.shape[1]
    Ls, Lb = len(batch.seed_layers), len(batch.build_layers)
    xyz = np.zeros((Ls + Lb, 3, n), np.float32)
    valid = np.zeros((Ls + Lb, n), np.uint8)
    xyz[:Ls], valid[:Ls] = batch.fit_hits.xyz, batch.fit_hits.valid
    for b in range(Lb):
        ids = hit_idx[b]
        ok = ids >= 0
        h = batch.layer_off[batch.seed_event * Lb + b] + ids
        xyz[Ls + b][:, ok] = batch.layer_xyz[:, h[ok]]
        valid[Ls + b, ok] = 1
    return xyz, valid


def correct_hits(batch, hit_idx):
    """Per seed, the number of chosen hits produced by the seed's own track."""
    n = batch.seeds.par.shape[1]
    Lb = len(batch.build_layers)
    seed_off = np.searchsorted(batch.seed_event, np.arange(batch.n_events + 1))
    track = np.arange(n) - seed_off[batch.seed_event]
    good = np.zeros(n, np.int64)
    for b in range(Lb):
        ids = hit_idx[b]
        ok = ids >= 0
        h = batch.layer_off[batch.seed_event * Lb + b] + ids
        good[ok] += batch.layer_truth[h[ok]] == track[ok]
    return good


@pytest.mark.parametrize("max_cands", [6, 1])
def test_refit_matches_oracle(cuda_ctx_factory, max_cands):
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    batch = S.make_build_batch(1620 + max_cands, 3, 500)
    hit_idx, g = pipeline(ctx, batch, max_cands)
    xyz, valid = host_gather(batch, hit_idx)
    r = oracle_fit(batch.seeds, xyz, valid, det)
    compare(g, r, det.radii[-1], label=f"refit N={max_cands}")
    assert np.all((g["status"] & ~16) == 0)  # only NO_HIT may appear (a layer without a hit)


def test_build_efficiency_and_refit_chi2(cuda_ctx_factory):
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    batch = S.make_build_batch(1630, 10, 5000)
    hit_idx, g = pipeline(ctx, batch, 6)
    Lb = len(batch.build_layers)
    good = correct_hits(batch, hit_idx)
    eff = float(np.mean(good >= 0.8 * Lb))
    print(f"build efficiency (>= 80 % correct hits): {eff:.4f}; all correct: {np.mean(good == Lb):.4f}")
    assert eff > 0.97
    full = (good == Lb) & (g["status"] == 0)
    c = g["chi2"][:, full]
    assert c.min() >= 0
    assert abs(c.mean() - 3.0) < 0.05, c.mean()


def test_refit_argument_checks(cuda_ctx_factory):
    import torch
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    batch = S.make_build_batch(1640, 1, 20)
    n = 20
    s = kf.Tracks(to_dev(batch.seeds.par), to_dev(batch.seeds.cov), to_dev(batch.seeds.charge))
    fh = kf.TrackHits(to_dev(batch.fit_hits.xyz), to_dev(batch.fit_hits.valid))
    lh_bad = kf.LayerHits(to_dev(batch.layer_xyz), to_dev(batch.layer_off), 1, 7, 2)  # first layer != 3
    idx = torch.full((7, n), -1, dtype=torch.int32, device="cuda")
    off = to_dev(np.array([0, n], np.int64))
    o = kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge)
    with pytest.raises(kf.KfError):
        kf.kf_refit(ctx, s, fh, off, lh_bad, idx, o)
    # no hit on any building layer: a plain fit over the seeding layers, then propagation only
    lh = kf.LayerHits(to_dev(batch.layer_xyz), to_dev(batch.layer_off), 1, 7, 3)
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    kf.kf_refit(ctx, s, fh, off, lh, idx, o, None, st)
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() & 16)

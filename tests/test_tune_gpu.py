"""Launch parameters (kf_tuning) change speed, never results: every setting
gives bitwise the same fit and build, including the build's per-warp hit
staging (window bin rows copied into shared memory) on wrapped and dense
windows; the autotuners keep a valid setting and leave identical outputs."""
import numpy as np
import pytest

from paper_1605_05508_gb300 import synth as S
from buildutil import gpu_build
from fitutil import gpu_fit

pytestmark = pytest.mark.gpu

DEFAULT = {"fit_block": 128, "build_hit_tile": 0, "build_list_width": 8, "build_scan": 4, "fit_chunk": 0,
           "fit_stage": 0, "bin_unordered": 0}
BUILD_KEYS = ("par", "cov", "chi2", "nhits", "status", "hits", "n_cands", "cand_hits", "cand_chi2", "cand_nhits")


def _same(a, b, keys):
    for k in keys:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_tuning_defaults_and_validation(cuda_ctx_factory):
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory(S.barrel().radii)
    assert kf.kf_get_tuning(ctx) == DEFAULT
    for bad in [(96, 0, 8, 0), (128, 256, 8, 0), (128, 0, 6, 0), (0, 0, 0, 0), (128, 0, 8, 5), (128, 512, 8, 2), (128, 512, 8, 3), (128, 512, 8, 4),
                (128, 0, 8, 0, 1000)]:
        with pytest.raises(kf.KfError):
            kf.kf_set_tuning(ctx, *bad)
    assert kf.kf_get_tuning(ctx) == DEFAULT
    kf.kf_set_tuning(ctx, 64, 512, 4, 1, 524288)
    assert kf.kf_get_tuning(ctx) == {"fit_block": 64, "build_hit_tile": 512, "build_list_width": 4, "build_scan": 1,
                                     "fit_chunk": 524288, "fit_stage": 0, "bin_unordered": 0}


@pytest.mark.parametrize("n", [7001, 64, 40_000])
def test_fit_block_sizes_bitwise(cuda_ctx_factory, n):
    """Block sizes 64 and 128, and the staged layer kernel (tensor copies of
    32-track tiles; batches not a multiple of 32 take the plain kernel): the
    same bits."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(91 + n, n, det, pt_range=(0.3, 10.0))
    res = []
    for b, stage in ((64, 0), (128, 0), (64, 1)):
        kf.kf_set_tuning(ctx, b, 0, 8, 0, 0, stage)
        res.append(gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "graph"))
    _same(res[0], res[1], ("par", "cov", "chi2", "status"))
    _same(res[0], res[2], ("par", "cov", "chi2", "status"))
    # the autotuner keeps one of the two and gives the same bits
    t = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "autotune")
    _same(res[0], t, ("par", "cov", "chi2", "status"))
    assert kf.kf_get_tuning(ctx)["fit_block"] in (64, 128)


def test_fit_l2_chunks_bitwise(cuda_ctx_factory):
    """fit_chunk: all layers of a chunk of tracks before the next chunk (three
    chunks of 262 144 tracks, the last one ragged): the same bits."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(95, 600_001, det, keep_truth=False)
    res = []
    for chunk in (0, 262144):
        kf.kf_set_tuning(ctx, 64, 0, 8, 0, chunk)
        res.append(gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "graph"))
    _same(res[0], res[1], ("par", "cov", "chi2", "status"))
    # the staged kernel over the same chunks (600 000 tracks: every chunk a multiple of 32)
    sub = S.Seeds(ev.seeds.par[:, :600_000], ev.seeds.cov[:, :600_000], ev.seeds.charge[:600_000])
    hx, hv = ev.hits.xyz[:, :, :600_000], ev.hits.valid[:, :600_000]
    kf.kf_set_tuning(ctx, 64, 0, 8, 0, 0)
    ref = gpu_fit(ctx, sub, hx, hv, "graph")
    for chunk in (0, 262144):
        kf.kf_set_tuning(ctx, 64, 0, 8, 0, chunk, 1)
        _same(ref, gpu_fit(ctx, sub, hx, hv, "graph"), ("par", "cov", "chi2", "status"))


def _batches():
    return {
        "config3-like": S.make_build_batch(1611, 4, 1500),
        "phi-wrap": S.make_build_batch(1612, 2, 300, phi_range=(np.pi - 0.06, np.pi + 0.06)),
        # dense hits: many warps' hulls exceed the staging tile and fall back
        "dense": S.make_build_batch(1613, 2, 1000, noise_factor=40),
    }


@pytest.mark.parametrize("max_cands", [8, 6, 3, 2, 1])
def test_build_settings_bitwise(cuda_ctx_factory, max_cands):
    """Every launch setting of the build step (hit staging, list width, thread
    layout: grouped per-lane, grouped cooperative, candidate-packed with 128 or
    64 seeds per block, register-resident with 8, 6, 4, 2 or 1 lanes a seed)
    gives the same bits."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    for name, batch in _batches().items():
        ref = None
        for tile in (0, 512):
            for lw in (8, 4):
                for scan in (0, 1, 2, 3, 4):
                    if (scan >= 2 and tile > 0) or (scan == 4 and lw == 4):
                        continue
                    kf.kf_set_tuning(ctx, 128, tile, lw, scan)
                    g = gpu_build(ctx, batch, max_cands)
                    if ref is None:
                        ref = g
                    else:
                        for k in BUILD_KEYS:
                            np.testing.assert_array_equal(ref[k], g[k],
                                                          err_msg=f"{name} tile={tile} list={lw} scan={scan} {k}")
        assert np.mean(ref["nhits"]) > 5.0, name


def test_build_autotune(cuda_ctx_factory):
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    batch = S.make_build_batch(1614, 3, 1200)
    ref = gpu_build(ctx, batch, 4)
    chosen = {}

    def tune(*args):
        chosen.update(kf.kf_autotune_build(*args))
    g = gpu_build(ctx, batch, 4, build_fn=tune)
    _same(ref, g, BUILD_KEYS)
    assert chosen["build_hit_tile"] in (0, 512) and chosen["build_list_width"] in (4, 8)
    assert chosen["build_scan"] in (0, 1, 2, 3, 4)
    assert kf.kf_get_tuning(ctx) == chosen


def test_unordered_bins_give_the_same_build(cuda_ctx_factory):
    """kf_tuning.bin_unordered leaves each bin in scatter order: the bins hold
    the same hits per bin, and kf_build's results are the same bits."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    for name, batch in _batches().items():
        res = []
        for unordered in (0, 1):
            kf.kf_set_tuning(ctx, 128, 0, 8, 2, 0, 0, unordered)
            res.append(gpu_build(ctx, batch, 6))
        _same(res[0], res[1], BUILD_KEYS)
        b0, b1 = res[0]["bins"], res[1]["bins"]
        assert np.array_equal(b0.bin_off.cpu().numpy(), b1.bin_off.cpu().numpy()), name
        ids0 = b0.hits.cpu().numpy()[:, 3].view(np.int32)
        ids1 = b1.hits.cpu().numpy()[:, 3].view(np.int32)
        off = b0.bin_off.cpu().numpy()
        pts1 = b1.hits.cpu().numpy()
        for s in range(off.shape[0]):  # per segment and bin: the same set of hits
            base = int(batch.layer_off[s])
            n = int(batch.layer_off[s + 1]) - base
            seg_ids = ids1[base:base + n]
            assert np.array_equal(np.sort(seg_ids), np.arange(n)), (name, s)  # a permutation
            np.testing.assert_array_equal(pts1[base:base + n, :3], batch.layer_xyz[:, base + seg_ids].T)
            for bb in np.nonzero(np.diff(off[s]) > 1)[0][:200]:
                lo, hi = base + off[s, bb], base + off[s, bb + 1]
                assert sorted(ids0[lo:hi]) == sorted(ids1[lo:hi]), (name, s, bb)
    kf.kf_set_tuning(ctx, 128, 0, 8, 0)


@pytest.mark.parametrize("max_cands", [8, 6, 3, 1])
def test_sub_bin_windows_give_the_same_build(cuda_ctx_factory, max_cands):
    """The register-resident layout looking its windows up by sub-bin (the
    unordered binning's 64 x 512 sub-bin starts) gives the same bits as by
    bin, with the first-layer launch (N > 2) and without (N = 1); the
    layer-stepping layouts, handed the sub-bin starts too, keep to the bins
    and give the same bits."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    for name, batch in _batches().items():
        kf.kf_set_tuning(ctx, 128, 0, 8, 4, 0, 0, 1)
        ref = gpu_build(ctx, batch, max_cands)
        g = gpu_build(ctx, batch, max_cands, fine=True)
        _same(ref, g, BUILD_KEYS)
        for scan in (0, 2):
            kf.kf_set_tuning(ctx, 128, 0, 8, scan, 0, 0, 1)
            _same(ref, gpu_build(ctx, batch, max_cands, fine=True), BUILD_KEYS)
    kf.kf_set_tuning(ctx, 128, 0, 8, 0)

"""The bounded waits of the staged fit layer kernel and of the build's hit
staging, made to run out without any GPU fault: the test hooks
kf_test_stage_fault / kf_test_build_stage_fault keep the copies of one
32-track tile (fit) or of one warp's window hits (build) from being issued,
so the warp waits for nothing until its poll limit.  The kernel must then
mark exactly the tracks or seeds it could not process with
KF_ST_DEVICE_TIMEOUT, drain only the copies it really issued, and leave every
other result bit for bit as without the fault; the context stays usable, and
clearing the hook restores the plain result."""
import numpy as np
import pytest

from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.gpu

WAIT_POLLS = 1 << 14  # far above the latency of a copy that was issued


def _fit(ctx, kf, ev):
    import torch
    from fitutil import to_dev
    n, L = ev.seeds.par.shape[1], ev.hits.xyz.shape[0]
    s = kf.Tracks(to_dev(ev.seeds.par), to_dev(ev.seeds.cov), to_dev(ev.seeds.charge))
    out = kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge,
                    torch.empty((3, n), device="cuda"))
    chi2 = torch.empty((L, n), device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    kf.kf_fit(ctx, s, kf.TrackHits(to_dev(ev.hits.xyz), to_dev(ev.hits.valid)), out, chi2, st)
    torch.cuda.synchronize()
    return (out.par.cpu().numpy(), out.par_lo.cpu().numpy(), out.cov.cpu().numpy(), chi2.cpu().numpy(),
            st.cpu().numpy())


@pytest.mark.parametrize("n_tiles,skip", [(1000, 5), (4000, 5)])
def test_stage_wait_runs_out_and_marks_only_its_tracks(cuda_ctx_factory, n_tiles, skip):
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    kf.kf_set_tuning(ctx, 64, 0, 8, 0, 0, 1)  # the staged layer kernel
    n = 32 * n_tiles
    ev = S.make_fit_batch(4242 + n_tiles, n, keep_truth=False)
    ref = _fit(ctx, kf, ev)
    assert not np.any(ref[4] & kf.ST_DEVICE_TIMEOUT)
    kf.kf_test_stage_fault(ctx, skip, WAIT_POLLS)
    got = _fit(ctx, kf, ev)
    kf.kf_test_stage_fault(ctx, -1, 0)
    timed_out = (got[4] & kf.ST_DEVICE_TIMEOUT) != 0
    tiles = np.nonzero(timed_out.reshape(n_tiles, 32).any(axis=1))[0]
    assert skip in tiles
    assert np.all(timed_out.reshape(n_tiles, 32)[tiles]), "a timed-out tile is flagged whole"
    # the flagged tiles are the skipped one and later tiles of the same warp:
    # tile indices congruent to it modulo the launch's warp count
    if len(tiles) > 1:
        stride = np.diff(tiles)
        assert np.all(stride == stride[0]) and tiles[0] == skip
    ok = ~timed_out
    for a, b in zip(got[:4], ref[:4]):
        np.testing.assert_array_equal(a[..., ok], b[..., ok])
    np.testing.assert_array_equal(got[4][ok], ref[4][ok])
    # the context and the device stay usable: the plain result again
    again = _fit(ctx, kf, ev)
    for a, b in zip(again, ref):
        np.testing.assert_array_equal(a, b)
    kf.kf_set_tuning(ctx, 128, 0, 8, 0)


@pytest.mark.parametrize("skip", [3, 40])
def test_build_stage_wait_runs_out_and_marks_only_its_seeds(cuda_ctx_factory, skip):
    """kf_build's hit staging (tile 512, grouped per-lane layout): the test hook
    kf_test_build_stage_fault keeps one warp of every layer step from issuing
    its copies, so that warp's wait for its staged hits runs out on the first
    layer where it stages.  Exactly its seeds (four at most) stop with
    KF_ST_DEVICE_TIMEOUT; every other seed's results are bit for bit those
    without the hook; the context stays usable and, the hook cleared, gives
    the plain results again."""
    from buildutil import gpu_build
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    batch = S.make_build_batch(5150 + skip, 2, 400)
    kf.kf_set_tuning(ctx, 128, 512, 8, 0)
    keys = ("par", "chi2", "nhits", "status", "hits")
    ref = gpu_build(ctx, batch, 6, want_cands=False)
    assert not np.any(ref["status"] & kf.ST_DEVICE_TIMEOUT)
    kf.kf_test_build_stage_fault(ctx, skip, WAIT_POLLS)
    got = gpu_build(ctx, batch, 6, want_cands=False)
    kf.kf_test_build_stage_fault(ctx, -1, 0)
    hit = (got["status"] & kf.ST_DEVICE_TIMEOUT) != 0
    assert 1 <= hit.sum() <= 4, hit.sum()
    for k in keys:
        np.testing.assert_array_equal(got[k][~hit], ref[k][~hit], err_msg=k)
    again = gpu_build(ctx, batch, 6, want_cands=False)
    for k in keys:
        np.testing.assert_array_equal(again[k], ref[k], err_msg=k)
    kf.kf_set_tuning(ctx, 128, 0, 8, 0)

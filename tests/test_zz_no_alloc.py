"""kf_fit_noalloc: the allocation-free variant of kf_fit for callers whose
device memory is planned up front (e.g. a trigger process that reserves the
GPU at start-up, or a host framework that owns device memory through its own
allocator) and who therefore cannot let the library call cudaMalloc.

Its scratch lives in libkf's static device memory. Checked through the C ABI
against kf_fit on two calls in a row (different batches, so the second call
runs over what the first one left in the shared array), plus the size limit.
This file is collected last on purpose."""
import numpy as np
import pytest

from fitutil import compare, oracle_fit, to_dev, unpack
from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _run(ctx, kf, ev, fn, with_lo, with_status):
    import torch
    n, L = ev.seeds.par.shape[1], ev.hits.xyz.shape[0]
    s = kf.Tracks(to_dev(ev.seeds.par), to_dev(ev.seeds.cov), to_dev(ev.seeds.charge))
    out = kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge,
                    torch.empty((3, n), device="cuda") if with_lo else None)
    chi2 = torch.empty((L, n), device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    fn(ctx, s, kf.TrackHits(to_dev(ev.hits.xyz), to_dev(ev.hits.valid)), out, chi2, st if with_status else None)
    torch.cuda.synchronize()
    return out, chi2, st


def _same_bits(kf_out, kf_chi2, ref_out, ref_chi2, label):
    """The allocation-free call runs the same layer kernel with the same
    arithmetic as kf_fit: the high parts of the state, the covariance and the
    chi2 are the same bits (only where the low parts are kept differs)."""
    import torch
    assert torch.equal(kf_out.par, ref_out.par), label
    assert torch.equal(kf_out.cov, ref_out.cov), label
    assert torch.equal(kf_chi2, ref_chi2), label


def test_noalloc_matches_kf_fit_on_two_calls(cuda_ctx_factory):
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    for seed, n in ((901, 20000), (902, 7001)):
        ev = S.make_fit_batch(seed, n, pt_range=(0.3, 10.0))
        ref_out, ref_chi2, ref_st = _run(ctx, kf, ev, kf.kf_fit, True, True)
        ref = unpack(ref_out, ref_chi2, ref_st)
        # scratch entirely from the static array: no status, no low-part buffer
        out, chi2, _ = _run(ctx, kf, ev, kf.kf_fit_noalloc, False, False)
        _same_bits(out, chi2, ref_out, ref_chi2, f"noalloc n={n}, scratch status and low parts")
        # status from the caller, low parts still from the static array
        out2, chi2_2, st2 = _run(ctx, kf, ev, kf.kf_fit_noalloc, False, True)
        _same_bits(out2, chi2_2, ref_out, ref_chi2, f"noalloc n={n}, caller status")
        got = unpack(out, chi2, st2)
        np.testing.assert_array_equal(got["status"], ref["status"])
        r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
        compare(got, r, det.radii[-1], label=f"noalloc n={n}")


def test_noalloc_batch_at_the_limit(cuda_ctx_factory):
    """A batch of exactly KF_NOALLOC_MAX_TRACKS tracks fills the low-part region
    of the static array up to the status words: with both taken from the
    array, the results are kf_fit's bits; and again with the status from the
    caller, whose status words equal kf_fit's."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    n = kf.NOALLOC_MAX_TRACKS
    ev = S.make_fit_batch(903, n, pt_range=(0.3, 10.0), keep_truth=False)
    ref_out, ref_chi2, ref_st = _run(ctx, kf, ev, kf.kf_fit, True, True)
    out, chi2, _ = _run(ctx, kf, ev, kf.kf_fit_noalloc, False, False)
    _same_bits(out, chi2, ref_out, ref_chi2, "noalloc at the limit")
    out2, chi2_2, st2 = _run(ctx, kf, ev, kf.kf_fit_noalloc, False, True)
    _same_bits(out2, chi2_2, ref_out, ref_chi2, "noalloc at the limit, caller status")
    import torch
    assert torch.equal(st2, ref_st)


def test_noalloc_rejects_batches_beyond_the_static_scratch(cuda_ctx_factory):
    import torch
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    n = kf.NOALLOC_MAX_TRACKS + 1
    z = lambda *sh: torch.empty(sh, device="cuda")
    s = kf.Tracks(z(6, n), z(21, n), torch.ones(n, dtype=torch.int8, device="cuda"))
    with pytest.raises(kf.KfError) as e:
        kf.kf_fit_noalloc(ctx, s, kf.TrackHits(z(det.n_layers, 3, n)), s)
    assert e.value.code == kf.KF_EINVAL

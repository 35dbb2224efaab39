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


def test_noalloc_matches_kf_fit_on_two_calls(cuda_ctx_factory):
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    for seed, n in ((901, 20000), (902, 7001)):
        ev = S.make_fit_batch(seed, n, pt_range=(0.3, 10.0))
        ref = unpack(*_run(ctx, kf, ev, kf.kf_fit, True, True))
        # scratch entirely from the static array: no status, no low-part buffer
        out, chi2, _ = _run(ctx, kf, ev, kf.kf_fit_noalloc, False, False)
        got = unpack(out, chi2, _run(ctx, kf, ev, kf.kf_fit_noalloc, False, True)[2])
        # same kernel, same arithmetic: identical up to the dropped low parts
        np.testing.assert_array_equal(got["status"], ref["status"])
        np.testing.assert_array_equal(got["chi2"], ref["chi2"])
        r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
        compare(got, r, det.radii[-1], chi2_frac=1e-3, label=f"noalloc n={n}")
        hi = out.par.double().cpu().numpy().T
        np.testing.assert_allclose(hi, ref["par"], rtol=0, atol=4e-6)


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

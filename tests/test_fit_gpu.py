"""GPU parity of the track fit (kf_fit, kf_fit_fused, kf_fit_f64, kf_fit_host)
against the FP64 oracle on the same seeded inputs, through the C ABI."""
import numpy as np
import pytest

from fitutil import compare, gpu_fit, oracle_fit, to_dev, unpack
from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def det():
    return S.barrel()


def test_config1_1000_tracks_graph(cuda_ctx_factory, det):
    """1 event of 1000 tracks, 10 layers (the plain-fit workload)."""
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(1605, 1000)
    g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "graph")
    r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
    st = compare(g, r, det.radii[-1], label="config1")
    print("config1", st)


@pytest.mark.parametrize("n", [1, 31, 257, 9001, 9008])
@pytest.mark.parametrize("mode", ["graph", "fused"])
def test_ragged_sizes(cuda_ctx_factory, det, n, mode):
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(2000 + n, n)
    g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, mode)
    r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
    compare(g, r, det.radii[-1], label=f"{mode} n={n}")


def test_fused_equals_graph_and_host_equals_device(cuda_ctx_factory, det):
    import torch
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(33, 5000)
    a = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "graph")
    b = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "fused")
    for k in ("par", "cov", "chi2", "status"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    # kf_fit_host: same bits through host buffers
    n, L = 5000, det.n_layers
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    s = kf.Tracks(pin(ev.seeds.par), pin(ev.seeds.cov), pin(ev.seeds.charge))
    out = kf.Tracks(torch.empty((6, n)).pin_memory(), torch.empty((21, n)).pin_memory(), s.charge,
                    torch.empty((3, n)).pin_memory())
    chi2 = torch.empty((L, n)).pin_memory()
    st = torch.empty(n, dtype=torch.int32).pin_memory()
    kf.kf_fit_host(ctx, s, kf.TrackHits(pin(ev.hits.xyz), pin(ev.hits.valid)), out, chi2, st)
    c = unpack(out, chi2, st)
    for k in ("par", "cov", "chi2", "status"):
        np.testing.assert_array_equal(a[k], c[k], err_msg=k)


def test_host_pipeline_chunks_equal_device_fit(cuda_ctx_factory, det):
    """kf_fit_host on a batch of seven chunks (65 536 tracks each, a ragged
    last one) on three streams, each reusing its staging slot: the same bits
    as kf_fit on the device; a separate charge output is the input's copy."""
    import torch
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory(det.radii)
    n = 400_003
    ev = S.make_fit_batch(4242, n, keep_truth=False)
    valid = ev.hits.valid.copy()
    valid[4, ::11] = 0
    a = gpu_fit(ctx, ev.seeds, ev.hits.xyz, valid, "graph")
    L = det.n_layers
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    s = kf.Tracks(pin(ev.seeds.par), pin(ev.seeds.cov), pin(ev.seeds.charge))
    out = kf.Tracks(torch.empty((6, n)).pin_memory(), torch.empty((21, n)).pin_memory(),
                    torch.zeros(n, dtype=torch.int8).pin_memory(), torch.empty((3, n)).pin_memory())
    chi2 = torch.empty((L, n)).pin_memory()
    st = torch.empty(n, dtype=torch.int32).pin_memory()
    for _ in range(2):  # the second call replays the cached per-chunk graphs
        kf.kf_fit_host(ctx, s, kf.TrackHits(pin(ev.hits.xyz), pin(valid)), out, chi2, st)
        c = unpack(out, chi2, st)
        for k in ("par", "cov", "chi2", "status"):
            np.testing.assert_array_equal(a[k], c[k], err_msg=k)
        np.testing.assert_array_equal(out.charge.numpy(), ev.seeds.charge)


@pytest.mark.parametrize("n", [4096, 40000, 40016])
def test_graph_equals_noalloc_bitwise(cuda_ctx_factory, det, n):
    """kf_fit (captured graph, scratch from the context) and kf_fit_noalloc
    (static scratch, direct launches): identical bits, also for ragged n."""
    import torch
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(3000 + n, n, pt_range=(0.3, 10.0))
    valid = ev.hits.valid.copy()
    valid[3, ::7] = 0
    res = []
    for fn in (kf.kf_fit, kf.kf_fit_noalloc):
        s = kf.Tracks(to_dev(ev.seeds.par), to_dev(ev.seeds.cov), to_dev(ev.seeds.charge))
        out = kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge,
                        torch.empty((3, n), device="cuda"))
        chi2 = torch.empty((10, n), device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        fn(ctx, s, kf.TrackHits(to_dev(ev.hits.xyz), to_dev(valid)), out, chi2, st)
        torch.cuda.synchronize()
        res.append(unpack(out, chi2, st))
    for k in ("par", "cov", "chi2", "status"):
        np.testing.assert_array_equal(res[0][k], res[1][k], err_msg=k)


def test_batch_invariance_bitwise(cuda_ctx_factory, det):
    """A track's result is bitwise the same alone, in a small batch, and in a
    large batch at another position."""
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(44, 6000)
    full = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "graph")
    idx = np.array([0, 17, 2999, 5999])
    sub = S.Seeds(ev.seeds.par[:, idx], ev.seeds.cov[:, idx], ev.seeds.charge[idx])
    part = gpu_fit(ctx, sub, ev.hits.xyz[:, :, idx], ev.hits.valid[:, idx], "graph")
    for k in ("par", "cov", "status"):
        np.testing.assert_array_equal(full[k][idx], part[k], err_msg=k)
    np.testing.assert_array_equal(full["chi2"][:, idx], part["chi2"])


def test_missing_hits_and_loopers(cuda_ctx_factory, det):
    """Layers without a hit are propagated only; low-pT loopers stop at the
    last reachable layer with the same status bits as the oracle."""
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(55, 3000, pt_range=(0.2, 2.0))
    valid = ev.hits.valid.copy()
    valid[2, ::5] = 0
    valid[7, 1::7] = 0
    g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, valid, "graph")
    r = oracle_fit(ev.seeds, ev.hits.xyz, valid, det)
    assert (r["status"] & 1).sum() > 50  # loopers present
    compare(g, r, det.radii[-1], label="missing+loopers")


def test_plain_f64_per_event_matches_oracle(cuda_ctx_factory, det):
    import torch
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory(det.radii)
    ev = S.make_fit_batch(66, 3000)
    n, L = 3000, det.n_layers
    s = kf.Tracks(to_dev(ev.seeds.par, torch.float64), to_dev(ev.seeds.cov, torch.float64), to_dev(ev.seeds.charge))
    out = kf.Tracks(torch.empty((6, n), dtype=torch.float64, device="cuda"),
                    torch.empty((21, n), dtype=torch.float64, device="cuda"), s.charge)
    chi2 = torch.empty((L, n), dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    kf.kf_fit_f64(ctx, s, kf.TrackHits(to_dev(ev.hits.xyz), to_dev(ev.hits.valid)), out, [0, 1000, 1001, 3000],
                  chi2, st)
    torch.cuda.synchronize()
    g = unpack(out, chi2, st)
    r = oracle_fit(ev.seeds, ev.hits.xyz, ev.hits.valid, det)
    np.testing.assert_array_equal(g["status"], r["status"])
    np.testing.assert_allclose(g["par"], r["par"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(g["chi2"], r["chi2"], rtol=1e-9, atol=1e-10)
    from fitutil import cov_error
    assert cov_error(g["cov"], r["cov"], r["par"]).max() < 1e-8


def test_empty_and_invalid_arguments(cuda_ctx_factory, det):
    import torch
    from paper_1605_05508_gb300 import kf
    ctx = cuda_ctx_factory(det.radii)
    z = lambda *sh: torch.empty(sh, device="cuda")
    empty = kf.Tracks(z(6, 0), z(21, 0), torch.empty(0, dtype=torch.int8, device="cuda"), z(3, 0))
    kf.kf_fit(ctx, empty, kf.TrackHits(z(10, 3, 0)), empty)  # n = 0 is a no-op
    s = kf.Tracks(z(6, 5), z(21, 5), torch.ones(5, dtype=torch.int8, device="cuda"))
    with pytest.raises(kf.KfError) as e:
        kf.kf_fit(ctx, s, kf.TrackHits(z(10, 3, 4)), s)  # hits for 4 tracks, seeds for 5
    assert e.value.code == kf.KF_EINVAL
    with pytest.raises(kf.KfError) as e:
        kf.kf_fit(ctx, s, kf.TrackHits(z(11, 3, 5)), s)  # more layers than configured
    assert e.value.code == kf.KF_EINVAL


def test_full_size_config2_sampled(cuda_ctx_factory, det):
    """200 events x 20000 tracks in one batch, in the benchmark's launch
    configuration (the autotuner's block size and L2 chunk on this batch); a
    random sample of tracks is checked against the oracle."""
    ctx = cuda_ctx_factory(det.radii)
    n = 200 * 20000
    ev = S.make_fit_batch(1606, n, keep_truth=False)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(n, 3000, replace=False))
    g = gpu_fit(ctx, ev.seeds, ev.hits.xyz, ev.hits.valid, "autotune", sample=idx)
    sub = S.Seeds(ev.seeds.par[:, idx], ev.seeds.cov[:, idx], ev.seeds.charge[idx])
    r = oracle_fit(sub, ev.hits.xyz[:, :, idx], ev.hits.valid[:, idx], det)
    compare(g, r, det.radii[-1], label="config2 sample")
    assert np.all(np.isfinite(g["par"])) and np.all(g["status"] == 0)
    assert np.all(g["chi2"] >= 0)

"""Serving (kf_serve_start / kf_submit / kf_poll): continuous batching of
build requests. Each event's result is bitwise the same alone, in a mix of
uneven events sharing build-step launches, and from the batch kf_build;
admission waits for device memory; failures are reported on the host."""
import threading
import time

import numpy as np
import pytest

from buildutil import gpu_build
from paper_1605_05508_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _event(seed, n, **kw):
    b = S.make_build_batch(seed, 1, n, **kw)
    ev = dict(seed_par=b.seeds.par, seed_cov=b.seeds.cov, seed_charge=b.seeds.charge, seed_hits=b.fit_hits.xyz,
              seed_valid=b.fit_hits.valid, layer_xyz=b.layer_xyz, layer_off=b.layer_off)
    return b, ev


def _poll_all(kf, ctx, tickets, sizes, timeout_us=60_000_000):
    return [kf.kf_poll(ctx, t, n, 7, timeout_us) for t, n in zip(tickets, sizes)]


SIZES = [700, 3100, 150, 5000, 1200, 60, 2300, 900]


@pytest.mark.parametrize("layout", [0, 2, 3, 4])
def test_alone_equals_mix_equals_batch_build(cuda_ctx_factory, layout):
    """layout: the build step's thread layout in the serving loop (grouped, or
    candidate-packed); the batch comparison runs the grouped layout."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    evs = [_event(100 + i, n) for i, n in enumerate(SIZES)]
    kf.kf_set_tuning(ctx, 128, 0, 8, layout)
    # pack_min_seeds=1: every step launch takes the configured layout, however few seeds
    kf.kf_serve_start(ctx, 3, 7, 6, max_slots=32, device_arena_bytes=1 << 30, host_arena_bytes=1 << 29,
                      pack_min_seeds=1)
    alone = []
    for (b, ev), n in zip(evs, SIZES):
        t = kf.kf_submit(ctx, ev)
        alone.append(kf.kf_poll(ctx, t, n, 7, 60_000_000))
    # the mix: every event in flight at once, sharing step launches
    tickets = [kf.kf_submit(ctx, ev) for _, ev in evs]
    mix = _poll_all(kf, ctx, tickets, SIZES)
    st = kf.kf_serve_stats_get(ctx)
    kf.kf_serve_stop(ctx)
    assert st["completed"] == 2 * len(SIZES) and st["max_resident"] >= 2
    for a, m in zip(alone, mix):
        for k in ("best_par", "chi2_tot", "n_hits", "status", "hit_idx"):
            np.testing.assert_array_equal(a[k], m[k], err_msg=k)
    # the batch API on the same events gives the same bits
    kf.kf_set_tuning(ctx, 128, 0, 8, 0)
    for (b, _), a in zip(evs, alone):
        g = gpu_build(ctx, b, 6, want_cands=False)
        np.testing.assert_array_equal(g["hits"].T, a["hit_idx"])
        np.testing.assert_array_equal(g["nhits"], a["n_hits"])
        np.testing.assert_array_equal(g["chi2"].astype(np.float32), a["chi2_tot"])


def test_admission_waits_for_device_memory(cuda_ctx_factory):
    """An arena that holds about one large event at a time: events queue,
    are admitted as memory frees, and all complete with unchanged results."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    sizes = [4000, 4000, 300, 4000, 300]
    evs = [_event(300 + i, n) for i, n in enumerate(sizes)]
    kf.kf_serve_start(ctx, 3, 7, 6, max_slots=8, device_arena_bytes=24 << 20, host_arena_bytes=1 << 28)
    tickets = [kf.kf_submit(ctx, ev) for _, ev in evs]
    mix = _poll_all(kf, ctx, tickets, sizes)
    st = kf.kf_serve_stats_get(ctx)
    kf.kf_serve_stop(ctx)
    assert st["completed"] == len(sizes)
    assert st["device_arena_peak"] <= 24 << 20
    assert max(r["queued_ms"] for r in mix) > 0.0
    kf.kf_serve_start(ctx, 3, 7, 6, device_arena_bytes=1 << 30, host_arena_bytes=1 << 28)
    for (_, ev), n, m in zip(evs, sizes, mix):
        a = kf.kf_poll(ctx, kf.kf_submit(ctx, ev), n, 7, 60_000_000)
        np.testing.assert_array_equal(a["hit_idx"], m["hit_idx"])
    kf.kf_serve_stop(ctx)


def test_oversized_event_cancel_timeout_and_bad_arguments(cuda_ctx_factory):
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    kf.kf_serve_start(ctx, 3, 7, 6, max_slots=1, device_arena_bytes=16 << 20, host_arena_bytes=1 << 28)
    _, big = _event(400, 20000)
    with pytest.raises(kf.KfError) as e:
        kf.kf_submit(ctx, big)  # needs more than the whole device arena: never admissible
    assert e.value.code == kf.KF_ENOMEM
    _, ev1 = _event(401, 3000)
    _, ev2 = _event(402, 50)
    t1 = kf.kf_submit(ctx, ev1)
    t2 = kf.kf_submit(ctx, ev2)
    t3 = kf.kf_submit(ctx, ev2)
    # one slot: t3 waits behind t1 and t2 and can be cancelled while queued
    rc = None
    try:
        kf.kf_cancel(ctx, t3)
        rc = kf.KF_OK
    except kf.KfError as err:
        rc = err.code
    assert rc in (kf.KF_OK, kf.KF_EAGAIN)
    try:
        kf.kf_poll(ctx, t2, 50, 7, 0)  # not waiting: may or may not be done
    except kf.KfError as err:
        assert err.code == kf.KF_ETIMEDOUT
        kf.kf_poll(ctx, t2, 50, 7, 60_000_000)  # the ticket stayed valid
    kf.kf_poll(ctx, t1, 3000, 7, 60_000_000)
    if rc == kf.KF_EAGAIN:
        kf.kf_poll(ctx, t3, 50, 7, 60_000_000)
    with pytest.raises(kf.KfError) as e:
        kf.kf_poll(ctx, 987654321, 1, 7, 0)
    assert e.value.code == kf.KF_EINVAL
    bad = dict(ev2)
    bad["layer_off"] = ev2["layer_off"][::-1].copy()  # decreasing offsets
    with pytest.raises(kf.KfError) as e:
        kf.kf_submit(ctx, bad)
    assert e.value.code == kf.KF_EINVAL
    st = kf.kf_serve_stats_get(ctx)
    kf.kf_serve_stop(ctx)
    assert st["max_resident"] == 1
    with pytest.raises(kf.KfError) as e:
        kf.kf_serve_start(ctx, 3, 7, 6, pack_min_seeds=-1)
    assert e.value.code == kf.KF_EINVAL


def test_concurrent_submitters_and_pollers(cuda_ctx_factory):
    """Several host threads submit and poll at once (the API is thread-safe)."""
    from paper_1605_05508_gb300 import kf
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    evs = [_event(500 + i, n) for i, n in enumerate([400, 900, 200, 1500])]
    kf.kf_serve_start(ctx, 3, 7, 6, device_arena_bytes=1 << 30, host_arena_bytes=1 << 29)
    ref = [kf.kf_poll(ctx, kf.kf_submit(ctx, ev), ev["seed_par"].shape[1], 7, 60_000_000) for _, ev in evs]
    errors = []

    def worker(w):
        try:
            for rep in range(3):
                i = (w + rep) % len(evs)
                ev = evs[i][1]
                r = kf.kf_poll(ctx, kf.kf_submit(ctx, ev), ev["seed_par"].shape[1], 7, 60_000_000)
                if not np.array_equal(r["hit_idx"], ref[i]["hit_idx"]):
                    errors.append((w, rep))
        except Exception as ex:  # noqa: BLE001
            errors.append(repr(ex))
    th = [threading.Thread(target=worker, args=(w,)) for w in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    kf.kf_serve_stop(ctx)
    assert not errors, errors


def test_served_refit_equals_batch_refit(cuda_ctx_factory):
    """refit = 1: each served request also fits its best candidates over all
    10 layers; the result is bitwise that of kf_build + kf_refit on the
    event alone."""
    from paper_1605_05508_gb300 import kf
    from test_refit_gpu import pipeline
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii)
    sizes = [500, 1700, 90, 2600]
    evs = [_event(300 + i, n) for i, n in enumerate(sizes)]
    kf.kf_serve_start(ctx, 3, 7, 6, max_slots=32, device_arena_bytes=1 << 30, host_arena_bytes=1 << 29, refit=True)
    tickets = [kf.kf_submit(ctx, ev) for _, ev in evs]
    res = [kf.kf_poll(ctx, t, n, 7, 60_000_000, refit_layers=10) for t, n in zip(tickets, sizes)]
    kf.kf_serve_stop(ctx)
    for (b, _), r in zip(evs, res):
        hit_idx, g = pipeline(ctx, b, 6, raw=True)
        np.testing.assert_array_equal(hit_idx, r["hit_idx"])
        np.testing.assert_array_equal(g["par"], r["refit_par"])
        np.testing.assert_array_equal(g["chi2"], r["refit_chi2"])
        np.testing.assert_array_equal(g["status"], r["refit_status"])
        assert np.mean(r["refit_chi2"][r["refit_chi2"] >= 0]) < 4.0


def test_native_driver_serves_every_request(tmp_path):
    """kf_serve_driver (the serving loop driven from native threads, as the
    benchmark measures it) completes every request of a small pool at
    saturation with two submitting threads and under Poisson arrivals, with
    latencies that are positive and ordered (p50 <= p99)."""
    import bench
    from paper_1605_05508_gb300 import build as B
    B.build()
    det = S.barrel()
    pool = []
    for i, n in enumerate([300, 2500, 800, 60]):
        b = S.make_build_batch(500 + i, 1, n)
        pool.append(dict(seed_par=b.seeds.par, seed_cov=b.seeds.cov, seed_charge=b.seeds.charge,
                         seed_hits=b.fit_hits.xyz, seed_valid=b.fit_hits.valid, layer_xyz=b.layer_xyz,
                         layer_off=b.layer_off))
    path = str(tmp_path / "pool.kfpool")
    bench.write_serve_pool(path, pool, det, 8, 1 << 30, 1 << 28)
    # build_scan 2 steps events one layer a launch; 4 takes each prepared
    # event through all 7 layers in one register-resident launch
    for scan, rate, threads in ((2, 0, 2), (2, 400.0, 1), (4, 0, 2), (4, 400.0, 1)):
        r = bench.run_serve_driver(path, 24, rate, threads, 3, tuning={"build_scan": scan, "build_list_width": 8})
        assert r["requests"] == 24 and r["events_per_s"] > 0, r
        assert 0 < r["p50_ms"] <= r["p99_ms"], r
        assert r["max_resident"] >= 1 and r["step_launches"] >= (7 if scan == 2 else 1), r
        # the scheduler thread's time split covers the run: each part >= 0,
        # together about the run's wall time (its clock runs from the first
        # submit; the scheduler's from the same counters read before and after)
        parts = [r["sched_busy_ms"], r["sched_gpu_wait_ms"], r["sched_idle_ms"]]
        assert all(p >= 0 for p in parts), r
        assert 0.5 * r["wall_s"] * 1e3 <= sum(parts) <= 1.5 * r["wall_s"] * 1e3 + 5.0, r


@pytest.mark.parametrize("n_build,max_cands", [(1, 6), (7, 1), (7, 3)])
def test_register_resident_serving_without_a_split_and_narrow(cuda_ctx_factory, n_build, max_cands):
    """Serving with the register-resident layout where it runs a single launch
    per iteration (one building layer, or one lane a seed at N = 1) and with
    W = 4 lanes (N = 3): each event's results are bitwise the batch build's."""
    from paper_1605_05508_gb300 import kf
    from test_build_gpu import _first_layer_only
    det = S.barrel()
    ctx = cuda_ctx_factory(det.radii, max_cands=8)
    evs = []
    for i, n in enumerate((400, 1500, 90)):
        b = S.make_build_batch(700 + i, 1, n)
        if n_build == 1:
            b = _first_layer_only(b)
        evs.append((b, dict(seed_par=b.seeds.par, seed_cov=b.seeds.cov, seed_charge=b.seeds.charge,
                            seed_hits=b.fit_hits.xyz, seed_valid=b.fit_hits.valid, layer_xyz=b.layer_xyz,
                            layer_off=b.layer_off)))
    kf.kf_set_tuning(ctx, 128, 0, 8, 4)
    kf.kf_serve_start(ctx, 3, n_build, max_cands, max_slots=8, device_arena_bytes=1 << 28,
                      host_arena_bytes=1 << 27)
    tickets = [kf.kf_submit(ctx, ev) for _, ev in evs]
    served = [kf.kf_poll(ctx, t, b.seeds.par.shape[1], n_build, 60_000_000) for t, (b, _) in zip(tickets, evs)]
    kf.kf_serve_stop(ctx)
    kf.kf_set_tuning(ctx, 128, 0, 8, 0)
    for (b, _), a in zip(evs, served):
        g = gpu_build(ctx, b, max_cands, want_cands=False)
        np.testing.assert_array_equal(g["hits"].T, a["hit_idx"])
        np.testing.assert_array_equal(g["nhits"], a["n_hits"])
        np.testing.assert_array_equal(g["status"], a["status"])
        np.testing.assert_array_equal(g["chi2"].astype(np.float32), a["chi2_tot"])

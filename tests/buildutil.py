"""Helpers of the build tests: the seed fit + build pipeline on the GPU
(through the binding) and on the oracle, on the same seeded inputs, and the
near-tie classification of differing chosen hits."""
import numpy as np

import oracle as O
from fitutil import f32, material, to_dev


def oracle_seed_fit(batch, idx=None):
    """The oracle's fit over the seeding layers (its own build seeds, FP64)."""
    det = batch.det
    sp, sc, q = batch.seeds.par, batch.seeds.cov, batch.seeds.charge
    xyz, val = batch.fit_hits.xyz, batch.fit_hits.valid
    if idx is not None:
        sp, sc, q, xyz, val = sp[:, idx], sc[:, idx], q[idx], xyz[:, :, idx], val[:, idx]
    L = len(batch.seed_layers)
    return O.fit(sp, sc, q, xyz, val, [f32(r) for r in det.radii[:L]], f32(det.bz), f32(det.sigma_xy),
                 f32(det.sigma_z), **material(det, range(L)))


def oracle_build(batch, max_cands, idx=None, cut=30.0):
    det = batch.det
    r = oracle_seed_fit(batch, idx)
    q = batch.seeds.charge if idx is None else batch.seeds.charge[idx]
    ev = batch.seed_event if idx is None else batch.seed_event[idx]
    radii = [f32(det.radii[l]) for l in batch.build_layers]
    b = O.build_tracks(r["par"], r["cov"], q, ev, batch.layer_xyz, batch.layer_off, radii, f32(det.bz),
                       f32(det.sigma_xy), f32(det.sigma_z), chi2_cut=cut, max_cands=max_cands,
                       **material(det, batch.build_layers))
    b["seed_par"], b["seed_cov"] = r["par"], r["cov"]
    return b


def gpu_build(ctx, batch, max_cands, want_cands=True, build_fn=None, fine=False, streams=False):
    """Seed fit (kf_fit over the seeding layers) -> kf_bin_hits -> kf_build
    (or build_fn with kf_build's arguments); fine: the binning also gives the
    sub-bin starts (unordered binning only), which the build then uses;
    streams: the seed fit and the binning run at once on two side streams,
    joined before the build.  Returns numpy arrays (hit_idx as [n, L])."""
    import torch
    from paper_1605_05508_gb300 import kf
    n = batch.seeds.par.shape[1]
    E, Lb = batch.n_events, len(batch.build_layers)
    s = kf.Tracks(to_dev(batch.seeds.par), to_dev(batch.seeds.cov), to_dev(batch.seeds.charge))
    fo = kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge,
                   torch.empty((3, n), device="cuda"))
    fst = torch.empty(n, dtype=torch.int32, device="cuda")
    th = kf.TrackHits(to_dev(batch.fit_hits.xyz), to_dev(batch.fit_hits.valid))
    if not streams:
        kf.kf_fit(ctx, s, th, fo, None, fst)
    seg_off = to_dev(batch.layer_off)
    lh = kf.LayerHits(to_dev(batch.layer_xyz), seg_off, E, Lb, batch.build_layers[0])
    nh = batch.layer_xyz.shape[1]
    bins = kf.HitBins(torch.empty((nh, 4), device="cuda"),
                      torch.empty((E * Lb, kf.NBINS + 1), dtype=torch.int32, device="cuda"),
                      fine_off=torch.empty((E * Lb, kf.NBINS_FINE + 1), dtype=torch.int32, device="cuda")
                      if fine else None)
    if streams:
        main = torch.cuda.current_stream()
        s_bin, s_fit = torch.cuda.Stream(), torch.cuda.Stream()
        fork = torch.cuda.Event()
        fork.record(main)
        s_bin.wait_event(fork)
        s_fit.wait_event(fork)
        kf.kf_bin_hits(ctx, lh, bins, s_bin)
        kf.kf_fit(ctx, s, th, fo, None, fst, s_fit)
        main.wait_stream(s_bin)
        main.wait_stream(s_fit)
    else:
        kf.kf_bin_hits(ctx, lh, bins)
    seed_off = to_dev(np.searchsorted(batch.seed_event, np.arange(E + 1)).astype(np.int64))
    N = max_cands
    i32 = dict(dtype=torch.int32, device="cuda")
    out = kf.BuildResult(
        best=kf.Tracks(torch.empty((6, n), device="cuda"), torch.empty((21, n), device="cuda"), s.charge,
                       torch.empty((3, n), device="cuda")),
        chi2_tot=torch.empty(n, device="cuda"), n_hits=torch.empty(n, **i32), status=torch.empty(n, **i32),
        hit_idx=torch.empty((Lb, n), **i32),
        n_cands=torch.empty(n, **i32) if want_cands else None,
        cand_hit_idx=torch.empty((Lb, n * N), **i32) if want_cands else None,
        cand_chi2_tot=torch.empty(n * N, device="cuda") if want_cands else None,
        cand_n_hits=torch.empty(n * N, **i32) if want_cands else None)
    (build_fn or kf.kf_build)(ctx, fo, seed_off, bins, N, out)
    torch.cuda.synchronize()
    res = dict(par=out.best.par.double().cpu().numpy().T + np.pad(out.best.par_lo.double().cpu().numpy().T,
                                                                     ((0, 0), (0, 3))),
               cov=O.full_cov_from_packed(out.best.cov.double().cpu().numpy()),
               chi2=out.chi2_tot.double().cpu().numpy(), nhits=out.n_hits.cpu().numpy(),
               status=out.status.cpu().numpy(), hits=out.hit_idx.cpu().numpy().T.copy(),
               fit_status=fst.cpu().numpy(), bins=bins)
    if want_cands:
        res["n_cands"] = out.n_cands.cpu().numpy()
        res["cand_hits"] = out.cand_hit_idx.cpu().numpy().reshape(Lb, n, N).transpose(1, 2, 0).copy()
        res["cand_chi2"] = out.cand_chi2_tot.double().cpu().numpy().reshape(n, N)
        res["cand_nhits"] = out.cand_n_hits.cpu().numpy().reshape(n, N)
    return res


def _path_args(batch):
    det = batch.det
    V = np.array([f32(det.sigma_xy) ** 2, f32(det.sigma_xy) ** 2, f32(det.sigma_z) ** 2])
    radii = [f32(det.radii[l]) for l in batch.build_layers]
    mat = material(det, batch.build_layers)
    return radii, V, mat.get("x_x0"), mat.get("mass", O.PION_MASS)


def classify(batch, g, r, idx=None, cut=30.0, rel=1e-4):
    """Compare best paths seed by seed (oracle.parity.classify). Returns
    (n_same, near_ties, bad) with GPU seed indices: a differing path is a near
    tie when, evaluated by the oracle, it has the oracle best's hit count and a
    chi2_tot within `rel` relative of it, or when a hit on either path sits
    within 1e-3 of the chi2 cut."""
    from oracle import parity
    n = len(r["n_cands"])
    idx = np.arange(n) if idx is None else np.asarray(idx)
    Lb = len(batch.build_layers)
    radii, V, x_x0, mass = _path_args(batch)
    a = O.a_coef(batch.seeds.charge[idx], f32(batch.det.bz))

    def hit_of(t, l, h):
        seg = int(batch.seed_event[idx[t]]) * Lb + l
        return batch.layer_xyz[:, batch.layer_off[seg] + h].astype(np.float64)
    same, ties, bad = parity.classify(g["hits"][idx], r["hits"][:, 0], r["seed_par"], r["seed_cov"], a, hit_of,
                                      radii, V, x_x0, mass, cut, rel)
    ties = [(int(idx[t]), ca, cb) for t, ca, cb in ties]
    bad = [(int(idx[t]), pa, pb, ca, cb) for t, pa, pb, ca, cb in bad]
    return same, ties, bad

"""Helpers shared by the GPU parity tests: run the CUDA pipeline and the
oracle on the same seeded batch and compare them.

Sets (cells, CA edges, n-tuplets) are compared exactly after mapping every
index to input hit indices (output order is unspecified).  Fitted
parameters are compared within the tolerance of the float32 path:
  kappa:                        |d| <= 1e-4 |kappa|
  phi0, tan(lambda), d0, z0:    |d| <= 1e-5 max(1, |value|)   (phi0 mod 2 pi)
covariance diagonal within 1e-3 relative, and chi2 within
CHI2_TOL sqrt(max(1, chi2)).  The chi2 bound is twice the largest departure
measured on every track of whole events of all the workloads (3.0e-3, a
stress event): its source is the float32 rounding of the arc lengths
(~1e-6 cm at 10-20 cm), which moves the s-z residuals by |tan lambda| times
that and chi2 by about twice that times sqrt(chi2).
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from synth import cuts as CU
from synth import geometry as G

DISK = [0] * 4 + [1] * 6
CHI2_TOL = 6e-3
KEYS = ("x", "y", "z", "r", "module", "ev_off")


def to_dev(batch, dev="cuda:0"):
    return {k: torch.as_tensor(np.ascontiguousarray(batch[k])).to(dev) for k in KEYS}


def make_pipeline(cuts, tuning=None):
    from paper_2008_13461_gb300.pipeline import Pipeline
    return Pipeline(G.layers(), G.module_layer_table(), cuts, CU.FIT_PARAMS, tuning=tuning, device="cuda:0")


def gpu_run(batch, cuts, tuning=None, capacity=None):
    pipe = make_pipeline(cuts, tuning)
    t = to_dev(batch)
    bufs = pipe.allocate(t["x"].numel(), t["ev_off"].numel() - 1, capacity) if capacity else None
    res, _ = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"], bufs=bufs)
    torch.cuda.synchronize()
    return res


def gpu_sets(res):
    order = res.hit_order.cpu().numpy()
    ci = order[res.cells["inner"].cpu().numpy()]
    co = order[res.cells["outer"].cpu().numpy()]
    pair = res.cells["pair"].cpu().numpy()
    alive = res.cells["alive"].cpu().numpy().astype(bool)
    cells = {(int(a), int(b)): (int(p), bool(al)) for a, b, p, al in zip(ci, co, pair, alive)}
    src = res.edges["src"].cpu().numpy().astype(np.int64)
    dst = res.edges["dst"].cpu().numpy().astype(np.int64)
    edges = {(int(ci[s]), int(co[s]), int(co[d])) for s, d in zip(src, dst)}
    assert all(ci[d] == co[s] for s, d in zip(src, dst)), "edge cells do not share a hit"
    n = res.tuples["n"].cpu().numpy()
    H = res.tuples["hits"].cpu().numpy()
    al = res.tuples["alive"].cpu().numpy().astype(bool)
    tuples = {}
    for t in range(len(n)):
        key = tuple(int(v) for v in H[t, :n[t]])
        assert key not in tuples, "duplicate n-tuplet"
        tuples[key] = bool(al[t])
    return cells, edges, tuples


def oracle_sets(want):
    C = want["cells"]
    cells = {(int(c[0]), int(c[1])): (int(c[2]), bool(a)) for c, a in zip(C, want["cell_alive"])}
    edges = {(int(C[e0][0]), int(C[e0][1]), int(C[e1][1])) for e0, e1 in want["edges"]}
    tuples = {tuple(int(v) for v in want["tuple_hits"][t, :want["tuple_n"][t]]): bool(want["tuple_alive"][t])
              for t in range(len(want["tuple_n"]))}
    return cells, edges, tuples


def compare_sets(res, want):
    gc, ge, gt = gpu_sets(res)
    wc, we, wt = oracle_sets(want)
    assert len(gc) == res.counts.n_cells
    assert gc == wc, f"cells differ: {len(set(gc) - set(wc))} extra, {len(set(wc) - set(gc))} missing"
    assert ge == we, f"edges differ: {len(ge - we)} extra, {len(we - ge)} missing"
    assert gt == wt, f"n-tuplets differ: {len(set(gt) - set(wt))} extra, {len(set(wt) - set(gt))} missing"
    return len(gc), len(ge), len(gt)


def compare_tracks(res, want, batch=None):
    """Match tracks by their hit sequence and compare parameters."""
    n = res.tuples["n"].cpu().numpy()
    H = res.tuples["hits"].cpu().numpy()
    tt = res.tracks["tuple"].cpu().numpy()
    P = res.tracks["params"].cpu().numpy().astype(np.float64)
    CV = res.tracks["cov"].cpu().numpy().astype(np.float64)
    X2 = res.tracks["chi2"].cpu().numpy().astype(np.float64)
    ND = res.tracks["ndf"].cpu().numpy()
    gmap = {tuple(int(v) for v in H[t, :n[t]]): k for k, t in enumerate(tt)}
    wmap = {tuple(int(v) for v in want["tuple_hits"][t, :want["tuple_n"][t]]): k
            for k, t in enumerate(want["track_tuple"])}
    assert set(gmap) == set(wmap), "different tracks were fitted"
    if not gmap:
        return {}
    gi = np.array([gmap[k] for k in wmap])
    wi = np.array(list(wmap.values()))
    return compare_params(P[gi], CV[gi], X2[gi], ND[gi], want["params"][wi], want["cov"][wi],
                          want["chi2"][wi], want["ndf"][wi])


def compare_params(P, CV, X2, ND, WP, WC, WX2, WND, kappa_abs=0.0):
    """Fitted tracks against the oracle's within the tolerances above.
    kappa_abs: an absolute term added to the curvature bound, for hits off
    the exactness grid (0 for hits on it)."""
    assert np.array_equal(ND.astype(np.int64), WND.astype(np.int64))
    err = {}
    d = np.abs(P[:, 0] - WP[:, 0])
    err["kappa_rel"] = d / np.abs(WP[:, 0])
    assert np.all(d <= 1e-4 * np.abs(WP[:, 0]) + kappa_abs), f"kappa max rel err {err['kappa_rel'].max():.3g}"
    for j, name in ((1, "phi0"), (2, "tanl"), (3, "d0"), (4, "z0")):
        dd = P[:, j] - WP[:, j]
        if j == 1:
            dd = (dd + np.pi) % (2 * np.pi) - np.pi
        sc = np.maximum(1.0, np.abs(WP[:, j]))
        err[name] = np.abs(dd) / sc
        assert np.all(np.abs(dd) <= 1e-5 * sc), f"{name} max err {err[name].max():.3g}"
    diag = [0, 2, 5, 9, 14]
    rel = np.abs(CV[:, diag] - WC[:, diag]) / np.abs(WC[:, diag])
    err["cov_diag_rel"] = rel
    assert np.all(rel <= 1e-3), f"cov diag max rel err {rel.max():.3g}"
    rc = np.abs(X2 - WX2) / np.sqrt(np.maximum(1.0, WX2))
    err["chi2_scaled"] = rc
    assert np.all(rc <= CHI2_TOL), f"chi2 max scaled err {rc.max():.3g}"
    return {k: (float(v.max()), float(np.percentile(v, 99))) for k, v in err.items()}


def oracle_run(batch, cuts, stage=4):
    return oracle.run(batch, cuts, CU.FIT_PARAMS, G.module_layer_table(), DISK, stage=stage)

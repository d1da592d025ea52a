"""Precision of the broken-line fit (Sec. 3.4).

The float64 solve is checked against the oracle's float64 fit of the same
n-tuplets on every track of one event of the stress configuration (pileup
200, soft tracks down to 0.3 GeV with loopers, noise): the worst-conditioned
normal equations of all the configurations.  The all-float32 variant
(solve_fp32 = 1) is characterised against the same oracle: how many of its
tracks stay within the float64 tolerances and how many break down.  That is
why the float64 solve is the default.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import cuts as CU
from synth import events as E
from synth import geometry as G

from parity import CHI2_TOL, compare_params, to_dev

pytestmark = pytest.mark.gpu


def _gpu_tracks(b, cuts, fp32):
    from paper_2008_13461_gb300.pipeline import Pipeline
    fit = dict(CU.FIT_PARAMS, solve_fp32=fp32)
    pipe = Pipeline(G.layers(), G.module_layer_table(), cuts, fit, device="cuda:0")
    t = to_dev(b)
    res, _ = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    torch.cuda.synchronize()
    n = res.tuples["n"].cpu().numpy()
    H = res.tuples["hits"].cpu().numpy()
    tt = res.tracks["tuple"].cpu().numpy()
    hits = [tuple(int(v) for v in H[t, :n[t]]) for t in tt]
    return (hits, res.tracks["params"].cpu().numpy().astype(np.float64),
            res.tracks["cov"].cpu().numpy().astype(np.float64),
            res.tracks["chi2"].cpu().numpy().astype(np.float64), res.tracks["ndf"].cpu().numpy())


@pytest.fixture(scope="module")
def stress():
    b = E.make_batch("pu200-stress-batch256", n_events=1)
    cuts = CU.cuts_for("pu200-stress-batch256")
    g64 = _gpu_tracks(b, cuts, 0)
    g32 = _gpu_tracks(b, cuts, 1)
    # the same tracks (their order follows atomics): put g32 in g64's order
    pos = {h: k for k, h in enumerate(g32[0])}
    assert set(pos) == set(g64[0])
    perm = np.array([pos[h] for h in g64[0]])
    g32 = (g64[0],) + tuple(a[perm] for a in g32[1:])
    lay = G.module_layer_table()[b["module"]]
    W = [oracle.fit(b["x"][list(h)], b["y"][list(h)], b["z"][list(h)], (lay[list(h)] >= 4).astype(int),
                    CU.FIT_PARAMS) for h in g64[0]]
    want = (np.array([w[0] for w in W]), np.array([w[1] for w in W]), np.array([w[2] for w in W]),
            np.array([w[3] for w in W]))
    # condition numbers of each track's normal matrices (line, circle)
    cond = np.array([[w[4][8], w[4][9]] for w in W])
    return g64, g32, want, cond


def test_fp64_solve_matches_the_oracle_on_every_stress_track(stress):
    g64, _, (WP, WC, WX, WN), _ = stress
    assert len(WP) > 10000
    err = compare_params(g64[1], g64[2], g64[3], g64[4], WP, WC, WX, WN)
    print("float64 solve vs oracle (max):", {k: float(np.max(v)) for k, v in err.items()})


def _outside(P, CV, X2, WP, WC, WX):
    """Per track: within the float64 tolerances of the fit parity contract?"""
    ok = np.isfinite(P).all(1) & np.isfinite(CV).all(1) & np.isfinite(X2)
    with np.errstate(invalid="ignore", divide="ignore"):
        ok &= np.abs(P[:, 0] - WP[:, 0]) <= 1e-4 * np.abs(WP[:, 0])
        for j in (1, 2, 3, 4):
            dd = P[:, j] - WP[:, j]
            if j == 1:
                dd = (dd + np.pi) % (2 * np.pi) - np.pi
            ok &= np.abs(dd) <= 1e-5 * np.maximum(1.0, np.abs(WP[:, j]))
        diag = [0, 2, 5, 9, 14]
        ok &= (np.abs(CV[:, diag] - WC[:, diag]) <= 1e-3 * np.abs(WC[:, diag])).all(1)
        ok &= np.abs(X2 - WX) <= CHI2_TOL * np.sqrt(np.maximum(1.0, WX))
    return ~ok


def test_fp32_variant_is_characterised(stress):
    _, g32, (WP, WC, WX, _), _ = stress
    P, CV, X2 = g32[1], g32[2], g32[3]
    finite = np.isfinite(P).all(1) & np.isfinite(CV).all(1) & np.isfinite(X2)
    out = _outside(P, CV, X2, WP, WC, WX)
    print(f"float32 variant: {len(P)} tracks, {np.mean(~finite):.2e} non-finite, "
          f"{np.mean(out):.2e} outside the float64 tolerances")
    for name, j in (("kappa", 0), ("tanl", 2), ("z0", 4)):
        e = np.abs(P[finite, j] - WP[finite, j]) / (np.abs(WP[finite, j]) if j == 0 else
                                                     np.maximum(1.0, np.abs(WP[finite, j])))
        print(f"  {name}: p50 {np.percentile(e, 50):.2e} p99 {np.percentile(e, 99):.2e} max {e.max():.2e}")
    # usable for most tracks but not for all (measured: 0.7% outside, a few
    # non-finite): the float64 solve is needed for the parity contract
    assert 0.0 < np.mean(out) < 0.02


def test_fp32_breakdown_follows_the_condition_number(stress):
    """Condition-number report per track: the all-float32 variant's
    departures from the float64 tolerances, by the 2-norm condition number
    of the worse of each track's two normal matrices (the oracle's)."""
    _, g32, (WP, WC, WX, _), cond = stress
    out = _outside(g32[1], g32[2], g32[3], WP, WC, WX)
    c = cond.max(1)
    print(f"condition number: p50 {np.percentile(c, 50):.2e} p90 {np.percentile(c, 90):.2e} "
          f"p99 {np.percentile(c, 99):.2e} max {c.max():.2e}")
    edges = [1.0, 1e4, 1e6, 1e8, 1e10, 1e12, np.inf]
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (c >= lo) & (c < hi)
        if sel.any():
            print(f"  cond [{lo:.0e}, {hi:.0e}): {sel.sum()} tracks, {out[sel].mean():.2e} outside")
    low, high = c < np.percentile(c, 50), c >= np.percentile(c, 99)
    assert out[high].mean() > 10 * out[low].mean()

"""Differentiation on the misaligned pileup-50 batch (needs a GB300).

All 32 events of the pileup-50 workload go through the four calls; the
n-tuplets found on the nominal hits are then refitted after every one of the
1856 modules has been moved by a seeded misalignment, shifts ~ N(0, 50 um)
and rotations ~ N(0, 0.1 mrad) per axis about the module centre.  Checked
against the oracle (float64):

  * the aligned hits (pt_align_hits) and the refit of every track on them.
    Aligned hits are off the 2^-14 cm grid, so the float32 differences of
    hit coordinates the fit starts from are no longer exact: each carries
    up to u |d| (u = 2^-24, |d| < 16 cm) of rounding, which moves the
    sagitta of an L ~ 10 cm track by ~2e-6 cm and its curvature by up to
    8 s / L^2 ~ 1e-7 /cm.  The curvature is therefore compared within
    1e-4 |kappa| + 1e-7 /cm (the relative bound alone cannot hold for the
    few tracks the misalignment makes nearly straight); every other
    tolerance is the on-grid one;
  * the adjoint's gradient with respect to the aligned hits, against plain
    central differences of the oracle fit with the 1e-4 cm step (within
    twice their own truncation error, estimated from the half step) and
    against the oracle's extrapolated gradient (within 1e-5);
  * the gradients with respect to the module shifts and rotations
    (pt_align_hits_grad after the adjoint), against central differences of
    the oracle's loss with the shift step 1e-4 cm and a rotation step that
    moves the hits by about as much.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import cuts as CU
from synth import events as E
from synth import geometry as G

from parity import compare_params, make_pipeline, to_dev

pytestmark = pytest.mark.gpu

SHIFT_SIGMA = 50e-4      # cm
ROT_SIGMA = 1e-4         # rad
H_SHIFT = 1e-4           # cm
H_ROT = 3e-5             # rad: hits ~3 cm from the centre move by ~1e-4 cm
MISALIGNMENT_SEED = 2008134610 + 4000 + 999
SCALE = np.array([1e3, 1e3, 1e3, 1e2, 1e2])   # a unit of each parameter ~ its resolution
KAPPA_OFF_GRID = 1e-7    # /cm: float32 rounding of off-grid hit differences (module docstring)


@pytest.fixture(scope="module")
def batch32():
    from paper_2008_13461_gb300.autograd import DifferentiableFit
    b = E.make_batch("pu50-batch32", workers=8)
    assert len(b["ev_off"]) == 33
    pipe = make_pipeline(CU.cuts_for("pu50-batch32"))
    t = to_dev(b)
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    n = res.tuples["n"].cpu().numpy()
    Ht = res.tuples["hits"].cpu().numpy()
    hits = [Ht[q, :n[q]].astype(np.int64) for q in res.tracks["tuple"].cpu().numpy()]
    rng = np.random.default_rng(MISALIGNMENT_SEED)
    nm = G.N_MODULES
    shift = rng.normal(0.0, SHIFT_SIGMA, size=(nm, 3)).astype(np.float32)
    rot = rng.normal(0.0, ROT_SIGMA, size=(nm, 3)).astype(np.float32)
    centres = G.module_centres().astype(np.float32)
    df = DifferentiableFit(pipe, bufs, t["r"], t["module"], t["ev_off"], centres=torch.as_tensor(centres))
    lay = G.module_layer_table()[b["module"]]
    return dict(b=b, t=t, hits=hits, df=df, shift=shift, rot=rot, centres=centres, disk=(lay >= 4).astype(int))


def _aligned(d):
    dev = d["t"]["x"].device
    with torch.no_grad():
        return d["df"].align(d["t"]["x"], d["t"]["y"], d["t"]["z"], torch.as_tensor(d["shift"], device=dev),
                             torch.as_tensor(d["rot"], device=dev))


def _disjoint(hits, rng, want):
    used, out = set(), []
    for k in rng.permutation(len(hits)):
        h = set(int(v) for v in hits[k])
        if used.isdisjoint(h):
            out.append(int(k))
            used |= h
        if len(out) == want:
            break
    return out


def _weights(d, n_pick, seed):
    rng = np.random.default_rng(seed)
    pick = _disjoint(d["hits"], rng, n_pick)
    K = len(d["hits"])
    gp = np.zeros((K, 5), np.float32)
    gc = np.zeros(K, np.float32)
    gp[pick] = rng.normal(size=(len(pick), 5)) / SCALE
    gc[pick] = rng.normal(size=len(pick)) * 1e-2
    return pick, gp, gc


def test_alignment_and_refit_of_every_track_match_the_oracle(batch32):
    d = batch32
    b = d["b"]
    xa, ya, za = (a.cpu().numpy() for a in _aligned(d))
    wx, wy, wz = oracle.align_hits(b["x"], b["y"], b["z"], b["module"], d["centres"].astype(np.float64),
                                   d["shift"].astype(np.float64), d["rot"].astype(np.float64))
    for got, want in ((xa, wx), (ya, wy), (za, wz)):
        assert np.all(np.abs(got - want) <= 4 * np.spacing(np.maximum(np.abs(want), 1.0).astype(np.float32)))
    moved = np.sqrt((xa - b["x"]) ** 2 + (ya - b["y"]) ** 2 + (za - b["z"]) ** 2)
    assert 20e-4 < np.median(moved) < 200e-4                     # the modules did move, by tens of um
    dev = d["t"]["x"].device
    params, chi2 = d["df"].fit(*(torch.as_tensor(a, device=dev) for a in (xa, ya, za)))
    K = len(d["hits"])
    P = params.double().cpu().numpy()
    X2 = chi2.double().cpu().numpy()
    CV = d["df"].cov[:K * 15].view(K, 15).double().cpu().numpy()
    ND = d["df"].ndf[:K].cpu().numpy()
    W = [oracle.fit(xa[h], ya[h], za[h], d["disk"][h], CU.FIT_PARAMS) for h in d["hits"]]
    WP = np.array([w[0] for w in W])
    err = compare_params(P, CV, X2, ND, WP, np.array([w[1] for w in W]), np.array([w[2] for w in W]),
                         np.array([w[3] for w in W]), kappa_abs=KAPPA_OFF_GRID)
    print(f"largest absolute curvature departure {np.abs(P[:, 0] - WP[:, 0]).max():.2e} /cm "
          f"(bound 1e-4 |kappa| + {KAPPA_OFF_GRID:g})")
    print(f"refit of {K} tracks on misaligned hits vs oracle (max, p99):", err)
    assert K > 50000


def test_hit_gradient_matches_oracle_central_differences(batch32):
    d = batch32
    pick, gp, gc = _weights(d, 150, 21)
    dev = d["t"]["x"].device
    xa, ya, za = (a.detach().clone().requires_grad_() for a in _aligned(d))
    params, chi2 = d["df"].fit(xa, ya, za)
    ((params * torch.as_tensor(gp, device=dev)).sum() + (chi2 * torch.as_tensor(gc, device=dev)).sum()).backward()
    gx, gy, gz = (a.grad.cpu().numpy() for a in (xa, ya, za))
    X, Y, Z = (a.detach().cpu().numpy() for a in (xa, ya, za))
    worst_c = worst_r = worst_t = 0.0
    for k in pick:
        h = d["hits"][k]
        args = (X[h], Y[h], Z[h], d["disk"][h], CU.FIT_PARAMS, gp[k].astype(np.float64), float(gc[k]))
        central = oracle.fit_grad_central(*args, h=1e-4)
        half = oracle.fit_grad_central(*args, h=5e-5)
        ref = oracle.fit_grad_fd(*args)
        got = np.stack([gx[h], gy[h], gz[h]])
        scale = np.abs(ref).max()
        # the central differences' truncation error, O(h^2): estimated per
        # component from the half step as (4/3) |c(h) - c(h/2)|
        trunc = 4.0 / 3.0 * np.abs(central - half)
        assert np.all(np.abs(got - central) <= 2.0 * trunc + 2e-5 * scale), k
        worst_c = max(worst_c, np.abs(got - central).max() / scale)
        worst_t = max(worst_t, trunc.max() / scale)
        worst_r = max(worst_r, np.abs(got - ref).max() / scale)
    print(f"adjoint vs oracle on {len(pick)} misaligned tracks, max relative to the track's largest component: "
          f"central differences (h = 1e-4 cm) {worst_c:.2e} (their own truncation error up to {worst_t:.2e}), "
          f"extrapolated {worst_r:.2e}")
    assert worst_r < 1e-5


def test_alignment_gradient_matches_oracle_central_differences(batch32):
    d = batch32
    b = d["b"]
    pick, gp, gc = _weights(d, 400, 22)
    dev = d["t"]["x"].device
    shift = torch.as_tensor(d["shift"], device=dev).requires_grad_()
    rot = torch.as_tensor(d["rot"], device=dev).requires_grad_()
    xa, ya, za = d["df"].align(d["t"]["x"], d["t"]["y"], d["t"]["z"], shift, rot)
    params, chi2 = d["df"].fit(xa, ya, za)
    ((params * torch.as_tensor(gp, device=dev)).sum() + (chi2 * torch.as_tensor(gc, device=dev)).sum()).backward()
    gs, gr = shift.grad.cpu().numpy(), rot.grad.cpu().numpy()
    mod = b["module"]
    counts = np.bincount(np.concatenate([mod[d["hits"][k]] for k in pick]), minlength=G.N_MODULES)
    C64, S64, R64 = (d[k].astype(np.float64) for k in ("centres", "shift", "rot"))
    for m in np.argsort(counts)[-4:]:
        ks = [k for k in pick if np.any(mod[d["hits"][k]] == m)]

        def fits(ds, dr):
            s, r = S64.copy(), R64.copy()
            s[m] += ds
            r[m] += dr
            out = []
            for k in ks:
                h = d["hits"][k]
                x, y, z = oracle.align_hits(b["x"][h], b["y"][h], b["z"][h], mod[h], C64, s, r)
                p, _, c2, _, _ = oracle.fit(x, y, z, d["disk"][h], CU.FIT_PARAMS)
                out.append((p, c2))
            return out

        def central(up, dn, step):
            tot = 0.0
            for k, (pu, cu), (pd, cd) in zip(ks, up, dn):
                dp = pu - pd
                dp[1] = (dp[1] + np.pi) % (2 * np.pi) - np.pi          # phi0 modulo 2 pi
                tot += float(np.dot(gp[k], dp)) + float(gc[k]) * (cu - cd)
            return tot / (2 * step)

        got = np.concatenate([gs[m], gr[m]])
        scale = np.abs(got).max()
        for j in range(6):
            e = np.zeros(3)
            e[j % 3] = 1.0
            if j < 3:
                fd = central(fits(H_SHIFT * e, 0 * e), fits(-H_SHIFT * e, 0 * e), H_SHIFT)
            else:
                fd = central(fits(0 * e, H_ROT * e), fits(0 * e, -H_ROT * e), H_ROT)
            assert abs(got[j] - fd) <= 2e-3 * abs(fd) + 2e-4 * scale, (int(m), j, float(got[j]), fd)
        print(f"module {int(m)} ({counts[m]} hits of the weighted tracks): shift and rotation gradients "
              f"match the oracle's central differences")

"""Gradients of the broken-line fit (the adjoint kernel, Sec. 3.4
differentiated) and of the per-module hit alignment, on two events of the
pileup-50 workload: against the oracle's float64 gradient, exact sum rules,
and finite differences of the GPU fit itself."""
import numpy as np
import pytest
import torch

import oracle
from synth import cuts as CU
from synth import events as E
from synth import geometry as G

from parity import make_pipeline, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pu50_pair():
    from paper_2008_13461_gb300.autograd import DifferentiableFit
    b = E.make_batch("pu50-batch32", n_events=2)
    cuts = CU.cuts_for("pu50-batch32")
    pipe = make_pipeline(cuts)
    t = to_dev(b)
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    n = res.tuples["n"].cpu().numpy()
    H = res.tuples["hits"].cpu().numpy()
    tt = res.tracks["tuple"].cpu().numpy()
    hits = [H[q, :n[q]].astype(np.int64) for q in tt]
    df = DifferentiableFit(pipe, bufs, t["r"], t["module"], t["ev_off"],
                           centres=torch.as_tensor(G.module_centres(), dtype=torch.float32))
    return b, t, hits, df


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


# output scales: a unit change of each parameter is weighted like one of
# its typical resolution, so no parameter dominates the loss
SCALE = np.array([1e3, 1e3, 1e3, 1e2, 1e2])


def _loss_grads(df, t, gp, gc):
    x, y, z = (t[k].clone().requires_grad_() for k in ("x", "y", "z"))
    params, chi2 = df.fit(x, y, z)
    loss = (params * gp).sum() + (chi2 * gc).sum()
    loss.backward()
    return params.detach(), chi2.detach(), x.grad.cpu().numpy(), y.grad.cpu().numpy(), z.grad.cpu().numpy()


def test_refit_reproduces_the_pipeline_fit(pu50_pair):
    b, t, hits, df = pu50_pair
    params, chi2 = df.fit(t["x"], t["y"], t["z"])
    assert params.shape[0] == len(hits)
    p2, c2 = df.fit(t["x"], t["y"], t["z"])          # same tracks, same order
    assert torch.equal(params, p2) and torch.equal(chi2, c2)


def test_adjoint_matches_the_oracle_gradient(pu50_pair):
    b, t, hits, df = pu50_pair
    rng = np.random.default_rng(5)
    pick = _disjoint(hits, rng, 120)
    K = len(hits)
    gp = np.zeros((K, 5), np.float32)
    gc = np.zeros(K, np.float32)
    gp[pick] = rng.normal(size=(len(pick), 5)) / SCALE
    gc[pick] = rng.normal(size=len(pick)) * 1e-2
    dev = t["x"].device
    _, _, gx, gy, gz = _loss_grads(df, t, torch.as_tensor(gp, device=dev), torch.as_tensor(gc, device=dev))
    lay = G.module_layer_table()[b["module"]]
    worst = 0.0
    for k in pick:
        h = hits[k]
        want = oracle.fit_grad_fd(b["x"][h], b["y"][h], b["z"][h], (lay[h] >= 4).astype(int), CU.FIT_PARAMS,
                                  gp[k].astype(np.float64), float(gc[k]))
        got = np.stack([gx[h], gy[h], gz[h]])
        scale = np.abs(want).max() + 1e-12
        err = np.abs(got - want).max() / scale
        worst = max(worst, err)
    print("adjoint vs oracle gradient, max relative to the track's largest component:", worst)
    assert worst < 1e-5


def test_adjoint_obeys_the_sum_rules(pu50_pair):
    b, t, hits, df = pu50_pair
    K = len(hits)
    dev = t["x"].device
    x = t["x"].cpu().numpy().astype(np.float64)
    y = t["y"].cpu().numpy().astype(np.float64)
    for o in range(6):
        gp = torch.zeros(K, 5, device=dev)
        gc = torch.zeros(K, device=dev)
        if o < 5:
            gp[:, o] = 1.0
        else:
            gc[:] = 1.0
        _, _, gx, gy, gz = _loss_grads(df, t, gp, gc)
        sz = gz.astype(np.float64).sum()
        rot = float(np.sum(x * gy - y * gx))
        scale = np.abs(gx).sum() + np.abs(gy).sum() + np.abs(gz).sum() + K
        # z translation moves every z0 by the shift; a rotation about the
        # beam line turns every phi0 by the angle; nothing else changes
        assert abs(sz - (K if o == 4 else 0.0)) < 1e-4 * scale, (o, sz)
        assert abs(rot - (K if o == 1 else 0.0)) < 1e-4 * scale, (o, rot)


def test_adjoint_matches_finite_differences_of_the_gpu_fit(pu50_pair):
    b, t, hits, df = pu50_pair
    rng = np.random.default_rng(9)
    K = len(hits)
    dev = t["x"].device
    gp = torch.as_tensor(rng.normal(size=(K, 5)) / SCALE, dtype=torch.float32, device=dev)
    gc = torch.as_tensor(rng.normal(size=K) * 1e-2, dtype=torch.float32, device=dev)
    _, _, gx, gy, gz = _loss_grads(df, t, gp, gc)
    used = np.unique(np.concatenate(hits))
    hs = rng.choice(used, size=20, replace=False)
    step = 1e-3
    for h in hs:
        # only the tracks through the hit depend on it; the others' float32
        # rounding would only add noise to the difference
        on = torch.as_tensor([bool(np.any(hk == h)) for hk in hits], device=dev)
        for axis, g in (("x", gx), ("y", gy), ("z", gz)):
            vals = []
            for sgn in (1.0, -1.0):
                tt = {k: t[k].clone() for k in ("x", "y", "z")}
                tt[axis][h] += sgn * step
                p, c = df.fit(tt["x"], tt["y"], tt["z"])
                v = (p.double() * gp.double()).sum(1) + c.double() * gc.double()
                vals.append(v[on].sum().item())
            fd = (vals[0] - vals[1]) / (2 * step)
            assert abs(fd - g[h]) <= 2e-2 * abs(g[h]) + 2e-2, (int(h), axis, fd, float(g[h]))


def test_alignment_gradient_matches_the_oracle(pu50_pair):
    b, t, hits, df = pu50_pair
    dev = t["x"].device
    nm = G.N_MODULES
    K = len(hits)
    shift = torch.zeros(nm, 3, device=dev, requires_grad=True)
    rot = torch.zeros(nm, 3, device=dev, requires_grad=True)
    xa, ya, za = df.align(t["x"], t["y"], t["z"], shift, rot)
    params, chi2 = df.fit(xa, ya, za)
    chi2.sum().backward()
    gs, gr = shift.grad.cpu().numpy(), rot.grad.cpu().numpy()
    # the modules with the most fitted hits
    mod = b["module"]
    counts = np.bincount(np.concatenate([mod[h] for h in hits]), minlength=nm)
    lay = G.module_layer_table()[mod]
    centres = G.module_centres()
    for m in np.argsort(counts)[-3:]:
        ks = [k for k in range(K) if np.any(mod[hits[k]] == m)]
        c = centres[m]

        def total(delta, omega):
            s = 0.0
            for k in ks:
                h = hits[k]
                P = np.stack([b["x"][h], b["y"][h], b["z"][h]], 1).astype(np.float64)
                on = mod[h] == m
                r = P[on] - c
                P[on] = P[on] + np.cross(omega, r) + delta
                s += oracle.fit(P[:, 0], P[:, 1], P[:, 2], (lay[h] >= 4).astype(int), CU.FIT_PARAMS)[2]
            return s

        for j in range(6):
            e = np.zeros(3)
            e[j % 3] = 1.0
            hstep = 1e-5 if j < 3 else 1e-6
            if j < 3:
                fd = (total(hstep * e, np.zeros(3)) - total(-hstep * e, np.zeros(3))) / (2 * hstep)
                got = gs[m, j]
            else:
                fd = (total(np.zeros(3), hstep * e) - total(np.zeros(3), -hstep * e)) / (2 * hstep)
                got = gr[m, j - 3]
            assert abs(got - fd) <= 1e-3 * abs(fd) + 1e-3 * (1.0 + np.abs(gs[m]).max()), (int(m), j, got, fd)


def test_a_refit_leaves_the_run_tracks_unchanged():
    from paper_2008_13461_gb300.autograd import DifferentiableFit
    b = E.make_batch("pu50-batch32", n_events=1)
    pipe = make_pipeline(CU.cuts_for("pu50-batch32"))
    t = to_dev(b)
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    before = {k: v.clone() for k, v in res.tracks.items()}
    df = DifferentiableFit(pipe, bufs, t["r"], t["module"], t["ev_off"])
    params, _ = df.fit(t["x"] + 1e-3, t["y"] - 2e-3, t["z"] + 5e-3)     # moved hits
    torch.cuda.synchronize()
    assert not torch.equal(params, before["params"])                      # the refit saw the moved hits
    for k, v in before.items():
        assert torch.equal(res.tracks[k], v), k                           # the run's tracks did not change

"""GPU vs oracle parity through the C ABI (needs a GB300).

Small configurations are compared element by element (exact sets, fits in
tolerance); the full PU200 batch is checked on sampled outputs the oracle
computes one by one, and through properties that hold at any size.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from synth import cuts as CU
from synth import events as E
from synth import geometry as G

from parity import compare_params, compare_sets, compare_tracks, gpu_run, make_pipeline, oracle_run, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pu50():
    return E.make_batch("pu50-ttbar-like")


@pytest.fixture(scope="module")
def pu50_oracle(pu50):
    return oracle_run(pu50, CU.cuts_for("pu50-ttbar-like"))


def test_noiseless_barrel_helices():
    b = E.make_batch("barrel-50-helices")
    cuts = CU.cuts_for("barrel-50-helices")
    res = gpu_run(b, cuts)
    want = oracle_run(b, cuts)
    compare_sets(res, want)
    compare_tracks(res, want)
    assert res.counts.n_tracks > 30


def test_pu50_event(pu50, pu50_oracle):
    res = gpu_run(pu50, CU.cuts_for("pu50-ttbar-like"))
    nc, ne, nt = compare_sets(res, pu50_oracle)
    err = compare_tracks(res, pu50_oracle)
    assert nc > 50000 and nt > 1000
    print("pu50-ttbar-like fit error (max, p99):", err)


def _concat(events):
    out = {}
    for k in ("x", "y", "z", "r", "module"):
        out[k] = np.concatenate([e[k] for e in events])
    off = np.zeros(len(events) + 1, dtype=np.int32)
    off[1:] = np.cumsum([e["x"].size for e in events])
    out["ev_off"] = off
    return out


def _slice(b, e):
    a, z = b["ev_off"][e], b["ev_off"][e + 1]
    return {k: b[k][a:z] for k in ("x", "y", "z", "r", "module")}


def test_ragged_batch_with_empty_and_tiny_events():
    b32 = E.make_batch("pu50-batch32", n_events=3)
    evs = [_slice(b32, 0), _slice(b32, 1), _slice(b32, 2)]
    empty = {k: v[:0] for k, v in evs[0].items()}
    one = {k: v[:1] for k, v in evs[1].items()}
    batch = _concat([empty, evs[0], one, evs[1], empty, empty, evs[2], one])
    cuts = CU.cuts_for("pu50-batch32")
    res = gpu_run(batch, cuts)
    want = oracle_run(batch, cuts)
    compare_sets(res, want)
    compare_tracks(res, want)


def test_all_empty_batch():
    batch = {k: np.zeros(0, dtype=np.float32) for k in ("x", "y", "z", "r")}
    batch["module"] = np.zeros(0, dtype=np.int32)
    batch["ev_off"] = np.zeros(3, dtype=np.int32)
    res = gpu_run(batch, CU.cuts_for("pu50-ttbar-like"))
    assert res.counts.n_cells == 0 and res.counts.n_tracks == 0


@pytest.mark.parametrize("tuning", [
    dict(n_phi_bins=16, n_t_bins=1, doublet_lanes=4, connect_lanes=4, blocks_per_sm=1),
    dict(n_phi_bins=1024, n_t_bins=64, doublet_lanes=32, connect_lanes=32, blocks_per_sm=2),
    dict(n_phi_bins=64, n_t_bins=8, doublet_lanes=16, connect_lanes=16, blocks_per_sm=16),
])
def test_results_do_not_depend_on_tuning(pu50, pu50_oracle, tuning):
    res = gpu_run(pu50, CU.cuts_for("pu50-ttbar-like"), tuning=tuning)
    compare_sets(res, pu50_oracle)
    compare_tracks(res, pu50_oracle)


def test_autotune_picks_a_tuning_with_unchanged_results(pu50, pu50_oracle):
    from paper_2008_13461_gb300.autotune import autotune
    pipe = make_pipeline(CU.cuts_for("pu50-ttbar-like"), tuning=dict(n_t_bins=32, doublet_lanes=8, n_phi_bins=128))
    t = to_dev(pu50)
    args = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    space = (("n_t_bins", (8, 32)), ("doublet_lanes", (4, 8)), ("n_phi_bins", (64, 128)))   # the base is inside
    best, timings = autotune(pipe, *args, reps=1, space=space)   # raises if a tuning changes a count
    assert len(timings) >= 4 and all(v > 0 for v in timings.values())
    assert best["n_t_bins"] in (8, 32) and best["doublet_lanes"] in (4, 8) and best["n_phi_bins"] in (64, 128)
    pipe.set_tuning(best)
    res, _ = pipe.run(*args)
    compare_sets(res, pu50_oracle)


def test_capacity_overflow_is_reported_then_retried(pu50, pu50_oracle):
    from paper_2008_13461_gb300 import _lib as L
    cuts = CU.cuts_for("pu50-ttbar-like")
    pipe = make_pipeline(cuts)
    t = to_dev(pu50)
    args = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    bufs = pipe.allocate(t["x"].numel(), 1, dict(cells=1000, edges=10, tuples=10, tracks=10))
    pipe.launch(bufs, *args)
    st, c = pipe.counts(bufs, *args)
    assert st == L.PT_ERR_CAPACITY
    assert c.flags & L.FLAG_CELLS
    assert c.n_cells == len(pu50_oracle["cells"])      # counting continues past the capacity
    res, _ = pipe.run(*args, bufs=bufs)             # grows the buffers and reruns
    compare_sets(res, pu50_oracle)


def test_input_contract_violations_are_flagged(pu50):
    from paper_2008_13461_gb300 import _lib as L
    cuts = CU.cuts_for("pu50-ttbar-like")
    pipe = make_pipeline(cuts)
    for what in ("offgrid", "module", "envelope"):
        b = {k: np.array(v, copy=True) for k, v in pu50.items() if k in ("x", "y", "z", "r", "module", "ev_off")}
        if what == "offgrid":
            b["x"][5] = np.float32(b["x"][5]) + np.float32(1e-6)
        elif what == "module":
            b["module"][7] = G.N_MODULES + 3
        else:
            b["z"][9] = np.float32(60.0)
        t = to_dev(b)
        args = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
        bufs = pipe.allocate(t["x"].numel(), 1)
        pipe.launch(bufs, *args)
        st, c = pipe.counts(bufs, *args)
        assert st == L.PT_ERR_INPUT and c.flags & L.FLAG_INPUT, what


def test_invalid_arguments_are_rejected_on_the_host(pu50):
    from paper_2008_13461_gb300 import _lib as L
    cuts = CU.cuts_for("pu50-ttbar-like")
    pipe = make_pipeline(cuts)
    t = to_dev(pu50)
    bufs = pipe.allocate(t["x"].numel(), 1)
    h = pipe._hits(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    cfg = pipe._cfg(bufs.capacity)
    cells, _, _, _ = bufs.structs()
    s = torch.cuda.current_stream().cuda_stream

    def call(ws_bytes, c):
        return L.lib().pt_build_doublets(bufs.ws.data_ptr(), ws_bytes, ctypes.byref(h), ctypes.byref(c),
                                         ctypes.byref(cells), s)

    assert call(16, cfg) == L.PT_ERR_INVALID_ARG                 # workspace too small
    bad = L.Config.from_buffer_copy(cfg)
    bad.tuning.doublet_lanes = 3
    assert call(bufs.ws.numel(), bad) == L.PT_ERR_INVALID_ARG    # bad tuning
    bad = L.Config.from_buffer_copy(cfg)
    bad.cuts.region[0].rmax2 = 0.0
    assert call(bufs.ws.numel(), bad) == L.PT_ERR_INVALID_ARG    # constant out of range
    bad = L.Config.from_buffer_copy(cfg)
    bad.cuts.pair[0].inner = bad.cuts.pair[0].outer
    assert call(bufs.ws.numel(), bad) == L.PT_ERR_INVALID_ARG    # degenerate pair
    assert call(bufs.ws.numel(), cfg) == L.PT_OK


# ------------------------------------------------------ full PU200 batch
@pytest.fixture(scope="module")
def pu200():
    b = E.make_batch("pu200-batch64")
    cuts = CU.cuts_for("pu200-batch64")
    res = gpu_run(b, cuts)
    return b, cuts, res


def _gpu_arrays(res):
    order = res.hit_order.cpu().numpy().astype(np.int64)
    ci = order[res.cells["inner"].cpu().numpy()]
    co = order[res.cells["outer"].cpu().numpy()]
    alive = res.cells["alive"].cpu().numpy().astype(bool)
    src = res.edges["src"].cpu().numpy().astype(np.int64)
    dst = res.edges["dst"].cpu().numpy().astype(np.int64)
    return ci, co, alive, src, dst


def test_pu200_sampled_doublets_and_fishbone(pu200):
    b, cuts, res = pu200
    ml = G.module_layer_table()
    lay = ml[b["module"]]
    H = np.stack([b["x"], b["y"], b["z"], b["r"]], 1).astype(np.float32)
    ci, co, alive, _, _ = _gpu_arrays(res)
    pair = res.cells["pair"].cpu().numpy()
    rng = np.random.default_rng(5)
    ev_of = np.searchsorted(b["ev_off"], np.arange(H.shape[0]), side="right") - 1
    outer_layers = {pp["outer"] for pp in cuts["pairs"]}
    outers = np.nonzero(np.isin(lay, list(outer_layers)))[0]
    for o in rng.choice(outers, size=30, replace=False):
        e = ev_of[o]
        lo, hi = b["ev_off"][e], b["ev_off"][e + 1]
        want = {}
        for p, pp in enumerate(cuts["pairs"]):
            if pp["outer"] != lay[o]:
                continue
            cand = lo + np.nonzero((lay[lo:hi] == pp["inner"]) & (H[lo:hi, 2] >= pp["zlo"]) &
                                   (H[lo:hi, 2] <= pp["zhi"]))[0]
            for i in cand:
                hh = H[[i, o]]
                if (oracle.pred("zip", hh, pp["zmax"]) and oracle.pred("phiw", hh, pp["tan2_dphi"])
                        and oracle.pred("pt", hh, pp["k_pt"])):
                    want[int(i)] = p
        sel = np.nonzero(co == o)[0]
        got = {int(ci[k]): int(pair[k]) for k in sel}
        assert got == want, f"outer hit {o}: doublets differ"
        # Fishbone by its definition on this complete sibling set
        for k in sel:
            i = ci[k]
            dead = False
            for k2 in sel:
                j = ci[k2]
                if j == i or lay[j] != lay[i]:
                    continue
                if not oracle.pred("fb", H[[i, j, o]], cuts["fishbone_eps2"]):
                    continue
                li = np.sum((H[i, :3].astype(np.float64) - H[o, :3]) ** 2)
                lj = np.sum((H[j, :3].astype(np.float64) - H[o, :3]) ** 2)
                dead |= bool(lj < li or (lj == li and j < i))
            assert alive[k] == (not dead), f"Fishbone verdict differs for cell ({i},{o})"


def test_pu200_sampled_edges_and_paths(pu200):
    b, cuts, res = pu200
    ml = G.module_layer_table()
    lay = ml[b["module"]]
    H = np.stack([b["x"], b["y"], b["z"], b["r"]], 1).astype(np.float32)
    ci, co, alive, src, dst = _gpu_arrays(res)
    assert np.all(co[src] == ci[dst]), "edge cells do not share a hit"
    assert np.all(alive[src]) and np.all(alive[dst])
    rng = np.random.default_rng(6)
    for k in rng.choice(src.size, size=min(400, src.size), replace=False):
        a, bb, c = ci[src[k]], ci[dst[k]], co[dst[k]]
        reg = cuts["region"][1 if lay[bb] >= 4 else 0]
        h3 = H[[a, bb, c]]
        assert (oracle.pred("dz", h3, reg["zmax"]) and oracle.pred("rz", h3, reg["tol_rz2"])
                and oracle.pred("curv", h3, reg["k_curv"]) and oracle.pred("beamspot", h3, reg["rmax2"]))
    nc = ci.size
    has_in = np.zeros(nc, bool)
    has_in[dst] = True
    has_out = np.zeros(nc, bool)
    has_out[src] = True
    root = alive & ((lay[ci] == 0) | (np.isin(lay[ci], [1, 4, 7]) & ~has_in))
    # number of maximal paths from each cell: fixed point of
    # paths(c) = 1 if c has no outer neighbour else sum of its neighbours' paths
    paths = np.ones(nc, dtype=np.int64)
    for _ in range(10):
        acc = np.bincount(src, weights=paths[dst], minlength=nc).astype(np.int64)
        new = np.where(has_out, acc, 1)
        if np.array_equal(new, paths):
            break
        paths = new
    total = int(paths[root & has_out].sum())
    n = res.tuples["n"].cpu().numpy()
    assert total == n.size
    # sampled n-tuplets are root-to-leaf paths of the graph
    Ht = res.tuples["hits"].cpu().numpy()
    Ct = res.tuples["cells"].cpu().numpy()
    for t in rng.choice(n.size, size=min(500, n.size), replace=False):
        cells_t = Ct[t, :n[t] - 1]
        hits_t = Ht[t, :n[t]]
        assert np.array_equal(ci[cells_t], hits_t[:-1]) and np.array_equal(co[cells_t], hits_t[1:])
        assert root[cells_t[0]] and not has_out[cells_t[-1]]


def test_pu200_sampled_fits(pu200):
    b, cuts, res = pu200
    ml = G.module_layer_table()
    lay = ml[b["module"]]
    n = res.tuples["n"].cpu().numpy()
    H = res.tuples["hits"].cpu().numpy()
    tt = res.tracks["tuple"].cpu().numpy()
    P = res.tracks["params"].cpu().numpy().astype(np.float64)
    CV = res.tracks["cov"].cpu().numpy().astype(np.float64)
    X2 = res.tracks["chi2"].cpu().numpy().astype(np.float64)
    ND = res.tracks["ndf"].cpu().numpy()
    rng = np.random.default_rng(7)
    ks = rng.choice(len(tt), size=min(2000, len(tt)), replace=False)
    WP, WC, WX, WN = [], [], [], []
    for k in ks:
        h = H[tt[k], :n[tt[k]]]
        p, cv, c2, nd, _ = oracle.fit(b["x"][h], b["y"][h], b["z"][h], (lay[h] >= 4).astype(int), CU.FIT_PARAMS)
        WP.append(p); WC.append(cv); WX.append(c2); WN.append(nd)
    err = compare_params(P[ks], CV[ks], X2[ks], ND[ks], np.array(WP), np.array(WC), np.array(WX), np.array(WN))
    print("PU200 fit error (max, p99):", err)


def test_kernel_timing_and_candidate_counts(pu50):
    """The per-kernel timing brackets every launch of the four calls, and
    the doublet search's candidate counts cover every cell it accepted."""
    from paper_2008_13461_gb300 import _lib as L
    cuts = CU.cuts_for("pu50-ttbar-like")
    pipe = make_pipeline(cuts)
    t = to_dev(pu50)
    args = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    res, bufs = pipe.run(*args)
    torch.cuda.synchronize()
    L.kernel_timing(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(3):
        pipe.launch(bufs, *args)
    ev[1].record()
    torch.cuda.synchronize()
    kt = L.kernel_timing_read()
    L.kernel_timing(False)
    for name in ("k_bin_count", "k_doublets", "k_fishbone_small", "k_connect", "k_dfs", "k_fit<3>"):
        assert kt[name][0] == 3, name
    assert sum(v[0] for v in kt.values()) == 3 * 23
    assert sum(v[1] for v in kt.values()) <= ev[0].elapsed_time(ev[1]) * 1.01
    st, c = pipe.counts(bufs, *args)
    assert st == L.PT_OK
    h = pipe._hits(*args)
    cand = L.doublet_candidates(bufs.ws.data_ptr(), bufs.ws.numel(), h, pipe._cfg(bufs.capacity),
                                torch.cuda.current_stream().cuda_stream)
    assert sum(cand) == c.n_doublet_candidates
    acc = np.bincount(res.cells["pair"].cpu().numpy(), minlength=len(cand))
    assert np.all(np.array(cand) >= acc) and c.n_doublet_candidates > c.n_cells

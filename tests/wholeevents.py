"""Oracle results of whole events, computed in background processes.

The whole-event parity tests compare one complete event of a large GPU
batch with the oracle's result on that event alone.  The oracle takes
minutes on a full pileup-200 event (its doublet search is quadratic in the
hits of an event), so the jobs start when pytest has collected those tests
(``start``, called from conftest) in a process pool started with ``spawn``
(safe whatever the main process has done with CUDA), and run while the
other tests use the GPU.  A job generates its event from the seeded
generator itself; nothing of the CUDA path is involved.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np

TEST_FILE = "test_gpu_whole_events.py"

# (workload, event) pairs compared whole: event 0 of the 64-event PU200
# batch, event 0 of the 256-event stress batch, all 32 PU50 events
JOBS = ([("pu200-batch64", 0), ("pu200-stress-batch256", 0)] +
        [("pu50-batch32", e) for e in range(32)])

_pool = None
_results = {}


def oracle_event(workload: str, event: int) -> dict:
    """The oracle's complete result (stages 1-4) on one event of a
    workload, with hit indices local to the event, and the seconds taken."""
    import oracle
    from synth import cuts as CU
    from synth import events as E
    from synth import geometry as G
    b = E.make_batch(workload, n_events=1, first=event)
    t = time.perf_counter()
    out = oracle.run(b, CU.cuts_for(workload), CU.FIT_PARAMS, G.module_layer_table(), [0] * 4 + [1] * 6)
    out["seconds"] = time.perf_counter() - t
    out["n_hits"] = int(b["x"].size)
    return out


def start(workers: int | None = None) -> None:
    """Submit every job to a spawn-started pool (idempotent); the longest
    jobs first."""
    global _pool
    if _pool is not None:
        return
    import oracle
    oracle.build()                      # once, before the workers load it
    n = workers or max(2, min(len(JOBS), (os.cpu_count() or 4) - 2))
    _pool = mp.get_context("spawn").Pool(n)
    for job in JOBS:
        _results[job] = _pool.apply_async(oracle_event, job)


def result(workload: str, event: int, timeout: float = 1800.0) -> dict:
    """The oracle's result of one job (starting the pool if the session did
    not)."""
    start()
    return _results[(workload, event)].get(timeout)


def stop() -> None:
    """End the pool without waiting for jobs still running."""
    global _pool
    if _pool is not None:
        _pool.terminate()
        _pool.join()
        _pool = None
        _results.clear()


# ------------------------------------------------------------ comparison
def _rows_sorted(rows: np.ndarray) -> np.ndarray:
    """Rows sorted lexicographically (first column most significant)."""
    if rows.shape[0] == 0:
        return rows
    return rows[np.lexsort(rows.T[::-1])]


def gpu_event(res, ev_off_host, e: int) -> dict:
    """The cells, edges, n-tuplets and tracks of event e of a batched GPU
    result, with hit indices local to the event (device-side selection,
    then host arrays)."""
    import torch
    a, b = int(ev_off_host[e]), int(ev_off_host[e + 1])
    order = res.hit_order.long()
    ci = order[res.cells["inner"].long()]
    co = order[res.cells["outer"].long()]
    cm = (ci >= a) & (ci < b)
    cells = torch.stack([ci[cm] - a, co[cm] - a, res.cells["pair"][cm].long()], 1).cpu().numpy()
    alive = res.cells["alive"][cm].cpu().numpy().astype(bool)
    src, dst = res.edges["src"].long(), res.edges["dst"].long()
    em = (ci[src] >= a) & (ci[src] < b)
    edges = torch.stack([ci[src][em] - a, co[src][em] - a, co[dst][em] - a,
                         ci[dst][em] - a], 1).cpu().numpy()
    n = res.tuples["n"].long()
    H = res.tuples["hits"].long()
    tm = (H[:, 0] >= a) & (H[:, 0] < b)
    k = torch.arange(H.shape[1], device=H.device)
    Ht = torch.where(k[None, :] < n[:, None], H - a, torch.full_like(H, -1))
    tuples = Ht[tm].cpu().numpy()
    talive = res.tuples["alive"][tm].cpu().numpy().astype(bool)
    tt = res.tracks["tuple"].long()
    km = tm[tt]
    return dict(cells=cells, cell_alive=alive, edges=edges, tuples=tuples, tuple_alive=talive,
                track_hits=Ht[tt[km]].cpu().numpy(),
                params=res.tracks["params"][km].double().cpu().numpy(),
                cov=res.tracks["cov"][km].double().cpu().numpy(),
                chi2=res.tracks["chi2"][km].double().cpu().numpy(),
                ndf=res.tracks["ndf"][km].cpu().numpy())


def oracle_rows(want: dict) -> dict:
    """The oracle's result in the form of gpu_event (local hit indices,
    n-tuplets padded with -1)."""
    C = want["cells"].astype(np.int64)
    E = want["edges"].astype(np.int64)
    nmax = want["tuple_hits"].shape[1]
    k = np.arange(nmax)
    T = np.where(k[None, :] < want["tuple_n"][:, None], want["tuple_hits"].astype(np.int64), -1)
    return dict(cells=C, cell_alive=want["cell_alive"].astype(bool),
                edges=np.stack([C[E[:, 0], 0], C[E[:, 0], 1], C[E[:, 1], 1], C[E[:, 1], 0]], 1) if len(E)
                else np.zeros((0, 4), np.int64),
                tuples=T, tuple_alive=want["tuple_alive"].astype(bool),
                track_hits=T[want["track_tuple"]], params=want["params"], cov=want["cov"], chi2=want["chi2"],
                ndf=want["ndf"])


def compare_event(got: dict, want: dict) -> dict:
    """Exact comparison of the sets (cells with pair and Fishbone flag, CA
    edges, n-tuplets with cleaning flag), then the fits of the same tracks
    within the fit tolerances.  Returns the counts, the per-parameter
    (max, p99) errors and the matched fit arrays (GPU params, cov, chi2,
    ndf, then the oracle's)."""
    from parity import compare_params
    w = oracle_rows(want)
    count = {}
    # cells: (inner, outer, pair) rows and the alive flag, sorted alike
    for name, flag in (("cells", "cell_alive"), ("tuples", "tuple_alive")):
        g = np.concatenate([got[name].astype(np.int64), got[flag][:, None].astype(np.int64)], 1)
        o = np.concatenate([w[name].astype(np.int64), w[flag][:, None].astype(np.int64)], 1)
        gs, os_ = _rows_sorted(g), _rows_sorted(o)
        assert gs.shape == os_.shape, f"{name}: {gs.shape[0]} on the GPU, {os_.shape[0]} in the oracle"
        assert len(np.unique(gs[:, :-1], axis=0)) == gs.shape[0], f"duplicate {name} on the GPU"
        bad = np.nonzero(np.any(gs != os_, 1))[0]
        assert bad.size == 0, f"{name} differ at {bad.size} rows, first GPU {gs[bad[0]]} oracle {os_[bad[0]]}"
        count[name] = int(gs.shape[0])
    ge, oe = _rows_sorted(got["edges"].astype(np.int64)), _rows_sorted(w["edges"])
    assert np.array_equal(got["edges"][:, 1], got["edges"][:, 3]), "edge cells do not share a hit"
    assert ge.shape == oe.shape and np.array_equal(ge, oe), \
        f"edges differ: {ge.shape[0]} on the GPU, {oe.shape[0]} in the oracle"
    # tracks: the same n-tuplets fitted, matched by their hit sequences
    gi = np.lexsort(got["track_hits"].T[::-1])
    wi = np.lexsort(w["track_hits"].T[::-1])
    assert np.array_equal(got["track_hits"][gi], w["track_hits"][wi]), "different n-tuplets were fitted"
    matched = (got["params"][gi], got["cov"][gi], got["chi2"][gi], got["ndf"][gi],
               w["params"][wi], w["cov"][wi], w["chi2"][wi], w["ndf"][wi])
    err = compare_params(*matched) if gi.size else {}
    return dict(cells=count["cells"], alive_cells=int(w["cell_alive"].sum()), edges=int(ge.shape[0]),
                tuples=count["tuples"], tracks=int(gi.size), fit_error=err, matched=matched)

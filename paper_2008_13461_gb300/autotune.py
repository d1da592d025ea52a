"""Autotuner for the speed knobs of ``pt_tuning``.

Tile counts (phi x z|r tiles per layer), lanes per outer hit and the
persistent grid size change how fast the kernels run, never what they
compute: every decision is exact and the search windows are supersets
whatever the tiles.  So the fastest setting on a representative batch can be
picked freely.  ``autotune`` times the four calls on the caller's batch for
one knob at a time around the current best (coordinate search), checks that
every candidate reproduces the counts of the first run, and returns the
fastest tuning.  ``coordinate_search`` is the search itself, independent of
the GPU.
"""
from __future__ import annotations

import statistics
from typing import Callable

import torch

SPACE = (
    ("n_t_bins", (24, 32, 48, 64)),
    ("n_phi_bins", (32, 48, 64, 96, 128, 192, 256)),
    ("doublet_lanes", (4, 8, 16)),
    ("blocks_per_sm", (8, 12, 16, 24, 32)),
)


def coordinate_search(evaluate: Callable[[dict], float], base: dict, space=SPACE, rounds: int = 2) -> tuple[dict, dict]:
    """Minimise evaluate(tuning) by varying one knob at a time around the
    best so far, for `rounds` passes over the knobs (stopping early when a
    pass changes nothing).  Each distinct tuning is evaluated once.  Returns
    (best tuning, {tuning as a sorted tuple: cost})."""
    seen: dict = {}

    def cost(t: dict) -> float:
        key = tuple(sorted(t.items()))
        if key not in seen:
            seen[key] = evaluate(dict(t))
        return seen[key]

    best = dict(base)
    best_cost = cost(best)
    for _ in range(rounds):
        changed = False
        for knob, values in space:
            for v in values:
                cand = dict(best, **{knob: v})
                c = cost(cand)
                if c < best_cost:
                    best, best_cost, changed = cand, c, True
        if not changed:
            break
    return best, seen


def autotune(pipe, x, y, z, r, module, ev_off, reps: int = 3, space=SPACE) -> tuple[dict, dict]:
    """Fastest tuning of `pipe` for this batch (device tensors), and the
    timings (ms per batch) of every tuning tried.  Raises if a tuning changes
    any count (which the exactness contract rules out)."""
    from .pipeline import Pipeline

    ref, bufs = pipe.run(x, y, z, r, module, ev_off)
    want = (ref.counts.n_cells, ref.counts.n_alive_cells, ref.counts.n_edges, ref.counts.n_tuples,
            ref.counts.n_tracks)
    capacity = dict(bufs.capacity)
    del bufs, ref

    def evaluate(tuning: dict) -> float:
        p = Pipeline.__new__(Pipeline)
        p.__dict__.update(pipe.__dict__)
        p.set_tuning(tuning)
        b = p.allocate(x.numel(), ev_off.numel() - 1, capacity)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        times = []
        for k in range(reps + 1):
            ev[0].record()
            p.launch(b, x, y, z, r, module, ev_off)
            ev[1].record()
            torch.cuda.synchronize()
            if k:
                times.append(ev[0].elapsed_time(ev[1]))
        st, c = p.counts(b, x, y, z, r, module, ev_off)
        got = (c.n_cells, c.n_alive_cells, c.n_edges, c.n_tuples, c.n_tracks)
        if got != want:
            raise RuntimeError(f"tuning {tuning} changed the results: {got} != {want}")
        del b
        return statistics.median(times)

    best, seen = coordinate_search(evaluate, dict(pipe.tuning), space)
    return best, {k: v for k, v in seen.items()}

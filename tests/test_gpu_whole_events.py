"""Whole-event parity at full size, taken from the batched runs (needs a
GB300).

Each test runs a complete batch through the four C-ABI calls on the GPU (one
launch per kernel over all events, per-event offsets) and compares whole
events of it with the oracle's result on that event alone, element by
element: every cell with its layer pair and Fishbone flag, every CA edge,
every n-tuplet with its cleaning flag, and the broken-line fit of every
track within the fit tolerances, with the error against the float64 oracle
printed per parameter (max and 99th percentile).  The oracle runs in
background processes started at collection (see wholeevents.py).

  * pu200-batch64: event 0 of the 64-event pileup-200 batch;
  * pu200-stress-batch256: event 0 of the 256-event stress batch (pT down
    to 0.3 GeV, 5% noise, 10% inefficiency), where the exact fallbacks of
    the predicates fire most;
  * pu50-batch32: all 32 events of the pileup-50 batch.
"""
import numpy as np
import pytest

from synth import cuts as CU
from synth import events as E

import wholeevents as W
from parity import compare_params, gpu_run

pytestmark = pytest.mark.gpu


def _batch_run(workload, cells_per_hit=96):
    b = E.make_batch(workload, workers=8)
    n = int(b["x"].size)
    cap = dict(cells=cells_per_hit * n, edges=12 * n, tuples=12 * n, tracks=12 * n)
    return b, gpu_run(b, CU.cuts_for(workload), capacity=cap)


def _report(label, out):
    print(f"{label}: {out['cells']} cells ({out['alive_cells']} alive), {out['edges']} edges, "
          f"{out['tuples']} n-tuplets, {out['tracks']} tracks identical to the oracle")
    for k, (mx, p99) in out["fit_error"].items():
        print(f"  {k:>12}: max {mx:.3e}  p99 {p99:.3e}")


def test_pu200_event0_of_the_64_event_batch():
    b, res = _batch_run("pu200-batch64")
    assert len(b["ev_off"]) == 65
    want = W.result("pu200-batch64", 0)
    out = W.compare_event(W.gpu_event(res, b["ev_off"], 0), want)
    _report(f"pu200-batch64 event 0 ({want['n_hits']} hits, oracle {want['seconds']:.0f} s)", out)
    assert out["cells"] > 10 ** 6 and out["tracks"] > 10 ** 4


def test_stress_event0_of_the_256_event_batch():
    b, res = _batch_run("pu200-stress-batch256", cells_per_hit=128)
    assert len(b["ev_off"]) == 257
    assert res.counts.n_exact_fallbacks > 0          # the exact path is exercised in this batch
    want = W.result("pu200-stress-batch256", 0)
    out = W.compare_event(W.gpu_event(res, b["ev_off"], 0), want)
    _report(f"pu200-stress-batch256 event 0 ({want['n_hits']} hits, oracle {want['seconds']:.0f} s; "
            f"{res.counts.n_exact_fallbacks} exact fallbacks in the batch)", out)
    assert out["cells"] > 10 ** 6 and out["tracks"] > 10 ** 4


def test_every_event_of_the_pu50_batch():
    b, res = _batch_run("pu50-batch32")
    ne = len(b["ev_off"]) - 1
    assert ne == 32
    matched, totals = [], dict(cells=0, edges=0, tuples=0, tracks=0)
    for e in range(ne):
        out = W.compare_event(W.gpu_event(res, b["ev_off"], e), W.result("pu50-batch32", e))
        matched.append(out["matched"])
        for k in totals:
            totals[k] += out[k]
    # every event's sets are in the batch: nothing else was produced
    assert totals["cells"] == res.counts.n_cells and totals["tracks"] == res.counts.n_tracks
    err = compare_params(*(np.concatenate([m[i] for m in matched]) for i in range(8)))
    _report("pu50-batch32, all 32 events", dict(totals, alive_cells=res.counts.n_alive_cells, fit_error=err))

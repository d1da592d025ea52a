"""Host logic of Pipeline.run without a GPU: the capacity retry grows the
buffers to what the counters asked for, and every other device status
raises (the library's calls are replaced by stand-ins)."""
import pytest
import torch

from paper_2008_13461_gb300 import _lib as L
from paper_2008_13461_gb300.pipeline import Pipeline
from synth import cuts as CU
from synth import geometry as G


def _pipe(monkeypatch, statuses, need, flags=None):
    pipe = Pipeline(G.layers(), G.module_layer_table(), CU.cuts_for("pu50-ttbar-like"), CU.FIT_PARAMS,
                    device="cpu")
    allocated, seq = [], iter(statuses)
    fl = iter(flags or [0] * len(statuses))
    needs = iter(need) if isinstance(need, list) else None

    class Bufs:
        def __init__(self, cap):
            self.capacity = dict(cap)

    def allocate(n_hits, n_events, capacity=None):
        cap = dict(capacity or pipe.default_capacity(n_hits))
        allocated.append(cap)
        return Bufs(cap)

    def counts(bufs, *hits, stream=None):
        c = L.Counts()
        n = next(needs) if needs else need
        c.n_cells, c.n_edges, c.n_tuples, c.n_tracks = n["cells"], n["edges"], n["tuples"], n["tracks"]
        c.flags = next(fl)
        return next(seq), c

    monkeypatch.setattr(pipe, "allocate", allocate)
    monkeypatch.setattr(pipe, "launch", lambda *a, **k: None)
    monkeypatch.setattr(pipe, "counts", counts)
    monkeypatch.setattr(pipe, "result", lambda bufs, c, *hits: ("result", bufs.capacity))
    hits = [torch.zeros(100) for _ in range(4)] + [torch.zeros(100, dtype=torch.int32),
                                                   torch.tensor([0, 100], dtype=torch.int32)]
    return pipe, hits, allocated


def test_capacity_overflow_grows_the_buffers_and_retries(monkeypatch):
    need = dict(cells=10 ** 6, edges=10, tuples=20, tracks=30)
    pipe, hits, allocated = _pipe(monkeypatch, [L.PT_ERR_CAPACITY, L.PT_OK], need)
    (tag, cap), _ = pipe.run(*hits)
    assert tag == "result" and len(allocated) == 2
    first = allocated[0]
    assert cap["cells"] == int(10 ** 6 * 1.25) + 1024                  # grown to the count asked for
    assert all(cap[k] == first[k] for k in ("edges", "tuples", "tracks"))   # never shrunk


def test_other_device_errors_raise(monkeypatch):
    pipe, hits, _ = _pipe(monkeypatch, [L.PT_ERR_INPUT], dict(cells=0, edges=0, tuples=0, tracks=0))
    with pytest.raises(L.PtError):
        pipe.run(*hits)


def test_retries_are_bounded(monkeypatch):
    pipe, hits, allocated = _pipe(monkeypatch, [L.PT_ERR_CAPACITY] * 10, dict(cells=5, edges=5, tuples=5, tracks=5))
    with pytest.raises(L.PtError):
        pipe.run(*hits, max_retries=2)
    assert len(allocated) == 3            # the first buffers and one growth per retry, none after the last


def test_a_four_stage_cascade_fits_in_the_default_retries(monkeypatch):
    # each stage overflows in turn; the stages after an overflowing one
    # report partial counts (here 0) and still grow with it
    base = Pipeline.default_capacity(100)
    seq = [dict(base, cells=2 * base["cells"], edges=0, tuples=0, tracks=0),
           dict(base, cells=10, edges=3 * base["edges"], tuples=0, tracks=0),
           dict(base, cells=10, edges=10, tuples=5 * base["tuples"], tracks=0),
           dict(base, cells=10, edges=10, tuples=10, tracks=7 * base["tracks"]),
           dict(cells=1, edges=1, tuples=1, tracks=1)]
    flags = [L.FLAG_CELLS, L.FLAG_EDGES, L.FLAG_TUPLES, L.FLAG_TRACKS, 0]
    pipe, hits, allocated = _pipe(monkeypatch, [L.PT_ERR_CAPACITY] * 4 + [L.PT_OK], seq, flags)
    (tag, cap), _ = pipe.run(*hits)
    assert tag == "result" and len(allocated) == 5
    a = allocated
    assert a[1]["cells"] == int(2 * base["cells"] * 1.25) + 1024
    # the downstream stages grew by the cells' ratio although their counts were 0
    for k in ("edges", "tuples", "tracks"):
        assert a[1][k] >= int(base[k] * a[1]["cells"] / base["cells"])
    assert a[2]["edges"] >= int(3 * base["edges"] * 1.25) and a[4]["tracks"] >= int(7 * base["tracks"] * 1.25)


def test_grown_capacities_stay_int32():
    from paper_2008_13461_gb300.pipeline import MAX_CAPACITY, grow_capacity
    cap = dict(cells=2 ** 30, edges=2 ** 30, tuples=10, tracks=10)
    out = grow_capacity(cap, dict(cells=2 ** 31 - 100, edges=5, tuples=5, tracks=5), L.FLAG_CELLS)
    assert out["cells"] == MAX_CAPACITY and max(out.values()) <= MAX_CAPACITY
    with pytest.raises(L.PtError):
        grow_capacity(cap, dict(cells=2 ** 31, edges=5, tuples=5, tracks=5), L.FLAG_CELLS)


def test_find_vertices_checks_its_tensors_before_any_call():
    from paper_2008_13461_gb300.pipeline import find_vertices
    k = 8
    good = dict(ev=torch.zeros(k, dtype=torch.int32), z0=torch.zeros(k), ez0=torch.ones(k), pt=torch.ones(k),
                nhits=torch.full((k,), 4, dtype=torch.uint8), keep=torch.ones(k, dtype=torch.uint8))
    order = ("ev", "z0", "ez0", "pt", "nhits", "keep")
    for name, bad in (("z0", torch.zeros(k, dtype=torch.float64)),       # wrong dtype
                      ("ev", torch.zeros(2 * k, dtype=torch.int32)[::2]),  # not contiguous
                      ("pt", torch.ones(k + 1)),                           # wrong length
                      ("keep", torch.ones(k, dtype=torch.bool))):          # keep must be uint8
        args = dict(good, **{name: bad})
        with pytest.raises(ValueError):
            find_vertices(*(args[n] for n in order), 1)

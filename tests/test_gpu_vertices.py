"""Pixel vertices on the GPU (Sec. 3.6) against the oracle.

Both sides read the same float32 track summaries (seeded, from
synth.vertices) and take every cut decision in float32 as written; the
vertex sums are float64 on both sides, in different orders, so z, ez, chi2
and sum pT^2 agree to float32 rounding (compared within 1e-5 relative, 1e-6
absolute) and counts, ndf and the track-to-vertex map exactly."""
import numpy as np
import pytest
import torch

from oracle import postfit
from synth import cuts as CU
from synth import events as E
from synth.vertices import vertex_tracks

from parity import make_pipeline, oracle_run, to_dev

pytestmark = pytest.mark.gpu

CUTS = dict(pt_min=0.5, min_hits=4, ez0_max=0.05, dz_cut=0.07, chi2_max=9.0, split_chi2=9.0, min_tracks=2)
KEYS = ("ev", "z0", "ez0", "pt", "nhits", "keep")


def _gpu(d, n_events, cuts=CUTS, max_vertices=256, keep=True):
    from paper_2008_13461_gb300.pipeline import find_vertices
    t = {k: torch.as_tensor(np.ascontiguousarray(d[k])).to("cuda:0") for k in KEYS}
    v = find_vertices(t["ev"], t["z0"], t["ez0"], t["pt"], t["nhits"], t["keep"] if keep else None, n_events,
                      cuts, max_vertices)
    torch.cuda.synchronize()
    return {k: x.cpu().numpy() for k, x in v.items() if k != "scratch"}


def _compare(g, want, vidx, n_events, max_vertices=256):
    assert int(g["status"][0]) == 0
    for e in range(n_events):
        wv = want[e]
        assert int(g["n"][e]) == len(wv), f"event {e}: {int(g['n'][e])} vertices, oracle {len(wv)}"
        for k, v in enumerate(wv):
            assert int(g["ntracks"][e, k]) == len(v["tracks"]) and int(g["ndf"][e, k]) == v["ndf"]
            for name in ("z", "ez", "chi2", "sumpt2"):
                assert abs(float(g[name][e, k]) - v[name]) <= 1e-6 + 1e-5 * abs(v[name]), (e, k, name)
    assert np.array_equal(g["track_vertex"].astype(np.int64), vidx)


@pytest.mark.parametrize("seed,n_events,pileup", [(1, 4, 20.0), (2, 3, 60.0), (3, 1, 1.0)])
def test_vertices_match_the_oracle(seed, n_events, pileup):
    d = vertex_tracks(seed, n_events, pileup=pileup)
    want, vidx = postfit.find_vertices(d["ev"], d["z0"], d["ez0"], d["pt"], d["nhits"], d["keep"], n_events, CUTS)
    assert sum(len(w) for w in want) > 0
    _compare(_gpu(d, n_events), want, vidx, n_events)


def test_vertices_full_size_pileup_200_batch_64():
    """The benchmark's vertex workload size: 64 events of pileup 200."""
    d = vertex_tracks(11, 64, pileup=200.0)
    g = _gpu(d, 64)
    sample = [0, 17, 63]                                  # oracle on a sample of events
    for e in sample:
        sel = d["ev"] == e
        idx = np.nonzero(sel)[0]
        sub = {k: d[k][sel] for k in KEYS}
        sub["ev"] = np.zeros(len(idx), np.int32)
        want, vidx = postfit.find_vertices(sub["ev"], sub["z0"], sub["ez0"], sub["pt"], sub["nhits"], sub["keep"], 1,
                                           CUTS)
        gs = {k: (v[e:e + 1] if k in ("n", "z", "ez", "chi2", "sumpt2", "ndf", "ntracks") else v)
              for k, v in g.items()}
        gs["track_vertex"] = g["track_vertex"][idx]
        _compare(gs, want, vidx, 1)
    # every event: the vertices partition their tracks, sorted by sum pT^2
    tv = g["track_vertex"]
    for e in range(64):
        n = int(g["n"][e])
        assert 50 < n <= 256
        sp = g["sumpt2"][e, :n]
        assert np.all(sp[:-1] >= sp[1:])
        cnt = np.bincount(tv[(d["ev"] == e) & (tv >= 0)], minlength=n)
        assert np.array_equal(cnt, g["ntracks"][e, :n])


def test_vertices_edge_cases():
    base = vertex_tracks(4, 2, pileup=10.0)
    # no tracks at all
    empty = {k: base[k][:0] for k in KEYS}
    g = _gpu(empty, 3)
    assert np.array_equal(g["n"], [0, 0, 0]) and int(g["status"][0]) == 0
    # keep = NULL means every track is kept
    d = dict(base)
    d["keep"] = np.ones_like(base["keep"])
    want, vidx = postfit.find_vertices(d["ev"], d["z0"], d["ez0"], d["pt"], d["nhits"], None, 2, CUTS)
    _compare(_gpu(base, 2, keep=False), want, vidx, 2)
    # exact ties in z0 and in errors, one dense cluster that needs a split
    n = 300
    rng = np.random.default_rng(5)
    z = np.where(rng.random(n) < 0.5, -0.02, 0.02).astype(np.float32)
    z[::7] = np.float32(0.0)
    t = dict(ev=np.zeros(n, np.int32), z0=z, ez0=np.full(n, 0.004, np.float32),
             pt=np.round(rng.uniform(0.6, 5.0, n), 1).astype(np.float32), nhits=np.full(n, 4, np.uint8),
             keep=np.ones(n, np.uint8))
    cuts = dict(CUTS, dz_cut=0.1, chi2_max=200.0)
    want, vidx = postfit.find_vertices(t["ev"], t["z0"], t["ez0"], t["pt"], t["nhits"], t["keep"], 1, cuts)
    assert len(want[0]) == 2                              # the split happened
    _compare(_gpu(t, 1, cuts), want, vidx, 1)
    # fewer output slots than vertices: the first max_vertices are reported
    d = vertex_tracks(6, 1, pileup=80.0)
    want, vidx = postfit.find_vertices(d["ev"], d["z0"], d["ez0"], d["pt"], d["nhits"], d["keep"], 1, CUTS)
    m = 5
    g = _gpu(d, 1, max_vertices=m)
    assert int(g["status"][0]) & 2 and int(g["n"][0]) == m
    for k in range(m):
        assert int(g["ntracks"][0, k]) == len(want[0][k]["tracks"])
    assert np.array_equal(g["track_vertex"].astype(np.int64), np.where(vidx < m, vidx, -1))


def test_track_summary_of_the_pipeline_tracks_matches_the_oracle():
    b = E.make_batch("pu50-batch32", n_events=2)                       # two pileup-50 events
    cuts = CU.cuts_for("pu50-batch32")
    want = oracle_run(b, cuts)
    pipe = make_pipeline(cuts)
    t = to_dev(b)
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    sm = pipe.track_summary(bufs, res.counts, t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    torch.cuda.synchronize()
    th = want["tuple_hits"][want["track_tuple"]]
    ws = postfit.track_summary(want["params"], want["cov"], want["tuple_n"][want["track_tuple"]], th[:, 0],
                               b["ev_off"], CU.FIT_PARAMS["bz"])
    n = res.tuples["n"].cpu().numpy()
    H = res.tuples["hits"].cpu().numpy()
    tt = res.tracks["tuple"].cpu().numpy()
    gmap = {tuple(int(v) for v in H[t_, :n[t_]]): k for k, t_ in enumerate(tt)}
    wk = [tuple(int(v) for v in th[k, :want["tuple_n"][want["track_tuple"][k]]]) for k in range(len(th))]
    gi = np.array([gmap[k] for k in wk])
    g = {k: v.cpu().numpy()[gi] for k, v in sm.items()}
    assert np.array_equal(g["ev"], ws["ev"]) and np.array_equal(g["nhits"], ws["nhits"])
    assert len(set(g["ev"].tolist())) == 2
    assert np.all(np.abs(g["z0"] - ws["z0"]) <= 1e-5 * np.maximum(1.0, np.abs(ws["z0"])))
    assert np.all(np.abs(g["pt"] - ws["pt"]) <= 1e-4 * ws["pt"])            # as kappa
    assert np.all(np.abs(g["ez0"] - ws["ez0"]) <= 5e-4 * ws["ez0"])         # half the covariance tolerance


def test_vertices_of_the_pipeline_tracks():
    """Sec. 3.5 + 3.6 on the fitted tracks of pileup events: every vertex's
    z is the weighted mean of the tracks assigned to it."""
    b = E.make_batch("pu50-batch32", n_events=2)
    pipe = make_pipeline(CU.cuts_for("pu50-batch32"))
    t = to_dev(b)
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    v, sm = pipe.find_vertices(bufs, res.counts, t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    torch.cuda.synchronize()
    assert int(v["status"][0]) == 0
    tv = v["track_vertex"].cpu().numpy()
    ev = sm["ev"].cpu().numpy()
    z0 = sm["z0"].cpu().numpy().astype(np.float64)
    ez = sm["ez0"].cpu().numpy().astype(np.float64)
    nv = v["n"].cpu().numpy()
    assert nv.sum() > 0
    for e in range(len(nv)):
        for k in range(int(nv[e])):
            m = (ev == e) & (tv == k)
            w = 1.0 / ez[m] ** 2
            assert m.sum() == int(v["ntracks"][e, k])
            assert abs(float(v["z"][e, k]) - np.sum(w * z0[m]) / np.sum(w)) <= 1e-5


def test_vertices_of_the_pipeline_tracks_match_the_oracle():
    """End to end on four pileup-50 events: the four calls, the ambiguity
    resolution, the track summaries and the vertex finder on the GPU; the
    oracle's vertex finder on the same summaries and keep flags gives the
    same vertices (counts, tracks, ndf and the track map exactly; z, ez,
    chi2 and sum pT^2 to float32 rounding)."""
    b = E.make_batch("pu50-batch32", n_events=4)
    pipe = make_pipeline(CU.cuts_for("pu50-batch32"))
    t = to_dev(b)
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    v, sm = pipe.find_vertices(bufs, res.counts, t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    torch.cuda.synchronize()
    g = {k: x.cpu().numpy() for k, x in v.items() if k != "scratch"}
    d = {k: sm[k].cpu().numpy() for k in KEYS}
    assert d["keep"].sum() < len(d["keep"])                  # the ambiguity resolution dropped tracks
    want, vidx = postfit.find_vertices(d["ev"], d["z0"], d["ez0"], d["pt"], d["nhits"], d["keep"], 4, CUTS)
    assert all(len(w) > 10 for w in want)
    _compare(g, want, vidx, 4)


def test_vertices_do_not_depend_on_the_order_of_the_tracks():
    d = vertex_tracks(10, 4, pileup=40.0)
    assert len(np.unique(d["z0"])) == len(d["z0"])          # distinct z0: no tie left to the index
    g1 = _gpu(d, 4)
    perm = np.random.default_rng(2).permutation(len(d["z0"]))
    g2 = _gpu({k: d[k][perm] for k in KEYS}, 4)
    assert np.array_equal(g1["n"], g2["n"])
    assert np.array_equal(g1["track_vertex"][perm], g2["track_vertex"])
    assert np.array_equal(g1["ntracks"], g2["ntracks"])
    assert np.allclose(g1["z"], g2["z"], rtol=1e-6, atol=1e-6)


def test_an_event_beyond_the_track_limit_is_reported_and_skipped():
    from paper_2008_13461_gb300 import _lib as L
    n0 = L.PT_VTX_MAX_TRACKS + 600
    rng = np.random.default_rng(12)
    big = dict(ev=np.zeros(n0, np.int32), z0=rng.uniform(-10, 10, n0).astype(np.float32),
               ez0=np.full(n0, 0.01, np.float32), pt=np.full(n0, 1.0, np.float32),
               nhits=np.full(n0, 4, np.uint8), keep=np.ones(n0, np.uint8))
    small = vertex_tracks(13, 1, pileup=5.0)
    small["ev"] = np.ones_like(small["ev"])
    d = {k: np.concatenate([big[k], small[k]]) for k in KEYS}
    g = _gpu(d, 2)
    assert int(g["status"][0]) & L.PT_VTX_EVENT_TOO_LARGE
    assert int(g["n"][0]) == 0 and np.all(g["track_vertex"][:n0] == -1)
    want, vidx = postfit.find_vertices(*(small[k] for k in KEYS), 2, CUTS)   # event 1 alone
    assert int(g["n"][1]) == len(want[1]) > 0
    assert np.array_equal(g["track_vertex"][n0:].astype(np.int64), vidx)

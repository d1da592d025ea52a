"""Synchronous argument checks of the four stage calls (include/pt.h: argument
errors are returned synchronously as PT_ERR_INVALID_ARG).

Every case starts from a valid configuration, hits and workspace size and
breaks exactly one thing; the call must refuse it before any device work.
Pointers are fake addresses that are never dereferenced when the checks
work, so the test only runs where no GPU is visible: there a check that let
a bad argument through would reach the CUDA runtime and come back as
PT_ERR_CUDA (no device), not touch memory."""
import ctypes as C

import pytest
import torch

from paper_2008_13461_gb300 import _lib as L
from paper_2008_13461_gb300.pipeline import Pipeline
from synth import cuts as CU
from synth import geometry as G

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="fake device pointers: host-only test")

WS = 0x10000000          # 256-byte aligned fake device address
PTR = 0x20000000         # fake array address


def _valid():
    pipe = Pipeline(G.layers(), G.module_layer_table(), CU.cuts_for("pu50-ttbar-like"), CU.FIT_PARAMS,
                    device="cpu")
    cfg = pipe._cfg(dict(cells=4096, edges=1024, tuples=1024, tracks=1024))
    hits = L.Hits(PTR, PTR, PTR, PTR, PTR, PTR, 5000, 2)
    nbytes = L.workspace_size(hits, cfg)
    assert nbytes > 0
    return cfg, hits, nbytes


def _build(cfg, hits, nbytes, ws=WS, cells=None):
    if cells is None:
        cells = L.Cells(PTR, PTR, PTR, PTR)
    return L.lib().pt_build_doublets(ws, nbytes, C.byref(hits), C.byref(cfg), C.byref(cells), None)


def _config_cases():
    """(name, mutate(cfg, hits) -> (cfg, hits)) pairs, each breaking one thing."""

    def tuning(**kw):
        def f(cfg, hits):
            for k, v in kw.items():
                setattr(cfg.tuning, k, v)
            return cfg, hits
        return f

    def pair(k, **kw):
        def f(cfg, hits):
            for a, v in kw.items():
                setattr(cfg.cuts.pair[k], a, v)
            return cfg, hits
        return f

    def cycle(cfg, hits):
        p = cfg.cuts.pair[0]
        n = cfg.cuts.n_pairs
        cfg.cuts.pair[n] = L.PairCuts(p.outer, p.inner, p.tan2_dphi, p.zlo, p.zhi, p.zmax, p.k_pt)
        cfg.cuts.n_pairs = n + 1
        return cfg, hits

    def duplicate(cfg, hits):
        n = cfg.cuts.n_pairs
        cfg.cuts.pair[n] = cfg.cuts.pair[0]
        cfg.cuts.n_pairs = n + 1
        return cfg, hits

    def setf(path, v):
        def f(cfg, hits):
            obj = cfg
            *head, last = path.split(".")
            for a in head:
                obj = getattr(obj, a)
            setattr(obj, last, v)
            return cfg, hits
        return f

    def region(i, **kw):
        def f(cfg, hits):
            for a, v in kw.items():
                setattr(cfg.cuts.region[i], a, v)
            return cfg, hits
        return f

    def layer(i, **kw):
        def f(cfg, hits):
            for a, v in kw.items():
                setattr(cfg.geometry.layer[i], a, v)
            return cfg, hits
        return f

    def hit(**kw):
        def f(cfg, hits):
            for a, v in kw.items():
                setattr(hits, a, v)
            return cfg, hits
        return f

    return [
        ("phi tiles below 16", tuning(n_phi_bins=8)),
        ("phi tiles above 1024", tuning(n_phi_bins=2048)),
        ("z|r tiles 0", tuning(n_t_bins=0)),
        ("doublet lanes 6", tuning(doublet_lanes=6)),
        ("connect lanes 64", tuning(connect_lanes=64)),
        ("blocks per SM 33", tuning(blocks_per_sm=33)),
        ("PhiW constant 0", pair(0, tan2_dphi=0.0)),
        ("ZIP constant inf", pair(1, zmax=float("inf"))),
        ("PT constant above 2^40", pair(2, k_pt=2.0 ** 41)),
        ("ZW window reversed", pair(3, zlo=5.0, zhi=-5.0)),
        ("pair on one layer", pair(0, outer=0, inner=0)),
        ("layer index 10", pair(0, outer=10)),
        ("layer-pair cycle", cycle),
        ("duplicate pair", duplicate),
        ("no pairs", setf("cuts.n_pairs", 0)),
        ("33 pairs", setf("cuts.n_pairs", 33)),
        ("CA constant nan", region(0, tol_rz2=float("nan"))),
        ("CA constant below 2^-30", region(1, k_curv=2.0 ** -31)),
        ("Fishbone eps^2 1", setf("cuts.fishbone_eps2", 1.0)),
        ("min hits 2", setf("cuts.min_hits", 2)),
        ("min hits 9", setf("cuts.min_hits", 9)),
        ("sigma_z 0", setf("fit.sigma_z", 0.0)),
        ("bz negative", setf("fit.bz", -3.8)),
        ("solve_fp32 2", setf("fit.solve_fp32", 2)),
        ("no module table", setf("geometry.module_layer", None)),
        ("no modules", setf("geometry.n_modules", 0)),
        ("layer rmin >= rmax", layer(2, rmin=20.0, rmax=10.0)),
        ("layer kind 7", layer(4, kind=7)),
        ("capacity negative", setf("capacity.cells", -1)),
        ("capacity above 2^31 - 1", setf("capacity.edges", 2 ** 31)),
        ("no events", hit(n_events=0)),
        ("negative hits", hit(n_hits=-1)),
        ("more than 2^30 hits", hit(n_hits=(1 << 30) + 1)),
        ("no event offsets", hit(ev_off=None)),
        ("no x", hit(x=None)),
        ("no module ids", hit(module=None)),
        ("tile count above 2^31", hit(n_events=1 << 20)),
    ]


@pytest.mark.parametrize("name,mutate", _config_cases(), ids=[c[0] for c in _config_cases()])
def test_build_doublets_rejects(name, mutate):
    cfg, hits, nbytes = _valid()
    cfg, hits = mutate(cfg, hits)
    assert _build(cfg, hits, 1 << 40) == L.PT_ERR_INVALID_ARG, name


def test_workspace_pointer_alignment_and_size():
    cfg, hits, nbytes = _valid()
    assert _build(cfg, hits, nbytes, ws=None) == L.PT_ERR_INVALID_ARG
    assert _build(cfg, hits, nbytes, ws=WS + 16) == L.PT_ERR_INVALID_ARG
    assert _build(cfg, hits, nbytes - 1) == L.PT_ERR_INVALID_ARG


def test_output_arrays_are_checked_by_their_writer():
    cfg, hits, nbytes = _valid()
    assert _build(cfg, hits, nbytes, cells=L.Cells(PTR, None, PTR, PTR)) == L.PT_ERR_INVALID_ARG
    lib = L.lib()
    cells = L.Cells(PTR, PTR, PTR, PTR)
    assert lib.pt_connect_cells(WS, nbytes, C.byref(hits), C.byref(cfg), C.byref(cells),
                                C.byref(L.Edges(PTR, None)), None) == L.PT_ERR_INVALID_ARG
    assert lib.pt_find_ntuplets(WS, nbytes, C.byref(hits), C.byref(cfg), C.byref(cells), C.byref(L.Edges(PTR, PTR)),
                                C.byref(L.Tuples(PTR, PTR, None, PTR)), None) == L.PT_ERR_INVALID_ARG
    assert lib.pt_fit_tracks(WS, nbytes, C.byref(hits), C.byref(cfg), C.byref(L.Tuples(PTR, PTR, PTR, PTR)),
                             C.byref(L.Tracks(PTR, PTR, None, PTR, PTR)), None) == L.PT_ERR_INVALID_ARG
    assert lib.pt_fit_tracks_grad(WS, nbytes, C.byref(hits), C.byref(cfg), C.byref(L.Tuples(PTR, PTR, PTR, PTR)),
                                  C.byref(L.Tracks(PTR, PTR, PTR, PTR, PTR)), PTR, None, PTR, None, PTR,
                                  None) == L.PT_ERR_INVALID_ARG


def test_read_counts_and_hit_order_check_the_workspace():
    cfg, hits, nbytes = _valid()
    lib = L.lib()
    out = L.Counts()
    assert lib.pt_read_counts(None, nbytes, C.byref(hits), C.byref(cfg), C.byref(out), None) == L.PT_ERR_INVALID_ARG
    assert lib.pt_read_counts(WS, nbytes - 1, C.byref(hits), C.byref(cfg), C.byref(out), None) == \
        L.PT_ERR_INVALID_ARG
    assert lib.pt_hit_order(WS, nbytes - 1, C.byref(hits), C.byref(cfg)) is None
    assert lib.pt_hit_order(WS, nbytes, C.byref(hits), C.byref(cfg)) is not None      # host arithmetic only


def test_allocation_free_binning_checks_its_arguments_and_limits():
    cfg, hits, _ = _valid()
    lib = L.lib()
    g = cfg.geometry

    def call(h=hits, geo=g, nphi=96, nt=48, binned=PTR, order=PTR, off=PTR, flags=PTR):
        return lib.pt_bin_hits_noalloc(C.byref(h), C.byref(geo), nphi, nt, binned, order, off, flags, None)

    bad = L.PT_ERR_INVALID_ARG
    assert call(binned=None) == bad and call(order=None) == bad and call(off=None) == bad and call(flags=None) == bad
    assert call(binned=PTR + 8) == bad                                   # float4 rows: 16-byte aligned
    assert call(nphi=15) == bad and call(nphi=1025) == bad and call(nt=0) == bad and call(nt=65) == bad
    assert call(h=L.Hits(PTR, PTR, PTR, PTR, PTR, None, 5000, 2)) == bad
    assert call(h=L.Hits(PTR, None, PTR, PTR, PTR, PTR, 5000, 2)) == bad
    assert call(h=L.Hits(PTR, PTR, PTR, PTR, PTR, PTR, 5000, 0)) == bad
    geo = L.Geometry.from_buffer_copy(g)
    geo.layer[3].zmin, geo.layer[3].zmax = 5.0, -5.0
    assert call(geo=geo) == bad
    # beyond the fixed scratch: 2^20 hits, 2^22 tiles
    assert call(h=L.Hits(PTR, PTR, PTR, PTR, PTR, PTR, (1 << 20) + 1, 2)) == L.PT_ERR_TOO_LARGE
    assert call(h=L.Hits(PTR, PTR, PTR, PTR, PTR, PTR, 5000, 100), nphi=96, nt=48) == L.PT_ERR_TOO_LARGE

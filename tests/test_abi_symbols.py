"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/pt.h declares (no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-z_]+)\s*\(", src)))


def test_header_lists_the_stage_entry_points():
    names = declared_functions()
    for n in ("pt_build_doublets", "pt_connect_cells", "pt_find_ntuplets", "pt_fit_tracks"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2008_13461_gb300 import _lib, build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTS) == set(declared_functions())


def test_status_strings_without_gpu():
    from paper_2008_13461_gb300 import _lib
    L = _lib.lib()
    assert L.pt_status_string(0) == b"ok"
    assert L.pt_status_string(2) == b"output capacity exceeded"


def test_workspace_size_is_host_only():
    from paper_2008_13461_gb300 import _lib as L
    cfg = L.Config()
    cfg.tuning = L.Tuning(128, 16, 8, 8, 8)
    cfg.capacity = L.Capacity(1000, 100, 100, 100)
    h = L.Hits(None, None, None, None, None, None, 5000, 4)
    n = L.workspace_size(h, cfg)
    assert n > 4 * 128 * 16 * 10 * 4
    cfg.tuning = L.Tuning(7, 16, 8, 8, 8)
    assert L.workspace_size(h, cfg) == 0


def test_post_fit_entry_points_reject_bad_arguments_without_gpu():
    """Argument checks return before any device call."""
    import ctypes as C
    from paper_2008_13461_gb300 import _lib as L
    lib = L.lib()
    bad = 1   # PT_ERR_INVALID_ARG
    assert lib.pt_vertex_scratch_size(-1, 4) == 0
    assert lib.pt_vertex_scratch_size(1000, 4) >= 4 * 3 * 1000
    trk = L.VertexTracks()
    out = L.Vertices()
    cuts = L.VertexCuts(0.5, 0.05, 0.07, 9.0, 9.0, 4, 2)
    assert lib.pt_find_vertices(None, 10, 1, C.byref(cuts), 8, None, 0, C.byref(out), None) == bad
    assert lib.pt_find_vertices(C.byref(trk), 10, 1, C.byref(cuts), 0, None, 0, C.byref(out), None) == bad
    cuts.min_tracks = 0
    assert lib.pt_find_vertices(C.byref(trk), 10, 1, C.byref(cuts), 8, None, 0, C.byref(out), None) == bad
    h = L.Hits(None, None, None, None, None, None, 10, 0)
    assert lib.pt_track_summary(C.byref(h), C.byref(L.Tuples()), C.byref(L.Tracks()), 5, 3.8,
                                None, None, None, None, None, None) == bad
    assert lib.pt_resolve_ambiguities(C.byref(L.Tuples()), None, -1, None, None, 5, 0, 0, None, None, None) == bad
    assert lib.pt_align_hits(10, None, None, None, None, 0, None, None, None, None, None, None, None) == bad


def test_a_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No fallback: without the CUDA library (and without a way to build it)
    the binding raises instead of running anything else."""
    import pytest
    from paper_2008_13461_gb300 import _lib, build
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libpt_gb300.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.lib(build_if_missing=False)

    def no_compiler():
        raise RuntimeError("nvcc not found")

    monkeypatch.setattr(build, "_stale", lambda: True)
    monkeypatch.setattr(build, "nvcc", no_compiler)
    with pytest.raises(RuntimeError, match="nvcc"):
        _lib.lib()


def test_kernel_timing_controls_without_gpu():
    from paper_2008_13461_gb300 import _lib as L
    lib = L.lib()
    assert lib.pt_kernel_timing(2) == L.PT_ERR_INVALID_ARG
    L.kernel_timing(True)                 # nothing launched: no totals, no device call
    assert L.kernel_timing_read() == {}
    L.kernel_timing(False)

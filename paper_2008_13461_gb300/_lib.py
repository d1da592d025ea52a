"""ctypes binding of the C ABI in include/pt.h (argument marshalling only).

Every function here forwards to the CUDA library libpt_gb300.so built in-tree
by ``paper_2008_13461_gb300.build``; there is no fallback implementation.  If
the library cannot be loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

N_LAYERS = 10
MAX_PAIRS = 32
NMAX = 8

PT_OK, PT_ERR_INVALID_ARG, PT_ERR_CAPACITY, PT_ERR_INPUT, PT_ERR_CUDA, PT_ERR_TOO_LARGE = range(6)
FLAG_CELLS, FLAG_EDGES, FLAG_TUPLES, FLAG_TRACKS, FLAG_INPUT = 1, 2, 4, 8, 16


class Layer(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rmin", C.c_float), ("rmax", C.c_float),
                ("zmin", C.c_float), ("zmax", C.c_float)]


class Geometry(C.Structure):
    _fields_ = [("layer", Layer * N_LAYERS), ("module_layer", C.c_void_p), ("n_modules", C.c_int32)]


class PairCuts(C.Structure):
    _fields_ = [("inner", C.c_int32), ("outer", C.c_int32), ("tan2_dphi", C.c_float),
                ("zlo", C.c_float), ("zhi", C.c_float), ("zmax", C.c_float), ("k_pt", C.c_float)]


class CaCuts(C.Structure):
    _fields_ = [("tol_rz2", C.c_float), ("k_curv", C.c_float), ("rmax2", C.c_float), ("zmax", C.c_float)]


class Cuts(C.Structure):
    _fields_ = [("n_pairs", C.c_int32), ("pair", PairCuts * MAX_PAIRS), ("region", CaCuts * 2),
                ("fishbone_eps2", C.c_float), ("min_hits", C.c_int32)]


class FitParams(C.Structure):
    _fields_ = [("bz", C.c_float), ("sigma_rphi", C.c_float), ("sigma_z", C.c_float),
                ("sigma_r", C.c_float), ("x0_barrel", C.c_float), ("x0_disk", C.c_float),
                ("solve_fp32", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("n_phi_bins", C.c_int32), ("n_t_bins", C.c_int32), ("doublet_lanes", C.c_int32),
                ("connect_lanes", C.c_int32), ("blocks_per_sm", C.c_int32)]


class Capacity(C.Structure):
    _fields_ = [("cells", C.c_int64), ("edges", C.c_int64), ("tuples", C.c_int64), ("tracks", C.c_int64)]


class Config(C.Structure):
    _fields_ = [("geometry", Geometry), ("cuts", Cuts), ("fit", FitParams), ("tuning", Tuning),
                ("capacity", Capacity)]


class Hits(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("r", C.c_void_p),
                ("module", C.c_void_p), ("ev_off", C.c_void_p), ("n_hits", C.c_int32),
                ("n_events", C.c_int32)]


class Cells(C.Structure):
    _fields_ = [("inner", C.c_void_p), ("outer", C.c_void_p), ("pair", C.c_void_p), ("alive", C.c_void_p)]


class Edges(C.Structure):
    _fields_ = [("src", C.c_void_p), ("dst", C.c_void_p)]


class Tuples(C.Structure):
    _fields_ = [("hits", C.c_void_p), ("cells", C.c_void_p), ("n", C.c_void_p), ("alive", C.c_void_p)]


class Tracks(C.Structure):
    _fields_ = [("params", C.c_void_p), ("cov", C.c_void_p), ("chi2", C.c_void_p), ("ndf", C.c_void_p),
                ("tuple", C.c_void_p)]


class VertexTracks(C.Structure):
    _fields_ = [("ev", C.c_void_p), ("z0", C.c_void_p), ("ez0", C.c_void_p), ("pt", C.c_void_p),
                ("nhits", C.c_void_p), ("keep", C.c_void_p)]


class VertexCuts(C.Structure):
    _fields_ = [("pt_min", C.c_float), ("ez0_max", C.c_float), ("dz_cut", C.c_float), ("chi2_max", C.c_float),
                ("split_chi2", C.c_float), ("min_hits", C.c_int32), ("min_tracks", C.c_int32)]


class Vertices(C.Structure):
    _fields_ = [("n", C.c_void_p), ("z", C.c_void_p), ("ez", C.c_void_p), ("chi2", C.c_void_p),
                ("sumpt2", C.c_void_p), ("ndf", C.c_void_p), ("ntracks", C.c_void_p),
                ("track_vertex", C.c_void_p), ("status", C.c_void_p)]


PT_VTX_MAX_TRACKS = 16384
PT_VTX_MAX_VERTICES = 512
PT_VTX_EVENT_TOO_LARGE, PT_VTX_TOO_MANY, PT_VTX_INTERNAL = 1, 2, 4


class Counts(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_edges", C.c_int64), ("n_tuples", C.c_int64),
                ("n_tracks", C.c_int64), ("n_alive_cells", C.c_int64), ("n_alive_tuples", C.c_int64),
                ("n_exact_fallbacks", C.c_int64), ("n_doublet_candidates", C.c_int64), ("flags", C.c_uint32)]


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double)]


# every symbol declared in include/pt.h
EXPORTS = ("pt_workspace_size", "pt_build_doublets", "pt_connect_cells", "pt_find_ntuplets",
           "pt_fit_tracks", "pt_fit_tracks_grad", "pt_align_hits", "pt_align_hits_grad",
           "pt_resolve_ambiguities", "pt_track_summary", "pt_vertex_scratch_size", "pt_find_vertices",
           "pt_fma_probe", "pt_read_counts",
           "pt_hit_order", "pt_status_string", "pt_bin_hits_noalloc", "pt_doublet_candidates",
           "pt_kernel_timing", "pt_kernel_timing_read")

_lib = None


def lib(build_if_missing: bool = True):
    """Load libpt_gb300.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2008_13461_gb300.build.build()")
    L = C.CDLL(path)
    P = C.POINTER
    L.pt_workspace_size.restype = C.c_size_t
    L.pt_workspace_size.argtypes = [P(Hits), P(Config)]
    common = [C.c_void_p, C.c_size_t, P(Hits), P(Config)]
    L.pt_build_doublets.restype = C.c_int
    L.pt_build_doublets.argtypes = common + [P(Cells), C.c_void_p]
    L.pt_connect_cells.restype = C.c_int
    L.pt_connect_cells.argtypes = common + [P(Cells), P(Edges), C.c_void_p]
    L.pt_find_ntuplets.restype = C.c_int
    L.pt_find_ntuplets.argtypes = common + [P(Cells), P(Edges), P(Tuples), C.c_void_p]
    L.pt_fit_tracks.restype = C.c_int
    L.pt_fit_tracks.argtypes = common + [P(Tuples), P(Tracks), C.c_void_p]
    L.pt_fit_tracks_grad.restype = C.c_int
    L.pt_fit_tracks_grad.argtypes = common + [P(Tuples), P(Tracks)] + [C.c_void_p] * 6
    L.pt_resolve_ambiguities.restype = C.c_int
    L.pt_resolve_ambiguities.argtypes = [P(Tuples), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                         C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.pt_track_summary.restype = C.c_int
    L.pt_track_summary.argtypes = [P(Hits), P(Tuples), P(Tracks), C.c_int32, C.c_float] + [C.c_void_p] * 6
    L.pt_vertex_scratch_size.restype = C.c_size_t
    L.pt_vertex_scratch_size.argtypes = [C.c_int32, C.c_int32]
    L.pt_find_vertices.restype = C.c_int
    L.pt_find_vertices.argtypes = [P(VertexTracks), C.c_int32, C.c_int32, P(VertexCuts), C.c_int32, C.c_void_p,
                                   C.c_size_t, P(Vertices), C.c_void_p]
    L.pt_align_hits.restype = C.c_int
    L.pt_align_hits.argtypes = [C.c_int32] + [C.c_void_p] * 4 + [C.c_int32] + [C.c_void_p] * 7
    L.pt_align_hits_grad.restype = C.c_int
    L.pt_align_hits_grad.argtypes = [C.c_int32] + [C.c_void_p] * 4 + [C.c_int32] + [C.c_void_p] * 11
    L.pt_fma_probe.restype = C.c_int
    L.pt_fma_probe.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p]
    L.pt_read_counts.restype = C.c_int
    L.pt_read_counts.argtypes = common + [P(Counts), C.c_void_p]
    L.pt_hit_order.restype = C.c_void_p
    L.pt_hit_order.argtypes = common
    L.pt_status_string.restype = C.c_char_p
    L.pt_status_string.argtypes = [C.c_int]
    L.pt_bin_hits_noalloc.restype = C.c_int
    L.pt_bin_hits_noalloc.argtypes = [P(Hits), P(Geometry), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
    L.pt_doublet_candidates.restype = C.c_int
    L.pt_doublet_candidates.argtypes = common + [P(C.c_int64), C.c_void_p]
    L.pt_kernel_timing.restype = C.c_int
    L.pt_kernel_timing.argtypes = [C.c_int32]
    L.pt_kernel_timing_read.restype = C.c_int32
    L.pt_kernel_timing_read.argtypes = [P(KernelTime), C.c_int32]
    _lib = L
    return L


class PtError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().pt_status_string(status).decode()
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


def check(status: int, what: str) -> None:
    if status != PT_OK:
        raise PtError(status, what)


# thin wrappers with the ABI's names -------------------------------------
def workspace_size(hits: Hits, cfg: Config) -> int:
    return int(lib().pt_workspace_size(C.byref(hits), C.byref(cfg)))


def build_doublets(ws, ws_bytes, hits, cfg, cells, stream) -> None:
    check(lib().pt_build_doublets(ws, ws_bytes, C.byref(hits), C.byref(cfg), C.byref(cells), stream),
          "pt_build_doublets")


def connect_cells(ws, ws_bytes, hits, cfg, cells, edges, stream) -> None:
    check(lib().pt_connect_cells(ws, ws_bytes, C.byref(hits), C.byref(cfg), C.byref(cells), C.byref(edges),
                                 stream), "pt_connect_cells")


def find_ntuplets(ws, ws_bytes, hits, cfg, cells, edges, tuples, stream) -> None:
    check(lib().pt_find_ntuplets(ws, ws_bytes, C.byref(hits), C.byref(cfg), C.byref(cells), C.byref(edges),
                                 C.byref(tuples), stream), "pt_find_ntuplets")


def fit_tracks(ws, ws_bytes, hits, cfg, tuples, tracks, stream) -> None:
    check(lib().pt_fit_tracks(ws, ws_bytes, C.byref(hits), C.byref(cfg), C.byref(tuples), C.byref(tracks),
                              stream), "pt_fit_tracks")


def fit_tracks_grad(ws, ws_bytes, hits, cfg, tuples, tracks, grad_params, grad_chi2, gx, gy, gz, stream) -> None:
    check(lib().pt_fit_tracks_grad(ws, ws_bytes, C.byref(hits), C.byref(cfg), C.byref(tuples), C.byref(tracks),
                                   grad_params, grad_chi2, gx, gy, gz, stream), "pt_fit_tracks_grad")


def resolve_ambiguities(tuples, track_tuple, n_tracks, chi2, tip, tip_stride, n_cells, n_hits, scratch, keep,
                        stream) -> None:
    check(lib().pt_resolve_ambiguities(C.byref(tuples), track_tuple, n_tracks, chi2, tip, tip_stride, n_cells, n_hits,
                                       scratch, keep, stream), "pt_resolve_ambiguities")


def track_summary(hits, tuples, tracks, n_tracks, bz, ev, z0, ez0, pt, nhits, stream) -> None:
    check(lib().pt_track_summary(C.byref(hits), C.byref(tuples), C.byref(tracks), n_tracks, bz, ev, z0, ez0, pt,
                                 nhits, stream), "pt_track_summary")


def vertex_scratch_size(n_tracks: int, n_events: int) -> int:
    return int(lib().pt_vertex_scratch_size(n_tracks, n_events))


def find_vertices(tracks: VertexTracks, n_tracks, n_events, cuts: VertexCuts, max_vertices, scratch, scratch_bytes,
                  out: Vertices, stream) -> None:
    check(lib().pt_find_vertices(C.byref(tracks), n_tracks, n_events, C.byref(cuts), max_vertices, scratch,
                                 scratch_bytes, C.byref(out), stream), "pt_find_vertices")


def align_hits(n_hits, x, y, z, module, n_modules, centre, shift, rot, xo, yo, zo, stream) -> None:
    check(lib().pt_align_hits(n_hits, x, y, z, module, n_modules, centre, shift, rot, xo, yo, zo, stream),
          "pt_align_hits")


def align_hits_grad(n_hits, x, y, z, module, n_modules, centre, rot, gxo, gyo, gzo, gx, gy, gz, gshift, grot,
                    stream) -> None:
    check(lib().pt_align_hits_grad(n_hits, x, y, z, module, n_modules, centre, rot, gxo, gyo, gzo, gx, gy, gz,
                                   gshift, grot, stream), "pt_align_hits_grad")


def fma_probe(fp64: bool, iters: int, n_threads: int, out, stream) -> None:
    check(lib().pt_fma_probe(1 if fp64 else 0, iters, n_threads, out, stream), "pt_fma_probe")


def read_counts(ws, ws_bytes, hits, cfg, stream) -> tuple[int, Counts]:
    c = Counts()
    st = lib().pt_read_counts(ws, ws_bytes, C.byref(hits), C.byref(cfg), C.byref(c), stream)
    return st, c


def hit_order(ws, ws_bytes, hits, cfg) -> int:
    return lib().pt_hit_order(ws, ws_bytes, C.byref(hits), C.byref(cfg))


def bin_hits_noalloc(hits, geometry, n_phi_bins, n_t_bins, binned, hit_order_out, tile_off, flags, stream) -> None:
    """Allocation-free binning (see pt_bin_hits_noalloc in pt.h)."""
    check(lib().pt_bin_hits_noalloc(C.byref(hits), C.byref(geometry), n_phi_bins, n_t_bins, binned, hit_order_out,
                                    tile_off, flags, stream), "pt_bin_hits_noalloc")


def doublet_candidates(ws, ws_bytes, hits, cfg, stream) -> list[int]:
    """Candidate inner hits tested per layer pair by the last doublet search
    (pt_doublet_candidates; synchronises the stream)."""
    out = (C.c_int64 * MAX_PAIRS)()
    check(lib().pt_doublet_candidates(ws, ws_bytes, C.byref(hits), C.byref(cfg), out, stream),
          "pt_doublet_candidates")
    return list(out)


def kernel_timing(enable: bool) -> None:
    """Start (clearing the totals) or stop per-kernel timing (pt_kernel_timing)."""
    check(lib().pt_kernel_timing(1 if enable else 0), "pt_kernel_timing")


def kernel_timing_read() -> dict:
    """{kernel name: (launches, total ms)} of the launches timed so far."""
    n = lib().pt_kernel_timing_read(None, 0)
    buf = (KernelTime * max(1, n))()
    n = lib().pt_kernel_timing_read(buf, n)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(n)}

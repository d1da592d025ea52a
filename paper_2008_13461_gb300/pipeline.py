"""Batched seeding + fitting pipeline over the C ABI (include/pt.h).

PyTorch provides device memory and streams; every step runs in the CUDA
library.  A ``Pipeline`` holds the configuration (geometry, cuts, fit
constants, tuning); ``Buffers`` holds the workspace and the output tensors for
one problem size; ``launch`` enqueues the four stages on a stream without any
host synchronisation (so it can be captured in a CUDA graph); ``run`` adds
the count read-back and grows the buffers when a capacity was exceeded.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _lib as L

DEFAULT_TUNING = dict(n_phi_bins=96, n_t_bins=48, doublet_lanes=8, connect_lanes=8, blocks_per_sm=24)

# Vertex-finder cuts (Sec. 3.6 fixes pT > 0.5 GeV, >= 4 hits, the split at
# chi2/ndf > 9 and >= 2 tracks per vertex; the z0-error, dz and chi2
# compatibility thresholds are configurable there without values).
DEFAULT_VERTEX_CUTS = dict(pt_min=0.5, min_hits=4, ez0_max=0.05, dz_cut=0.07, chi2_max=9.0, split_chi2=9.0,
                           min_tracks=2)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


@dataclasses.dataclass
class Buffers:
    n_hits: int
    n_events: int
    capacity: dict
    ws: torch.Tensor
    cell_inner: torch.Tensor
    cell_outer: torch.Tensor
    cell_pair: torch.Tensor
    cell_alive: torch.Tensor
    edge_src: torch.Tensor
    edge_dst: torch.Tensor
    tup_hits: torch.Tensor
    tup_cells: torch.Tensor
    tup_n: torch.Tensor
    tup_alive: torch.Tensor
    trk_params: torch.Tensor
    trk_cov: torch.Tensor
    trk_chi2: torch.Tensor
    trk_ndf: torch.Tensor
    trk_tuple: torch.Tensor

    def structs(self):
        cells = L.Cells(_ptr(self.cell_inner), _ptr(self.cell_outer), _ptr(self.cell_pair), _ptr(self.cell_alive))
        edges = L.Edges(_ptr(self.edge_src), _ptr(self.edge_dst))
        tuples = L.Tuples(_ptr(self.tup_hits), _ptr(self.tup_cells), _ptr(self.tup_n), _ptr(self.tup_alive))
        tracks = L.Tracks(_ptr(self.trk_params), _ptr(self.trk_cov), _ptr(self.trk_chi2), _ptr(self.trk_ndf),
                          _ptr(self.trk_tuple))
        return cells, edges, tuples, tracks


def find_vertices(ev, z0, ez0, pt, nhits, keep, n_events: int, cuts: dict | None = None, max_vertices: int = 256,
                  stream: torch.cuda.Stream | None = None) -> dict:
    """Pixel vertices (Sec. 3.6) of per-track summaries (device tensors of
    n_tracks: ev int32, z0 / ez0 / pt float32, nhits uint8, keep uint8 or
    None), enqueued on `stream`.  Returns device tensors: n[E], z, ez, chi2,
    sumpt2, ndf, ntracks [E, max_vertices] (event e's first n[e] rows, in
    decreasing sum pT^2), track_vertex[n_tracks] and status[1] (PT_VTX_*)."""
    c = dict(DEFAULT_VERTEX_CUTS, **(cuts or {}))
    dev = z0.device
    k = z0.numel()
    for t, dt in ((ev, torch.int32), (z0, torch.float32), (ez0, torch.float32), (pt, torch.float32),
                  (nhits, torch.uint8)) + (((keep, torch.uint8),) if keep is not None else ()):
        if t.dtype != dt or not t.is_contiguous() or t.numel() != k:
            raise ValueError("find_vertices: per-track tensors must be contiguous, of equal length and dtypes "
                             "int32 / float32 x3 / uint8 / uint8")
    s = (stream or torch.cuda.current_stream(dev)).cuda_stream
    E, M = n_events, max_vertices
    out = dict(n=torch.empty(max(1, E), dtype=torch.int32, device=dev),
               z=torch.empty(max(1, E * M), dtype=torch.float32, device=dev),
               ez=torch.empty(max(1, E * M), dtype=torch.float32, device=dev),
               chi2=torch.empty(max(1, E * M), dtype=torch.float32, device=dev),
               sumpt2=torch.empty(max(1, E * M), dtype=torch.float32, device=dev),
               ndf=torch.empty(max(1, E * M), dtype=torch.int32, device=dev),
               ntracks=torch.empty(max(1, E * M), dtype=torch.int32, device=dev),
               track_vertex=torch.empty(max(1, k), dtype=torch.int32, device=dev),
               status=torch.zeros(1, dtype=torch.int32, device=dev))
    nbytes = L.vertex_scratch_size(k, E)
    scratch = torch.empty(2 * ((nbytes + 15) // 16), dtype=torch.int64, device=dev)     # 16-byte units
    assert scratch.numel() * scratch.element_size() >= nbytes
    trk = L.VertexTracks(ev.data_ptr(), z0.data_ptr(), ez0.data_ptr(), pt.data_ptr(), nhits.data_ptr(),
                         _ptr(keep))
    vc = L.VertexCuts(c["pt_min"], c["ez0_max"], c["dz_cut"], c["chi2_max"], c["split_chi2"], int(c["min_hits"]),
                      int(c["min_tracks"]))
    vo = L.Vertices(*(out[n].data_ptr() for n in ("n", "z", "ez", "chi2", "sumpt2", "ndf", "ntracks",
                                                    "track_vertex", "status")))
    L.find_vertices(trk, k, E, vc, M, scratch.data_ptr(), scratch.numel() * scratch.element_size(), vo, s)
    if stream is not None:
        scratch.record_stream(stream)
    out["scratch"] = scratch                                   # kept alive until the stream has used it
    res = {n: (t[:E * M].view(E, M) if n in ("z", "ez", "chi2", "sumpt2", "ndf", "ntracks") else t)
           for n, t in out.items()}
    res["n"] = out["n"][:E]
    res["track_vertex"] = out["track_vertex"][:k]
    return res


STAGES = ("cells", "edges", "tuples", "tracks")
_STAGE_FLAG = dict(cells=L.FLAG_CELLS, edges=L.FLAG_EDGES, tuples=L.FLAG_TUPLES, tracks=L.FLAG_TRACKS)
MAX_CAPACITY = 0x7FFFFFFF          # int32 indices


def grow_capacity(cap: dict, need: dict, flags: int) -> dict:
    """Capacities for the rerun after an overflow.  A stage that overflowed
    keeps counting, so its count is what it needs: it gets that plus a
    quarter and a margin.  The stages after it ran on incomplete inputs
    (or not at all), so their counts say nothing: each grows at least by the
    largest ratio an earlier stage grew by.  No capacity shrinks; none may
    pass 2^31 - 1 (int32 indices), which raises PT_ERR_CAPACITY."""
    out, ratio = {}, 1.0
    for k in STAGES:
        if need[k] > MAX_CAPACITY:
            raise L.PtError(L.PT_ERR_CAPACITY, f"pipeline: {need[k]} {k} needed, above the int32 limit")
        want = max(cap[k], int(need[k] * 1.25) + 1024)
        if ratio > 1.0:
            want = max(want, int(cap[k] * ratio) + 1024)
        want = min(want, MAX_CAPACITY)
        if flags & _STAGE_FLAG[k]:
            ratio = max(ratio, want / max(1, cap[k]))
        out[k] = want
    return out


@dataclasses.dataclass
class Result:
    counts: L.Counts
    cells: dict
    edges: dict
    tuples: dict
    tracks: dict
    hit_order: torch.Tensor


class Pipeline:
    def __init__(self, layers, module_layer, cuts: dict, fit: dict, tuning: dict | None = None,
                 device: str | torch.device = "cuda"):
        self.device = torch.device(device)
        self.module_layer = torch.as_tensor(module_layer, dtype=torch.int32).to(self.device).contiguous()
        self.tuning = dict(DEFAULT_TUNING, **(tuning or {}))
        cfg = L.Config()
        for i, ly in enumerate(layers):
            cfg.geometry.layer[i] = L.Layer(ly.kind, ly.rmin, ly.rmax, ly.zmin, ly.zmax)
        cfg.geometry.module_layer = self.module_layer.data_ptr()
        cfg.geometry.n_modules = self.module_layer.numel()
        cfg.cuts.n_pairs = len(cuts["pairs"])
        for i, p in enumerate(cuts["pairs"]):
            cfg.cuts.pair[i] = L.PairCuts(p["inner"], p["outer"], p["tan2_dphi"], p["zlo"], p["zhi"], p["zmax"],
                                          p["k_pt"])
        for i, rg in enumerate(cuts["region"]):
            cfg.cuts.region[i] = L.CaCuts(rg["tol_rz2"], rg["k_curv"], rg["rmax2"], rg["zmax"])
        cfg.cuts.fishbone_eps2 = cuts["fishbone_eps2"]
        cfg.cuts.min_hits = cuts["min_hits"]
        cfg.fit = L.FitParams(fit["bz"], fit["sigma_rphi"], fit["sigma_z"], fit["sigma_r"], fit["x0_barrel"],
                              fit["x0_disk"], int(fit.get("solve_fp32", 0)))
        self.cfg = cfg
        self.set_tuning(self.tuning)
        L.lib()

    def set_tuning(self, tuning: dict) -> None:
        """Replace the speed knobs (results do not depend on them); buffers
        must be allocated again, since the workspace size depends on the
        tile counts.  (A copy of the configuration is made, so a pipeline
        sharing this one's dictionary is not changed.)"""
        self.tuning = dict(DEFAULT_TUNING, **tuning)
        t = self.tuning
        self.cfg = L.Config.from_buffer_copy(self.cfg)
        self.cfg.tuning = L.Tuning(t["n_phi_bins"], t["n_t_bins"], t["doublet_lanes"], t["connect_lanes"],
                                   t["blocks_per_sm"])

    def autotune(self, x, y, z, r, module, ev_off, reps: int = 3) -> dict:
        """Pick the fastest tuning for this batch (see autotune.py), adopt it
        and return the timings of the tunings tried."""
        from .autotune import autotune
        best, timings = autotune(self, x, y, z, r, module, ev_off, reps=reps)
        self.set_tuning(best)
        return timings

    # ------------------------------------------------------------ buffers
    @staticmethod
    def default_capacity(n_hits: int) -> dict:
        n = max(n_hits, 64)
        return dict(cells=96 * n, edges=12 * n, tuples=12 * n, tracks=12 * n)

    def _hits(self, x, y, z, r, module, ev_off) -> L.Hits:
        return L.Hits(x.data_ptr(), y.data_ptr(), z.data_ptr(), r.data_ptr(), module.data_ptr(), ev_off.data_ptr(),
                      x.numel(), ev_off.numel() - 1)

    def _cfg(self, capacity: dict) -> L.Config:
        c = L.Config.from_buffer_copy(self.cfg)
        c.capacity = L.Capacity(capacity["cells"], capacity["edges"], capacity["tuples"], capacity["tracks"])
        return c

    def allocate(self, n_hits: int, n_events: int, capacity: dict | None = None) -> Buffers:
        cap = dict(capacity or self.default_capacity(n_hits))
        cfg = self._cfg(cap)
        h = L.Hits(None, None, None, None, None, None, n_hits, n_events)
        nbytes = L.workspace_size(h, cfg)
        if nbytes == 0:
            raise ValueError("invalid sizes or tuning for the workspace")
        d, i32, u8 = self.device, torch.int32, torch.uint8
        ws = torch.empty(nbytes, dtype=u8, device=d)
        nc, ne, nt, nk = (max(1, int(cap[k])) for k in ("cells", "edges", "tuples", "tracks"))
        return Buffers(
            n_hits, n_events, cap, ws,
            torch.empty(nc, dtype=i32, device=d), torch.empty(nc, dtype=i32, device=d),
            torch.empty(nc, dtype=u8, device=d), torch.empty(nc, dtype=u8, device=d),
            torch.empty(ne, dtype=i32, device=d), torch.empty(ne, dtype=i32, device=d),
            torch.empty(nt * L.NMAX, dtype=i32, device=d), torch.empty(nt * L.NMAX, dtype=i32, device=d),
            torch.empty(nt, dtype=u8, device=d), torch.empty(nt, dtype=u8, device=d),
            torch.empty(nk * 5, dtype=torch.float32, device=d), torch.empty(nk * 15, dtype=torch.float32, device=d),
            torch.empty(nk, dtype=torch.float32, device=d), torch.empty(nk, dtype=torch.int8, device=d),
            torch.empty(nk, dtype=i32, device=d))

    # ------------------------------------------------------------- launch
    def launch(self, bufs: Buffers, x, y, z, r, module, ev_off, stream: torch.cuda.Stream | None = None) -> None:
        """Enqueue the four stages on `stream` (default: current stream); no sync."""
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        h = self._hits(x, y, z, r, module, ev_off)
        cfg = self._cfg(bufs.capacity)
        cells, edges, tuples, tracks = bufs.structs()
        ws, nb = bufs.ws.data_ptr(), bufs.ws.numel()
        L.build_doublets(ws, nb, h, cfg, cells, s)
        L.connect_cells(ws, nb, h, cfg, cells, edges, s)
        L.find_ntuplets(ws, nb, h, cfg, cells, edges, tuples, s)
        L.fit_tracks(ws, nb, h, cfg, tuples, tracks, s)

    def counts(self, bufs: Buffers, x, y, z, r, module, ev_off, stream=None) -> tuple[int, L.Counts]:
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        return L.read_counts(bufs.ws.data_ptr(), bufs.ws.numel(), self._hits(x, y, z, r, module, ev_off),
                             self._cfg(bufs.capacity), s)

    def hit_order(self, bufs: Buffers, x, y, z, r, module, ev_off) -> torch.Tensor:
        """Binned position -> input hit index (a view into the workspace)."""
        h = self._hits(x, y, z, r, module, ev_off)
        ptr = L.hit_order(bufs.ws.data_ptr(), bufs.ws.numel(), h, self._cfg(bufs.capacity))
        off = ptr - bufs.ws.data_ptr()
        return bufs.ws[off:off + 4 * max(1, x.numel())].view(torch.int32)[:x.numel()]

    def result(self, bufs: Buffers, counts: L.Counts, x, y, z, r, module, ev_off) -> Result:
        nc, ne, nt, nk = counts.n_cells, counts.n_edges, counts.n_tuples, counts.n_tracks
        return Result(
            counts=counts,
            cells=dict(inner=bufs.cell_inner[:nc], outer=bufs.cell_outer[:nc], pair=bufs.cell_pair[:nc],
                       alive=bufs.cell_alive[:nc]),
            edges=dict(src=bufs.edge_src[:ne], dst=bufs.edge_dst[:ne]),
            tuples=dict(hits=bufs.tup_hits[:nt * L.NMAX].view(-1, L.NMAX), cells=bufs.tup_cells[:nt * L.NMAX]
                        .view(-1, L.NMAX), n=bufs.tup_n[:nt], alive=bufs.tup_alive[:nt]),
            tracks=dict(params=bufs.trk_params[:nk * 5].view(-1, 5), cov=bufs.trk_cov[:nk * 15].view(-1, 15),
                        chi2=bufs.trk_chi2[:nk], ndf=bufs.trk_ndf[:nk], tuple=bufs.trk_tuple[:nk]),
            hit_order=self.hit_order(bufs, x, y, z, r, module, ev_off),
        )

    def resolve_ambiguities(self, bufs: Buffers, counts: L.Counts, n_hits: int,
                            stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """Post-fit ambiguity resolution (Sec. 3.5) of the fitted tracks:
        uint8 keep[n_tracks] (1 = kept), enqueued on `stream`."""
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        k, nc = counts.n_tracks, counts.n_cells
        keep = torch.empty(max(1, k), dtype=torch.uint8, device=self.device)
        scratch = torch.empty(max(1, nc + n_hits), dtype=torch.int32, device=self.device)
        _, _, tuples, _ = bufs.structs()
        L.resolve_ambiguities(tuples, bufs.trk_tuple.data_ptr(), k, bufs.trk_chi2.data_ptr(),
                              bufs.trk_params.data_ptr() + 3 * 4, 5, nc, n_hits, scratch.data_ptr(), keep.data_ptr(), s)
        if stream is not None:
            scratch.record_stream(stream)      # freed here, used by `stream`: keep it until the work is done
        return keep[:k]

    def track_summary(self, bufs: Buffers, counts: L.Counts, x, y, z, r, module, ev_off,
                      stream: torch.cuda.Stream | None = None) -> dict:
        """Per-track inputs of the vertex finder for the fitted tracks:
        ev, z0, ez0, pt, nhits (device tensors of n_tracks)."""
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        k = counts.n_tracks
        o = dict(ev=torch.empty(max(1, k), dtype=torch.int32, device=self.device),
                 z0=torch.empty(max(1, k), dtype=torch.float32, device=self.device),
                 ez0=torch.empty(max(1, k), dtype=torch.float32, device=self.device),
                 pt=torch.empty(max(1, k), dtype=torch.float32, device=self.device),
                 nhits=torch.empty(max(1, k), dtype=torch.uint8, device=self.device))
        _, _, tuples, tracks = bufs.structs()
        L.track_summary(self._hits(x, y, z, r, module, ev_off), tuples, tracks, k, self.cfg.fit.bz,
                        o["ev"].data_ptr(), o["z0"].data_ptr(), o["ez0"].data_ptr(), o["pt"].data_ptr(),
                        o["nhits"].data_ptr(), s)
        return {n: t[:k] for n, t in o.items()}

    def find_vertices(self, bufs: Buffers, counts: L.Counts, x, y, z, r, module, ev_off, cuts: dict | None = None,
                      max_vertices: int = 256, stream: torch.cuda.Stream | None = None) -> tuple[dict, dict]:
        """Sec. 3.5 + 3.6 on the fitted tracks: ambiguity resolution, track
        summaries, vertices.  Returns (vertices, summaries incl. keep)."""
        keep = self.resolve_ambiguities(bufs, counts, x.numel(), stream)
        sm = self.track_summary(bufs, counts, x, y, z, r, module, ev_off, stream)
        sm["keep"] = keep
        v = find_vertices(sm["ev"], sm["z0"], sm["ez0"], sm["pt"], sm["nhits"], keep.contiguous(),
                          ev_off.numel() - 1, cuts, max_vertices, stream)
        return v, sm

    def run(self, x, y, z, r, module, ev_off, bufs: Buffers | None = None, max_retries: int = 4):
        """Run the batch and read the counts back; grow buffers on overflow
        (``grow_capacity``) and rerun, at most ``max_retries`` times (one per
        stage covers the worst cascade).  Returns (Result, Buffers)."""
        if bufs is None:
            bufs = self.allocate(x.numel(), ev_off.numel() - 1)
        for attempt in range(max_retries + 1):
            self.launch(bufs, x, y, z, r, module, ev_off)
            st, c = self.counts(bufs, x, y, z, r, module, ev_off)
            if st == L.PT_OK:
                return self.result(bufs, c, x, y, z, r, module, ev_off), bufs
            if st != L.PT_ERR_CAPACITY:
                raise L.PtError(st, f"pipeline (flags 0x{c.flags:x})")
            if attempt == max_retries:
                break
            need = dict(cells=c.n_cells, edges=c.n_edges, tuples=c.n_tuples, tracks=c.n_tracks)
            bufs = self.allocate(x.numel(), ev_off.numel() - 1, grow_capacity(bufs.capacity, need, c.flags))
        raise L.PtError(L.PT_ERR_CAPACITY, "pipeline: capacity still exceeded after retries")

    def run_per_event(self, x, y, z, r, module, ev_off_host):
        """The plain per-event form: the same kernels on one event at a time,
        with a host read of the counts after each stage."""
        out = []
        for e in range(len(ev_off_host) - 1):
            a, b = int(ev_off_host[e]), int(ev_off_host[e + 1])
            off = torch.tensor([0, b - a], dtype=torch.int32, device=self.device)
            out.append(self.run(x[a:b], y[a:b], z[a:b], r[a:b], module[a:b], off)[0])
        return out

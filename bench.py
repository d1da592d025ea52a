"""Throughput benchmark of the pixel seeding + broken-line fitting path.

One step = the four stages (doublets + Fishbone, CA connection, n-tuplets +
cleaning, broken-line fit) over one batch of 64 synthetic PU200 events (about
1.7 M hits), inputs resident on the GPU.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs under torchrun, one rank per GPU, each rank on its own 64 events
(weak scaling, no collective on the data path).  --impl reference times the
CPU oracle (the plain FP64 / exact-integer implementation the GPU path is
checked against) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s and tracks/s at PU200 (1 GB300) vs plain per-event GPU; % HBM roofline"
WORKLOAD = "pu200-batch64: 64 synthetic ttbar-like events, pileup Poisson(200), ~1.7M hits"
EVENTS_PER_STEP = 64
SECTOR = 16          # oracle sample: 1/SECTOR of the azimuth of one PU200 event


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------- CPU oracle
def _oracle_sample(batch, sector: int = 0):
    import numpy as np
    phi = np.arctan2(batch["y"], batch["x"]) + np.pi
    a, b = batch["ev_off"][0], batch["ev_off"][1]
    m = np.zeros(batch["x"].size, bool)
    m[a:b] = True
    lo = (sector + SECTOR // 2) % SECTOR            # sector 0 is phi in [0, 2 pi / SECTOR)
    m &= (phi >= lo * 2 * np.pi / SECTOR) & (phi < (lo + 1) * 2 * np.pi / SECTOR)
    s = {k: batch[k][m] for k in ("x", "y", "z", "r", "module")}
    s["ev_off"] = np.array([0, int(m.sum())], dtype=np.int32)
    return s


def _time_oracle(sample, repeats):
    import oracle
    from synth import cuts as CU
    from synth import geometry as G
    oracle.build()
    times = []
    for _ in range(repeats):
        t = time.perf_counter()
        oracle.run(sample, CU.cuts_for("pu200-batch64"), CU.FIT_PARAMS, G.module_layer_table(), [0] * 4 + [1] * 6)
        times.append(time.perf_counter() - t)
    return times


def _oracle_sector_worker(sample):
    """One sector through the oracle in a worker process; seconds taken."""
    import oracle
    from synth import cuts as CU
    from synth import geometry as G
    t = time.perf_counter()
    oracle.run(sample, CU.cuts_for("pu200-batch64"), CU.FIT_PARAMS, G.module_layer_table(), [0] * 4 + [1] * 6)
    return time.perf_counter() - t


def _time_oracle_all_cores(batch):
    """Wall time of the oracle over the SECTOR azimuthal sectors of PU200
    event 0, one sector per worker process (spawned), on all host cores."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()
    samples = [_oracle_sample(batch, k) for k in range(SECTOR)]
    workers = max(1, min(SECTOR, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_sector_worker, samples[:workers]))          # warm the workers up
        t = time.perf_counter()
        list(ex.map(_oracle_sector_worker, samples))
        wall = time.perf_counter() - t
    return wall, workers, sum(int(x["x"].size) for x in samples)


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _cpu_desc(n_hits):
    return (f"1/{SECTOR} azimuthal sector (phi in [0, 2pi/{SECTOR})) of PU200 event 0, {n_hits} hits, all "
            f"stages; events/s = 1/({SECTOR} x sector time), which overstates the oracle's full-event rate "
            f"because its doublet search is quadratic in the hits of an event")


# ------------------------------------------------------------ clock sampling
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, tmp_dir: str | None = None):
        self.proc = None
        self.path = None
        self.idx = gpu_index
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv", dir=tmp_dir)
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            if getattr(self, "f", None):
                self.f.close()
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
            self.path = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) < 9:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "nvidia-smi every 200 ms from the first warm-up step to the end of the timed steps"}


# ------------------------------------------------------------------ bytes
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "dram_traffic_pu200_batch8.md")


# the sources of the four seeding and fitting calls (whose DRAM traffic the
# profile summary records); the post-fit and adjoint kernels are not among them
PIPELINE_SOURCES = ("pt_common.cuh", "pt_kernels.cuh", "pt_bin.cu", "pt_doublets.cu", "pt_fishbone.cu",
                    "pt_connect.cu", "pt_ntuplets.cu", "pt_fit.cu", "pt_abi.cu")


def kernel_source_hash() -> str:
    """Hash of the code (comments and blank space removed) of the pipeline's
    CUDA sources and the ABI header: which kernels a profile summary was
    taken on."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2008_13461_gb300", "csrc")
    for p in [os.path.join(csrc, f) for f in PIPELINE_SOURCES] + [os.path.join(ROOT, "include", "pt.h")]:
        with open(p) as fh:
            code = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        h.update(os.path.basename(p).encode())
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def _profile_entry(key: str):
    """Value list of `key:` in the committed ncu summary, or None when the
    kernels changed since it was taken."""
    try:
        with open(TRAFFIC_PROFILE) as fh:
            lines = fh.read().splitlines()
    except OSError:
        return None
    src = next((l.split(":", 1)[1].strip() for l in lines if l.startswith("kernel_sources:")), None)
    val = next((l.split(":", 1)[1].split() for l in lines if l.startswith(key + ":")), None)
    return val if src == kernel_source_hash() and val else None


def measured_traffic(kernel: str, cells: int):
    """DRAM bytes of one launch of a kernel, scaled by cells from the
    committed ncu summary; None when the kernels changed since it was taken."""
    per = _profile_entry("traffic_bytes_per_cell")
    if not per:
        return None
    table = dict(kv.split("=") for kv in per)
    return float(table[kernel]) * cells if kernel in table else None


def measured_issue(kernel: str):
    """Warp instructions issued per SM cycle of a kernel (of the 4 the SM's
    schedulers can issue) from the committed ncu summary, or None."""
    per = _profile_entry("issue_per_sm_cycle")
    if not per:
        return None
    table = dict(kv.split("=") for kv in per)
    return float(table[kernel]) if kernel in table else None


def measure_alu_peaks(dev, stream):
    """The GPU's float32 and float64 fused-multiply-add peaks, from the
    library's probe (8 independent FMA chains per thread, 2048 threads per
    SM), best of 5 launches after one warm-up."""
    import torch
    from paper_2008_13461_gb300 import _lib as L
    n = torch.cuda.get_device_properties(dev).multi_processor_count * 2048
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    out = {}
    for fp64, iters in ((False, 4096), (True, 256)):
        buf = torch.empty(n, dtype=torch.float64 if fp64 else torch.float32, device=dev)
        times = []
        for k in range(6):
            ev[0].record(stream)
            L.fma_probe(fp64, iters, n, buf.data_ptr(), stream.cuda_stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            if k:
                times.append(ev[0].elapsed_time(ev[1]))
        out["fp64_tflops" if fp64 else "fp32_tflops"] = 16.0 * iters * n / (min(times) * 1e-3) / 1e12
    out["method"] = "pt_fma_probe: dependent FMA chains, 8 per thread, 2048 threads per SM, best of 5"
    return out


# Algorithmic bytes per unit of each step (each input read once, each
# output written once), with H hits, D cells, E edges, T n-tuplets, K
# tracks (K_n of them with n hits):
#   a0 binning      20 H read + 24 H written
#   a1 doublets     16 H x 3.4 (layer pairs per hit's layer) read + 9 D (cells) + 4 D (incoming lists) written
#   a2 Fishbone     8 D + 16 H read + 1 D written
#   a3 connection   8 D + 4 D read + 4 E (neighbour lists) + 1 D written
#   a4 search       4 E + 8 D read + 36 T written
#   a5 cleaning     36 T read + 12 T (per-cell maxima) + 1 T written
#   a6 fit          (36 + 16 n + 84 + 1) K_n
STAGE_KERNELS = {
    "a0_binning": ("k_bin_count", "k_scan_reduce", "k_scan_partials", "k_scan_apply", "k_bin_fill"),
    "a1_doublets": ("k_doublets", "k_doublets_exact"),
    "a2_fishbone": ("k_fishbone_small", "k_fishbone_medium", "k_fishbone_large", "k_fishbone_exact"),
    "a3_connect": ("k_connect", "k_connect_exact"),
    "a4_search": ("k_edge_records", "k_dfs"),
    "a5_cleaning": ("k_clean_max", "k_clean_keep"),
    "a6_fit": ("k_count_tracks", "k_select_tracks", "k_fit<3>", "k_fit<4>", "k_fit<5>", "k_fit<6..8>"),
}
FB_CLASS_MAX = {"k_fishbone_small": 192, "k_fishbone_medium": 320, "k_fishbone_large": 512}


def stage_bytes(H, D, E, T, K_by_n):
    return {
        "a0_binning": 44 * H,
        "a1_doublets": 16 * 3.4 * H + 13 * D,
        "a2_fishbone": 9 * D + 16 * H,
        "a3_connect": 13 * D + 4 * E,
        "a4_search": 4 * E + 8 * D + 36 * T,
        "a5_cleaning": 49 * T,
        "a6_fit": sum((121 + 16 * n) * k for n, k in K_by_n.items()),
    }


def kernel_bytes(H, D, E, T, K_by_n, fb_cells):
    """Algorithmic bytes of one launch of each kernel: its stage's bytes
    for the units it processes.  The main kernel of a stage processes all
    of its units (its exact pass repeats a few and gets none); the
    Fishbone's three kernels split the cells by their outer hit's cell count
    (fb_cells: cells of each kernel); each fit kernel has its tracks."""
    sb = stage_bytes(H, D, E, T, K_by_n)
    out = {"k_bin_count": 20 * H, "k_bin_fill": 24 * H, "k_doublets": sb["a1_doublets"],
           "k_connect": sb["a3_connect"], "k_dfs": sb["a4_search"], "k_clean_max": 36 * T + 12 * T,
           "k_clean_keep": 36 * T + 1 * T}
    for k, c in fb_cells.items():
        out[k] = sb["a2_fishbone"] * (c / D if D else 0.0)
    names = {3: "k_fit<3>", 4: "k_fit<4>", 5: "k_fit<5>"}
    for n, k in K_by_n.items():
        name = names.get(n, "k_fit<6..8>")
        out[name] = out.get(name, 0.0) + (121 + 16 * n) * k
    return out


def fit_flops_per_track(n: int) -> float:
    """Floating-point operations of the broken-line fit of one n-hit track,
    counted on the method as written (dense algebra): the s-z line system
    (n unknowns, 3-point slope kinks) and the circle system (n offsets plus
    the curvature correction, 4-term kinks), each assembled (2 flops per
    measurement, 2 per entry of each kink's outer product), factorised by
    Cholesky (m^3/3 + m^2/2) and solved forward and back (2 m^2 each), plus
    the pre-fit circle and the arc lengths and offsets of the hits (~30 +
    20 n)."""
    total = 30.0 + 20.0 * n
    for m, kink in ((n, 3), (n + 1, 4)):
        total += 2 * n + 2 * kink * kink * max(0, n - 2) + m ** 3 / 3.0 + m * m / 2.0 + 4.0 * m * m
    return total


class Ctx:
    """Everything the extra measurements need from the main run."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def measure_graph(c, args):
    """Median time of a CUDA-graph replay of the four stages (L2 flushed
    before each; 3 warm-up replays, then at least 20 timed)."""
    import torch
    from paper_2008_13461_gb300 import _lib as L
    try:
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(c.dev)
        side.wait_stream(c.stream)
        with torch.cuda.stream(side):
            ss = side.cuda_stream
            with torch.cuda.graph(g, stream=side):
                L.build_doublets(c.ws, c.nb, c.h, c.cfg, c.cells, ss)
                L.connect_cells(c.ws, c.nb, c.h, c.cfg, c.cells, c.edges, ss)
                L.find_ntuplets(c.ws, c.nb, c.h, c.cfg, c.cells, c.edges, c.tuples, ss)
                L.fit_tracks(c.ws, c.nb, c.h, c.cfg, c.tuples, c.tracks, ss)
        c.stream.wait_stream(side)
        torch.cuda.synchronize()
        ge = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        gms = []
        for k in range(3 + max(20, args.steps)):        # 3 warm-up replays, then at least 20 timed
            c.flush.zero_()
            ge[0].record(c.stream)
            g.replay()
            ge[1].record(c.stream)
            torch.cuda.synchronize()
            if k >= 3:
                gms.append(ge[0].elapsed_time(ge[1]))
        st, c3 = L.read_counts(c.ws, c.nb, c.h, c.cfg, c.s)
        assert st == L.PT_OK and c3.n_tracks == c.counts.n_tracks
        return statistics.median(gms)
    except Exception as exc:   # reported, never required
        return f"unavailable: {exc}"


def measure_e2e(c, args, batch, world):
    """Events/s through the public API with host buffers: pinned host inputs
    copied to the device, the four stages, counts and track parameters copied
    back to pinned host memory, every step."""
    import torch
    host = {k: torch.as_tensor(batch[k]).pin_memory() for k in ("x", "y", "z", "r", "module", "ev_off")}
    out_host = torch.empty(max(1, c.counts.n_tracks) * 5 * 2, dtype=torch.float32).pin_memory()
    dbuf = {k: torch.empty_like(v, device=c.dev) for k, v in host.items()}
    dargs = (dbuf["x"], dbuf["y"], dbuf["z"], dbuf["r"], dbuf["module"], dbuf["ev_off"])
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    times, d2h = [], 0
    for k in range(args.warmup + args.steps):
        c.flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for key in host:
            dbuf[key].copy_(host[key], non_blocking=True)
        c.pipe.launch(c.bufs, *dargs)
        st, c4 = c.pipe.counts(c.bufs, *dargs)
        n5 = c4.n_tracks * 5
        out_host[:n5].copy_(c.bufs.trk_params[:n5], non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            d2h = n5 * 4 + 64
    n_events = (len(batch["ev_off"]) - 1) * world
    slowest = max_over_ranks(statistics.mean(times), world, c.dev)      # the slowest rank's step
    return {"value": n_events / slowest, "unit": "events/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def measure_differentiable(c, args):
    """The differentiable form on the same batch: a refit of every track from
    the hits (its n-tuplets fixed) and the adjoint pass giving the gradient
    of a loss of all parameters and chi2 with respect to every hit; median
    milliseconds of each, CUDA events, after warm-up."""
    import torch
    from paper_2008_13461_gb300 import _lib as L
    K = c.counts.n_tracks
    g = torch.Generator(device=c.dev).manual_seed(3)
    gp = torch.randn(max(K, 1), 5, device=c.dev, generator=g) * 1e-3
    gc = torch.randn(max(K, 1), device=c.dev, generator=g) * 1e-2
    gx, gy, gz = (torch.zeros(c.bufs.n_hits, device=c.dev) for _ in range(3))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf, tb = [], []
    for k in range(args.warmup + args.steps):
        for a in (gx, gy, gz):
            a.zero_()
        ev[0].record(c.stream)
        L.fit_tracks(c.ws, c.nb, c.h, c.cfg, c.tuples, c.tracks, c.s)
        ev[1].record(c.stream)
        L.fit_tracks_grad(c.ws, c.nb, c.h, c.cfg, c.tuples, c.tracks, gp.data_ptr(), gc.data_ptr(), gx.data_ptr(),
                          gy.data_ptr(), gz.data_ptr(), c.s)
        ev[2].record(c.stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            tf.append(ev[0].elapsed_time(ev[1]))
            tb.append(ev[1].elapsed_time(ev[2]))
    fit_ms, adj_ms = statistics.median(tf), statistics.median(tb)
    ta = []
    for k in range(args.warmup + args.steps):
        ev[0].record(c.stream)
        keep = c.pipe.resolve_ambiguities(c.bufs, c.counts, c.bufs.n_hits, c.stream)
        ev[1].record(c.stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            ta.append(ev[0].elapsed_time(ev[1]))
    c.ambiguity = {"ms": statistics.median(ta), "tracks_kept": int(keep.sum().item()), "tracks": K}
    tv = []
    t = c.t
    hits = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            L.kernel_timing(True)
        ev[0].record(c.stream)
        v, sm = c.pipe.find_vertices(c.bufs, c.counts, *hits, stream=c.stream)
        ev[1].record(c.stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            tv.append(ev[0].elapsed_time(ev[1]))
    kt = L.kernel_timing_read()
    L.kernel_timing(False)
    nv = v["n"].cpu()
    elig = int((v["track_vertex"] >= 0).sum().item())
    c.vertexing = {"ms": statistics.median(tv), "vertices_per_event": float(nv.float().mean().item()),
                   "kernels_ms_per_launch": {k: round(ms / n, 4) for k, (n, ms) in kt.items()},
                   "tracks_in_vertices": elig, "status": int(v["status"].item()),
                   "note": "ambiguity resolution + track summary + vertex finding on the fitted tracks, "
                           "default vertex cuts"}
    return {"tracks": K, "refit_ms": fit_ms, "adjoint_ms": adj_ms,
            "tracks_per_s_refit_plus_adjoint": K / ((fit_ms + adj_ms) * 1e-3),
            "note": "gradient of a loss of all track parameters and chi2 with respect to every hit"}


MISALIGNMENT_SEED = 2008134610 + 4000 + 999


def measure_misaligned(args, dev, stream):
    """The differentiable form on the misaligned pileup-50 workload: 32
    events, every module shifted ~ N(0, 50 um) and rotated ~ N(0, 0.1 mrad)
    per axis (seeded); per step, the alignment of every hit, the refit of
    every track (its n-tuplets found on the nominal hits), the adjoint of
    the fit for a loss of all parameters and chi2, and the adjoint of the
    alignment down to every module's shift and rotation.  Median ms of each
    phase over the steps (CUDA events, after warm-up)."""
    import numpy as np
    import torch
    from synth import cuts as CU
    from synth import events as E
    from synth import geometry as G
    from paper_2008_13461_gb300 import _lib as L
    from paper_2008_13461_gb300.autograd import DifferentiableFit
    from paper_2008_13461_gb300.pipeline import Pipeline
    b = E.make_batch("pu50-batch32", workers=max(1, min(16, os.cpu_count() or 4)))
    pipe = Pipeline(G.layers(), G.module_layer_table(), CU.cuts_for("pu50-batch32"), CU.FIT_PARAMS, device=dev)
    t = {k: torch.as_tensor(b[k]).to(dev) for k in ("x", "y", "z", "r", "module", "ev_off")}
    res, bufs = pipe.run(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    K, n = res.counts.n_tracks, t["x"].numel()
    nm = G.N_MODULES
    rng = np.random.default_rng(MISALIGNMENT_SEED)
    shift = torch.as_tensor(rng.normal(0.0, 50e-4, size=(nm, 3)), dtype=torch.float32, device=dev)
    rot = torch.as_tensor(rng.normal(0.0, 1e-4, size=(nm, 3)), dtype=torch.float32, device=dev)
    centres = torch.as_tensor(G.module_centres(), dtype=torch.float32, device=dev)
    df = DifferentiableFit(pipe, bufs, t["r"], t["module"], t["ev_off"], centres=centres)
    g = torch.Generator(device=dev).manual_seed(4)
    gp = torch.randn(max(K, 1), 5, device=dev, generator=g) * 1e-3
    gc = torch.randn(max(K, 1), device=dev, generator=g) * 1e-2
    xa, ya, za, gx, gy, gz, hx, hy, hz = (torch.empty(n, device=dev) for _ in range(9))
    gshift, grot = torch.empty(nm, 3, device=dev), torch.empty(nm, 3, device=dev)
    s = stream.cuda_stream
    cfg = pipe._cfg(bufs.capacity)
    ws, nb = bufs.ws.data_ptr(), bufs.ws.numel()
    _, _, tuples, _ = bufs.structs()
    tracks = df._tracks()
    ptr = lambda a: a.data_ptr()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    times = [[] for _ in range(4)]
    for k in range(args.warmup + args.steps):
        ev[0].record(stream)
        L.align_hits(n, ptr(t["x"]), ptr(t["y"]), ptr(t["z"]), ptr(t["module"]), nm, ptr(centres), ptr(shift),
                     ptr(rot), ptr(xa), ptr(ya), ptr(za), s)
        ev[1].record(stream)
        h = pipe._hits(xa, ya, za, t["r"], t["module"], t["ev_off"])
        L.fit_tracks(ws, nb, h, cfg, tuples, tracks, s)
        ev[2].record(stream)
        for a in (gx, gy, gz, hx, hy, hz, gshift, grot):
            a.zero_()
        L.fit_tracks_grad(ws, nb, h, cfg, tuples, tracks, ptr(gp), ptr(gc), ptr(gx), ptr(gy), ptr(gz), s)
        ev[3].record(stream)
        L.align_hits_grad(n, ptr(t["x"]), ptr(t["y"]), ptr(t["z"]), ptr(t["module"]), nm, ptr(centres), ptr(rot),
                          ptr(gx), ptr(gy), ptr(gz), ptr(hx), ptr(hy), ptr(hz), ptr(gshift), ptr(grot), s)
        ev[4].record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            for i in range(4):
                times[i].append(ev[i].elapsed_time(ev[i + 1]))
    ms = [statistics.median(v) for v in times]
    total = sum(ms)
    return {"workload": "pu50-batch32: 32 synthetic pileup-50 events, every module misaligned "
                        "(shifts ~ N(0, 50 um), rotations ~ N(0, 0.1 mrad) per axis)",
            "events": len(b["ev_off"]) - 1, "hits": n, "tracks": K, "modules": nm,
            "align_ms": ms[0], "refit_ms": ms[1], "adjoint_ms": ms[2], "align_adjoint_ms": ms[3],
            "ms_per_step": total, "events_per_s": (len(b["ev_off"]) - 1) / (total * 1e-3),
            "tracks_per_s": K / (total * 1e-3),
            "note": "the adjoint phase includes zeroing the gradient arrays; n-tuplets from the nominal hits"}


def grow_capacity(cap: dict, need: dict) -> dict:
    """Capacities after an overflow: the sizes needed plus a quarter and a
    margin, never smaller than before."""
    return {k: max(cap[k], int(need[k] * 1.25) + 1024) for k in cap}


def measure_per_event(c, batch, max_retries: int = 4):
    """Seconds for the plain per-event GPU form over the batch: the same
    kernels one event at a time, with a host read of the counts after every
    stage.  The per-event buffers start at 1/8 of the batch's capacities and
    grow until every event of the batch fits (an untimed pass, which also
    warms up); the timed pass then runs on them."""
    import numpy as np
    import torch
    from paper_2008_13461_gb300 import _lib as L
    ev_host = batch["ev_off"]
    sizes = np.diff(ev_host)
    offs = [torch.tensor([0, int(n)], dtype=torch.int32, device=c.dev) for n in sizes]
    t, s = c.t, c.s

    def setup(cap):
        ebufs = c.pipe.allocate(int(sizes.max()), 1, cap)
        return ebufs, c.pipe._cfg(ebufs.capacity), ebufs.structs()

    def one_pass(env):
        """Every event through the four calls; (all fitted, sizes needed)."""
        ebufs, ecfg, (ec, ee, et, ek) = env
        ews, enb = ebufs.ws.data_ptr(), ebufs.ws.numel()
        ok, need = True, dict.fromkeys(("cells", "edges", "tuples", "tracks"), 0)
        for e in range(len(sizes)):
            a, b = int(ev_host[e]), int(ev_host[e + 1])
            eh = c.pipe._hits(t["x"][a:b], t["y"][a:b], t["z"][a:b], t["r"][a:b], t["module"][a:b], offs[e])
            L.build_doublets(ews, enb, eh, ecfg, ec, s)
            L.read_counts(ews, enb, eh, ecfg, s)
            L.connect_cells(ews, enb, eh, ecfg, ec, ee, s)
            L.read_counts(ews, enb, eh, ecfg, s)
            L.find_ntuplets(ews, enb, eh, ecfg, ec, ee, et, s)
            L.read_counts(ews, enb, eh, ecfg, s)
            L.fit_tracks(ews, enb, eh, ecfg, et, ek, s)
            stc, n = L.read_counts(ews, enb, eh, ecfg, s)     # the flags of all four calls of this event
            if stc == L.PT_ERR_CAPACITY:
                ok = False
            elif stc != L.PT_OK:
                raise L.PtError(stc, f"per-event form, event {e}")
            for k, v in (("cells", n.n_cells), ("edges", n.n_edges), ("tuples", n.n_tuples),
                         ("tracks", n.n_tracks)):
                need[k] = max(need[k], int(v))
        return ok, need

    cap = {k: max(v // 8, 1 << 20) for k, v in c.bufs.capacity.items()}
    env = setup(cap)
    for _ in range(max_retries + 1):
        ok, need = one_pass(env)
        if ok:
            break
        cap = grow_capacity(cap, need)
        env = setup(cap)
    else:
        raise L.PtError(L.PT_ERR_CAPACITY, "per-event form: capacity still exceeded after retries")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok, _ = one_pass(env)
    torch.cuda.synchronize()
    assert ok, "per-event form: an event overflowed buffers it fitted before"
    return time.perf_counter() - t0


# ------------------------------------------------------------ sharding
def shard_first_event(rank: int, n_ev: int) -> int:
    """First event of a rank's shard: ranks take consecutive, disjoint blocks
    of n_ev events (events are independent, so ranks exchange no data)."""
    return rank * n_ev


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest value over the ranks (the slowest rank's time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Units per second of the whole job: every rank's units over the
    slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3)


# ---------------------------------------------------------------- native
def run_native(args, rank, world, local_rank):
    import numpy as np
    from synth import cuts as CU
    from synth import events as E
    from synth import geometry as G

    workers = max(1, min(16, (os.cpu_count() or 4) // max(1, world)))
    n_ev = args.events
    batch = E.make_batch("pu200-batch64", n_events=n_ev, first=shard_first_event(rank, n_ev), workers=workers)
    import torch
    import torch.distributed as dist
    from paper_2008_13461_gb300 import _lib as L
    from paper_2008_13461_gb300.pipeline import Pipeline

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    pipe = Pipeline(G.layers(), G.module_layer_table(), CU.cuts_for("pu200-batch64"), CU.FIT_PARAMS, device=dev)
    t = {k: torch.as_tensor(batch[k]).to(dev) for k in ("x", "y", "z", "r", "module", "ev_off")}
    args6 = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    tune = "defaults"
    if args.tuning:
        pipe.set_tuning(dict((k, int(v)) for k, v in (kv.split("=") for kv in args.tuning.split(","))))
        tune = "given"
    elif args.autotune:
        # tile counts, lanes and grid size picked on this batch (results do
        # not depend on them; the tuner checks that every count is unchanged)
        timings = pipe.autotune(*args6)
        tune = f"autotuned over {len(timings)} settings"
    res, bufs = pipe.run(*args6)
    counts = res.counts
    stream = torch.cuda.current_stream(dev)
    s = stream.cuda_stream
    h = pipe._hits(*args6)
    cfg = pipe._cfg(bufs.capacity)
    cells, edges, tuples, tracks = bufs.structs()
    ws, nb = bufs.ws.data_ptr(), bufs.ws.numel()
    stages = (lambda: L.build_doublets(ws, nb, h, cfg, cells, s),
              lambda: L.connect_cells(ws, nb, h, cfg, cells, edges, s),
              lambda: L.find_ntuplets(ws, nb, h, cfg, cells, edges, tuples, s),
              lambda: L.fit_tracks(ws, nb, h, cfg, tuples, tracks, s))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        for i, f in enumerate(stages):
            f()
            if evs:
                evs[i + 1].record(stream)

    # the clock sampler starts with the warm-up steps (the same work as the
    # timed ones): nvidia-smi takes a few hundred ms to report its first
    # sample, longer than the timed steps of a short run
    clocks = Clocks(local_rank) if rank == 0 else None
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    st, c2 = L.read_counts(ws, nb, h, cfg, s)
    assert st == L.PT_OK and c2.n_tracks == counts.n_tracks, "results changed between runs"
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # per-kernel CUDA events around every launch of the library, on the
    # launching stream, over the timed steps (pt_kernel_timing)
    L.kernel_timing(True)
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    kt = L.kernel_timing_read()
    L.kernel_timing(False)
    clk = clocks.stop() if clocks else None
    step_ms = [e[0].elapsed_time(e[4]) for e in evs]
    stage_ms = [statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i in range(4)]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    ctx = Ctx(dev=dev, stream=stream, s=s, ws=ws, nb=nb, h=h, cfg=cfg, cells=cells, edges=edges, tuples=tuples,
              tracks=tracks, flush=flush, counts=counts, pipe=pipe, bufs=bufs, t=t)

    graph_ms = e2e = per_event_s = diff_form = diff_misaligned = "skipped"
    if not args.no_extras:
        graph_ms = measure_graph(ctx, args)
        diff_form = measure_differentiable(ctx, args)
        diff_misaligned = measure_misaligned(args, dev, stream)
        e2e = measure_e2e(ctx, args, batch, world)
        if rank == 0:
            per_event_s = measure_per_event(ctx, batch)

    # roofline of the dominant kernel (the one with the most time in the
    # timed steps), per launch, from the per-kernel events
    H, D, Ed, T, K = bufs.n_hits, counts.n_cells, counts.n_edges, counts.n_tuples, counts.n_tracks
    n_t = res.tuples["n"].long()
    n_of_track = n_t[res.tracks["tuple"].long()].cpu().numpy() if K else np.zeros(0, int)
    K_by_n = {int(v): int((n_of_track == v).sum()) for v in np.unique(n_of_track)}
    # cells per Fishbone kernel: by their outer hit's cell count
    per_outer = torch.bincount(res.cells["outer"].long(), minlength=H)
    fb_cells, lo = {}, 0
    for name, hi in FB_CLASS_MAX.items():
        fb_cells[name] = int(per_outer[(per_outer > lo) & (per_outer <= hi)].sum().item())
        lo = hi
    kb = kernel_bytes(H, D, Ed, T, K_by_n, fb_cells)
    peak, peak_kind = _peaks()
    total_kernel_ms = sum(ms for _, ms in kt.values())
    kernels = {}
    for name, (launches, ms) in sorted(kt.items(), key=lambda kv: -kv[1][1]):
        per_launch = ms / launches
        e = {"launches": launches, "ms_per_launch": per_launch, "share": ms / total_kernel_ms}
        if name in kb and kb[name] > 0:
            e["algorithmic_bytes"] = kb[name]
            e["gbs"] = kb[name] / (per_launch * 1e-3) / 1e9
            e["frac"] = e["gbs"] / peak
        kernels[name] = e
    dom = max(kt, key=lambda k: kt[k][1])
    dom_ms = kt[dom][1] / kt[dom][0]
    dom_bytes = kb.get(dom)
    sb = stage_bytes(H, D, Ed, T, K_by_n)
    stages = {}
    for st_name, names in STAGE_KERNELS.items():
        ms = sum(kt[k][1] / kt[k][0] for k in names if k in kt)
        stages[st_name] = {"ms": ms, "algorithmic_bytes": sb[st_name],
                           "frac": sb[st_name] / (ms * 1e-3) / 1e9 / peak if ms > 0 else None}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": (dom_bytes / (dom_ms * 1e-3) / 1e9) if dom_bytes else None,
                "peak": peak, "unit": "GB/s", "peak_source": peak_kind, "launch_ms": dom_ms,
                "algorithmic_bytes": dom_bytes, "traffic": measured_traffic(dom, D),
                "traffic_source": "profiles/dram_traffic_pu200_batch8.md (ncu, 8 events), scaled by cells",
                "issue_per_sm_cycle": measured_issue(dom),
                "timing": "CUDA events around each launch on the launching stream, over the timed steps"}
    roofline["frac"] = roofline["achieved"] / peak if roofline["achieved"] else None

    # the fit is bound by the float64 pipe: its arithmetic roofline
    alu = measure_alu_peaks(dev, stream)
    fit_flops = sum(fit_flops_per_track(n) * k for n, k in K_by_n.items())
    fit_ms = sum(kt[k][1] / kt[k][0] for k in ("k_fit<3>", "k_fit<4>", "k_fit<5>", "k_fit<6..8>") if k in kt)
    fit_roofline = {"bound": "alu", "kernel": "k_fit<3..8>", "unit": "TFLOP/s", "precision": "f64",
                    "peak": alu["fp64_tflops"], "peak_source": alu["method"], "fp32_peak": alu["fp32_tflops"],
                    "algorithmic_flops": fit_flops, "ms": fit_ms,
                    "flops_source": "the method's dense-algebra count per track (bench.fit_flops_per_track)",
                    "note": "the closed-form triplet and quadruplet fits and the float32 covariance transform "
                            "execute fewer float64 operations than this count, so the method's rate can pass "
                            "the pipe's peak; the pipe itself is bound (ncu: float64 pipe busy)"}
    if fit_ms > 0:
        fit_roofline["achieved"] = fit_flops / (fit_ms * 1e-3) / 1e12
        fit_roofline["frac"] = fit_roofline["achieved"] / alu["fp64_tflops"]

    # the doublet search's candidates per accepted cell, per layer pair
    cand = L.doublet_candidates(ws, nb, h, cfg, s)
    acc = torch.bincount(res.cells["pair"].long(), minlength=len(cand)).cpu().numpy()
    cuts = CU.cuts_for("pu200-batch64")
    cand_pairs = {f"{pp['inner']}-{pp['outer']}": {"candidates": int(cand[i]), "cells": int(acc[i]),
                                                   "per_cell": cand[i] / max(1, int(acc[i]))}
                  for i, pp in enumerate(cuts["pairs"])}

    if rank != 0:
        return None
    cpu = cpu_all = None
    if world == 1 and not args.no_cpu_baseline:
        sample = _oracle_sample(batch)
        times = _time_oracle(sample, repeats=3)
        tm = statistics.median(times)
        cpu = {"value": 1.0 / (SECTOR * tm), "unit": "events/s", "cores": 1, "kind": "oracle",
               "sample": _cpu_desc(int(sample["x"].size)), "seconds_per_sample": tm, "cpu": _cpu_model()}
        try:
            wall, workers, nh = _time_oracle_all_cores(batch)
            cpu_all = {"value": 1.0 / wall, "unit": "events/s", "cores": workers, "kind": "oracle",
                       "sample": f"PU200 event 0 as {SECTOR} azimuthal sectors ({nh} hits), one sector per "
                                 f"process on {workers} host cores; events/s = 1 / wall time",
                       "cpu": _cpu_model()}
        except Exception as exc:   # reported, never required
            cpu_all = f"unavailable: {exc}"
    value = whole_job_rate(n_ev, world, ms_per_step)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "events/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (graph predicates exact; fit normal equations f64)",
        "data": "synthetic (seeded helical-track events; the paper's CMS Open Data sample is not available)",
        "config": {"workload": WORKLOAD if n_ev == EVENTS_PER_STEP else f"pu200-batch{n_ev} (profiling size)",
                   "events_per_step": n_ev, "hits_per_step": H,
                   "parallelism": f"replicas x{world} (events sharded per rank)",
                   "l2": "512 MiB buffer written between timed steps (L2 flush)",
                   "tuning": pipe.tuning, "tuning_source": tune},
        "tracks_per_s": K * world / (ms_per_step * 1e-3),
        "counts_per_step": {"hits": H, "cells": D, "alive_cells": counts.n_alive_cells, "edges": Ed,
                            "ntuplets": T, "alive_ntuplets": counts.n_alive_tuples, "tracks": K,
                            "tracks_by_hits": K_by_n, "exact_fallbacks": counts.n_exact_fallbacks,
                            "doublet_candidates": counts.n_doublet_candidates,
                            "doublet_candidates_per_cell": counts.n_doublet_candidates / max(1, D),
                            "doublet_candidates_by_pair": cand_pairs},
        "stage_ms": dict(zip(("build_doublets", "connect_cells", "find_ntuplets", "fit_tracks"), stage_ms)),
        "graph_ms_per_step": graph_ms,
        "graph_events_per_s": (n_ev / (graph_ms * 1e-3)) if isinstance(graph_ms, float) else graph_ms,
        "per_event_form": per_event_s if isinstance(per_event_s, str) else {
            "events_per_s": n_ev / per_event_s,
            "note": "same kernels one event at a time, host read of counts after every stage"},
        "e2e": e2e,
        "differentiable_form": diff_form,
        "differentiable_form_misaligned_pu50_batch32": diff_misaligned,
        "ambiguity_resolution": getattr(ctx, "ambiguity", "skipped"),
        "vertexing": getattr(ctx, "vertexing", "skipped"),
        "roofline": roofline,
        "kernels": kernels,
        "stage_roofline": stages,
        "fit_roofline": fit_roofline,
        "gpu_launches": sum(v[0] for v in kt.values()),
        "clocks": clk,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
    }
    return line


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from synth import events as E
    batch = E.make_batch("pu200-batch64", n_events=1)
    sample = _oracle_sample(batch)
    times = _time_oracle(sample, repeats=args.warmup + args.steps)[args.warmup:]
    value = args.steps / (SECTOR * sum(times))
    cpu = {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
           "sample": _cpu_desc(int(sample["x"].size)), "cpu": _cpu_model()}
    return {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 / exact integer", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": cpu["sample"]},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--events", type=int, default=EVENTS_PER_STEP,
                    help="events per step (default 64; smaller batches are for profiling runs)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="time the default tuning instead of picking tile counts, lanes and grid size on the batch")
    ap.add_argument("--tuning", default="",
                    help="explicit pt_tuning as k=v,k=v (skips the autotuner), e.g. to profile a tuned run")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the CUDA-graph, end-to-end and per-event measurements")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        line = run_native(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

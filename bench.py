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
# kernels the pipeline launches per step: binning 5 (count, 3 scan passes,
# fill), doublets 2 (main, exact pass), Fishbone 4 (small, medium, large,
# exact pass), connection 2 (main, exact pass), n-tuplets 4 (edge records,
# search, 2 cleaning), fit 6 (count and selection, one per hit count 3, 4,
# 5, 6..8)
KERNELS_PER_STEP = 23
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


def measured_traffic(stage: str, cells: int):
    """DRAM bytes of one launch of an ABI call, scaled by cells from the
    committed ncu summary; None when the kernels changed since it was taken."""
    per = _profile_entry("traffic_bytes_per_cell")
    if not per:
        return None
    table = dict(kv.split("=") for kv in per)
    return float(table[stage]) * cells if stage in table else None


def measured_fit_flops(tracks: int):
    """float64 flops of one pt_fit_tracks call (FMA = 2, add, multiply),
    scaled by tracks from the ncu instruction counts of the summary."""
    per = _profile_entry("fit_fp64_flops_per_track")
    return float(per[0]) * tracks if per else None


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


def algorithmic_bytes(H, D, E, T, K, nbar):
    """Bytes each stage must move at least (each input read once, each output
    written once): binning 20H + 24H; doublets 16H per layer-pair slot
    (3.4 on average) + 9D (cell) + 8H (per-hit cell range); Fishbone 8D read +
    1D write; connection 13D + 4E + 4E (edge src, dst); n-tuplets 8E + 8D read
    + 66T written (hits, cells, n, alive); cleaning 66T; fit 36K + 12 nbar K
    read + 88K written."""
    return {
        "binning": 44 * H,
        "doublets": 16 * 3.4 * H + 9 * D + 8 * H,
        "fishbone": 9 * D,
        "connect": 13 * D + 8 * E,
        "ntuplets": 8 * E + 8 * D + 66 * T + 66 * T,
        "fit": 36 * K + 12 * nbar * K + 88 * K,
    }



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
        ev[0].record(c.stream)
        v, sm = c.pipe.find_vertices(c.bufs, c.counts, *hits, stream=c.stream)
        ev[1].record(c.stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            tv.append(ev[0].elapsed_time(ev[1]))
    nv = v["n"].cpu()
    elig = int((v["track_vertex"] >= 0).sum().item())
    c.vertexing = {"ms": statistics.median(tv), "vertices_per_event": float(nv.float().mean().item()),
                   "tracks_in_vertices": elig, "status": int(v["status"].item()),
                   "note": "ambiguity resolution + track summary + vertex finding on the fitted tracks, "
                           "default vertex cuts"}
    return {"tracks": K, "refit_ms": fit_ms, "adjoint_ms": adj_ms,
            "tracks_per_s_refit_plus_adjoint": K / ((fit_ms + adj_ms) * 1e-3),
            "note": "gradient of a loss of all track parameters and chi2 with respect to every hit"}


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
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [e[0].elapsed_time(e[4]) for e in evs]
    stage_ms = [statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i in range(4)]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    ms_per_step = total_ms / args.steps
    ctx = Ctx(dev=dev, stream=stream, s=s, ws=ws, nb=nb, h=h, cfg=cfg, cells=cells, edges=edges, tuples=tuples,
              tracks=tracks, flush=flush, counts=counts, pipe=pipe, bufs=bufs, t=t)

    graph_ms = e2e = per_event_s = diff_form = "skipped"
    if not args.no_extras:
        graph_ms = measure_graph(ctx, args)
        diff_form = measure_differentiable(ctx, args)
        e2e = measure_e2e(ctx, args, batch, world)
        if rank == 0:
            per_event_s = measure_per_event(ctx, batch)

    # roofline of the dominant kernel
    H, D, Ed, T, K = bufs.n_hits, counts.n_cells, counts.n_edges, counts.n_tuples, counts.n_tracks
    n = res.tuples["n"].cpu().numpy()
    nbar = float(n[res.tracks["tuple"].cpu().numpy()].mean()) if K else 0.0
    ab = algorithmic_bytes(H, D, Ed, T, K, nbar)
    stage_bytes = [ab["binning"] + ab["doublets"] + ab["fishbone"], ab["connect"], ab["ntuplets"], ab["fit"]]
    stage_names = ["build_doublets", "connect_cells", "find_ntuplets", "fit_tracks"]
    dom = max(range(4), key=lambda i: stage_ms[i])
    peak, peak_kind = _peaks()
    achieved = stage_bytes[dom] / (stage_ms[dom] * 1e-3) / 1e9

    # the fit is bound by the float64 pipe: its arithmetic roofline
    alu = measure_alu_peaks(dev, stream)
    fit_flops = measured_fit_flops(K)
    fit_roofline = {"bound": "alu", "kernel": "fit_tracks", "unit": "TFLOP/s", "precision": "f64",
                    "peak": alu["fp64_tflops"], "peak_source": alu["method"], "fp32_peak": alu["fp32_tflops"],
                    "algorithmic_flops": fit_flops,
                    "flops_source": "ncu float64 instruction counts, profiles/dram_traffic_pu200_batch8.md"}
    if fit_flops is not None:
        fit_roofline["achieved"] = fit_flops / (stage_ms[3] * 1e-3) / 1e12
        fit_roofline["frac"] = fit_roofline["achieved"] / alu["fp64_tflops"]

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
                            "exact_fallbacks": counts.n_exact_fallbacks},
        "stage_ms": dict(zip(stage_names, stage_ms)),
        "graph_ms_per_step": graph_ms,
        "graph_events_per_s": (n_ev / (graph_ms * 1e-3)) if isinstance(graph_ms, float) else graph_ms,
        "per_event_form": per_event_s if isinstance(per_event_s, str) else {
            "events_per_s": n_ev / per_event_s,
            "note": "same kernels one event at a time, host read of counts after every stage"},
        "e2e": e2e,
        "differentiable_form": diff_form,
        "ambiguity_resolution": getattr(ctx, "ambiguity", "skipped"),
        "vertexing": getattr(ctx, "vertexing", "skipped"),
        "roofline": {"bound": "hbm", "kernel": stage_names[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "algorithmic_bytes": stage_bytes[dom], "traffic": measured_traffic(stage_names[dom], D),
                     "traffic_source": "profiles/dram_traffic_pu200_batch8.md, scaled by cells"},
        "fit_roofline": fit_roofline,
        "gpu_launches": KERNELS_PER_STEP * args.steps,
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

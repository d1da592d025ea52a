"""Host-side helpers of the benchmark (no GPU): the profile lookup is keyed
to the pipeline's kernel code, and the byte model adds up."""
import bench


def test_profile_entries_require_the_current_kernel_code(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    good = tmp_path / "good.md"
    good.write_text(f"kernel_sources: {h}\ntraffic_bytes_per_cell: k_doublets=20.0 k_fit<3>=2.0\n"
                    f"issue_per_sm_cycle: k_doublets=2.5\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(good))
    assert bench.measured_traffic("k_doublets", 1000) == 20000.0
    assert bench.measured_traffic("k_connect", 1000) is None
    assert bench.measured_issue("k_doublets") == 2.5
    stale = tmp_path / "stale.md"
    stale.write_text("kernel_sources: 0000000000000000\ntraffic_bytes_per_cell: k_doublets=20.0\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(stale))
    assert bench.measured_traffic("k_doublets", 1000) is None


def test_byte_model_per_stage_and_kernel():
    H, D, E, T = 100, 1000, 50, 20
    K_by_n = {3: 6, 4: 4}
    sb = bench.stage_bytes(H, D, E, T, K_by_n)
    assert sb["a0_binning"] == 44 * H
    assert sb["a1_doublets"] == 16 * 3.4 * H + 13 * D
    assert sb["a2_fishbone"] == 9 * D + 16 * H
    assert sb["a3_connect"] == 13 * D + 4 * E
    assert sb["a4_search"] == 4 * E + 8 * D + 36 * T
    assert sb["a5_cleaning"] == 49 * T
    assert sb["a6_fit"] == (121 + 48) * 6 + (121 + 64) * 4
    fb = {"k_fishbone_small": 700, "k_fishbone_medium": 200, "k_fishbone_large": 100}
    kb = bench.kernel_bytes(H, D, E, T, K_by_n, fb)
    # the Fishbone's kernels split its stage by cells; the fit kernels by tracks
    assert abs(sum(kb[k] for k in fb) - sb["a2_fishbone"]) < 1e-6
    assert kb["k_fit<3>"] + kb["k_fit<4>"] == sb["a6_fit"]
    assert kb["k_bin_count"] + kb["k_bin_fill"] == sb["a0_binning"]
    assert kb["k_clean_max"] + kb["k_clean_keep"] == 36 * T + sb["a5_cleaning"]


def test_fit_flop_count():
    # n = 3: line (3 unknowns, one 3-point kink) and circle (4 unknowns,
    # one 4-term kink), plus the pre-fit
    line = 2 * 3 + 2 * 9 * 1 + 27 / 3 + 9 / 2 + 4 * 9
    circle = 2 * 3 + 2 * 16 * 1 + 64 / 3 + 16 / 2 + 4 * 16
    assert abs(bench.fit_flops_per_track(3) - (30 + 60 + line + circle)) < 1e-9
    assert bench.fit_flops_per_track(5) > bench.fit_flops_per_track(4) > bench.fit_flops_per_track(3)


class _FakeBufs:
    def __init__(self, capacity):
        import torch
        self.capacity = dict(capacity)
        self.ws = torch.zeros(16, dtype=torch.uint8)

    def structs(self):
        return ("cells", "edges", "tuples", "tracks")


class _FakePipe:
    """allocate / _cfg / _hits of the pipeline, recording the capacities."""

    def __init__(self):
        self.allocated = []

    def allocate(self, n_hits, n_events, cap):
        self.allocated.append(dict(cap))
        return _FakeBufs(cap)

    def _cfg(self, cap):
        return dict(cap)

    def _hits(self, x, *rest):
        return int(x.numel())


def _per_event_setup(monkeypatch, ev_off, per_hit, fail_status=None):
    """A fake library whose events need `per_hit` x hits of every capacity
    and report PT_ERR_CAPACITY when a buffer is smaller."""
    import numpy as np
    import torch
    from paper_2008_13461_gb300 import _lib as L
    calls = []
    for name in ("build_doublets", "connect_cells", "find_ntuplets", "fit_tracks"):
        monkeypatch.setattr(L, name, lambda *a, _n=name: calls.append(_n))

    def read_counts(ws, nb, n_hits, cfg, s):
        c = L.Counts()
        c.n_cells, c.n_edges, c.n_tuples, c.n_tracks = (per_hit * n_hits,) * 4
        if fail_status is not None:
            return fail_status, c
        over = any(per_hit * n_hits > cfg[k] for k in ("cells", "edges", "tuples", "tracks"))
        return (L.PT_ERR_CAPACITY if over else L.PT_OK), c

    monkeypatch.setattr(L, "read_counts", read_counts)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    n = int(ev_off[-1])
    t = {k: torch.zeros(n) for k in ("x", "y", "z", "r", "module")}
    pipe = _FakePipe()
    ctx = bench.Ctx(dev="cpu", t=t, s=0, pipe=pipe,
                    bufs=_FakeBufs({k: per_hit * n for k in ("cells", "edges", "tuples", "tracks")}))
    return ctx, {"ev_off": np.asarray(ev_off)}, pipe, calls


def test_per_event_form_grows_its_buffers_until_every_event_fits(monkeypatch):
    # a batch of 3 events, the middle one large: 1/8 of the batch's
    # capacities (and the 2^20 floor) is too small for it
    ctx, batch, pipe, calls = _per_event_setup(monkeypatch, [0, 100, 5000, 5100], per_hit=1000)
    sec = bench.measure_per_event(ctx, batch)
    assert sec >= 0.0
    assert pipe.allocated[0]["cells"] == max(1000 * 5100 // 8, 1 << 20)
    final = pipe.allocated[-1]
    assert all(v >= 1000 * 4900 for v in final.values())          # the largest event fits
    assert len(pipe.allocated) == 2                                 # one growth step sufficed
    assert calls[:4] == ["build_doublets", "connect_cells", "find_ntuplets", "fit_tracks"]


def test_per_event_form_keeps_buffers_that_fit(monkeypatch):
    ctx, batch, pipe, _ = _per_event_setup(monkeypatch, [0, 100, 200], per_hit=10)
    bench.measure_per_event(ctx, batch)
    assert len(pipe.allocated) == 1


def test_per_event_form_raises_on_other_errors(monkeypatch):
    import pytest
    from paper_2008_13461_gb300 import _lib as L
    ctx, batch, _, _ = _per_event_setup(monkeypatch, [0, 100], per_hit=10, fail_status=L.PT_ERR_INPUT)
    with pytest.raises(L.PtError):
        bench.measure_per_event(ctx, batch)


def test_grow_capacity_never_shrinks():
    cap = {"cells": 100, "edges": 5000}
    assert bench.grow_capacity(cap, {"cells": 1000, "edges": 10}) == {"cells": 2274, "edges": 5000}


def test_clock_sampler_parses_nvidia_smi_lines(tmp_path, monkeypatch):
    """The sampler's reading of nvidia-smi's CSV (a stand-in script prints
    three samples in the same format and keeps running until stopped)."""
    import os
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 1001.7, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = bench.Clocks(0, tmp_dir=str(tmp_path))
    for _ in range(100):                       # until the three lines are written
        with open(c.path) as fh:
            if fh.read().count("\n") >= 3:
                break
        time.sleep(0.05)
    got = c.stop()
    assert got["samples"] == 3 and got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi_reports_nothing(monkeypatch, tmp_path):
    monkeypatch.setenv("PATH", str(tmp_path))
    assert bench.Clocks(0, tmp_dir=str(tmp_path)).stop() is None
    assert list(tmp_path.iterdir()) == []           # its sample file is removed


def test_kernel_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    """The key that ties the committed traffic summary to the kernels: a
    comment edit keeps it, a code edit changes it."""
    import os
    import shutil
    for sub in ("include", os.path.join("paper_2008_13461_gb300", "csrc")):
        shutil.copytree(os.path.join(bench.ROOT, sub), tmp_path / sub)
    real = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    assert h0 == real                                 # the copy hashes like the tree
    f = tmp_path / "paper_2008_13461_gb300" / "csrc" / "pt_connect.cu"
    src = f.read_text()
    f.write_text("// a new comment line\n" + src.replace("\n", "\n/* block comment */\n", 1))
    assert bench.kernel_source_hash() == h0
    f.write_text(src.replace("kCaQueue", "kCaQueueX"))
    assert bench.kernel_source_hash() != h0

"""Allocation-free hit binning (pt_bin_hits_noalloc) agrees with the binning
that pt_build_doublets performs in its workspace.

Callers that cannot allocate device memory use pt_bin_hits_noalloc, whose
scratch is a fixed array inside the library.  Its tile offsets and the set
of hits in every tile must equal those of the workspace path (the order
inside a tile is unspecified on both paths), its binned coordinates must be
the input coordinates of the hits it lists, and this must hold on
consecutive calls, since every call reuses the same fixed array.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import cuts as CU
from synth import events as E

from parity import make_pipeline, to_dev

pytestmark = pytest.mark.gpu


def _reference_order(batch, cuts):
    pipe = make_pipeline(cuts)
    t = to_dev(batch)
    args = (t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    res, bufs = pipe.run(*args)
    torch.cuda.synchronize()
    return pipe, t, res.hit_order.cpu().numpy().copy()


def _noalloc(pipe, t):
    from paper_2008_13461_gb300 import _lib as L
    n = t["x"].numel()
    n_ev = t["ev_off"].numel() - 1
    nphi, nt = pipe.tuning["n_phi_bins"], pipe.tuning["n_t_bins"]
    T = n_ev * 10 * nphi * nt
    binned = torch.full((max(n, 1), 4), float("nan"), dtype=torch.float32, device="cuda:0")
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda:0")
    tile_off = torch.full((T + 1,), -7, dtype=torch.int32, device="cuda:0")
    flags = torch.full((1,), -7, dtype=torch.int32, device="cuda:0")
    hits = pipe._hits(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    L.bin_hits_noalloc(hits, pipe.cfg.geometry, nphi, nt, binned.data_ptr(), order.data_ptr(),
                       tile_off.data_ptr(), flags.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return binned.cpu().numpy()[:n], order.cpu().numpy()[:n], tile_off.cpu().numpy(), int(flags.item())


def _check(batch, pipe, t, ref_order):
    binned, order, tile_off, flags = _noalloc(pipe, t)
    n = batch["x"].size
    assert flags == 0
    assert tile_off[0] == 0 and tile_off[-1] == n
    assert np.all(np.diff(tile_off) >= 0)
    assert np.array_equal(np.sort(order), np.arange(n))
    # the same hits in every tile as the workspace path
    for a, b in zip(tile_off[:-1], tile_off[1:]):
        if b > a:
            assert np.array_equal(np.sort(order[a:b]), np.sort(ref_order[a:b]))
    want = np.stack([batch["x"], batch["y"], batch["z"], batch["r"]], 1)[order]
    assert np.array_equal(binned, want)


def test_noalloc_binning_matches_the_workspace_path_on_consecutive_calls():
    b2 = E.make_batch("pu50-ttbar-like")
    pipe2, t2, ref2 = _reference_order(b2, CU.cuts_for("pu50-ttbar-like"))
    b4 = E.make_batch("pu50-batch32", n_events=3)
    pipe4, t4, ref4 = _reference_order(b4, CU.cuts_for("pu50-batch32"))
    _check(b2, pipe2, t2, ref2)     # first call
    _check(b4, pipe4, t4, ref4)     # second call: different sizes, same fixed array
    _check(b2, pipe2, t2, ref2)     # third call: stale contents of the array must not matter


def test_noalloc_call_allocates_no_device_memory():
    b = E.make_batch("pu50-batch32", n_events=2)
    pipe, t, _ = _reference_order(b, CU.cuts_for("pu50-batch32"))
    _noalloc(pipe, t)                                   # warm-up: the library's kernels are loaded
    from paper_2008_13461_gb300 import _lib as L
    n = t["x"].numel()
    nphi, nt = pipe.tuning["n_phi_bins"], pipe.tuning["n_t_bins"]
    binned = torch.empty((n, 4), dtype=torch.float32, device="cuda:0")
    order = torch.empty(n, dtype=torch.int32, device="cuda:0")
    tile_off = torch.empty(2 * 10 * nphi * nt + 1, dtype=torch.int32, device="cuda:0")
    flags = torch.empty(1, dtype=torch.int32, device="cuda:0")
    hits = pipe._hits(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    L.bin_hits_noalloc(hits, pipe.cfg.geometry, nphi, nt, binned.data_ptr(), order.data_ptr(),
                       tile_off.data_ptr(), flags.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # no device allocation by the library
    assert torch.cuda.memory_allocated() == alloc0        # nor through torch
    assert int(flags.item()) == 0 and int(tile_off[-1].item()) == n


def test_noalloc_rejects_problems_beyond_its_fixed_scratch():
    from paper_2008_13461_gb300 import _lib as L
    b = E.make_batch("barrel-50-helices")
    pipe = make_pipeline(CU.cuts_for("barrel-50-helices"))
    t = to_dev(b)
    hits = pipe._hits(t["x"], t["y"], t["z"], t["r"], t["module"], t["ev_off"])
    hits.n_hits = (1 << 20) + 1          # rejected on the host, before any launch
    out = torch.empty((16, 4), dtype=torch.float32, device="cuda:0")
    i32 = torch.empty(16, dtype=torch.int32, device="cuda:0")
    st = L.lib().pt_bin_hits_noalloc(ctypes.byref(hits), ctypes.byref(pipe.cfg.geometry), 128, 16,
                                     out.data_ptr(), i32.data_ptr(), i32.data_ptr(), i32.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert st == L.PT_ERR_TOO_LARGE

"""Post-fit steps on the GPU (Sec. 3.5-3.6) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import postfit
from synth import cuts as CU
from synth import events as E

from parity import oracle_run, gpu_run

pytestmark = pytest.mark.gpu


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device="cuda:0")


def _gpu_ambiguities(hits8, cells8, n, track_tuple, chi2, tip, n_cells, n_hits):
    from paper_2008_13461_gb300 import _lib as L
    H, Cc, N = _dev(hits8, np.int32), _dev(cells8, np.int32), _dev(n, np.uint8)
    tt, c2, tp = _dev(track_tuple, np.int32), _dev(chi2, np.float32), _dev(tip, np.float32)
    scratch = torch.empty(max(1, n_cells + n_hits), dtype=torch.int32, device="cuda:0")
    keep = torch.empty(max(1, len(track_tuple)), dtype=torch.uint8, device="cuda:0")
    tuples = L.Tuples(H.data_ptr(), Cc.data_ptr(), N.data_ptr(), N.data_ptr())
    L.resolve_ambiguities(tuples, tt.data_ptr(), len(track_tuple), c2.data_ptr(), tp.data_ptr(), 1, n_cells, n_hits,
                          scratch.data_ptr(), keep.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return keep.cpu().numpy()[:len(track_tuple)].astype(bool)


def test_ambiguity_resolution_matches_the_oracle():
    b = E.make_batch("pu50-ttbar-like")
    want = oracle_run(b, CU.cuts_for("pu50-ttbar-like"))
    T = len(want["tuple_n"])
    cells8 = np.full((T, 8), -1, np.int32)
    cells8[:, :want["tuple_cells"].shape[1]] = want["tuple_cells"]
    tt = want["track_tuple"]
    chi2 = want["chi2"].astype(np.float32)               # both sides decide on float32 values
    tip = want["params"][:, 3].astype(np.float32)
    keep_o = postfit.resolve_ambiguities(want["tuple_hits"], cells8, want["tuple_n"], tt, chi2, tip)
    keep_g = _gpu_ambiguities(want["tuple_hits"], cells8, want["tuple_n"], tt, chi2, tip, len(want["cells"]),
                              len(b["x"]))
    assert 0 < keep_o.sum() < len(keep_o)
    assert np.array_equal(keep_g, keep_o)


def test_ambiguity_resolution_of_the_pipeline_tracks_obeys_the_rule():
    b = E.make_batch("pu50-ttbar-like")
    res = gpu_run(b, CU.cuts_for("pu50-ttbar-like"))
    from paper_2008_13461_gb300 import _lib as L
    K, nc, nh = res.counts.n_tracks, res.counts.n_cells, len(b["x"])
    scratch = torch.empty(nc + nh, dtype=torch.int32, device="cuda:0")
    keep = torch.empty(K, dtype=torch.uint8, device="cuda:0")
    tup = res.tuples
    tuples = L.Tuples(tup["hits"].data_ptr(), tup["cells"].data_ptr(), tup["n"].data_ptr(), tup["alive"].data_ptr())
    par = res.tracks["params"].contiguous()
    L.resolve_ambiguities(tuples, res.tracks["tuple"].data_ptr(), K, res.tracks["chi2"].data_ptr(),
                          par.data_ptr() + 3 * 4, 5, nc, nh, scratch.data_ptr(), keep.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    keep = keep.cpu().numpy().astype(bool)
    tt = res.tracks["tuple"].cpu().numpy()
    n = tup["n"].cpu().numpy()[tt]
    C = tup["cells"].cpu().numpy()[tt]
    Hh = tup["hits"].cpu().numpy()[tt]
    c2 = res.tracks["chi2"].cpu().numpy()
    tip = np.abs(par.cpu().numpy()[:, 3])
    # rule 1: a kept track has the smallest chi2 at each of its cells
    best = {}
    for k in range(K):
        for c in C[k, :n[k] - 1]:
            best[c] = min(best.get(c, np.inf), c2[k])
    keep1 = np.array([all(c2[k] == best[c] for c in C[k, :n[k] - 1]) for k in range(K)])
    assert np.all(keep <= keep1)
    # rule 2 among the triplets kept by rule 1
    bh = {}
    for k in np.nonzero(keep1 & (n == 3))[0]:
        for h in Hh[k, :3]:
            bh[h] = min(bh.get(h, np.inf), tip[k])
    want = keep1.copy()
    for k in np.nonzero(keep1 & (n == 3))[0]:
        want[k] = all(tip[k] == bh[h] for h in Hh[k, :3])
    assert np.array_equal(keep, want)
    assert 0 < keep.sum() < K

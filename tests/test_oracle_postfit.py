"""Pins of the oracle's post-fit steps (Sec. 3.5-3.6) on hand-built cases."""
import numpy as np

from oracle import postfit


def _tuples(rows):
    """rows: list of hit lists; cells are numbered by their hit pair."""
    T = len(rows)
    H = np.full((T, 8), -1, np.int32)
    Cc = np.full((T, 8), -1, np.int32)
    ids = {}
    n = np.zeros(T, np.int32)
    for t, hs in enumerate(rows):
        n[t] = len(hs)
        H[t, :len(hs)] = hs
        for j in range(len(hs) - 1):
            Cc[t, j] = ids.setdefault((hs[j], hs[j + 1]), len(ids))
    return H, Cc, n


def test_ambiguity_resolution_by_shared_doublet_and_shared_hit():
    rows = [
        [1, 2, 3, 4],      # A: shares cell (3,4) with B, worse chi2 -> dropped
        [9, 3, 4, 5],      # B: kept
        [20, 21, 22],      # C: triplet, shares hit 22 with D, smaller |tip| -> kept
        [23, 24, 22],      # D: dropped by C
        [30, 31, 32, 33],  # E: shares nothing -> kept
        [40, 41, 42],      # F: shares cell (41,42) with G, equal chi2: both kept by step 1;
        [43, 41, 42],      # G:   then they share hits 41, 42: F has the smaller |tip|
        [50, 51, 52],      # H: shares hit 51 with I (equal |tip|): both kept
        [53, 51, 54],      # I
    ]
    H, Cc, n = _tuples(rows)
    tt = np.arange(len(rows))
    chi2 = np.array([5.0, 2.0, 1.0, 1.0, 3.0, 1.5, 1.5, 0.5, 0.7], np.float32)
    tip = np.array([0.1, 0.1, 0.01, -0.02, 0.0, -0.003, 0.004, 0.05, -0.05], np.float32)
    keep = postfit.resolve_ambiguities(H, Cc, n, tt, chi2, tip)
    assert keep.tolist() == [False, True, True, False, True, True, False, True, True]
    # independent of the order of the tracks
    perm = np.random.default_rng(1).permutation(len(rows))
    keep_p = postfit.resolve_ambiguities(H, Cc, n, tt[perm], chi2[perm], tip[perm])
    assert np.array_equal(keep_p, keep[perm])


def test_ambiguity_resolution_triplets_only_compete_after_the_doublet_step():
    # [7,8,9] has the smallest |tip| but shares cell (7,8) with [1,7,8] at a
    # worse chi2, so the doublet step drops it first; then [5,6,7] shares hit
    # 7 with the surviving [1,7,8], whose |tip| is smaller: dropped
    rows = [[5, 6, 7], [7, 8, 9], [1, 7, 8]]
    H, Cc, n = _tuples(rows)
    keep = postfit.resolve_ambiguities(H, Cc, n, np.arange(3), np.float32([1, 9, 2]),
                                       np.float32([0.5, 0.01, 0.02]))
    assert keep.tolist() == [False, False, True]


def test_nan_chi2_never_wins():
    rows = [[1, 2, 3, 4], [0, 2, 3, 5]]
    H, Cc, n = _tuples(rows)
    keep = postfit.resolve_ambiguities(H, Cc, n, np.arange(2), np.float32([np.nan, 3.0]), np.float32([0, 0]))
    assert keep.tolist() == [False, True]

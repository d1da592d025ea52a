"""Post-fit steps of the pixel chain (Sec. 3.5-3.6), plain and slow.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Decisions that compare
floating-point track quantities are taken in float32, the precision of the
GPU's track outputs, so that both sides decide alike on the same inputs.
"""
from __future__ import annotations

import numpy as np


def _key(v) -> np.float32:
    """Comparison key of a non-negative quantity; NaN or negative -> +inf."""
    v = np.float32(v)
    return v if v >= 0 else np.float32(np.inf)


def resolve_ambiguities(tuple_hits, tuple_cells, tuple_n, track_tuple, chi2, tip) -> np.ndarray:
    """Ambiguity resolution (Sec. 3.5), read as:

    1. tracks sharing a hit-doublet (a cell, i.e. two consecutive hits) are
       ambiguous: a track is kept only if no track sharing one of its cells
       has a smaller chi2 (equal chi2: both kept);
    2. among the tracks kept by 1, triplets (3 hits) sharing a hit are
       ambiguous: a triplet is kept only if no such triplet sharing one of
       its hits has a smaller |transverse impact parameter| (equal: both
       kept).

    Returns keep[K] (bool), K = len(track_tuple); chi2, tip per track."""
    K = len(track_tuple)
    cells = [[int(c) for c in tuple_cells[t, :tuple_n[t] - 1]] for t in track_tuple]
    hits = [[int(h) for h in tuple_hits[t, :tuple_n[t]]] for t in track_tuple]
    n = [int(tuple_n[t]) for t in track_tuple]
    c2 = [_key(v) for v in chi2]
    tp = [_key(abs(np.float32(v))) for v in tip]
    best = {}
    for k in range(K):
        for c in cells[k]:
            best[c] = min(best.get(c, np.float32(np.inf)), c2[k])
    keep = np.array([all(c2[k] == best[c] for c in cells[k]) for k in range(K)], dtype=bool)
    best_h = {}
    for k in range(K):
        if keep[k] and n[k] == 3:
            for h in hits[k]:
                best_h[h] = min(best_h.get(h, np.float32(np.inf)), tp[k])
    for k in range(K):
        if keep[k] and n[k] == 3:
            keep[k] = all(tp[k] == best_h[h] for h in hits[k])
    return keep

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


def _vfit(z0, w):
    """Weighted mean, its error, chi2 (float64 sums)."""
    sw = float(np.sum(w))
    z = float(np.sum(w * z0)) / sw
    return z, 1.0 / np.sqrt(sw), float(np.sum(w * (z0 - z) ** 2))


def find_vertices(ev, z0, ez0, pt, nhits, keep, n_events, cuts: dict):
    """Pixel vertices (Sec. 3.6), read as:

    * eligible tracks: kept, nhits >= min_hits, pt > pt_min, ez0 < ez0_max;
    * density rho_i: the number of eligible tracks j of the same event
      compatible with i, i itself included: |z0_i - z0_j| < dz_cut and
      (z0_i - z0_j)^2 < chi2_max (ez0_i^2 + ez0_j^2) (so rho > 1, the seed
      condition, means at least one compatible neighbour, and a 2-track
      cluster can form a vertex);
    * each eligible track links to its nearest compatible track (smallest
      |dz|, then smallest index) ranking higher: larger rho, or equal rho
      and smaller index; tracks without such a track are roots;
    * a root with rho > 1 seeds a vertex candidate made of every track whose
      links lead to it; a candidate with at least min_tracks tracks is a
      vertex: z = weighted mean of z0 (w = 1/ez0^2), ez = 1/sqrt(sum w),
      chi2 = sum w (z0 - z)^2, ndf = n - 1;
    * a vertex with chi2/ndf > split_chi2 is split in two by 2-means in z
      (centres started at the weighted means of its tracks below and above
      z, tracks assigned to the nearer centre (ties: the lower one), centres
      recomputed, until no assignment changes, at most 20 rounds); the split
      is kept if both parts have at least min_tracks tracks;
    * vertices of an event are sorted by sum of pt^2, descending (ties by
      z).

    Distances and cuts are evaluated in float32 in the order written above
    (dz = z0_i - z0_j; dz*dz against chi2_max*(ez_i*ez_i + ez_j*ez_j)), sums
    in float64.  Returns (vertices: list per event of dicts with z, ez,
    chi2, ndf, sumpt2, tracks (sorted track indices)), vertex index per track
    within its event (-1: none))."""
    f = np.float32
    z0 = np.asarray(z0, f)
    ez0 = np.asarray(ez0, f)
    pt = np.asarray(pt, f)
    K = len(z0)
    dzc, c2m = f(cuts["dz_cut"]), f(cuts["chi2_max"])
    elig = np.array([bool(keep[i]) and int(nhits[i]) >= cuts["min_hits"] and pt[i] > f(cuts["pt_min"]) and
                     ez0[i] < f(cuts["ez0_max"]) for i in range(K)])
    out_v, vidx = [[] for _ in range(n_events)], np.full(K, -1, np.int64)
    for e in range(n_events):
        ids = [i for i in range(K) if elig[i] and ev[i] == e]

        def compatible(i, j):
            dz = f(z0[i] - z0[j])
            return abs(dz) < dzc and f(dz * dz) < f(c2m * f(f(ez0[i] * ez0[i]) + f(ez0[j] * ez0[j])))

        rho = {i: 1 + sum(1 for j in ids if j != i and compatible(i, j)) for i in ids}
        parent = {}
        for i in ids:
            best = None
            for j in ids:
                if j == i or not compatible(i, j):
                    continue
                if not (rho[j] > rho[i] or (rho[j] == rho[i] and j < i)):
                    continue
                key = (abs(f(z0[i] - z0[j])), j)
                if best is None or key < best[0]:
                    best = (key, j)
            parent[i] = None if best is None else best[1]

        def root(i):
            while parent[i] is not None:
                i = parent[i]
            return i

        groups = {}
        for i in ids:
            groups.setdefault(root(i), []).append(i)
        verts = []
        for r, tr in groups.items():
            if rho[r] <= 1 or len(tr) < cuts["min_tracks"]:
                continue
            tr = sorted(tr)
            zz, ww = z0[tr].astype(np.float64), 1.0 / ez0[tr].astype(np.float64) ** 2
            z, ez, chi2 = _vfit(zz, ww)
            parts = [tr]
            if len(tr) > 1 and chi2 / (len(tr) - 1) > cuts["split_chi2"]:
                lo, hi = zz < z, zz >= z
                if lo.any() and hi.any():
                    c = [_vfit(zz[lo], ww[lo])[0], _vfit(zz[hi], ww[hi])[0]]
                    assign = None
                    for _ in range(20):
                        a = np.abs(zz - c[1]) < np.abs(zz - c[0])      # True: the upper centre
                        if assign is not None and np.array_equal(a, assign):
                            break
                        assign = a
                        if a.all() or (~a).all():
                            break
                        c = [_vfit(zz[~a], ww[~a])[0], _vfit(zz[a], ww[a])[0]]
                    if assign is not None and (~assign).sum() >= cuts["min_tracks"] and \
                            assign.sum() >= cuts["min_tracks"]:
                        parts = [[t for t, u in zip(tr, assign) if not u], [t for t, u in zip(tr, assign) if u]]
            for pr in parts:
                zz, ww = z0[pr].astype(np.float64), 1.0 / ez0[pr].astype(np.float64) ** 2
                z, ez, chi2 = _vfit(zz, ww)
                verts.append(dict(z=z, ez=ez, chi2=chi2, ndf=len(pr) - 1, tracks=pr,
                                  sumpt2=float(np.sum(pt[pr].astype(np.float64) ** 2))))
        verts.sort(key=lambda v: (-v["sumpt2"], v["z"]))
        for k, v in enumerate(verts):
            vidx[v["tracks"]] = k
        out_v[e] = verts
    return out_v, vidx

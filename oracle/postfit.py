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


def track_summary(params, cov, tuple_n, first_hit, ev_off, bz):
    """Per-track inputs of the vertex finder from fitted tracks (Sec. 3.6):
    the event of the track's first hit, z0, its error sqrt(cov[z0, z0]),
    pT = 0.299792458 B R with R = 1 / (100 |kappa|) m (kappa in 1/cm, B in
    T, pT in GeV), and the hit count.  cov rows hold the lower triangle of
    the 5x5 covariance (kappa, phi0, tan lambda, d0, z0) row by row, so
    (z0, z0) is entry 14.  float64."""
    params = np.asarray(params, np.float64)
    cov = np.asarray(cov, np.float64)
    ev = np.searchsorted(np.asarray(ev_off), np.asarray(first_hit), side="right") - 1
    return dict(ev=ev.astype(np.int64), z0=params[:, 4].copy(), ez0=np.sqrt(cov[:, 14]),
                pt=0.299792458 * bz / (100.0 * np.abs(params[:, 0])), nhits=np.asarray(tuple_n).astype(np.int64))


def find_vertices(ev, z0, ez0, pt, nhits, keep, n_events, cuts: dict):
    """Pixel vertices (Sec. 3.6), read as:

    * eligible tracks: kept (keep None: all), nhits >= min_hits,
      pt > pt_min, 0 < ez0 < ez0_max, z0 finite (a track without a finite
      z0 or a positive error has no place in the clustering);
    * density rho_i: the number of eligible tracks j of the same event
      compatible with i, i itself included: |z0_i - z0_j| < dz_cut and
      (z0_i - z0_j)^2 < chi2_max (ez0_i^2 + ez0_j^2) (so rho > 1, the seed
      condition, means at least one compatible neighbour, and a 2-track
      cluster can form a vertex);
    * each eligible track links to its nearest compatible track (smallest
      |dz|, then smaller z0, then smallest index) ranking higher: larger
      rho, or equal rho and smaller z0, or equal rho and z0 and smaller
      index; tracks without such a track are roots (ties go by z0 before
      the index, so the result does not depend on the order of the tracks
      unless two share a z0);
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
    keep = np.ones(K, bool) if keep is None else np.asarray(keep).astype(bool)
    ev = np.asarray(ev)
    elig = keep & (np.asarray(nhits).astype(np.int64) >= cuts["min_hits"]) & (pt > f(cuts["pt_min"])) & \
        (ez0 > 0) & (ez0 < f(cuts["ez0_max"])) & np.isfinite(z0)
    out_v, vidx = [[] for _ in range(n_events)], np.full(K, -1, np.int64)
    for e in range(n_events):
        ids = np.nonzero(elig & (ev == e))[0].astype(np.int64)
        zs, es = z0[ids], ez0[ids]
        es2 = es * es                                           # float32 products

        def compatible_row(a):
            """compatible(ids[a], ids[b]) for every b (float32, as written)."""
            dz = zs[a] - zs                                     # float32
            return (np.abs(dz) < dzc) & (dz * dz < c2m * (es2[a] + es2))

        rows = [compatible_row(a) for a in range(len(ids))]
        for a in range(len(ids)):
            rows[a][a] = False                                  # j != i
        R = np.array([1 + int(rows[a].sum()) for a in range(len(ids))], dtype=np.int64)
        rho = {int(ids[a]): int(R[a]) for a in range(len(ids))}
        parent = {}
        for a, i in enumerate(ids.tolist()):
            higher = (R > R[a]) | ((R == R[a]) & ((zs < zs[a]) | ((zs == zs[a]) & (ids < i))))
            cand = np.nonzero(rows[a] & higher)[0]
            if len(cand) == 0:
                parent[i] = None
                continue
            d = np.abs(zs[a] - zs[cand])                        # float32 |dz|
            near = cand[d == d.min()]                           # nearest,
            near = near[zs[near] == zs[near].min()]             # then smaller z0,
            parent[i] = int(ids[near].min())                    # then smallest index

        def root(i):
            while parent[i] is not None:
                i = parent[i]
            return i

        groups = {}
        for i in ids.tolist():
            groups.setdefault(root(i), []).append(i)
        verts = []
        for r, tr in groups.items():
            if rho[r] <= 1 or len(tr) < cuts["min_tracks"]:
                continue
            tr = sorted(tr)
            zz, ww = z0[tr].astype(np.float64), 1.0 / ez0[tr].astype(np.float64) ** 2
            z, ez, chi2 = _vfit(zz, ww)
            parts = [tr]
            if len(tr) > 1 and chi2 / (len(tr) - 1) > float(f(cuts["split_chi2"])):
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

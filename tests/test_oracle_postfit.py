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


VCUTS = dict(pt_min=0.5, min_hits=4, ez0_max=0.5, dz_cut=0.1, chi2_max=9.0, split_chi2=9.0, min_tracks=2)


def _tracks(zs, ez=0.01, pt=1.0, nh=4, ev=0):
    n = len(zs)
    return (np.full(n, ev), np.float32(zs), np.full(n, ez, np.float32), np.full(n, pt, np.float32),
            np.full(n, nh), np.ones(n, bool))


def _cat(*parts):
    return tuple(np.concatenate(a) for a in zip(*parts))


def test_vertices_two_separated_clusters_and_noise():
    a = _tracks([1.000, 1.004, 0.998, 1.002], pt=2.0)
    b = _tracks([-3.0, -3.006, -2.995], pt=1.0)
    iso = _tracks([5.0, 7.0])                              # isolated: no vertex
    soft = _tracks([1.001, 1.003], pt=0.4)                 # below pt_min: ignored
    short = _tracks([1.0015], nh=3)                        # too few hits: ignored
    ev, z0, ez, pt, nh, keep = _cat(a, b, iso, soft, short)
    V, vi = postfit.find_vertices(ev, z0, ez, pt, nh, keep, 1, VCUTS)
    V = V[0]
    assert len(V) == 2
    # sorted by sum pt^2: the 4-track cluster at pt 2 first
    assert V[0]["tracks"] == [0, 1, 2, 3] and V[1]["tracks"] == [4, 5, 6]
    w = 1 / np.float64(np.float32(0.01)) ** 2
    assert abs(V[0]["z"] - np.mean(np.float32([1.000, 1.004, 0.998, 1.002]).astype(np.float64))) < 1e-12
    assert abs(V[0]["ez"] - 1 / np.sqrt(4 * w)) < 1e-12
    assert V[0]["sumpt2"] == 16.0 and V[1]["sumpt2"] == 3.0
    # chi2 = sum of squared pulls about the mean, ndf = n - 1, by hand
    zb = np.float32([-3.0, -3.006, -2.995]).astype(np.float64)
    assert abs(V[1]["chi2"] - w * np.sum((zb - zb.mean()) ** 2)) < 1e-9 * V[1]["chi2"]
    assert V[0]["ndf"] == 3 and V[1]["ndf"] == 2
    assert vi.tolist() == [0, 0, 0, 0, 1, 1, 1, -1, -1, -1, -1, -1]


def test_vertex_with_a_large_chi2_is_split_by_two_means():
    # two groups 0.06 cm apart, linked into one candidate (dz_cut 0.1 and
    # loose errors), whose chi2/ndf is large -> split into the two groups
    zs = [0.0, 0.002, -0.002, 0.06, 0.062, 0.058]
    ev, z0, ez, pt, nh, keep = _tracks(zs, ez=0.008)
    cuts = dict(VCUTS, chi2_max=100.0)
    V, vi = postfit.find_vertices(ev, z0, ez, pt, nh, keep, 1, cuts)
    assert sorted(v["tracks"] for v in V[0]) == [[0, 1, 2], [3, 4, 5]]
    # without the split threshold being passed, one vertex
    V2, _ = postfit.find_vertices(ev, z0, ez, pt, nh, keep, 1, dict(cuts, split_chi2=1e9))
    assert len(V2[0]) == 1 and len(V2[0][0]["tracks"]) == 6


def test_vertices_are_found_per_event():
    a = _tracks([0.5, 0.502, 0.499], ev=0)
    b = _tracks([0.5, 0.501], ev=1)
    ev, z0, ez, pt, nh, keep = _cat(a, b)
    V, vi = postfit.find_vertices(ev, z0, ez, pt, nh, keep, 2, VCUTS)
    assert [len(v) for v in V] == [1, 1]
    assert V[0][0]["tracks"] == [0, 1, 2] and V[1][0]["tracks"] == [3, 4]


def test_track_summary_inverts_the_generator_curvature_and_reads_the_z0_variance():
    from synth import events as E
    pt = np.array([0.5, 1.0, 7.3, 42.0])
    kappa = 1.0 / E.rho_of_pt(pt)                     # the generator's radius of curvature (cm) for pT
    params = np.zeros((4, 5))
    params[:, 0] = kappa * np.array([1, -1, 1, -1])   # either charge
    params[:, 4] = [0.1, -3.0, 2.5, 0.0]
    cov = np.zeros((4, 15))
    for k in range(4):                                # lower triangle of a 5x5, row by row
        M = np.arange(25, dtype=np.float64).reshape(5, 5) + k
        M = M + M.T
        cov[k] = [M[i, j] for i in range(5) for j in range(i + 1)]
    ev_off = np.array([0, 10, 10, 25])                # the middle event is empty
    first = np.array([0, 9, 10, 24])
    s = postfit.track_summary(params, cov, np.array([3, 4, 5, 6]), first, ev_off, E.BZ_TESLA)
    assert np.allclose(s["pt"], pt, rtol=1e-12)
    assert np.array_equal(s["ev"], [0, 0, 2, 2])
    assert np.allclose(s["ez0"] ** 2, [2 * (24 + k) for k in range(4)])   # M[4, 4] = 2 (24 + k)
    assert np.array_equal(s["z0"], params[:, 4])
    assert np.array_equal(s["nhits"], [3, 4, 5, 6])


def test_vertices_do_not_depend_on_the_order_of_the_tracks():
    from synth.vertices import vertex_tracks
    d = vertex_tracks(8, 2, pileup=30.0)
    keys = ("ev", "z0", "ez0", "pt", "nhits", "keep")
    assert len(np.unique(d["z0"])) == len(d["z0"])          # distinct z0: no tie left to the index
    v1, i1 = postfit.find_vertices(*(d[k] for k in keys), 2, VCUTS)
    perm = np.random.default_rng(1).permutation(len(d["z0"]))
    v2, i2 = postfit.find_vertices(*(d[k][perm] for k in keys), 2, VCUTS)
    assert np.array_equal(i1[perm], i2)
    for a, b in zip(v1, v2):                                # the sums only change their order
        assert [len(v["tracks"]) for v in a] == [len(v["tracks"]) for v in b]
        assert np.allclose([v["z"] for v in a], [v["z"] for v in b], rtol=0, atol=1e-12)


def _vertices_by_definition(ev, z0, ez0, pt, nh, keep, n_events, cuts):
    """The vertex finder's rules as plain per-pair loops (float32 scalars for
    the cuts, tuple keys for the orders, union-find for the groups): the
    track sets of the vertices of each event, split included, as a sorted
    list of tuples, and the order of the vertices by sum pT^2."""
    f = np.float32
    dzc, c2m = f(cuts["dz_cut"]), f(cuts["chi2_max"])
    out = []
    for e in range(n_events):
        ids = [i for i in range(len(z0)) if ev[i] == e and keep[i] and nh[i] >= cuts["min_hits"]
               and f(pt[i]) > f(cuts["pt_min"]) and f(0) < f(ez0[i]) < f(cuts["ez0_max"]) and np.isfinite(z0[i])]

        def compat(i, j):
            dz = f(z0[i]) - f(z0[j])
            return abs(dz) < dzc and dz * dz < c2m * (f(ez0[i]) * f(ez0[i]) + f(ez0[j]) * f(ez0[j]))

        rho = {i: 1 + sum(compat(i, j) for j in ids if j != i) for i in ids}
        rank = {i: (-rho[i], f(z0[i]), i) for i in ids}              # smaller tuple = higher rank
        parent = {}
        for i in ids:
            up = [j for j in ids if j != i and compat(i, j) and rank[j] < rank[i]]
            parent[i] = min(up, key=lambda j: (abs(f(z0[i]) - f(z0[j])), f(z0[j]), j)) if up else i
        root = {i: i for i in ids}                                  # union-find over the links

        def find(i):
            while root[i] != i:
                root[i] = root[root[i]]
                i = root[i]
            return i

        for i in ids:
            a, b = find(i), find(parent[i])
            if a != b:
                root[a] = b
        groups = {}
        for i in ids:
            groups.setdefault(find(i), []).append(i)
        verts = []
        for members in groups.values():
            r = next(i for i in members if parent[i] == i)           # the group's root: links only go up
            if rho[r] <= 1 or len(members) < cuts["min_tracks"]:
                continue
            members = sorted(members)
            zz = np.array([float(f(z0[i])) for i in members])
            ww = np.array([1.0 / float(f(ez0[i])) ** 2 for i in members])
            z = float(np.sum(ww * zz) / np.sum(ww))
            chi2 = float(np.sum(ww * (zz - z) ** 2))
            parts = [members]
            if len(members) > 1 and chi2 / (len(members) - 1) > float(f(cuts["split_chi2"])):
                side = [int(zi >= z) for zi in zz]                  # 1: at or above the mean
                if 0 < sum(side) < len(side):
                    for it in range(20):
                        c = [float(np.sum(ww[[s == k for s in side]] * zz[[s == k for s in side]]) /
                                   np.sum(ww[[s == k for s in side]])) for k in (0, 1)]
                        new = [int(abs(zi - c[1]) < abs(zi - c[0])) for zi in zz]
                        if new == side and it > 0:
                            break
                        side = new
                        if sum(side) in (0, len(side)):
                            break
                    lo = [m for m, s in zip(members, side) if s == 0]
                    hi = [m for m, s in zip(members, side) if s == 1]
                    if len(lo) >= cuts["min_tracks"] and len(hi) >= cuts["min_tracks"]:
                        parts = [lo, hi]
            for part in parts:
                zp = np.array([float(f(z0[i])) for i in part])
                wp = np.array([1.0 / float(f(ez0[i])) ** 2 for i in part])
                verts.append((-float(np.sum(np.float64(f(pt[part])) ** 2)), float(np.sum(wp * zp) / np.sum(wp)),
                              tuple(part)))
        out.append([v[2] for v in sorted(verts)])
    return out


def test_vertices_match_the_rules_written_as_pair_loops():
    """Random small events, with z0 values on a coarse grid so that ties of
    z0 (and of distances) occur and the tie-breaks decide: the oracle's
    vectorised finder gives the vertices of the pair-loop definition, in the
    same order."""
    rng = np.random.default_rng(12)
    for trial in range(30):
        n_events = 3
        K = int(rng.integers(0, 60))
        ev = rng.integers(0, n_events, K)
        centres = rng.uniform(-1.0, 1.0, 4)
        z0 = np.float32(np.round((centres[rng.integers(0, 4, K)] + rng.normal(0, 0.02, K)) * 500) / 500)
        ez0 = np.float32(rng.choice([0.004, 0.008, 0.012], K))
        pt = np.float32(rng.uniform(0.3, 3.0, K))
        nh = rng.integers(3, 6, K)
        keep = rng.uniform(size=K) < 0.9
        cuts = dict(VCUTS, dz_cut=float(rng.choice([0.02, 0.05, 0.1])), chi2_max=float(rng.choice([4.0, 9.0, 25.0])),
                    split_chi2=float(rng.choice([2.0, 9.0])), min_tracks=int(rng.integers(1, 4)))
        V, _ = postfit.find_vertices(ev, z0, ez0, pt, nh, keep, n_events, cuts)
        want = _vertices_by_definition(ev, z0, ez0, pt, nh, keep, n_events, cuts)
        got = [[tuple(v["tracks"]) for v in vs] for vs in V]
        assert got == want, (trial, got, want)


def test_a_bridge_track_at_equal_distance_joins_the_cluster_with_the_smaller_z0():
    """Two clusters of six tracks (z0 = 0..5 u and 15..20 u, u = 2^-7 cm,
    dz_cut = 6 u: every pair inside a cluster is compatible) and one track B
    at 10 u, compatible only with the two clusters' inner edges (5 u and
    15 u, both at 5 u from it).  Those two edge tracks have the largest
    density of their clusters (7, with B) and are not compatible with each
    other, so they are the two roots; B's nearest higher-ranked tracks are
    both at 5 u and the tie goes to the smaller z0: B joins the lower
    cluster.  Both the pair-loop definition and the oracle say so."""
    u = 2.0 ** -7
    zs = [k * u for k in range(6)] + [10 * u] + [k * u for k in range(15, 21)]
    ev, z0, ez, pt, nh, keep = _tracks(zs, ez=0.01)
    cuts = dict(VCUTS, dz_cut=6 * u, chi2_max=1e4, min_tracks=2, split_chi2=1e9)   # no split to mask the links
    V, vi = postfit.find_vertices(ev, z0, ez, pt, nh, keep, 1, cuts)
    groups = sorted(tuple(v["tracks"]) for v in V[0])
    assert groups == [(0, 1, 2, 3, 4, 5, 6), (7, 8, 9, 10, 11, 12)]
    assert _vertices_by_definition(ev, z0, ez, pt, nh, keep, 1, cuts) == [[tuple(v["tracks"]) for v in V[0]]]


def test_equal_densities_rank_by_the_smaller_z0():
    """u = 2^-7 cm, dz_cut = 6 u.  P' (-4 u), P (0) and X (2 u) form a short
    chain; X is also compatible with Q (7 u), the densest track of a cluster
    Q, R at 7..12 u.  P and X both have density 3, and P ranks above X
    because its z0 is smaller, so X links to its nearest higher-ranked
    track, P (2 u away, Q is 5 u away): two vertices, {P', P, X} and the
    cluster.  (Were the larger z0 to rank higher, X would link to Q and P to
    X, and everything would form one vertex; the split is switched off so
    that it cannot undo that.)"""
    u = 2.0 ** -7
    zs = [-4 * u, 0.0, 2 * u] + [k * u for k in range(7, 13)]
    ev, z0, ez, pt, nh, keep = _tracks(zs, ez=0.01)
    cuts = dict(VCUTS, dz_cut=6 * u, chi2_max=1e4, min_tracks=2, split_chi2=1e9)   # no split to mask the links
    V, vi = postfit.find_vertices(ev, z0, ez, pt, nh, keep, 1, cuts)
    assert sorted(tuple(v["tracks"]) for v in V[0]) == [(0, 1, 2), (3, 4, 5, 6, 7, 8)]
    assert _vertices_by_definition(ev, z0, ez, pt, nh, keep, 1, cuts) == [[tuple(v["tracks"]) for v in V[0]]]


def test_ambiguity_resolution_matches_its_rules_written_as_pair_loops():
    """Random n-tuplets over few hits (so cells and hits are shared a lot),
    chi2 and |tip| on coarse grids (so ties occur), a few NaN chi2: the
    oracle's keep flags equal the two rules evaluated pair by pair."""
    rng = np.random.default_rng(4)
    for trial in range(40):
        T = int(rng.integers(1, 40))
        rows = [list(rng.choice(12, size=int(rng.integers(3, 6)), replace=False)) for _ in range(T)]
        H, Cc, n = _tuples(rows)
        tt = rng.permutation(T)[:int(rng.integers(1, T + 1))]      # the tuples that became tracks
        chi2 = np.float32(rng.integers(0, 4, len(tt)) * 0.5)
        chi2[rng.uniform(size=len(tt)) < 0.1] = np.nan
        tip = np.float32(rng.integers(-3, 4, len(tt)) * 0.01)
        keep = postfit.resolve_ambiguities(H, Cc, n, tt, chi2, tip)

        def key(v):
            return float("inf") if not (v >= 0) else float(v)

        cells = [set(Cc[t, :n[t] - 1].tolist()) for t in tt]
        hits = [set(H[t, :n[t]].tolist()) for t in tt]
        K = len(tt)
        k1 = [all(key(chi2[k]) <= key(chi2[j]) for j in range(K) if cells[k] & cells[j]) for k in range(K)]
        want = [k1[k] and (n[tt[k]] != 3 or all(abs(float(tip[k])) <= abs(float(tip[j])) for j in range(K)
                                                if k1[j] and n[tt[j]] == 3 and hits[k] & hits[j]))
                for k in range(K)]
        assert keep.tolist() == want, trial

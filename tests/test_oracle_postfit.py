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

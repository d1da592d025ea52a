"""Pins of the CPU oracle against what the paper's definitions and plain
mathematics fix, independently of the oracle's own code:

* every exact predicate on hand-derived boundary configurations (equality is
  accepted, the next float32 constant on the strict side rejects);
* every predicate against its geometric meaning evaluated another way
  (angles, circumcentres, distances in float64) on random hits away from the
  boundary;
* the graph stages (doublets, Fishbone, CA connection, roots, DFS, cleaning)
  against brute-force enumeration of hit sequences on a small event;
* 100 % finding of noiseless helices (Sec. 4.2's efficiency definition);
* the broken-line fit (Sec. 3.4) against exact helices (chi2 = 0, parameters
  equal to the truth), the rigid limit (closed-form least squares), and the
  statistics of fits of simulated scattered tracks (pulls ~ N(0,1)).
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from synth import cuts as CU
from synth import events as E
from synth import geometry as G

HERE = os.path.dirname(os.path.abspath(__file__))
DISK = [0] * 4 + [1] * 6
F32 = np.float32


# ------------------------------------------------------------ boundaries
def _golden_boundaries():
    out = []
    with open(os.path.join(HERE, "golden", "predicate_boundaries.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            t = line.split()
            name, k = t[0], float(t[1])
            v = [float(a) for a in t[2:]]
            out.append((name, k, np.array(v, dtype=np.float32).reshape(-1, 4)))
    return out


# direction in which a larger constant loosens the cut
_LOOSER_UP = dict(phiw=True, zip=True, pt=False, rz=True, curv=False, beamspot=True, dz=True, fb=True)


@pytest.mark.parametrize("name,k,hits", _golden_boundaries(), ids=lambda v: v if isinstance(v, str) else "")
def test_predicate_boundaries(name, k, hits):
    assert oracle.pred(name, hits, k), f"{name} must accept exactly on its boundary"
    strict = np.nextafter(F32(k), F32(0) if _LOOSER_UP[name] else F32(np.inf))
    assert not oracle.pred(name, hits, float(strict)), f"{name} must reject one ulp past the boundary"


# ------------------------------------------------- geometric meanings (f64)
def _snap(v):
    return np.rint(np.asarray(v, dtype=np.float64) * 16384.0) / 16384.0


def _hit(rng, r_lo, r_hi, z_lo, z_hi, phi_c=0.0, phi_w=0.3):
    r = rng.uniform(r_lo, r_hi)
    ph = phi_c + rng.uniform(-phi_w, phi_w)
    x, y, z = _snap(r * math.cos(ph)), _snap(r * math.sin(ph)), _snap(rng.uniform(z_lo, z_hi))
    return np.array([x, y, z, _snap(math.hypot(x, y))])


def _circum(a, b, c):
    A = 2 * np.array([[b[0] - a[0], b[1] - a[1]], [c[0] - a[0], c[1] - a[1]]])
    rhs = np.array([b[0] ** 2 + b[1] ** 2 - a[0] ** 2 - a[1] ** 2,
                    c[0] ** 2 + c[1] ** 2 - a[0] ** 2 - a[1] ** 2])
    ctr = np.linalg.solve(A, rhs)
    return ctr, float(np.hypot(a[0] - ctr[0], a[1] - ctr[1]))


def _meaning(name, h):
    """Return (value, threshold_transform) so that accept <=> value <= f(k)."""
    if name == "phiw":
        i, o = h
        d = math.atan2(o[1], o[0]) - math.atan2(i[1], i[0])
        d = (d + math.pi) % (2 * math.pi) - math.pi
        return abs(d), lambda k: math.atan(math.sqrt(k)) if abs(d) < math.pi / 2 else -1
    if name in ("zip", "dz"):
        i, o = (h[0], h[1]) if name == "zip" else (h[0], h[2])
        if o[3] <= i[3]:
            return 1.0, lambda k: -1.0
        zint = i[2] - i[3] * (o[2] - i[2]) / (o[3] - i[3])
        return abs(zint), lambda k: k
    if name == "pt":
        i, o = h
        _, R = _circum(np.zeros(2), i[:2], o[:2])
        return -R, lambda k: -math.sqrt(k) / 2
    if name == "curv":
        _, R = _circum(h[0][:2], h[1][:2], h[2][:2])
        return -R, lambda k: -math.sqrt(k) / 2
    if name == "beamspot":
        ctr, R = _circum(h[0][:2], h[1][:2], h[2][:2])
        pw = ctr @ ctr - R * R
        return abs(pw) / (2 * R), lambda k: math.sqrt(k)
    if name == "rz":
        a, b, c = [np.array([p[3], p[2]]) for p in h]
        ac = c - a
        dist = abs(ac[0] * (b - a)[1] - ac[1] * (b - a)[0]) / np.linalg.norm(ac)
        return dist, lambda k: math.sqrt(k)
    if name == "fb":
        h1, h2, hh = [p[:3] for p in h]
        u, v = h1 - hh, h2 - hh
        cs = u @ v / (np.linalg.norm(u) * np.linalg.norm(v))
        sn = np.linalg.norm(np.cross(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v))
        return (sn if cs > 0 else 2.0), lambda k: math.sqrt(k)
    raise KeyError(name)


def _random_case(name, rng):
    if name in ("phiw", "pt"):
        i = _hit(rng, 2.8, 7, -20, 20)
        o = _hit(rng, 7.5, 16, -26, 26)
        return [i, o]
    if name == "zip":
        return [_hit(rng, 2.8, 7, -20, 20), _hit(rng, 7.5, 16, -26, 26)]
    if name in ("rz", "curv", "beamspot", "dz"):
        a = _hit(rng, 2.8, 3.2, -10, 10, phi_w=0.05)
        b = _hit(rng, 6.6, 7.0, a[2] * 2.2 - 3, a[2] * 2.2 + 3, phi_w=0.08)
        c = _hit(rng, 10.6, 11.2, a[2] * 3.7 - 5, a[2] * 3.7 + 5, phi_w=0.15)
        return [a, b, c]
    if name == "fb":
        hh = _hit(rng, 10, 11, -5, 5, phi_w=0.1)
        d = np.array([hh[0], hh[1], hh[2]]) * -0.4
        h1 = _snap(hh[:3] + d + rng.normal(0, 0.003, 3))
        h2 = _snap(hh[:3] + 1.1 * d + rng.normal(0, 0.003, 3))
        return [np.append(h1, _snap(np.hypot(*h1[:2]))), np.append(h2, _snap(np.hypot(*h2[:2]))), hh]
    raise KeyError(name)


_K_RANGE = dict(phiw=(1e-3, 0.05), zip=(2.0, 20.0), pt=(1e2, 1e5), rz=(1e-3, 30.0),
                curv=(1e2, 1e5), beamspot=(1e-4, 1e-1), dz=(0.02, 3.0), fb=(1e-7, 1e-4))


@pytest.mark.parametrize("name", list(_K_RANGE))
def test_predicate_meaning(name):
    rng = np.random.default_rng(20081346 + len(name))
    n_acc = n_rej = 0
    for _ in range(1500):
        h = _random_case(name, rng)
        lo, hi = _K_RANGE[name]
        k = float(F32(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        val, thr = _meaning(name, h)
        t = thr(k)
        if abs(val - t) <= 1e-9 * max(1.0, abs(t)):
            continue  # too close to call in float64
        want = val <= t
        got = oracle.pred(name, np.array(h, dtype=np.float32), k)
        assert got == want, (name, h, k, val, t)
        n_acc += want
        n_rej += not want
    assert n_acc > 50 and n_rej > 50, (n_acc, n_rej)


# ------------------------------------------------- graph vs brute force
def _small_event():
    cfg = dataclasses.replace(E.WORKLOADS["pu50-ttbar-like"], name="small", index=90, pileup=0, hard_tracks=0,
                              fixed_tracks=40, noise_frac=0.15)
    return E.make_batch(cfg)


def test_graph_stages_against_brute_force():
    b = _small_event()
    cuts = CU.cuts_for("pu50-ttbar-like")
    ml = G.module_layer_table()
    res = oracle.run(b, cuts, CU.FIT_PARAMS, ml, DISK, stage=3)
    lay = ml[b["module"]]
    H = np.stack([b["x"], b["y"], b["z"], b["r"]], 1).astype(np.float32)
    n = H.shape[0]
    # doublets
    cells = {}
    for p, pp in enumerate(cuts["pairs"]):
        for o in np.nonzero(lay == pp["outer"])[0]:
            for i in np.nonzero(lay == pp["inner"])[0]:
                if not (pp["zlo"] <= b["z"][i] <= pp["zhi"]):
                    continue
                hh = H[[i, o]]
                if (oracle.pred("zip", hh, pp["zmax"]) and oracle.pred("phiw", hh, pp["tan2_dphi"])
                        and oracle.pred("pt", hh, pp["k_pt"])):
                    cells[(int(i), int(o))] = p
    got = {(int(c[0]), int(c[1])): int(c[2]) for c in res["cells"]}
    assert got == cells
    # Fishbone by definition
    alive = {}
    for (i, o) in cells:
        dead = False
        for (j, o2) in cells:
            if o2 != o or j == i or lay[j] != lay[i]:
                continue
            if not oracle.pred("fb", H[[i, j, o]], cuts["fishbone_eps2"]):
                continue
            li = float(np.sum((H[i, :3].astype(np.float64) - H[o, :3]) ** 2))
            lj = float(np.sum((H[j, :3].astype(np.float64) - H[o, :3]) ** 2))
            if lj < li or (lj == li and j < i):
                dead = True
        alive[(i, o)] = not dead
    got_alive = {(int(c[0]), int(c[1])): bool(a) for c, a in zip(res["cells"], res["cell_alive"])}
    assert got_alive == alive
    live = {c for c, a in alive.items() if a}

    def ca_ok(a, bb, c):
        reg = cuts["region"][1 if lay[bb] >= 4 else 0]
        h3 = H[[a, bb, c]]
        return (oracle.pred("dz", h3, reg["zmax"]) and oracle.pred("rz", h3, reg["tol_rz2"])
                and oracle.pred("curv", h3, reg["k_curv"]) and oracle.pred("beamspot", h3, reg["rmax2"]))

    edges = {(a, bb, c) for (a, bb) in live for (b2, c) in live if b2 == bb and ca_ok(a, bb, c)}
    C = res["cells"]
    got_edges = {(int(C[e0][0]), int(C[e0][1]), int(C[e1][1])) for e0, e1 in res["edges"]}
    assert got_edges == edges
    # maximal paths from roots by enumeration of hit sequences
    nxt = {}
    for (a, bb, c) in edges:
        nxt.setdefault((a, bb), []).append(c)
    has_in = {(bb, c) for (a, bb, c) in edges}
    paths = set()

    def extend(seq):
        ext = nxt.get((seq[-2], seq[-1]), [])
        if not ext or len(seq) == oracle.NMAX:
            if len(seq) >= 3:
                paths.add(tuple(int(v) for v in seq))
            if not ext:
                return
            return
        for c in ext:
            extend(seq + [c])

    for (a, bb) in live:
        root = lay[a] == 0 or (lay[a] in (1, 4, 7) and (a, bb) not in has_in)
        if root:
            extend([a, bb])
    got_paths = {tuple(int(v) for v in res["tuple_hits"][t, :res["tuple_n"][t]])
                 for t in range(len(res["tuple_n"]))}
    assert got_paths == paths
    assert len(paths) > 10
    # shared-doublet cleaning by definition
    best = {}
    for p in paths:
        for q in range(len(p) - 1):
            best[p[q:q + 2]] = max(best.get(p[q:q + 2], 0), len(p))
    keep = {p for p in paths if all(len(p) >= best[p[q:q + 2]] for q in range(len(p) - 1))}
    got_keep = {tuple(int(v) for v in res["tuple_hits"][t, :res["tuple_n"][t]])
                for t in range(len(res["tuple_n"])) if res["tuple_alive"][t]}
    assert got_keep == keep


def test_cleaning_keeps_only_the_quadruplet():
    """A lone barrel track crossing all four layers yields the quadruplet
    B1B2B3B4 and, through the skip pairs, the triplets B1B3B4 and B1B2B4, which
    share a cell with it; only the quadruplet survives (Sec. 3.3)."""
    cfg = dataclasses.replace(E.WORKLOADS["barrel-50-helices"], name="one", index=91, fixed_tracks=1, eta_max=0.3,
                              pt_min=5.0, pt_max=6.0)
    b = E.make_batch(cfg)
    assert b["x"].size == 4
    res = oracle.run(b, CU.cuts_for("barrel-50-helices"), CU.FIT_PARAMS, G.module_layer_table(), DISK, stage=3)
    lay = G.module_layer_table()[b["module"]]
    seqs = sorted(tuple(int(lay[h]) for h in res["tuple_hits"][t, :res["tuple_n"][t]])
                  for t in range(len(res["tuple_n"])))
    assert seqs == [(0, 1, 2, 3), (0, 1, 3), (0, 2, 3)]
    alive = [tuple(int(lay[h]) for h in res["tuple_hits"][t, :res["tuple_n"][t]])
             for t in range(len(res["tuple_n"])) if res["tuple_alive"][t]]
    assert alive == [(0, 1, 2, 3)]


def test_full_finding_on_noiseless_helices():
    """50 noiseless barrel helices: every generated track leaving >= 3 hits
    is found exactly once as a tuple holding all its hits; no surviving tuple
    mixes tracks."""
    b = E.make_batch("barrel-50-helices")
    res = oracle.run(b, CU.cuts_for("barrel-50-helices"), CU.FIT_PARAMS, G.module_layer_table(), DISK, stage=4)
    tid = b["track"]
    counts = np.bincount(tid[tid >= 0], minlength=b["trk_pt"].size)
    want = {t for t in range(counts.size) if counts[t] >= 3}
    found = {}
    for t in res["track_tuple"]:
        hits = res["tuple_hits"][t, :res["tuple_n"][t]]
        ids = set(tid[hits].tolist())
        assert len(ids) == 1 and -1 not in ids, "fake track"
        (k,) = ids
        assert res["tuple_n"][t] == counts[k], "track found without all its hits"
        found[k] = found.get(k, 0) + 1
    assert set(found) == want
    assert all(v == 1 for v in found.values()), "duplicates"
    assert len(want) >= 30


# ------------------------------------------------------------------ fit
def _helix_points(kappa, phi0, tanl, d0, z0, s_list):
    """Points of the exact helix with perigee parameters (kappa = q/rho,
    positive bending clockwise; PCA = d0 (sin phi0, -cos phi0))."""
    k = -kappa
    px, py = d0 * math.sin(phi0), -d0 * math.cos(phi0)
    out = []
    for s in s_list:
        h = 0.5 * k * s
        f = s * (math.sin(h) / h if h != 0 else 1.0)
        out.append((px + f * math.cos(phi0 + h), py + f * math.sin(phi0 + h), z0 + s * tanl))
    return np.array(out)


@pytest.mark.parametrize("kappa", [1 / 30.0, -1 / 45.0, 1 / 400.0, -1 / 8000.0])
@pytest.mark.parametrize("n", [3, 4, 5])
def test_fit_exact_helix(kappa, n):
    phi0, tanl, d0, z0 = 0.7, 1.3, 0.004, -2.5
    s = [3.0, 6.9, 11.0, 15.5, 19.0][:n]
    P = _helix_points(kappa, phi0, tanl, d0, z0, s)
    disk = [0, 0, 1, 1, 1][:n]
    p, cov, chi2, ndf, ex = oracle.fit(P[:, 0], P[:, 1], P[:, 2], disk, CU.FIT_PARAMS)
    assert ndf == 2 * n - 5
    assert chi2 < 1e-12
    assert abs(p[0] - kappa) <= 1e-9 * abs(kappa)
    assert abs(p[1] - phi0) < 1e-10 and abs(p[2] - tanl) < 1e-10
    assert abs(p[3] - d0) < 1e-10 and abs(p[4] - z0) < 1e-10
    # covariance diagonal positive
    diag = cov[[0, 2, 5, 9, 14]]
    assert np.all(diag > 0)


def test_fit_rigid_limit_is_least_squares():
    """With scattering almost switched off the s-z line fit is the weighted
    straight-line regression of z on s and the circle fit is the weighted
    parabola fit of the offsets, whose second coefficient is dk/2.  The
    scattering variance is scaled by 1e-8: the broken line then departs from
    the rigid solution by ~1e-7 of the measurement weight ratio while the
    normal matrix (condition ~1e6 w.r.t. the measurement scale) stays well
    inside double precision; at 1e-12 the condition number reaches 1e12 and
    rounding, not the model, dominates."""
    rng = np.random.default_rng(7)
    s = np.array([3.0, 6.9, 11.0, 15.5, 19.0])
    P = _helix_points(1 / 60.0, 0.2, 0.8, 0.0, 1.0, s)
    P[:, 2] += rng.normal(0, 20e-4, 5)
    nrm = np.stack([-np.sin(0.2 + 0 * s), np.cos(0.2 + 0 * s)], 1)
    P[:, :2] += rng.normal(0, 10e-4, (5, 1)) * nrm
    p, cov, chi2, ndf, ex = oracle.fit(P[:, 0], P[:, 1], P[:, 2], [0] * 5, CU.FIT_PARAMS, ms_scale=1e-8)
    # arc lengths and offsets as the fit defines them (prefit through 0, 2, 4)
    k0, psi0 = ex[2], ex[3]
    d = P[:, :2] - P[0, :2]
    dist = np.hypot(d[:, 0], d[:, 1])
    sx = np.where(dist > 0, 2 * np.arcsin(np.clip(k0 * dist / 2, -1, 1)) / np.where(k0 != 0, k0, 1), 0)
    t = np.array([math.cos(psi0), math.sin(psi0)])
    nn = np.array([-t[1], t[0]])
    X, Y = d @ t, d @ nn
    U = k0 * (X * X + Y * Y) - 2 * Y
    m = -U / (1 + np.sqrt(1 + k0 * U))
    slope, icpt = np.polyfit(sx, P[:, 2], 1)          # equal weights (all barrel)
    assert abs(p[2] - slope) < 1e-8
    c2, c1, c0 = np.polyfit(sx, m, 2)
    assert abs(ex[5] - 2 * c2) < 1e-10
    res_line = P[:, 2] - (slope * sx + icpt)
    res_circ = m - np.polyval([c2, c1, c0], sx)
    want = np.sum(res_line ** 2) / (20e-4) ** 2 + np.sum(res_circ ** 2) / (10e-4) ** 2
    assert abs(chi2 - want) < 1e-3 * want + 1e-6
    # the line block of the covariance is the regression's: var(slope) =
    # sigma^2 / Sxx, var(icpt) = sigma^2 (1/n + mean^2 / Sxx), cov = -sigma^2
    # mean / Sxx, carried to z0 = icpt + slope * arc (arc to the perigee)
    sig2, n = (20e-4) ** 2, len(sx)
    sxx = np.sum((sx - sx.mean()) ** 2)
    v_sl, v_ic, c_si = sig2 / sxx, sig2 * (1 / n + sx.mean() ** 2 / sxx), -sig2 * sx.mean() / sxx
    # (the residual scattering, 1e-8 of nominal, adds ~5e-6 relative)
    arc = ex[6]
    assert abs(cov[5] - v_sl) < 2e-5 * v_sl                                   # (tan lambda, tan lambda)
    assert abs(cov[12] - (c_si + arc * v_sl)) < 2e-5 * v_ic                    # (z0, tan lambda)
    assert abs(cov[14] - (v_ic + 2 * arc * c_si + arc ** 2 * v_sl)) < 2e-5 * v_ic   # (z0, z0)
    # and the curvature's variance is the parabola's: kappa = -(k0 + dk),
    # dk = 2 c2, var(c2) from (X^T X)^-1 sigma_rphi^2 with X = [1, s, s^2]
    Xp = np.stack([np.ones_like(sx), sx, sx * sx], 1)
    v_c2 = np.linalg.inv(Xp.T @ Xp)[2, 2] * (10e-4) ** 2
    assert abs(cov[0] - 4 * v_c2) < 2e-5 * 4 * v_c2                         # (kappa, kappa)


def test_fit_three_hits_has_zero_circle_chi2():
    P = _helix_points(1 / 50.0, -1.0, 0.3, 0.01, 0.5, [3.0, 7.0, 11.0])
    P[:, :2] += np.array([[1e-3, -2e-3], [0, 1e-3], [-1e-3, 0]])
    _, _, chi2, ndf, ex = oracle.fit(P[:, 0], P[:, 1], P[:, 2], [0, 0, 0], CU.FIT_PARAMS)
    assert ndf == 1
    assert abs(ex[1]) < 1e-9


def test_fit_pulls_on_scattered_tracks():
    """Tracks simulated with scattering kinks at inner hits: residuals of the
    fitted parameters divided by their fitted errors are N(0,1) and chi2
    averages ndf (tracks matched to one simulated particle)."""
    cfg = dataclasses.replace(E.WORKLOADS["pu50-ttbar-like"], ms_skip_first=True, noise_frac=0.0, overlaps=False)
    b = E.make_batch(cfg)
    res = oracle.run(b, CU.cuts_for("pu50-ttbar-like"), CU.FIT_PARAMS, G.module_layer_table(), DISK, stage=4)
    tt = res["track_tuple"]
    n = res["tuple_n"][tt]
    Hh = res["tuple_hits"][tt]
    tid = b["track"]
    per_track = np.bincount(tid[tid >= 0], minlength=b["trk_pt"].size)
    # tuples made of all the hits of one simulated particle (a tuple that
    # skips one of its hits would put an unmodelled kink in a segment)
    match = np.array([tid[Hh[i, 0]] if (np.all(tid[Hh[i, :n[i]]] == tid[Hh[i, 0]])
                                        and per_track[tid[Hh[i, 0]]] == n[i]) else -1
                      for i in range(len(tt))])
    g = match >= 0
    assert g.sum() > 1000
    P, cv, mt = res["params"][g], res["cov"][g], match[g]
    q, pt, eta, phi = b["trk_q"][mt], b["trk_pt"][mt], b["trk_eta"][mt], b["trk_phi"][mt]
    vtx = b["trk_vertex"][mt]
    tanl = np.sinh(eta)
    arc = -(vtx[:, 0] * np.cos(phi) + vtx[:, 1] * np.sin(phi))
    truth = [q / E.rho_of_pt(pt), phi, tanl, vtx[:, 0] * np.sin(phi) - vtx[:, 1] * np.cos(phi),
             vtx[:, 2] + tanl * arc]
    var = cv[:, [0, 2, 5, 9, 14]]
    for j in range(5):
        d = P[:, j] - truth[j]
        if j == 1:
            d = (d + np.pi) % (2 * np.pi) - np.pi
        pull = d / np.sqrt(var[:, j])
        assert abs(np.mean(pull)) < 0.1, j
        assert 0.9 < np.std(pull) < 1.15, (j, np.std(pull))
    c2 = res["chi2"][g] / res["ndf"][g]
    assert 0.85 < np.mean(res["chi2"][g]) / np.mean(res["ndf"][g]) < 1.15, np.mean(c2)


# ------------------------------------------------------ fit gradient
def _smeared_helix(rng, n):
    kappa = rng.choice([1, -1]) / rng.uniform(40.0, 3000.0)
    s = np.cumsum(rng.uniform(3.0, 5.0, n))
    P = _helix_points(kappa, rng.uniform(-3, 3), rng.uniform(-2.0, 2.0), rng.normal(0, 0.01),
                      rng.normal(0, 3.0), s)
    P[:, :2] += rng.normal(0, 10e-4, (n, 2))
    P[:, 2] += rng.normal(0, 20e-4, n)
    disk = list((rng.uniform(size=n) < 0.3).astype(int))
    return P, disk


def test_fit_gradient_sum_rules():
    """The fit commutes with a translation of all hits along z (z0 moves by
    the shift, the other parameters and chi2 stay) and with a rotation about
    the beam line (phi0 turns by the angle, the rest stays), so the gradient
    with respect to the hits obeys exact sum rules: sum_i dF/dz_i = [F = z0]
    and sum_i (x_i dF/dy_i - y_i dF/dx_i) = [F = phi0].  Checked on the
    oracle's float64 finite-difference gradient for smeared helices of 3, 4
    and 5 hits (barrel and disk hits mixed)."""
    rng = np.random.default_rng(11)
    for n in (3, 4, 5, 5):
        P, disk = _smeared_helix(rng, n)
        for o in range(6):
            gp = np.zeros(5)
            gc = 0.0
            if o < 5:
                gp[o] = 1.0
            else:
                gc = 1.0
            Gr = oracle.fit_grad_fd(P[:, 0], P[:, 1], P[:, 2], disk, CU.FIT_PARAMS, gp, gc)
            sz = Gr[2].sum()
            rot = float(np.sum(P[:, 0] * Gr[1] - P[:, 1] * Gr[0]))
            scale = 1.0 + np.abs(Gr).sum()
            assert abs(sz - (1.0 if o == 4 else 0.0)) < 1e-7 * scale, (n, o, sz)
            assert abs(rot - (1.0 if o == 1 else 0.0)) < 1e-7 * scale, (n, o, rot)


def test_fit_gradient_rigid_limit_is_the_regression_hat_matrix():
    """With scattering almost off, the s-z line fit of barrel hits is the
    straight-line regression of z on the arc lengths s (which depend on x and
    y only), so its z-gradients have closed forms: d tanl/dz_i = (s_i - m)/Sxx,
    d icpt/dz_i = 1/n - m (s_i - m)/Sxx, z0 = icpt + tanl * arc, and
    d chi2/dz_i = 2 r_i / sigma_z^2 with r_i the regression residual (the
    minimum's own gradient, parameters held).  Every hit's entry is checked,
    so a wrong index, sign or dropped term in the oracle's gradient fails.
    The step is 2e-3 cm: the fit is linear in z except through the first and
    last hits' pre-fit dip, which sets the (tiny) scattering variances, and
    with them 1e12-sized entries of the normal matrix whose rounding a
    2e-5 cm difference would amplify at those two hits."""
    rng = np.random.default_rng(5)
    s = np.array([3.0, 6.9, 11.0, 15.5, 19.0])
    P = _helix_points(-1 / 80.0, -0.9, -0.6, 0.0, 2.0, s)
    P[:, 2] += rng.normal(0, 20e-4, 5)
    nrm = np.stack([-np.sin(-0.9 + 0 * s), np.cos(-0.9 + 0 * s)], 1)
    P[:, :2] += rng.normal(0, 10e-4, (5, 1)) * nrm
    _, _, _, _, ex = oracle.fit(P[:, 0], P[:, 1], P[:, 2], [0] * 5, CU.FIT_PARAMS, ms_scale=1e-8)
    k0 = ex[2]
    d = P[:, :2] - P[0, :2]
    dist = np.hypot(d[:, 0], d[:, 1])
    sx = np.where(dist > 0, 2 * np.arcsin(np.clip(k0 * dist / 2, -1, 1)) / np.where(k0 != 0, k0, 1), 0)
    n, m = len(sx), sx.mean()
    sxx = np.sum((sx - m) ** 2)
    d_slope = (sx - m) / sxx
    d_icpt = 1.0 / n - m * d_slope
    slope, icpt = np.polyfit(sx, P[:, 2], 1)
    resid = P[:, 2] - (slope * sx + icpt)
    arc = ex[6]
    want = {2: d_slope, 4: d_icpt + arc * d_slope, "chi2": 2 * resid / (20e-4) ** 2}
    for o, w in want.items():
        gp = np.zeros(5)
        if o != "chi2":
            gp[o] = 1.0
        Gr = oracle.fit_grad_fd(P[:, 0], P[:, 1], P[:, 2], [0] * 5, CU.FIT_PARAMS, gp,
                                1.0 if o == "chi2" else 0.0, h=2e-3, ms_scale=1e-8)
        assert np.abs(Gr[2] - w).max() < 1e-4 * np.abs(w).max(), (o, Gr[2], w)


def _circumcentre(a, b, c):
    d = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux = ((a @ a) * (b[1] - c[1]) + (b @ b) * (c[1] - a[1]) + (c @ c) * (a[1] - b[1])) / d
    uy = ((a @ a) * (c[0] - b[0]) + (b @ b) * (a[0] - c[0]) + (c @ c) * (b[0] - a[0])) / d
    return np.array([ux, uy])


@pytest.mark.parametrize("kappa,n,tol", [(1 / 1000.0, 5, 1e-4), (-1 / 1000.0, 4, 1e-4), (1 / 2000.0, 3, 1e-4),
                                         (-1 / 60.0, 3, 1e-2), (1 / 60.0, 5, 1e-2)])
def test_fit_circle_covariance_is_the_propagated_measurement_error(kappa, n, tol):
    """In the rigid limit the transverse parameters (kappa, phi0, d0) are a
    function of the hits' offsets across the track, each measured with
    sigma_rphi, so their covariance must equal sigma_rphi^2 sum_i g_i g_i^T,
    g_i the derivative of the parameters with respect to a move of hit i
    along the pre-fit circle's normal (the oracle's gradient, projected).
    This ties the fit's covariance (inverse normal matrix carried to the
    perigee) to the estimator it describes, entry by entry, including the
    phi0 and d0 rows.  The broken line is a small-angle model of the arc, so
    the two agree to O((kappa s)^2): 1e-4 for stiff tracks, 1e-2 at a 60 cm
    radius (measured 2e-5 and 6e-3), both far below what a wrong sign,
    index or dropped term would give."""
    rng = np.random.default_rng(3)
    s = np.array([3.0, 6.9, 11.0, 15.5, 19.0])[:n]
    P = _helix_points(kappa, 0.5, 0.7, 0.003, 1.0, s)
    P[:, :2] += rng.normal(0, 10e-4, (n, 2))
    P[:, 2] += rng.normal(0, 20e-4, n)
    _, cov, _, _, _ = oracle.fit(P[:, 0], P[:, 1], P[:, 2], [0] * n, CU.FIT_PARAMS, ms_scale=1e-8)
    nrm = P[:, :2] - _circumcentre(P[0, :2], P[n // 2, :2], P[-1, :2])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    idx = (0, 1, 3)                                     # kappa, phi0, d0
    g = []
    for j in idx:
        gp = np.zeros(5)
        gp[j] = 1.0
        Gr = oracle.fit_grad_fd(P[:, 0], P[:, 1], P[:, 2], [0] * n, CU.FIT_PARAMS, gp, 0.0, h=2e-3,
                                ms_scale=1e-8)
        g.append(Gr[0] * nrm[:, 0] + Gr[1] * nrm[:, 1])
    g = np.array(g)
    want = (10e-4) ** 2 * g @ g.T

    def packed(r, c):                                   # lower triangle of the 5x5, row by row
        r, c = max(r, c), min(r, c)
        return cov[r * (r + 1) // 2 + c]

    for a, i in enumerate(idx):
        for b, j in enumerate(idx):
            scale = math.sqrt(packed(i, i) * packed(j, j))
            assert abs(packed(i, j) - want[a, b]) <= tol * scale, (i, j, packed(i, j), want[a, b])


def test_fit_gradient_of_chi2_vanishes_on_exact_helices():
    """chi2 is zero, its minimum, on the hits of an exact helix, so its
    gradient with respect to the hits vanishes there."""
    P = _helix_points(1 / 60.0, 0.4, 0.8, 0.002, 1.0, [3.0, 7.0, 11.0, 15.5])
    Gr = oracle.fit_grad_fd(P[:, 0], P[:, 1], P[:, 2], [0, 0, 0, 0], CU.FIT_PARAMS, np.zeros(5), 1.0)
    assert np.abs(Gr).max() < 1e-3


def test_condition_numbers_match_the_library_eigenvalues():
    """The oracle's Jacobi condition number against numpy's singular values,
    on symmetric positive definite matrices up to 9 x 9 spanning 1 to 1e12."""
    rng = np.random.default_rng(3)
    assert abs(oracle.sym_condition(np.diag([2.0, 8.0, 0.5])) - 16.0) < 1e-12
    for n in range(2, 10):
        for decades in (0, 4, 8, 12):
            Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
            lam = np.logspace(0, decades, n)
            M = (Q * lam) @ Q.T
            M = 0.5 * (M + M.T)
            want = np.linalg.cond(M)
            got = oracle.sym_condition(M)
            # the smallest eigenvalue carries an error of ~1e-16 lambda_max on
            # either side: relative error up to ~1e-16 cond
            assert abs(got - want) <= (1e-9 + 1e-13 * want) * want, (n, decades, got, want)


def test_fit_reports_the_condition_of_its_normal_matrices():
    P = _helix_points(1 / 200.0, 0.3, 0.5, 0.001, 1.0, [3.0, 6.9, 11.0, 15.5])
    ex = oracle.fit(P[:, 0], P[:, 1], P[:, 2], [0, 0, 0, 0], CU.FIT_PARAMS)[4]
    assert len(ex) == 10 and ex[8] >= 1.0 and ex[9] >= 1.0 and np.isfinite(ex[8:]).all()


# ------------------------------------------------------------- alignment
def test_alignment_moves_each_module_rigidly_to_first_order():
    """The oracle's per-module alignment: no correction leaves the hits in
    place; a shift moves exactly the hits of its module by it; a small
    rotation turns a module's hits about its centre, equal to the exact
    rotation matrix up to second order in the angle."""
    rng = np.random.default_rng(11)
    n, nm = 400, 5
    centres = rng.normal(size=(nm, 3)) * 5.0
    module = rng.integers(0, nm, size=n)
    P = centres[module] + rng.normal(size=(n, 3)) * 2.0
    zero = np.zeros((nm, 3))
    got = np.stack(oracle.align_hits(P[:, 0], P[:, 1], P[:, 2], module, centres, zero, zero), 1)
    assert np.array_equal(got, P)
    shift = zero.copy()
    shift[2] = (1e-3, -2e-3, 5e-4)
    got = np.stack(oracle.align_hits(P[:, 0], P[:, 1], P[:, 2], module, centres, shift, zero), 1)
    on = module == 2
    assert np.allclose(got[on] - P[on], shift[2], atol=1e-15) and np.array_equal(got[~on], P[~on])
    axis = np.array([0.3, -0.5, 0.8])
    axis /= np.linalg.norm(axis)
    theta = 1e-4
    rot = zero.copy()
    rot[3] = theta * axis
    got = np.stack(oracle.align_hits(P[:, 0], P[:, 1], P[:, 2], module, centres, zero, rot), 1)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + math.sin(theta) * K + (1 - math.cos(theta)) * K @ K          # Rodrigues
    on = module == 3
    exact = centres[3] + (P[on] - centres[3]) @ R.T
    r = np.linalg.norm(P[on] - centres[3], axis=1)
    assert np.all(np.linalg.norm(got[on] - exact, axis=1) <= theta ** 2 * r + 1e-14)
    assert np.array_equal(got[~on], P[~on])


def test_plain_central_differences_agree_with_the_extrapolated_gradient():
    """The plain central differences at the 1e-4 cm step agree with the
    Richardson-extrapolated gradient to the step's O(h^2) error (here
    ~3e-5 of the largest component: the fit bends on the scale of the hit
    resolution, tens of um), and halving the step divides the departure
    by about four."""
    b = E.make_batch("barrel-50-helices")
    lay = G.module_layer_table()[b["module"]]
    idx = np.nonzero(b["track"] == 3)[0]
    idx = idx[np.argsort(b["r"][idx])]
    gp = np.array([1e-3, 1e-3, 1e-3, 1e-2, 1e-2])
    args = (b["x"][idx], b["y"][idx], b["z"][idx], (lay[idx] >= 4).astype(int), CU.FIT_PARAMS, gp, 0.3)
    a = oracle.fit_grad_central(*args, h=1e-4)
    ref = oracle.fit_grad_fd(*args)
    e1 = np.abs(a - ref).max()
    assert e1 <= 1e-4 * np.abs(ref).max()
    e2 = np.abs(oracle.fit_grad_central(*args, h=5e-5) - ref).max()
    assert 3.0 < e1 / e2 < 5.0

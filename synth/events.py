"""Seeded synthetic pixel events (input data shared by the oracle, the CUDA
path, the tests and the benchmark).  Holds no arithmetic of the seeding or
fitting method: it only simulates charged helices crossing the detector of
``synth.geometry`` and writes the hits they leave.

Physics of the simulation (a stand-in for the CMS Open Data ttbar sample of
Sec. 4.1, which is not available here):
  * vertices: z ~ N(0, 3.5 cm), x, y ~ N(0, 15 um); pileup vertices carry
    Poisson(30) tracks; an optional hard vertex carries Poisson(60) harder ones;
  * pT from a 1/pT^2 spectrum on [pt_min, 100] GeV (or log-uniform), eta
    uniform in [-eta_max, eta_max], phi uniform, charge +-1;
  * helices in B = 3.8 T along +z, stepped surface to surface; at every module
    crossing an optional Gaussian multiple-scattering kink (Highland width,
    x/X0 = 0.02 per barrel module, 0.03 per disk module, divided by the cosine
    of the incidence angle); loopers stop after half a turn;
  * hit smear 10 um in r-phi and 20 um in z (barrel) or r (disks);
  * every coordinate snapped to the grid g = 2^-14 cm and stored as float32;
    r is the snapped sqrt(x^2 + y^2), given as data;
  * optional uniform noise hits and per-hit inefficiency.

Hits are shuffled within each event.  Seeds: event e of configuration k uses
numpy PCG64 seeded with 2008134610 + 1000 k + e.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import geometry as G

GRID = 2.0 ** -14            # cm
BZ_TESLA = 3.8
C_LIGHT = 0.299792458        # GeV / (T m)
SIGMA_RPHI = 10e-4           # cm
SIGMA_Z = 20e-4              # cm (barrel z, disk r)
X0_BARREL = 0.02
X0_DISK = 0.03
SEED_BASE = 2008134610


def rho_of_pt(pt_gev, bz=BZ_TESLA):
    """Radius of curvature in cm for transverse momentum pt (GeV)."""
    return np.asarray(pt_gev) / (C_LIGHT * bz) * 100.0


@dataclasses.dataclass(frozen=True)
class EventConfig:
    name: str
    index: int                      # seeds the workload's events
    n_events: int
    pileup: float                   # mean number of pileup vertices
    pileup_poisson: bool
    tracks_per_vertex: float = 30.0
    hard_tracks: float = 0.0        # mean tracks of an extra hard vertex (0: none)
    pt_min: float = 0.5
    pt_max: float = 100.0
    pt_spectrum: str = "inv2"       # "inv2" or "loguniform"
    eta_max: float = 2.5
    barrel_only: bool = False
    overlaps: bool = True
    noise_frac: float = 0.0
    ineff: float = 0.0
    multiple_scattering: bool = True
    vertex_at_origin: bool = False
    fixed_tracks: int = 0           # >0: exactly this many tracks, one vertex
    ms_skip_first: bool = False     # no scattering at a track's first hit


# the synthetic workloads by name; each index only seeds its events
WORKLOADS = {c.name: c for c in (
    EventConfig("barrel-50-helices", 1, 1, 0, False, pt_min=1.0, pt_max=10.0,
                pt_spectrum="loguniform", eta_max=2.0, barrel_only=True,
                overlaps=False, multiple_scattering=False, vertex_at_origin=True,
                fixed_tracks=50),
    EventConfig("pu50-ttbar-like", 2, 1, 50, False, hard_tracks=60.0, noise_frac=0.02),
    EventConfig("pu200-batch64", 3, 64, 200, True, hard_tracks=60.0, noise_frac=0.02),
    EventConfig("pu50-batch32", 4, 32, 50, False, hard_tracks=60.0, noise_frac=0.02),
    EventConfig("pu200-stress-batch256", 5, 256, 200, True, hard_tracks=60.0,
                pt_min=0.3, noise_frac=0.05, ineff=0.10),
)}


def snap(v):
    return (np.rint(np.asarray(v, dtype=np.float64) / GRID) * GRID)


# ------------------------------------------------------------------ tracks
def _draw_tracks(cfg: EventConfig, rng: np.random.Generator):
    if cfg.fixed_tracks:
        nv = 1
        ntrk = np.array([cfg.fixed_tracks])
        hard = np.array([False])
    else:
        nv = rng.poisson(cfg.pileup) if cfg.pileup_poisson else int(cfg.pileup)
        ntrk = rng.poisson(cfg.tracks_per_vertex, size=nv)
        hard = np.zeros(nv, dtype=bool)
        if cfg.hard_tracks > 0:
            ntrk = np.concatenate([[rng.poisson(cfg.hard_tracks)], ntrk])
            hard = np.concatenate([[True], hard])
            nv += 1
    if cfg.vertex_at_origin:
        vtx = np.zeros((nv, 3))
    else:
        vtx = np.stack([rng.normal(0, 15e-4, nv), rng.normal(0, 15e-4, nv),
                        rng.normal(0, 3.5, nv)], axis=1)
    vid = np.repeat(np.arange(nv), ntrk)
    n = int(ntrk.sum())
    u = rng.random(n)
    if cfg.pt_spectrum == "loguniform":
        pt = np.exp(np.log(cfg.pt_min) + u * (np.log(cfg.pt_max) - np.log(cfg.pt_min)))
    else:
        pmin = np.where(hard[vid], max(1.0, cfg.pt_min), cfg.pt_min)
        pt = pmin / (1.0 - u * (1.0 - pmin / cfg.pt_max))
    eta = rng.uniform(-cfg.eta_max, cfg.eta_max, n)
    phi = rng.uniform(-math.pi, math.pi, n)
    q = rng.choice(np.array([-1.0, 1.0]), n)
    return dict(vertex=vtx, vid=vid, pt=pt, eta=eta, phi=phi, q=q)


# ------------------------------------------------------------- propagation
def _sinc(x):
    out = np.ones_like(x)
    m = np.abs(x) > 1e-8
    out[m] = np.sin(x[m]) / x[m]
    return out


def _pos(x0, y0, phi, k, s):
    """Position after transverse arc length s on a circle of signed (left
    turning positive) curvature k starting at (x0, y0) with direction phi."""
    h = 0.5 * k * s
    f = s * _sinc(h)
    return x0 + f * np.cos(phi + h), y0 + f * np.sin(phi + h)


def _asinc(x):
    out = np.ones_like(x)
    m = np.abs(x) > 1e-8
    out[m] = np.arcsin(np.clip(x[m], -1, 1)) / x[m]
    return out


def _cyl_crossing(x0, y0, phi, k, R):
    """Smallest s > 0 with |p(s)| = R on the outgoing branch, or nan."""
    r0 = np.hypot(x0, y0)
    ak = np.abs(k)
    reach = 0.5 * R * ak <= 1.0
    arc = lambda r: r * _asinc(np.minimum(0.5 * r * ak, 1.0))
    s = np.where(reach, arc(R) - arc(r0), np.nan)
    for _ in range(12):
        xs, ys = _pos(x0, y0, phi, k, s)
        f = xs * xs + ys * ys - R * R
        ang = phi + k * s
        fp = 2.0 * (xs * np.cos(ang) + ys * np.sin(ang))
        fp = np.where(np.abs(fp) < 1e-12, np.nan, fp)
        s = s - f / fp
    xs, ys = _pos(x0, y0, phi, k, s)
    ang = phi + k * s
    ok = (np.abs(xs * xs + ys * ys - R * R) < 1e-9 * R * R) & (s > 1e-7) & \
         ((xs * np.cos(ang) + ys * np.sin(ang)) > 0) & (r0 < R)
    return np.where(ok, s, np.nan)


def _surfaces(cfg: EventConfig):
    """List of (layer, kind, value, parity): kind 0 = cylinder radius value,
    kind 1 = plane at z = value.  parity selects which alternate modules sit
    on that surface (-1: all modules, no overlaps)."""
    out = []
    for L, r in enumerate(G.BARREL_R):
        if cfg.overlaps:
            out.append((L, 0, r - G.BARREL_DR, 0))
            out.append((L, 0, r + G.BARREL_DR, 1))
        else:
            out.append((L, 0, r, -1))
    if not cfg.barrel_only:
        for side, base in ((+1, 4), (-1, 7)):
            for d, z in enumerate(G.DISK_Z):
                if cfg.overlaps:
                    out.append((base + d, 1, side * (z - G.DISK_DZ), 0))
                    out.append((base + d, 1, side * (z + G.DISK_DZ), 1))
                else:
                    out.append((base + d, 1, side * z, -1))
    return out


def _highland(p, xx0):
    return 0.0136 / p * np.sqrt(xx0) * (1.0 + 0.038 * np.log(xx0))


def _simulate(cfg: EventConfig, trk, rng):
    """Propagate all tracks; return hit arrays (x, y, z, layer, module, tid)."""
    n = trk["pt"].size
    vtx = trk["vertex"][trk["vid"]]
    x, y, z = vtx[:, 0].copy(), vtx[:, 1].copy(), vtx[:, 2].copy()
    phi = trk["phi"].copy()
    tanl = np.sinh(trk["eta"])
    p = trk["pt"] * np.cosh(trk["eta"])
    q = trk["q"]
    k = -q / rho_of_pt(trk["pt"])
    turned = np.zeros(n)
    surfs = _surfaces(cfg)
    done = np.zeros((n, len(surfs)), dtype=bool)
    alive = np.ones(n, dtype=bool)
    nhit = np.zeros(n, dtype=np.int64)
    hx, hy, hz, hl, hm, ht = [], [], [], [], [], []
    for _step in range(len(surfs)):
        best = np.full(n, np.inf)
        which = np.full(n, -1)
        for j, (L, kind, val, par) in enumerate(surfs):
            if kind == 0:
                s = _cyl_crossing(x, y, phi, k, val)
            else:
                with np.errstate(divide="ignore", invalid="ignore"):
                    s = (val - z) / tanl
                s = np.where(s > 1e-7, s, np.nan)
            s = np.where(done[:, j] | ~alive, np.nan, s)
            better = np.isfinite(s) & (s < best)
            best = np.where(better, s, best)
            which = np.where(better, j, which)
        go = which >= 0
        # stop loopers after half a turn
        go &= (turned + np.abs(k) * np.where(go, best, 0)) <= math.pi
        if not go.any():
            break
        idx = np.nonzero(go)[0]
        s = best[idx]
        nx, ny = _pos(x[idx], y[idx], phi[idx], k[idx], s)
        nz = z[idx] + s * tanl[idx]
        x[idx], y[idx], z[idx] = nx, ny, nz
        phi[idx] = phi[idx] + k[idx] * s
        turned[idx] += np.abs(k[idx]) * s
        w = which[idx]
        done[idx, w] = True
        alive &= ~(~go & (which >= 0))   # a track that could not go on stops
        # acceptance per surface
        for j in np.unique(w):
            L, kind, val, par = surfs[j]
            m = idx[w == j]
            px, py, pz = x[m], y[m], z[m]
            hphi = np.arctan2(py, px)
            if kind == 0:
                nl = G.BARREL_LADDERS[L]
                inz = np.abs(pz) < G.BARREL_HALF_Z
                if par < 0:
                    wlad = 2 * math.pi / nl
                    lad = np.floor(np.mod(hphi, 2 * math.pi) / wlad).astype(np.int64) % nl
                    cov = np.ones(m.size, dtype=bool)
                else:
                    cov, lad = G.covering_module(hphi, nl, par)
                acc = inz & cov
                mod = G.barrel_module_id(L, lad, pz)
                # incidence: normal is radial
                r = np.hypot(px, py)
                cosl = 1.0 / np.sqrt(1.0 + tanl[m] ** 2)
                cos_a = np.abs(cosl * (np.cos(phi[m]) * px + np.sin(phi[m]) * py) / r)
                xx0 = X0_BARREL / np.maximum(cos_a, 1e-3)
            else:
                r = np.hypot(px, py)
                ring = (r >= G.DISK_RING_SPLIT).astype(np.int64)
                nm = np.where(ring == 0, G.DISK_RING_MODULES[0], G.DISK_RING_MODULES[1])
                inr = (r >= G.DISK_RMIN) & (r <= G.DISK_RMAX)
                kk = np.zeros(m.size, dtype=np.int64)
                cov = np.zeros(m.size, dtype=bool)
                for ri in (0, 1):
                    sel = ring == ri
                    if not sel.any():
                        continue
                    nmod = G.DISK_RING_MODULES[ri]
                    if par < 0:
                        wm = 2 * math.pi / nmod
                        kk[sel] = np.floor(np.mod(hphi[sel], 2 * math.pi) / wm).astype(np.int64) % nmod
                        cov[sel] = True
                    else:
                        c, kq = G.covering_module(hphi[sel], nmod, par)
                        cov[sel], kk[sel] = c, kq
                acc = inr & cov
                mod = G.disk_module_id(L, ring, kk)
                sinl = np.abs(tanl[m]) / np.sqrt(1.0 + tanl[m] ** 2)
                xx0 = X0_DISK / np.maximum(sinl, 1e-3)
            if not acc.any():
                continue
            ma = m[acc]
            hx.append(px[acc]); hy.append(py[acc]); hz.append(pz[acc])
            hl.append(np.full(ma.size, L)); hm.append(mod[acc]); ht.append(ma)
            first = nhit[ma] == 0
            nhit[ma] += 1
            if cfg.multiple_scattering:
                th0 = _highland(p[ma], xx0[acc])
                if cfg.ms_skip_first:
                    th0 = np.where(first, 0.0, th0)
                cosl = 1.0 / np.sqrt(1.0 + tanl[ma] ** 2)
                lam = np.arctan(tanl[ma]) + rng.normal(0, 1, ma.size) * th0
                phi[ma] = phi[ma] + rng.normal(0, 1, ma.size) * th0 / cosl
                tanl[ma] = np.tan(lam)
                pt_new = p[ma] * np.cos(lam)
                k[ma] = -q[ma] / rho_of_pt(pt_new)
    if not hx:
        e = np.zeros(0)
        return e, e, e, e.astype(np.int64), e.astype(np.int64), e.astype(np.int64)
    return (np.concatenate(hx), np.concatenate(hy), np.concatenate(hz),
            np.concatenate(hl), np.concatenate(hm), np.concatenate(ht))


def _smear(x, y, z, layer, rng):
    disk = layer >= 4
    r = np.hypot(x, y)
    phi = np.arctan2(y, x)
    phi = phi + rng.normal(0, SIGMA_RPHI, x.size) / r
    r2 = np.where(disk, r + rng.normal(0, SIGMA_Z, x.size), r)
    z2 = np.where(disk, z, z + rng.normal(0, SIGMA_Z, x.size))
    return r2 * np.cos(phi), r2 * np.sin(phi), z2


def _noise(cfg, layer_counts, rng, overlaps):
    n_sig = int(layer_counts.sum())
    n_noise = rng.poisson(cfg.noise_frac * n_sig) if cfg.noise_frac > 0 else 0
    if n_noise == 0:
        e = np.zeros(0)
        return e, e, e, e.astype(np.int64), e.astype(np.int64)
    prob = layer_counts / max(1, layer_counts.sum())
    lay = rng.choice(np.arange(G.N_LAYERS), size=n_noise, p=prob)
    phi = rng.uniform(-math.pi, math.pi, n_noise)
    x = np.empty(n_noise); y = np.empty(n_noise); z = np.empty(n_noise)
    mod = np.empty(n_noise, dtype=np.int64)
    for L in range(G.N_LAYERS):
        m = lay == L
        if not m.any():
            continue
        ph = phi[m]
        if L < 4:
            nl = G.BARREL_LADDERS[L]
            c0, k0 = G.covering_module(ph, nl, 0)
            c1, k1 = G.covering_module(ph, nl, 1)
            if overlaps:
                rr = np.where(c0, G.BARREL_R[L] - G.BARREL_DR, G.BARREL_R[L] + G.BARREL_DR)
                lad = np.where(c0, k0, k1)
            else:
                rr = np.full(ph.size, G.BARREL_R[L])
                lad = np.floor(np.mod(ph, 2 * math.pi) / (2 * math.pi / nl)).astype(np.int64) % nl
            zz = rng.uniform(-G.BARREL_HALF_Z + 0.01, G.BARREL_HALF_Z - 0.01, ph.size)
            x[m], y[m], z[m] = rr * np.cos(ph), rr * np.sin(ph), zz
            mod[m] = G.barrel_module_id(L, lad, zz)
        else:
            side = 1.0 if L < 7 else -1.0
            zd = G.DISK_Z[(L - 4) % 3]
            rr = np.sqrt(rng.uniform(G.DISK_RMIN ** 2 + 0.01, G.DISK_RMAX ** 2 - 0.01, ph.size))
            ring = (rr >= G.DISK_RING_SPLIT).astype(np.int64)
            kk = np.zeros(ph.size, dtype=np.int64)
            zz = np.full(ph.size, side * zd)
            for ri in (0, 1):
                sel = ring == ri
                if not sel.any():
                    continue
                nmod = G.DISK_RING_MODULES[ri]
                c0, k0 = G.covering_module(ph[sel], nmod, 0)
                _, k1 = G.covering_module(ph[sel], nmod, 1)
                if overlaps:
                    kk[sel] = np.where(c0, k0, k1)
                    zz[sel] = side * np.where(c0, zd - G.DISK_DZ, zd + G.DISK_DZ)
                else:
                    kk[sel] = np.floor(np.mod(ph[sel], 2 * math.pi) /
                                       (2 * math.pi / nmod)).astype(np.int64) % nmod
            x[m], y[m], z[m] = rr * np.cos(ph), rr * np.sin(ph), zz
            mod[m] = G.disk_module_id(L, ring, kk)
    return x, y, z, lay.astype(np.int64), mod


def make_event(cfg: EventConfig, e: int) -> dict:
    """One event of configuration cfg (event index e within the batch)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * cfg.index + e))
    trk = _draw_tracks(cfg, rng)
    x, y, z, layer, module, tid = _simulate(cfg, trk, rng)
    if cfg.ineff > 0 and x.size:
        keep = rng.random(x.size) >= cfg.ineff
        x, y, z, layer, module, tid = x[keep], y[keep], z[keep], layer[keep], module[keep], tid[keep]
    x, y, z = _smear(x, y, z, layer, rng)
    counts = np.bincount(layer, minlength=G.N_LAYERS).astype(np.float64)
    nx, ny, nz, nl, nm = _noise(cfg, counts, rng, cfg.overlaps)
    x = np.concatenate([x, nx]); y = np.concatenate([y, ny]); z = np.concatenate([z, nz])
    layer = np.concatenate([layer, nl]); module = np.concatenate([module, nm])
    tid = np.concatenate([tid, np.full(nx.size, -1)])
    perm = rng.permutation(x.size)
    x, y, z, layer, module, tid = x[perm], y[perm], z[perm], layer[perm], module[perm], tid[perm]
    xs, ys, zs = snap(x), snap(y), snap(z)
    rs = snap(np.hypot(xs, ys))
    return dict(
        x=xs.astype(np.float32), y=ys.astype(np.float32), z=zs.astype(np.float32),
        r=rs.astype(np.float32), module=module.astype(np.int32),
        layer=layer.astype(np.int32), track=tid.astype(np.int32),
        trk_pt=trk["pt"], trk_eta=trk["eta"], trk_phi=trk["phi"], trk_q=trk["q"],
        trk_vertex=trk["vertex"][trk["vid"]],
    )


def _make_event_args(args):
    return make_event(*args)


def make_batch(cfg: EventConfig | str, n_events: int | None = None, first: int = 0,
               workers: int = 0) -> dict:
    """Concatenate events first .. first+n_events-1 into one SoA batch.

    Returns x, y, z, r (float32), module (int32), ev_off (int32[N+1]) plus
    truth: layer, track (index into the batch-wide track arrays, -1 noise),
    trk_* arrays.  workers > 1 generates events in a spawn-started process
    pool (safe before or after CUDA initialisation in the caller).  `cfg`
    is a workload or its name (a key of WORKLOADS)."""
    if isinstance(cfg, str):
        cfg = WORKLOADS[cfg]
    n = cfg.n_events if n_events is None else n_events
    if workers > 1 and n > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            evs = list(ex.map(_make_event_args, [(cfg, first + e) for e in range(n)]))
    else:
        evs = [make_event(cfg, first + e) for e in range(n)]
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([ev["x"].size for ev in evs])
    toff = np.zeros(n + 1, dtype=np.int64)
    toff[1:] = np.cumsum([ev["trk_pt"].size for ev in evs])
    out = {}
    for key in ("x", "y", "z", "r", "module", "layer"):
        out[key] = np.concatenate([ev[key] for ev in evs]) if n else np.zeros(0, np.float32)
    out["track"] = np.concatenate(
        [np.where(ev["track"] >= 0, ev["track"] + toff[i], -1) for i, ev in enumerate(evs)]
    ).astype(np.int64) if n else np.zeros(0, np.int64)
    for key in ("trk_pt", "trk_eta", "trk_phi", "trk_q"):
        out[key] = np.concatenate([ev[key] for ev in evs]) if n else np.zeros(0)
    out["trk_vertex"] = np.concatenate([ev["trk_vertex"] for ev in evs]) if n else np.zeros((0, 3))
    out["ev_off"] = off.astype(np.int32)
    out["config"] = cfg
    return out

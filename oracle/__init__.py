"""Python access to the CPU oracle (oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, exact/FP64
implementation of the seeding + broken-line fitting path of arXiv 2008.13461
(Sec. 3.2-3.4).  Only tests/, the smoke check and the CPU-baseline leg of the
benchmark may import this package; the library never does.  It imports
nothing from the CUDA package: inputs come from the separate ``synth``
package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NMAX = 8
NLAYERS = 10
MAX_PAIRS = 32
PRED = dict(phiw=0, zip=1, pt=2, rz=3, curv=4, beamspot=5, dz=6, fb=7)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no -ffast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC,
                               "-o", _LIB + ".tmp", "-lm"])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Pair(C.Structure):
    _fields_ = [("inner", C.c_int32), ("outer", C.c_int32), ("tan2_dphi", C.c_float),
                ("zlo", C.c_float), ("zhi", C.c_float), ("zmax", C.c_float), ("k_pt", C.c_float)]


class _Region(C.Structure):
    _fields_ = [("tol_rz2", C.c_float), ("k_curv", C.c_float), ("rmax2", C.c_float),
                ("zmax", C.c_float)]


class _Cuts(C.Structure):
    _fields_ = [("n_pairs", C.c_int32), ("pair", _Pair * MAX_PAIRS), ("region", _Region * 2),
                ("fishbone_eps2", C.c_float), ("min_hits", C.c_int32)]


class _FitPar(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("bz", "sigma_rphi", "sigma_z", "sigma_r", "x0_barrel", "x0_disk", "ms_scale")]


class _Input(C.Structure):
    _fields_ = [("x", C.POINTER(C.c_float)), ("y", C.POINTER(C.c_float)),
                ("z", C.POINTER(C.c_float)), ("r", C.POINTER(C.c_float)),
                ("module", C.POINTER(C.c_int32)), ("n_hits", C.c_int32),
                ("ev_off", C.POINTER(C.c_int32)), ("n_events", C.c_int32),
                ("module_layer", C.POINTER(C.c_int32)), ("n_modules", C.c_int32),
                ("layer_is_disk", C.c_int32 * NLAYERS),
                ("cuts", C.POINTER(_Cuts)), ("fitpar", C.POINTER(_FitPar))]


class _Tuple(C.Structure):
    _fields_ = [("n", C.c_int32), ("hits", C.c_int32 * NMAX), ("cells", C.c_int32 * (NMAX - 1))]


class _Result(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("cells", C.POINTER(C.c_int32)),
                ("cell_alive", C.POINTER(C.c_uint8)),
                ("n_edges", C.c_int64), ("edges", C.POINTER(C.c_int64)),
                ("n_tuples", C.c_int64), ("tuples", C.POINTER(_Tuple)),
                ("tuple_alive", C.POINTER(C.c_uint8)),
                ("n_tracks", C.c_int64), ("track_tuple", C.POINTER(C.c_int64)),
                ("params", C.POINTER(C.c_double)), ("cov", C.POINTER(C.c_double)),
                ("chi2", C.POINTER(C.c_double)), ("ndf", C.POINTER(C.c_int32))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_pred.restype = C.c_int
        _lib.oracle_pred.argtypes = [C.c_int, C.POINTER(C.c_float), C.c_int, C.c_float]
        _lib.oracle_fit.restype = C.c_int
        _lib.oracle_fit.argtypes = [C.c_int] + [C.POINTER(C.c_double)] * 3 + [
            C.POINTER(C.c_int), C.POINTER(_FitPar), C.POINTER(C.c_double), C.POINTER(C.c_double),
            C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_double)]
        _lib.oracle_sym_condition.restype = C.c_double
        _lib.oracle_sym_condition.argtypes = [C.c_int, C.POINTER(C.c_double)]
        _lib.oracle_run.restype = C.c_int
        _lib.oracle_run.argtypes = [C.POINTER(_Input), C.c_int, C.POINTER(_Result)]
        _lib.oracle_free.restype = None
        _lib.oracle_free.argtypes = [C.POINTER(_Result)]
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def make_cuts(cuts: dict) -> _Cuts:
    c = _Cuts()
    c.n_pairs = len(cuts["pairs"])
    for i, p in enumerate(cuts["pairs"]):
        c.pair[i] = _Pair(p["inner"], p["outer"], p["tan2_dphi"], p["zlo"], p["zhi"],
                          p["zmax"], p["k_pt"])
    for i, rg in enumerate(cuts["region"]):
        c.region[i] = _Region(rg["tol_rz2"], rg["k_curv"], rg["rmax2"], rg["zmax"])
    c.fishbone_eps2 = cuts["fishbone_eps2"]
    c.min_hits = cuts["min_hits"]
    return c


def make_fitpar(fp: dict, ms_scale: float = 1.0) -> _FitPar:
    return _FitPar(fp["bz"], fp["sigma_rphi"], fp["sigma_z"], fp["sigma_r"],
                   fp["x0_barrel"], fp["x0_disk"], ms_scale)


def pred(which: str, hits, k: float) -> bool:
    """Evaluate one exact predicate on 2 or 3 hits given as rows (x, y, z, r)."""
    h = np.ascontiguousarray(np.asarray(hits, dtype=np.float32).reshape(-1, 4))
    v = lib().oracle_pred(PRED[which], _ptr(h, C.c_float), h.shape[0], C.c_float(k))
    if v < 0:
        raise ValueError(which)
    return bool(v)


def fit(hx, hy, hz, is_disk, fitpar: dict, ms_scale: float = 1.0):
    """Broken-line fit of one track (hits inner to outer).  Returns
    (params[5], cov[15], chi2, ndf, extra[10]); extra holds chi2 of the line
    and circle fits, k0, psi0, tanl0, dk, the arc to the perigee, 0, and the
    condition numbers of the line and circle normal matrices."""
    n = len(hx)
    hx = np.ascontiguousarray(hx, dtype=np.float64)
    hy = np.ascontiguousarray(hy, dtype=np.float64)
    hz = np.ascontiguousarray(hz, dtype=np.float64)
    dk = np.ascontiguousarray(is_disk, dtype=np.int32)
    fp = make_fitpar(fitpar, ms_scale)
    p = np.zeros(5); cv = np.zeros(15); chi2 = C.c_double(); ndf = C.c_int(); ex = np.zeros(10)
    rc = lib().oracle_fit(n, _ptr(hx, C.c_double), _ptr(hy, C.c_double), _ptr(hz, C.c_double),
                          _ptr(dk, C.c_int), C.byref(fp), _ptr(p, C.c_double), _ptr(cv, C.c_double),
                          C.byref(chi2), C.byref(ndf), _ptr(ex, C.c_double))
    if rc != 0:
        raise ValueError("oracle_fit: bad number of hits")
    return p, cv, chi2.value, ndf.value, ex


def sym_condition(M) -> float:
    """2-norm condition number of a symmetric matrix (the oracle's Jacobi
    eigenvalues)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    return float(lib().oracle_sym_condition(M.shape[0], _ptr(M, C.c_double)))


def fit_grad_fd(hx, hy, hz, is_disk, fitpar: dict, gparams, gchi2: float = 0.0, h: float = 2e-5,
                ms_scale: float = 1.0) -> np.ndarray:
    """Gradient of  gparams . params + gchi2 * chi2  of the broken-line fit
    (Sec. 3.4) with respect to the hit coordinates, float[3, n] (x, y, z rows):
    the derivative's plain definition evaluated numerically, by Richardson
    extrapolation of central differences of the float64 fit with steps h and
    h/2 cm (error O(h^4); phi0 differences taken modulo 2 pi).  `ms_scale`
    scales the scattering variance as in fit()."""
    base = [np.array(a, dtype=np.float64) for a in (hx, hy, hz)]
    gp = np.asarray(gparams, dtype=np.float64)
    n = len(base[0])

    def central(a, i, step):
        up = [b.copy() for b in base]
        dn = [b.copy() for b in base]
        up[a][i] += step
        dn[a][i] -= step
        pu, _, cu, _, _ = fit(up[0], up[1], up[2], is_disk, fitpar, ms_scale)
        pd, _, cd, _, _ = fit(dn[0], dn[1], dn[2], is_disk, fitpar, ms_scale)
        d = pu - pd
        d[1] = (d[1] + np.pi) % (2 * np.pi) - np.pi
        return (float(np.dot(gp, d)) + gchi2 * (cu - cd)) / (2 * step)

    G = np.zeros((3, n))
    for a in range(3):
        for i in range(n):
            G[a, i] = (4.0 * central(a, i, h / 2) - central(a, i, h)) / 3.0
    return G


def align_hits(x, y, z, module, centres, shift, rot):
    """Per-module alignment of hits (the corrections whose gradient a
    track-based alignment of the pixel detector needs, differentiated with
    the fit of Sec. 3.4): a hit on module m moves to
        x' = c_m + (I + [w_m]x) (x - c_m) + d_m = x + w_m x (x - c_m) + d_m,
    the module rotated by the small angle vector w_m (to first order) about
    its centre c_m and shifted by d_m.  float64 arrays (x', y', z')."""
    P = np.stack([np.asarray(a, dtype=np.float64) for a in (x, y, z)], 1)
    m = np.asarray(module)
    c = np.asarray(centres, dtype=np.float64)[m]
    out = P + np.cross(np.asarray(rot, dtype=np.float64)[m], P - c) + np.asarray(shift, dtype=np.float64)[m]
    return out[:, 0], out[:, 1], out[:, 2]


def fit_grad_central(hx, hy, hz, is_disk, fitpar: dict, gparams, gchi2: float = 0.0, h: float = 1e-4,
                     ms_scale: float = 1.0) -> np.ndarray:
    """Gradient of  gparams . params + gchi2 * chi2  of the broken-line fit
    with respect to the hit coordinates, float[3, n]: plain central
    differences (f(x + h) - f(x - h)) / 2h of the float64 fit with step h cm
    (phi0 differences taken modulo 2 pi)."""
    base = [np.array(a, dtype=np.float64) for a in (hx, hy, hz)]
    gp = np.asarray(gparams, dtype=np.float64)
    n = len(base[0])
    G = np.zeros((3, n))
    for a in range(3):
        for i in range(n):
            up = [b.copy() for b in base]
            dn = [b.copy() for b in base]
            up[a][i] += h
            dn[a][i] -= h
            pu, _, cu, _, _ = fit(up[0], up[1], up[2], is_disk, fitpar, ms_scale)
            pd, _, cd, _, _ = fit(dn[0], dn[1], dn[2], is_disk, fitpar, ms_scale)
            d = pu - pd
            d[1] = (d[1] + np.pi) % (2 * np.pi) - np.pi
            G[a, i] = (float(np.dot(gp, d)) + gchi2 * (cu - cd)) / (2 * h)
    return G


def run(batch: dict, cuts: dict, fitpar: dict, module_layer: np.ndarray,
        layer_is_disk, stage: int = 4, ms_scale: float = 1.0) -> dict:
    """Run the oracle chain up to `stage` (1 doublets+Fishbone, 2 connect,
    3 n-tuplets+cleaning, 4 fit) over a batch of events."""
    x = np.ascontiguousarray(batch["x"], dtype=np.float32)
    y = np.ascontiguousarray(batch["y"], dtype=np.float32)
    z = np.ascontiguousarray(batch["z"], dtype=np.float32)
    r = np.ascontiguousarray(batch["r"], dtype=np.float32)
    mod = np.ascontiguousarray(batch["module"], dtype=np.int32)
    off = np.ascontiguousarray(batch["ev_off"], dtype=np.int32)
    ml = np.ascontiguousarray(module_layer, dtype=np.int32)
    c = make_cuts(cuts)
    fp = make_fitpar(fitpar, ms_scale)
    inp = _Input()
    inp.x, inp.y, inp.z, inp.r = (_ptr(a, C.c_float) for a in (x, y, z, r))
    inp.module = _ptr(mod, C.c_int32)
    inp.n_hits = x.size
    inp.ev_off = _ptr(off, C.c_int32)
    inp.n_events = off.size - 1
    inp.module_layer = _ptr(ml, C.c_int32)
    inp.n_modules = ml.size
    for i in range(NLAYERS):
        inp.layer_is_disk[i] = int(layer_is_disk[i])
    inp.cuts = C.pointer(c)
    inp.fitpar = C.pointer(fp)
    res = _Result()
    rc = lib().oracle_run(C.byref(inp), stage, C.byref(res))
    if rc != 0:
        raise ValueError(f"oracle_run failed ({rc})")
    try:
        nc, ne, nt, nk = res.n_cells, res.n_edges, res.n_tuples, res.n_tracks

        def arr(p, n, dt, shape=None):
            if n == 0:
                return np.zeros((0,) + (shape or ()), dtype=dt)
            a = np.ctypeslib.as_array(p, shape=(n,) + (shape or ())).copy()
            return a.astype(dt, copy=False)

        out = dict(
            cells=arr(res.cells, nc, np.int32, (3,)),
            cell_alive=arr(res.cell_alive, nc, np.uint8).astype(bool),
            edges=arr(res.edges, ne, np.int64, (2,)),
        )
        if nt:
            tb = np.ctypeslib.as_array(C.cast(res.tuples, C.POINTER(C.c_int32)),
                                       shape=(nt, 1 + NMAX + NMAX - 1)).copy()
        else:
            tb = np.zeros((0, 2 * NMAX), dtype=np.int32)
        out["tuple_n"] = tb[:, 0].astype(np.int32)
        out["tuple_hits"] = tb[:, 1:1 + NMAX].astype(np.int32)
        out["tuple_cells"] = tb[:, 1 + NMAX:].astype(np.int32)
        out["tuple_alive"] = arr(res.tuple_alive, nt, np.uint8).astype(bool) if stage >= 3 else \
            np.zeros(0, bool)
        out["track_tuple"] = arr(res.track_tuple, nk, np.int64)
        out["params"] = arr(res.params, nk, np.float64, (5,))
        out["cov"] = arr(res.cov, nk, np.float64, (15,))
        out["chi2"] = arr(res.chi2, nk, np.float64)
        out["ndf"] = arr(res.ndf, nk, np.int32)
        return out
    finally:
        lib().oracle_free(C.byref(res))

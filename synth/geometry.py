"""Detector description for synthetic pixel events (input data, not method).

Layer numbering (fixed throughout the project):

    0..3  barrel layers BPix1..BPix4, nominal r = 2.9, 6.8, 10.9, 16.0 cm, |z| < 26.7 cm
    4..6  forward disks FPix+1..3 at z = +32, +39.5, +48.8 cm, r in [4.5, 16] cm
    7..9  forward disks FPix-1..3 at z = -32, -39.5, -48.8 cm

The paper (Sec. 3.1) describes the Phase-1 pixel detector as 1856 sensors in
four barrel layers and three disks per side, with azimuthal sensor overlaps
that make hermetic coverage (and that the Fishbone step of Sec. 3.3 exists
for).  Here each barrel layer is built from ladders that alternate between
two radii (r - DR, r + DR) and overlap in phi, and each disk from modules that
alternate between two z planes and overlap in phi, so a track near a module
edge leaves two hits on one layer.

Module count: barrel ladders 12/28/44/64 x 8 modules along z = 1184, plus
6 disks x (44 inner + 68 outer) = 672, total 1856.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_LAYERS = 10
BARREL_R = (2.9, 6.8, 10.9, 16.0)
BARREL_HALF_Z = 26.7
BARREL_LADDERS = (12, 28, 44, 64)
BARREL_ZSEG = 8
BARREL_DR = 0.15          # ladders alternate at r - DR / r + DR
DISK_Z = (32.0, 39.5, 48.8)
DISK_RMIN, DISK_RMAX = 4.5, 16.0
DISK_RING_SPLIT = 10.0    # inner ring r < split, outer ring r >= split
DISK_RING_MODULES = (44, 68)
DISK_DZ = 0.2             # modules alternate at |z| - DZ / |z| + DZ
PHI_OVERLAP = 0.08        # fractional phi overlap of neighbouring modules

LAYER_BARREL = 0
LAYER_DISK = 1

# Envelope margins so that every generated hit lies strictly inside the
# layer envelope the binning kernel validates against.
_ENV_MARGIN_R = 0.05
_ENV_MARGIN_Z = 0.05


@dataclasses.dataclass(frozen=True)
class Layer:
    index: int
    kind: int              # LAYER_BARREL or LAYER_DISK
    r_nom: float           # barrel radius (0 for disks)
    z_nom: float           # disk z (0 for barrel)
    rmin: float            # envelope of hit positions on this layer
    rmax: float
    zmin: float
    zmax: float


def layers(barrel_only: bool = False) -> list[Layer]:
    out = []
    for i, r in enumerate(BARREL_R):
        out.append(Layer(i, LAYER_BARREL, r, 0.0,
                         r - BARREL_DR - _ENV_MARGIN_R, r + BARREL_DR + _ENV_MARGIN_R,
                         -BARREL_HALF_Z - _ENV_MARGIN_Z, BARREL_HALF_Z + _ENV_MARGIN_Z))
    for side, base in ((+1, 4), (-1, 7)):
        for d, z in enumerate(DISK_Z):
            zc = side * z
            out.append(Layer(base + d, LAYER_DISK, 0.0, zc,
                             DISK_RMIN - _ENV_MARGIN_R, DISK_RMAX + _ENV_MARGIN_R,
                             zc - DISK_DZ - _ENV_MARGIN_Z, zc + DISK_DZ + _ENV_MARGIN_Z))
    return out


def layer_is_disk(layer: int) -> bool:
    return layer >= 4


# ---------------------------------------------------------------- modules
def _barrel_module_base() -> list[int]:
    base, acc = [], 0
    for n in BARREL_LADDERS:
        base.append(acc)
        acc += n * BARREL_ZSEG
    return base


N_BARREL_MODULES = sum(n * BARREL_ZSEG for n in BARREL_LADDERS)          # 1184
N_DISK_MODULES_PER_DISK = sum(DISK_RING_MODULES)                           # 112
N_MODULES = N_BARREL_MODULES + 6 * N_DISK_MODULES_PER_DISK                 # 1856
_BARREL_BASE = _barrel_module_base()


def module_layer_table() -> np.ndarray:
    """int32[N_MODULES]: layer index of each module id."""
    t = np.empty(N_MODULES, dtype=np.int32)
    for L, n in enumerate(BARREL_LADDERS):
        b = _BARREL_BASE[L]
        t[b:b + n * BARREL_ZSEG] = L
    for d in range(6):
        b = N_BARREL_MODULES + d * N_DISK_MODULES_PER_DISK
        t[b:b + N_DISK_MODULES_PER_DISK] = 4 + d
    return t


def module_centres() -> np.ndarray:
    """float64[N_MODULES, 3]: the centre of each module (barrel: ladder axis
    at the module's mid z; disks: mid radius of the ring, mid azimuth), the
    reference point about which alignment rotations act."""
    c = np.zeros((N_MODULES, 3))
    hz = 2 * BARREL_HALF_Z / BARREL_ZSEG
    for L, n in enumerate(BARREL_LADDERS):
        for k in range(n):
            phi = (k + 0.5) * 2 * math.pi / n
            r = BARREL_R[L] - BARREL_DR if k % 2 == 0 else BARREL_R[L] + BARREL_DR
            for j in range(BARREL_ZSEG):
                c[_BARREL_BASE[L] + k * BARREL_ZSEG + j] = (r * math.cos(phi), r * math.sin(phi),
                                                          -BARREL_HALF_Z + (j + 0.5) * hz)
    rings = ((DISK_RMIN + DISK_RING_SPLIT) / 2, (DISK_RING_SPLIT + DISK_RMAX) / 2)
    for layer in range(4, 10):
        side = 1.0 if layer < 7 else -1.0
        zd = DISK_Z[(layer - 4) % 3]
        for ring, nm in enumerate(DISK_RING_MODULES):
            for k in range(nm):
                phi = (k + 0.5) * 2 * math.pi / nm
                z = side * (zd - DISK_DZ if k % 2 == 0 else zd + DISK_DZ)
                m = disk_module_id(layer, np.array([ring]), np.array([k]))[0]
                c[m] = (rings[ring] * math.cos(phi), rings[ring] * math.sin(phi), z)
    return c


def barrel_module_id(layer: int, ladder: np.ndarray, z: np.ndarray) -> np.ndarray:
    zseg = np.clip(np.floor((z + BARREL_HALF_Z) / (2 * BARREL_HALF_Z / BARREL_ZSEG)), 0,
                   BARREL_ZSEG - 1).astype(np.int64)
    return _BARREL_BASE[layer] + ladder.astype(np.int64) * BARREL_ZSEG + zseg


def disk_module_id(layer: int, ring: np.ndarray, k: np.ndarray) -> np.ndarray:
    b = N_BARREL_MODULES + (layer - 4) * N_DISK_MODULES_PER_DISK
    return b + np.where(ring == 0, k, DISK_RING_MODULES[0] + k)


def covering_module(phi: np.ndarray, n_mod: int, parity: int) -> tuple[np.ndarray, np.ndarray]:
    """For modules k = 0..n_mod-1 spanning phi in
    [k*w - ov*w/2, (k+1)*w + ov*w/2], w = 2pi/n_mod, return (covered, k) where k is
    the module of the requested parity (k % 2 == parity) covering phi, if any."""
    w = 2.0 * math.pi / n_mod
    p = np.mod(phi, 2.0 * math.pi)
    k0 = np.floor(p / w).astype(np.int64) % n_mod
    frac = p / w - np.floor(p / w)
    half = PHI_OVERLAP / 2.0
    cand = [k0, (k0 - 1) % n_mod, (k0 + 1) % n_mod]
    inside = [np.ones_like(frac, dtype=bool), frac <= half, frac >= 1.0 - half]
    covered = np.zeros(phi.shape, dtype=bool)
    kk = np.zeros(phi.shape, dtype=np.int64)
    for c, ins in zip(cand, inside):
        ok = ins & (c % 2 == parity) & ~covered
        kk = np.where(ok, c, kk)
        covered |= ok
    return covered, kk


# ------------------------------------------------------------ layer pairs
# The paper's figure of layer pairs did not survive; the reading used is
# adjacent pairs plus skip-one pairs (B = barrel, F = forward disk):
#   adjacent: B1B2 B2B3 B3B4 B1F1+- B2F1+- F1F2+- F2F3+-
#   skip:     B1B3 B2B4 B1F2+- F1F3+-
PAIRS_FULL = (
    (0, 1), (1, 2), (2, 3),
    (0, 4), (0, 7), (1, 4), (1, 7),
    (4, 5), (7, 8), (5, 6), (8, 9),
    (0, 2), (1, 3), (0, 5), (0, 8), (4, 6), (7, 9),
)
PAIRS_BARREL = ((0, 1), (1, 2), (2, 3), (0, 2), (1, 3))

"""Cut tables: the constants the seeding predicates compare against.

The paper (Sec. 3.2, Table 1) names the doublet cuts (PhiW, ZW, ZIP, PT) and
the Cellular Automaton criteria (R-z alignment, curvature above pT_min,
beamspot compatibility within R_max, barrel/endcap CA cut sets), and the
general criteria pT_min, R_max, z_max and n_hits, but prints no values.  This
module derives one value per layer pair and per CA region from pT_min,
R_max and z_max with a safety margin; the values change efficiencies, never
the agreement between two implementations, because both read this same
table.  Every constant is rounded to float32 here; its exact binary value is
the constant of the predicate.

Stored forms (so that no further rounding is needed on either side):
  pair p:  tan2_dphi = tan^2(dphi_max)     PhiW
           zlo, zhi                        ZW window on the inner hit's z
           zmax                            ZIP: |z-intercept at r=0| <= zmax
           k_pt = 4 rho_min^2              PT: circle through origin, i, o
  region:  tol_rz2 = tol^2                 R-z alignment distance
           k_curv = 4 rho_min^2            CA curvature
           rmax2 = R_max^2                 CA beamspot compatibility
           zmax                            CA dz compatibility
  fishbone_eps2 = eps^2                    Fishbone alignment (sin^2 of angle)
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry as G
from .events import rho_of_pt

REGION_BARREL = 0
REGION_ENDCAP = 1


def _f32(v) -> float:
    return float(np.float32(v))


def make_cuts(pt_min: float = 0.5, barrel_only: bool = False, min_hits: int = 3,
              zmax: float = 12.0, rmax_doublet: float = 0.01, pt_factor: float = 0.9,
              ca_tol=(0.02, 0.03), ca_rmax=(0.05, 0.1), ca_curv_factor: float = 0.8,
              dphi_scale: float = 1.0) -> dict:
    """Cut table for tracks above pt_min (GeV).  zmax: luminous-region half
    length (12 cm = 3.4 sigma of the vertex z spread); rmax_doublet: transverse
    impact allowance in the doublet phi window; pt_factor / ca_curv_factor:
    fraction of the pt_min radius used by the PT and CA curvature cuts;
    ca_tol / ca_rmax: R-z alignment distance and beamspot R_max (cm) for the
    barrel and endcap CA cut sets.  Defaults were chosen on the PU50 sample
    for ~99% efficiency of tracks leaving >= 3 layer hits."""
    lay = {L.index: L for L in G.layers()}
    pairs = G.PAIRS_BARREL if barrel_only else G.PAIRS_FULL
    rho = float(rho_of_pt(pt_min))
    soft = max(1.0, 0.5 / pt_min)
    out_pairs = []
    for (li, lo) in pairs:
        Li, Lo = lay[li], lay[lo]
        ri_min, ro_max = Li.rmin, Lo.rmax
        ro_min = max(Lo.rmin, ri_min)
        rr = 0.9 * rho
        dphi = (math.asin(min(1.0, ro_max / (2 * rr))) - math.asin(min(1.0, ri_min / (2 * rr)))
                + math.asin(min(1.0, rmax_doublet / ri_min))
                + math.asin(min(1.0, rmax_doublet / ro_min)))
        dphi = dphi_scale * dphi + 0.005
        dphi = min(dphi, 1.2)
        zlo, zhi = Li.zmin, Li.zmax
        if Li.kind == G.LAYER_BARREL and Lo.kind == G.LAYER_DISK:
            if Lo.z_nom > 0:
                zlo = max(zlo, -zmax + (Lo.zmin + zmax) * Li.rmin / Lo.rmax - 0.5)
            else:
                zhi = min(zhi, zmax + (Lo.zmax - zmax) * Li.rmin / Lo.rmax + 0.5)
        out_pairs.append(dict(
            inner=li, outer=lo,
            tan2_dphi=_f32(math.tan(dphi) ** 2),
            zlo=_f32(zlo), zhi=_f32(zhi),
            zmax=_f32(zmax),
            k_pt=_f32(4.0 * (pt_factor * rho) ** 2),
        ))
    region = []
    for tol, rmax in zip(ca_tol, ca_rmax):
        region.append(dict(
            tol_rz2=_f32((tol * soft) ** 2),
            k_curv=_f32(4.0 * (ca_curv_factor * rho) ** 2),
            rmax2=_f32((rmax * soft) ** 2),
            zmax=_f32(zmax),
        ))
    return dict(pairs=out_pairs, region=region,
                fishbone_eps2=_f32(math.tan(2e-3) ** 2),
                min_hits=int(min_hits), pt_min=float(pt_min))


def cuts_for(workload: str) -> dict:
    """The cut set of a synthetic workload (by its name): the noiseless
    barrel helices above 1 GeV take barrel pairs and a 0.9 GeV threshold,
    the stress workload with tracks down to 0.3 GeV a 0.3 GeV threshold, the
    pileup workloads 0.5 GeV."""
    if workload == "barrel-50-helices":
        return make_cuts(pt_min=0.9, barrel_only=True)
    if workload == "pu200-stress-batch256":
        return make_cuts(pt_min=0.3)
    if workload in ("pu50-ttbar-like", "pu200-batch64", "pu50-batch32"):
        return make_cuts(pt_min=0.5)
    raise KeyError(f"no cut set for workload {workload!r}")


# Fit constants (measurement errors and material, matching the simulation).
FIT_PARAMS = dict(
    bz=3.8,
    sigma_rphi=10e-4,
    sigma_z=20e-4,       # barrel z
    sigma_r=20e-4,       # disk r
    x0_barrel=0.02,
    x0_disk=0.03,
)

"""The doublet search's per-outer-hit azimuth window (CPU, against the oracle).

The search narrows each layer pair's PhiW window to the outer hit with the
PT cut (Sec. 3.2, Table 1): the cut accepts a doublet when the circle through
the beam line and its two hits has a radius of at least R (k_pt = 4 R^2).  On
such a circle a chord from the beam line of length r makes the angle
asin(r / 2R) with the tangent there, so two hits at radii r_i, r_o on a
circle of radius R differ in azimuth by |asin(r_o / 2R) - asin(r_i / 2R)| or
by pi - asin(r_o / 2R) - asin(r_i / 2R), and a larger radius only shrinks the
first difference.  The window is therefore the first bound, taken over the
inner layer's radii (plus 1e-4 rad), wherever the second lies beyond the
pair's PhiW window.  These tests check that claim where it matters: every
doublet the oracle accepts lies inside the narrowed window, and the window
is narrower than the pair's (so it saves work).
"""
import math

import numpy as np
import pytest

from synth import cuts as CU
from synth import events as E
from synth import geometry as G

from parity import oracle_run


def narrowed_window(pc, inner_layer, ro):
    """The azimuth half-window of the doublet search for outer hits at radii
    ro (float64 restatement of the search's bound)."""
    pdphi = math.atan(math.sqrt(float(pc["tan2_dphi"]))) + 1e-4
    if float(pc["k_pt"]) <= 0.0:
        return np.full_like(ro, pdphi)
    pa = 1.0 / math.sqrt(float(pc["k_pt"]))
    so = np.arcsin(np.minimum(ro * pa, 1.0))
    si = math.asin(min(inner_layer.rmin * pa, 1.0))
    sx = math.asin(min(inner_layer.rmax * pa, 1.0))
    guard = (ro * pa < 1.0) & (inner_layer.rmax * pa < 1.0) & (math.pi - so - sx > pdphi + 1e-3)
    return np.where(guard, np.minimum(pdphi, np.maximum(so - si, sx - so) + 1e-4), pdphi)


@pytest.mark.parametrize("workload", ["pu50-batch32", "barrel-50-helices"])
def test_every_oracle_doublet_lies_inside_the_narrowed_window(workload):
    b = E.make_batch(workload, n_events=1)
    cuts = CU.cuts_for(workload)
    cells = np.asarray(oracle_run(b, cuts, stage=1)["cells"])
    assert len(cells) > 100
    x, y = b["x"].astype(np.float64), b["y"].astype(np.float64)
    inner, outer, pair = cells[:, 0], cells[:, 1], cells[:, 2]
    dphi = np.abs((np.arctan2(y[outer], x[outer]) - np.arctan2(y[inner], x[inner]) + np.pi) % (2 * np.pi) - np.pi)
    ro = np.hypot(x[outer], y[outer])
    layers = {L.index: L for L in G.layers()}
    narrower = 0
    for k, pc in enumerate(cuts["pairs"]):
        sel = pair == k
        if not sel.any():
            continue
        w = narrowed_window(pc, layers[pc["inner"]], ro[sel])
        assert np.all(dphi[sel] <= w), (pc["inner"], pc["outer"], float((dphi[sel] - w).max()))
        pdphi = math.atan(math.sqrt(float(pc["tan2_dphi"]))) + 1e-4
        narrower += int(np.median(w) < 0.95 * pdphi)
    assert narrower >= 1


def test_the_bound_is_the_pt_cut_boundary():
    """Hits placed on a circle of radius exactly R through the beam line sit
    on the bound: the first branch's azimuth difference equals
    |asin(r_o/2R) - asin(r_i/2R)| and the circumradius computed as the PT
    predicate does (|d| r_i r_o / 2|C|) equals R."""
    R = 40.0
    for r_i, r_o in ((3.0, 7.0), (7.0, 11.0), (12.0, 6.0)):
        # points on the circle centred at (0, R) through the origin: polar
        # angle psi from the tangent (the x axis), radius 2R sin(psi)
        psi_i, psi_o = math.asin(r_i / (2 * R)), math.asin(r_o / (2 * R))
        hi = np.array([r_i * math.cos(psi_i), r_i * math.sin(psi_i)])
        ho = np.array([r_o * math.cos(psi_o), r_o * math.sin(psi_o)])
        d = np.linalg.norm(ho - hi)
        C = hi[0] * ho[1] - hi[1] * ho[0]
        assert abs(d * r_i * r_o / (2 * abs(C)) - R) < 1e-9 * R
        dphi = abs(math.atan2(ho[1], ho[0]) - math.atan2(hi[1], hi[0]))
        assert abs(dphi - abs(psi_o - psi_i)) < 1e-12

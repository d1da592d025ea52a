"""Seeded per-track inputs for the vertex finder (Sec. 3.6), shaped like the
fitted pixel tracks of pileup events.  Holds no arithmetic of the method: it
only draws track summaries (event, z0 and its error, pT, hit count, the
ambiguity-resolution flag) around simulated vertices.

Recipe (same vertex model as ``synth.events``):
  * per event Poisson(pileup) vertices with z ~ N(0, 3.5 cm), each carrying
    Poisson(tracks_per_vertex) tracks;
  * pT from a 1/pT^2 spectrum on [pt_lo, 100] GeV, eta uniform in [-2.5, 2.5];
  * z0 error ez0 = sigma_z0 (1 + |eta|) sqrt(1 + (1 GeV / pT)^2), z0 drawn
    from N(z_vertex, ez0);
  * hit counts 3, 4, 5 with probabilities 0.35, 0.55, 0.10;
  * a fraction `fake_fraction` of extra tracks with z0 uniform in +-15 cm and
    a five times larger error (fakes and badly measured tracks);
  * keep = 1 with probability keep_prob; tracks of a batch in random order.
Seed: numpy PCG64 seeded with 2008134610 + 7000 + seed.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2008134610 + 7000


def vertex_tracks(seed: int, n_events: int, pileup: float = 200.0, tracks_per_vertex: float = 30.0,
                  pt_lo: float = 0.3, sigma_z0: float = 0.002, fake_fraction: float = 0.1,
                  keep_prob: float = 0.9) -> dict:
    """Track summaries of n_events events: dict of numpy arrays ev (int32),
    z0, ez0, pt (float32), nhits, keep (uint8), plus the true vertex z per
    event (list of float64 arrays) and each track's true vertex index within
    its event (-1: fake)."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + seed))
    cols = {k: [] for k in ("ev", "z0", "ez0", "pt", "nhits", "keep", "truth")}
    vz_all = []
    for e in range(n_events):
        nv = max(1, int(rng.poisson(pileup)))
        vz = rng.normal(0.0, 3.5, nv)
        vz_all.append(vz)
        ntr = rng.poisson(tracks_per_vertex, nv)
        truth = np.repeat(np.arange(nv), ntr)
        nf = int(round(fake_fraction * len(truth)))
        n = len(truth) + nf
        u = rng.random(n)
        pt = pt_lo / (1.0 - u * (1.0 - pt_lo / 100.0))             # 1/pT^2 on [pt_lo, 100]
        eta = rng.uniform(-2.5, 2.5, n)
        ez = sigma_z0 * (1.0 + np.abs(eta)) * np.sqrt(1.0 + (1.0 / pt) ** 2)
        ez[len(truth):] *= 5.0
        z0 = np.concatenate([rng.normal(vz[truth], ez[:len(truth)]), rng.uniform(-15.0, 15.0, nf)])
        cols["ev"].append(np.full(n, e))
        cols["z0"].append(z0)
        cols["ez0"].append(ez)
        cols["pt"].append(pt)
        cols["nhits"].append(rng.choice([3, 4, 5], size=n, p=[0.35, 0.55, 0.10]))
        cols["keep"].append(rng.random(n) < keep_prob)
        cols["truth"].append(np.concatenate([truth, np.full(nf, -1)]))
    perm = rng.permutation(sum(len(c) for c in cols["ev"]))
    cat = {k: np.concatenate(v)[perm] for k, v in cols.items()}
    return dict(ev=cat["ev"].astype(np.int32), z0=cat["z0"].astype(np.float32),
                ez0=cat["ez0"].astype(np.float32), pt=cat["pt"].astype(np.float32),
                nhits=cat["nhits"].astype(np.uint8), keep=cat["keep"].astype(np.uint8),
                truth=cat["truth"].astype(np.int64), vertex_z=vz_all)

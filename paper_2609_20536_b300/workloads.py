"""Seeded synthetic workloads: (beta, Delta, D_cut) point sets.

This module holds none of the method's arithmetic; it only draws parameter
sets, so both the CUDA path and the oracle can be fed the same inputs.  The
inputs of the method are parameters only (no dataset): the thesis scans
temperature and Delta (Table 3.1 spans Delta = 0.04 .. 0.80, T ~ 0.08 .. 1.0).
"""

from dataclasses import dataclass

import numpy as np

SEED = 20536


@dataclass(frozen=True)
class Point:
    beta: float
    delta: float
    n_max: int
    d_cut: int
    n_steps: int
    h: float = 0.0
    h1: float = 0.0


# single-point configurations
SMALL = Point(1.0, 0.5, 2, 16, 20)            # n_max = 2 (D0 = 5), D_cut = 16, 20 steps
MEDIUM = Point(1.1, 0.5, 5, 48, 30)           # n_max = 5 (D0 = 11), D_cut = 48, 30 steps


def headline_points(n, seed=SEED, d_cut=64, n_max=4, n_steps=25):
    """n distinct points, beta ~ U[0.5, 2.0], Delta ~ U[0, 1], at one D_cut.

    The pairs are drawn one point at a time, so the first k points are the
    same for every n >= k (a run of any length starts on the same points).
    """
    rng = np.random.default_rng(seed)
    bd = rng.uniform((0.5, 0.0), (2.0, 1.0), size=(n, 2))
    return [Point(float(b), float(d), n_max, d_cut, n_steps) for b, d in bd]


def grid_points(nb=64, nd=64, seed=SEED, n_max=4, n_steps=25, dcuts=(24, 32, 48, 64)):
    """nb x nd linspace grid over beta in [0.5, 2.0] and Delta in [0, 1]; D_cut drawn per point."""
    rng = np.random.default_rng(seed)
    betas = np.linspace(0.5, 2.0, nb)
    deltas = np.linspace(0.0, 1.0, nd)
    cuts = rng.choice(np.asarray(dcuts), size=(nb, nd))
    return [Point(float(b), float(d), n_max, int(cuts[i, j]), n_steps)
            for i, b in enumerate(betas) for j, d in enumerate(deltas)]


def beta_sweep(delta=0.3, lo=0.8, hi=1.6, step=0.01, n_max=6, d_cut=96, n_steps=30):
    n = int(round((hi - lo) / step)) + 1
    return [Point(float(lo + i * step), delta, n_max, d_cut, n_steps) for i in range(n)]

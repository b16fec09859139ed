"""An 8-seed ensemble of oracle runs of the 1D faux-shock box and the
per-bin comparison of one more run against it (test infrastructure).

The statistical outputs of a particle-in-cell run depend on its seed, so a
single run of another implementation is judged against the spread of the
oracle ensemble: per bin, |x - mean| <= 3 sigma (sigma the ensemble's sample
standard deviation, floored) for at least 95 % of the bins, and no bin
beyond 8 sigma. With eight members the sample sigma is itself uncertain
(Student t with 7 degrees of freedom), which is why a few bins past 3 sigma
are allowed.
"""
from __future__ import annotations

import functools

import numpy as np

from oracle import oracle as o
from tests import workloads as W

ENSEMBLE_SEEDS = tuple(range(101, 109))
STEPS = W.CONFIG_1D_STEPS


def coarse(a: np.ndarray, k: int) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a[: len(a) // k * k].reshape(-1, k).mean(1)


def observables(profile_n, profile_db2, hist) -> dict:
    """Coarse-binned precursor profiles and x-p_x histogram of one run."""
    h = np.asarray(hist, dtype=np.float64)
    nx, npx = h.shape
    return {
        "n": coarse(profile_n[: len(profile_n) - 1], 16),
        "db2": coarse(profile_db2, 16),
        "hist": h.reshape(nx // 4, 4, npx // 4, 4).sum((1, 3)).ravel(),
    }


def oracle_run(seed: int, **kw):
    sim = o.Oracle(**W.scaled(W.CONFIG_1D, seed=seed, **kw))
    sim.step(STEPS)
    obs = observables(sim.grid(o.GRID_PROFILE_N), sim.grid(o.GRID_PROFILE_DB2),
                      sim.histogram())
    parts = sim.particles()
    diag = sim.diag()
    sim.close()
    return obs, parts, diag


@functools.lru_cache(maxsize=1)
def ensemble():
    return [oracle_run(s) for s in ENSEMBLE_SEEDS]


def compare(x: np.ndarray, members: np.ndarray, floor: float):
    """(fraction of bins within 3 sigma, largest |z|) of x against members."""
    mu = members.mean(0)
    sd = np.maximum(members.std(0, ddof=1), floor)
    z = np.abs(x - mu) / sd
    return float(np.mean(z <= 3.0)), float(z.max())


# sigma floors: a histogram bin holds whole counts; the profiles are means
# over 16 cells of smooth quantities
FLOORS = {"n": 1e-3, "db2": 1e-4, "hist": 1.0}

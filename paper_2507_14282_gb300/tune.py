"""Tile-shape autotuner: picks the particles per tile of the push by timed
sweeps on the GPU and caches the choice per (dimension, ppc, precision).

A tile's particle count sets the push's chunk fill, the halo overhead of the
deposit and the number of persistent-CTA work items; the tuner times the two
phases it affects (push and movers). The best count depends
on ppc and precision more than on the box length, so the tuner times a few
candidate counts on a representative box of each class and applies the
winner to any box of that class (tile width = the divisor of nx whose mean
particle count is closest to it). All timing runs the library's own kernels.
"""
from __future__ import annotations

import json
import os

from . import fs

TARGETS = (128, 256, 512, 1024)  # mean particles per tile tried
MAX_NX = 65535                    # longest box the library accepts


def divisors(n: int, lo: int = 2, hi: int = 256) -> list:
    return [c for c in range(lo, min(hi, n) + 1) if n % c == 0]


def tile_for(nx: int, ppc: int, target: int) -> int:
    """Tile width (1D) whose mean particle count is closest to target."""
    ds = divisors(nx)
    if not ds:
        return nx
    return min(ds, key=lambda c: (abs(c * ppc - target), c))


class Autotuner:
    def __init__(self, cache_path: str | None = None, probe_particles: int = 1 << 22,
                 warm: int = 3, steps: int = 8):
        self.cache_path = cache_path
        self.probe_particles = probe_particles
        self.warm, self.steps = warm, steps
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)
        self.log = []

    @staticmethod
    def key(dim: int, ppc: int, precision: int) -> str:
        return f"dim{dim}-ppc{ppc}-{'fp64' if precision == fs.FS_FP64 else 'fp32'}"

    def _time(self, params: dict) -> float:
        """ms per step of the phases the tile shape sets (push and movers),
        from the library's own CUDA-event phase timing."""
        sim = fs.FauxShock(**params)
        try:
            sim.step(self.warm)
            sim.profile(True)
            sim.profile_read()
            sim.step(self.steps)
            ph = sim.profile_read()
            sim.profile(False)
            return sum(ph[k][0] / max(ph[k][1], 1) for k in ("push", "movers"))
        finally:
            sim.close()

    def best_target(self, base: dict) -> int:
        """Particles per tile for the class of base (1D parameter dict)."""
        prec = base.get("precision", fs.FS_FP64)
        k = self.key(base.get("dim", 1), base["ppc"], prec)
        if k in self.cache:
            return self.cache[k]
        probe = dict(base)
        # a box of about probe_particles particles (large enough that the
        # kernels, not launch latency, set the time), nx a multiple of 1024
        probe["nx"] = min(max(1024, (self.probe_particles // base["ppc"]) // 1024 * 1024),
                          MAX_NX // 1024 * 1024)
        best, best_ms = None, None
        for target in TARGETS:
            tx = tile_for(probe["nx"], probe["ppc"], target)
            ms = self._time(dict(probe, tile_x=tx, tile_y=1))
            self.log.append({"class": k, "target": target, "tile_x": tx, "ms_per_step": ms})
            if best_ms is None or ms < best_ms:
                best, best_ms = target, ms
        self.cache[k] = best
        if self.cache_path:
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
        return best

    def tile(self, params: dict) -> dict:
        """params with tile_x / tile_y chosen (1D boxes)."""
        if params.get("dim", 1) != 1:
            return dict(params)
        target = self.best_target(params)
        return dict(params, tile_x=tile_for(params["nx"], params["ppc"], target), tile_y=1)

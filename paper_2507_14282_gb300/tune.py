"""Push autotuner: picks the tile shape and the push's launch shape by timed
sweeps on the GPU and caches the choice per (dimension, ppc, precision).

A tile's shape sets the push's chunk fill, the share of particles that leave
the tile (the deposit's halo cells and the mover list) and the number of
persistent-CTA work items; the launch shape is the shared-memory chunk size
with its pipeline depth (512 particles in three stages or 576 in two, FP32)
and the number of persistent CTAs per SM. The tuner times the phases these
set (push and movers) with the library's own CUDA-event phase timing, in two
stages: the tile over a set of candidates at the library's default launch
shape, then every launch shape on the winning tile. The best choice depends
on ppc and precision more than on the box size, so it is timed on a
representative probe box of each class and applied to any box of that
class: in 1D as a mean particle count per tile (tile width = the divisor of
nx whose mean count is closest), in 2D as a tile shape (used where its sides
divide the box; otherwise the library chooses). All timing runs the
library's own kernels.
"""
from __future__ import annotations

import json
import os

from . import fs

TARGETS = (128, 256, 512, 1024)  # 1D: mean particles per tile tried
MAX_NX = 65535                    # longest box the library accepts


def divisors(n: int, lo: int = 2, hi: int = 256) -> list:
    return [c for c in range(lo, min(hi, n) + 1) if n % c == 0]


def tile_for(nx: int, ppc: int, target: int) -> int:
    """Tile width (1D) whose mean particle count is closest to target."""
    ds = divisors(nx)
    if not ds:
        return nx
    return min(ds, key=lambda c: (abs(c * ppc - target), c))


def targets_1d(nx: int, ppc: int, widths=None) -> list:
    """1D targets (mean particles per tile) tried on an nx-cell box: all of
    TARGETS, or, with widths, those whose tile width is one of them (all if
    none is)."""
    if not widths:
        return list(TARGETS)
    within = [t for t in TARGETS if tile_for(nx, ppc, t) in widths]
    return within or list(TARGETS)


def tile_candidates_2d(nx: int, ny: int, ppc: int, lo: int = 128, hi: int = 1024) -> list:
    """2D tile shapes (tx, ty) with tx >= 2 dividing nx (at most 64), ty
    dividing ny (at most 32) and a mean particle count in [lo, hi], ordered by
    count, then squareness."""
    out = []
    for ty in [d for d in range(1, min(32, ny) + 1) if ny % d == 0]:
        for tx in divisors(nx, 2, 64):
            n = tx * ty * ppc
            if lo <= n <= hi:
                out.append((tx, ty))
    return sorted(out, key=lambda s: (s[0] * s[1], abs(s[0] - 2 * s[1]), s))


def launch_shapes(precision: int) -> list:
    """(push_chunk, push_ctas_per_sm) pairs tried on the winning tile; (0, 0)
    is the library's choice."""
    if precision == fs.FS_FP64:
        return [(0, 0), (512, 1)]
    return [(0, 0), (512, 0), (576, 0), (576, 3), (512, 2)]


class Autotuner:
    """widths: 1D tile widths the choice is limited to where a candidate gives
    one (e.g. FsBatch.COMPILED_WIDTHS for runs that are stepped in a batch,
    whose push has those widths compiled in; the standalone probe timing does
    not see that)."""

    def __init__(self, cache_path: str | None = None, probe_particles: int = 1 << 22,
                 warm: int = 3, steps: int = 16, shapes: bool = True, widths=None):
        self.cache_path = cache_path
        self.probe_particles = probe_particles
        self.warm, self.steps = warm, steps
        self.shapes = shapes  # also tune the launch shape
        self.widths = tuple(widths) if widths else None
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)
        self.log = []

    def key(self, dim: int, ppc: int, precision: int) -> str:
        k = f"dim{dim}-ppc{ppc}-{'fp64' if precision == fs.FS_FP64 else 'fp32'}"
        return k + (f"-w{'.'.join(map(str, self.widths))}" if self.widths and dim == 1 else "")

    def _time(self, params: dict) -> float:
        """ms per step of the phases the tile and launch shapes set (push and
        movers), from the library's own CUDA-event phase timing."""
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

    def _probe(self, base: dict) -> dict:
        """A box of the class of base with about probe_particles particles
        (large enough that the kernels, not launch latency, set the time)."""
        probe = dict(base)
        ppc = base["ppc"]
        if base.get("dim", 1) == 1:
            probe["nx"] = min(max(1024, (self.probe_particles // ppc) // 1024 * 1024),
                              MAX_NX // 1024 * 1024)
        else:
            probe["ny"] = 64
            probe["nx"] = min(max(256, (self.probe_particles // (ppc * 64)) // 256 * 256),
                              MAX_NX // 256 * 256)
        for k in ("tile_x", "tile_y", "push_chunk", "push_ctas_per_sm"):
            probe.pop(k, None)
        return probe

    def _sweep(self, k: str, cands: list) -> tuple:
        best, best_ms = None, None
        for label, params in cands:
            try:
                ms = self._time(params)
            except fs.FsError as e:  # a shape the library rejects for this box
                self.log.append({"class": k, **label, "error": str(e)})
                continue
            self.log.append({"class": k, **label, "ms_per_step": ms})
            if best_ms is None or ms < best_ms:
                best, best_ms = label, ms
        return best, best_ms

    def best(self, base: dict) -> dict:
        """The tuned choice for the class of base: {"target": n} (1D) or
        {"tile": [tx, ty]} (2D), plus "push_chunk" and "push_ctas_per_sm"."""
        prec = base.get("precision", fs.FS_FP64)
        dim = base.get("dim", 1)
        k = self.key(dim, base["ppc"], prec)
        hit = self.cache.get(k)
        if isinstance(hit, dict):
            return hit
        probe = self._probe(base)
        if dim == 1:
            targets = targets_1d(probe["nx"], probe["ppc"], self.widths)
            cands = [({"target": t}, dict(probe, tile_x=tile_for(probe["nx"], probe["ppc"], t),
                                          tile_y=1)) for t in targets]
        else:
            shapes = tile_candidates_2d(probe["nx"], probe["ny"], probe["ppc"]) or [(0, 0)]
            cands = [({"tile": [tx, ty]}, dict(probe, tile_x=tx, tile_y=ty))
                     for tx, ty in shapes]
        choice, _ = self._sweep(k, cands)
        choice = dict(choice or ({"target": 512} if dim == 1 else {"tile": [0, 0]}))
        choice.update(push_chunk=0, push_ctas_per_sm=0)
        if self.shapes:
            tiled = dict(cands[0][1])
            for label, params in cands:
                if all(label.get(x) == choice.get(x) for x in ("target", "tile")):
                    tiled = params
            launch = [({"push_chunk": c, "push_ctas_per_sm": n},
                       dict(tiled, push_chunk=c, push_ctas_per_sm=n))
                      for c, n in launch_shapes(prec)]
            best_launch, _ = self._sweep(k, launch)
            if best_launch:
                choice.update(best_launch)
        self.cache[k] = choice
        if self.cache_path:
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
        return choice

    def tile(self, params: dict) -> dict:
        """params with the tuned tile (tile_x, tile_y) and launch shape
        (push_chunk, push_ctas_per_sm) set for its class."""
        c = self.best(params)
        out = dict(params, push_chunk=c["push_chunk"], push_ctas_per_sm=c["push_ctas_per_sm"])
        if params.get("dim", 1) == 1:
            out.update(tile_x=tile_for(params["nx"], params["ppc"], c["target"]), tile_y=1)
        else:
            tx, ty = c["tile"]
            if tx and params["nx"] % tx == 0 and params.get("ny", 1) % ty == 0:
                out.update(tile_x=tx, tile_y=ty)
        return out

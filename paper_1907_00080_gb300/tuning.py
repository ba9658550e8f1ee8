"""Tile shape of the fused LB kernel.

The fused kernel processes tiles of (32 * vec) x ty nodes: vec consecutive x
nodes per thread, one warp per row, ty rows per block.  Small lattices want
small vec (more threads to hide latency); large lattices want 16-byte vectors.
``TABLE`` holds shapes measured on GB300 for the benchmarked workloads;
anything else uses the library's default rule.  ``autotune`` times candidates
through the C ABI.
"""
from __future__ import annotations

import time

# (precision, nx, ny) -> (vec, ty), measured with autotune() on a GB300
TABLE = {}


def candidates(precision: str, nx: int):
    vecs = {"f64": (1, 2), "f32": (1, 2, 4), "f16": (2, 4, 8), "bf16": (2, 4, 8)}[precision]
    out = []
    for v in vecs:
        if nx % v:
            continue
        for ty in (1, 2, 4, 8):
            out.append((v, ty))
    return out


def bench_tiling(wl):
    """Tiling used by the benchmark (and by the parity test of the same
    workload): the measured table entry, else None (library default)."""
    return TABLE.get((wl.precision, wl.nx, wl.ny))


def autotune(make_sim, precision: str, nx: int, steps: int = 400, reps: int = 2):
    """Time every candidate tiling; returns (best, {tiling: seconds per step})."""
    import torch
    res = {}
    for t in candidates(precision, nx):
        sim = make_sim(t)
        sim.step(32)
        sim.sync()
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.step(steps)
            sim.sync()
            best = min(best, (time.perf_counter() - t0) / steps)
        res[t] = best
        sim.close()
    return min(res, key=res.get), res

"""Tile shape of the fused LB kernel.

The fused kernel processes tiles of (32 * vec) x ty nodes: vec consecutive x
nodes per thread, one warp per row, ty rows per block; or, with ty = 0, runs
its persistent bulk-copy form with segments of 256 * vec nodes.  Small
lattices want small vec (more threads to hide latency); large lattices want
16-byte vectors and, beyond L2, the persistent form.
``TABLE`` holds shapes measured on GB300 for the benchmarked workloads;
anything else uses the library's default rule.  ``autotune`` times candidates
through the C ABI.
"""
from __future__ import annotations

import time

# (precision, nx, ny) -> (vec, ty), measured with autotune() on a GB300
# (whole time steps, graph-launched, 3 x 2000 steps per candidate)
TABLE = {
    ("f32", 640, 160): (1, 4),  # 20.89 us/step; library default (1, 2): 21.26
}


def candidates(precision: str, nx: int):
    """Row tiles (vec, ty) and the persistent bulk-copy form (npt, 0)."""
    vecs = {"f64": (1, 2), "f32": (1, 2, 4), "f16": (2, 4, 8), "bf16": (2, 4, 8)}[precision]
    out = []
    for v in vecs:
        if nx % v:
            continue
        for ty in (1, 2, 4, 8):
            out.append((v, ty))
    halo = {"f64": 2, "f32": 4, "f16": 8, "bf16": 8}[precision]
    npts = {"f64": (1, 2), "f32": (1, 2, 4), "f16": (2, 4, 8), "bf16": (2, 4, 8)}[precision]
    if nx % halo == 0:
        out += [(n, 0) for n in npts]
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

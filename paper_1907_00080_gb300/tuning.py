"""Tile shape of the fused LB kernel, and the shape of batched ensembles.

The fused kernel processes tiles of (32 * vec) x ty nodes: vec consecutive x
nodes per thread, one warp per row, ty rows per block; or, with ty = 0, runs
its persistent bulk-copy form with segments of 256 * vec nodes.  Small
lattices want small vec (more threads to hide latency); large lattices want
16-byte vectors and, beyond L2, the persistent form.
``TABLE`` holds shapes measured on GB300 for the benchmarked workloads;
anything else uses the library's default rule.  ``autotune`` times candidates
through the C ABI.

Ensembles in the batched form share one fused-kernel shape (row tiles or the
persistent form) and are split into groups that run as independent graph
branches.  ``autotune_ensemble`` times every (shape, groups) candidate on the
ensemble itself; ``ENSEMBLE_TABLE`` keeps the choices measured on GB300 for
the benchmarked ensembles, and ``ensemble_shape`` returns the stored choice or
tunes on the spot.
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


# (precision, members, total nodes) -> ((vec, ty), groups), measured with
# autotune_ensemble() on a GB300 (3 x 320 time steps per candidate, CUDA
# events); ensemble of 64 coarse capillaries, NX 512-1008 x NY 160
ENSEMBLE_TABLE = {
    # 0.2500 ms per step; (2, 0) x 2: 0.2507, (2, 0) x 4: 0.2519, row tiles (4, 1) x 4: 0.2521,
    # (1, 0) x 4: 0.2550, (1, 0) x 1: 0.2786
    ("f32", 64, 8033280): ((2, 0), 1),
}


def ensemble_candidates(precision: str):
    """(tiling, groups) candidates of a batched ensemble: row tiles with
    16-byte vectors and the persistent form, each in 1, 2 or 4 groups."""
    shapes = {"f64": [(1, 2), (2, 1), (1, 0), (2, 0)],
              "f32": [(4, 1), (4, 2), (2, 2), (1, 0), (2, 0)],
              "f16": [(8, 1), (4, 2), (2, 0), (4, 0)],
              "bf16": [(8, 1), (4, 2), (2, 0), (4, 0)]}[precision]
    return [(t, g) for t in shapes for g in (1, 2, 4)]


def ensemble_key(workloads):
    return (workloads[0].precision, len(workloads), int(sum(wl.nx * wl.ny for wl in workloads)))


def autotune_ensemble(workloads, steps: int = 320, reps: int = 3, cuda_stream=None):
    """Time every candidate on the ensemble itself (batched form, one graph
    launch per 16 steps); returns (best (tiling, groups), {candidate: ms per
    step}).  Candidates whose tiling a member cannot take are skipped."""
    import torch
    from . import lbib
    res = {}
    prec = workloads[0].precision
    by_tiling = {}
    for t, g in ensemble_candidates(prec):
        by_tiling.setdefault(t, []).append(g)
    stream = torch.cuda.Stream() if cuda_stream is None else cuda_stream
    with torch.cuda.stream(stream):
        for t, groups in by_tiling.items():
            try:
                ens = lbib.Ensemble(workloads, cuda_stream=stream.cuda_stream, tiling=t)
            except lbib.LbibError:
                continue
            if ens.form != 1:
                ens.close()
                continue
            for g in groups:
                if g > len(workloads):
                    continue
                ens.set_groups(g)
                ens.step(32)
                ens.sync()
                best = float("inf")
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ens.step(steps)
                    e1.record(stream)
                    e1.synchronize()
                    best = min(best, e0.elapsed_time(e1) / steps)
                res[(t, g)] = best
            ens.close()
    return min(res, key=res.get), res


def ensemble_shape(workloads, cuda_stream=None):
    """(tiling, groups) for a batched ensemble: the stored choice for these
    workloads, else the autotuner's (returned with its measurements)."""
    key = ensemble_key(workloads)
    if key in ENSEMBLE_TABLE:
        return ENSEMBLE_TABLE[key], None
    best, res = autotune_ensemble(workloads, cuda_stream=cuda_stream)
    return best, res

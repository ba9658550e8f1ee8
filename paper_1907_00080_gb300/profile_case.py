"""Run one small, fixed case of the solver for a profiler (ncu) or a quick timing.

  python -m paper_1907_00080_gb300.profile_case --case probe --nx 8192 --ny 1024 --launches 3
  python -m paper_1907_00080_gb300.profile_case --case capillary --steps 40
  python -m paper_1907_00080_gb300.profile_case --case adjoint --steps 40 --checkpoint-every 20
  python -m paper_1907_00080_gb300.profile_case --case fine --precision f16 --steps 20
  python -m paper_1907_00080_gb300.profile_case --case dynamic --steps 40

``probe``: a channel of nx x ny nodes with soft circular carriers spread over
it (the coarse capillary's share of nodes under a marker stencil), stepped twice, then ``--launches``
launches of the fused collide-stream kernel alone (``lbib_profile_fused``).
``capillary``: the 640 x 160 coarse capillary stepped ``--steps`` time steps
(all kernels of the time step).  ``adjoint``: the 320 x 160 sensitivity case
(FP64) recorded for ``--steps`` steps with checkpoints every
``--checkpoint-every`` steps, then one backward sweep.  ``fine``: the 2000 x 667
fine capillary stepped ``--steps`` time steps.  ``dynamic``: the 640 x 160
capillary with dynamic carriers (Sec. 2.4) stepped ``--steps`` time steps.
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1907_00080_gb300 import build, inputs, lbib  # noqa: E402

ALG_BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}


def probe_workload(nx, ny, precision, n_carriers=None, seed=1):
    wl = inputs.Workload(name="probe_%dx%d" % (nx, ny), nx=nx, ny=ny,
                         body_force=(inputs.body_force_for(1e-5, ny), 0.0), walls=1,
                         init="poiseuille", precision=precision, membranes=[], receptors=None)
    rng = np.random.Generator(np.random.PCG64(seed))
    if n_carriers is None:
        # same share of nodes under a marker stencil as the 640 x 160 capillary
        n_carriers = max(1, int(round(256 * nx * ny / (8192 * 2048))))
    for _ in range(n_carriers):
        cx, cy = rng.uniform(0, nx), rng.uniform(20, ny - 20)
        wl.membranes.append(inputs.Membrane(xy=inputs.circle(cx, cy, 8.0, 50), ks=1e-4, kb=0.0, ka=1.0))
    return wl


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--case", choices=["probe", "capillary", "adjoint", "fine", "dynamic"], default="probe")
    p.add_argument("--nx", type=int, default=8192)
    p.add_argument("--ny", type=int, default=1024)
    p.add_argument("--precision", default="f32")
    p.add_argument("--tiling", default=None, help="vec,ty of the fused kernel")
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--checkpoint-every", type=int, default=20)
    args = p.parse_args(argv)
    build.build()
    lbib.load()
    tiling = tuple(int(v) for v in args.tiling.split(",")) if args.tiling else None
    out = {"case": args.case, "precision": args.precision}
    if args.case == "probe":
        wl = probe_workload(args.nx, args.ny, args.precision)
        sim = lbib.Simulation(wl, tiling=tiling)
        sim.step(2)
        sim.sync()
        ms = lbib.lbib_profile_fused(sim.ctx, args.launches)
        alg = ALG_BYTES_PER_NODE[args.precision] * wl.nx * wl.ny
        out.update(nx=wl.nx, ny=wl.ny, tiling=list(sim.tiling), launches=args.launches,
                   ms_per_launch=ms, algorithmic_bytes_per_launch=alg, gbs=alg / (ms * 1e-3) / 1e9)
    elif args.case == "adjoint":
        from paper_1907_00080_gb300 import sensitivity
        rec = sensitivity.Recording(sensitivity.default_params(), args.steps, args.checkpoint_every)
        try:
            g = rec.gradient((1.0, 1.0))
        finally:
            rec.close()
        out.update(precision="f64", steps=args.steps, checkpoint_every=args.checkpoint_every,
                   gradient=[float(v) for v in g])
        print(json.dumps(out))
        return 0
    else:
        if args.case == "fine":
            wl = inputs.fine_capillary_2000x667(args.precision)
        elif args.case == "dynamic":
            wl = inputs.coarse_capillary_640x160(args.precision, carrier_model="dynamic")
        else:
            wl = inputs.coarse_capillary_640x160(args.precision)
        sim = lbib.Simulation(wl, tiling=tiling)
        sim.step(args.steps)
        sim.sync()
        out.update(nx=wl.nx, ny=wl.ny, steps=args.steps, tiling=list(sim.tiling))
    sim.close()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python3
"""Benchmark of the LB-IB hot path on GB300.

Workload (the largest single-GPU configuration): an ensemble of 64 coarse
capillaries -- 10 um wide, 32-64 um long at dx = 62.5 nm (NX 512-1008 x NY
160, 8.03 M nodes in all), red cells at 20 % of the 10 x 40 um capillary's
count per length (200 markers each), 4 adhesive 1 um carriers each (50
markers; rigid or soft, sigma swept), receptors on both walls, FP32 --
synthetic, seeded inputs -- advanced in the batched form (three launches per
time step for all members, shape from the autotuner).  One benchmark "step"
advances every member by T time steps (each: forces, IB weights and
spreading, fused collide-stream, interpolation + advance, bonds).  Metric:
MLUPS including IB and adhesion (lattice nodes x time steps / s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbib|reference]
  python bench.py --profile-case probe|capillary|ensemble|fine|adjoint|dynamic ...

N > 1 runs under torchrun, one independent ensemble per GPU (weak scaling,
different seeds, no collective on the data path).  ``--impl reference`` times
the FP64 CPU oracle on all host cores on one member of the same ensemble (a
bounded sample per step).  ``--profile-case`` runs one small fixed case for a
profiler (ncu) and prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MLUPS incl. IB+adhesion"
UNIT = "MLUPS"
WORKLOAD = ("ensemble of 64 coarse capillaries (10 um x 32-64 um at dx = 62.5 nm: NX 512-1008 x NY 160, "
            "8.03 M nodes, 138,600 markers, 4 carriers each, receptors on both walls), batched form")
C2_WORKLOAD = "coarse capillary 640x160: 8 RBC x 200 markers, 4 carriers x 50 markers, receptors on both walls"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
ENSEMBLE_N = 64


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="lbib", choices=["lbib", "reference"])
    p.add_argument("--timesteps-per-step", type=int, default=200)
    p.add_argument("--precision", default="f32")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-probe", action="store_true")
    p.add_argument("--no-forms", action="store_true")
    p.add_argument("--no-c2", action="store_true", help="skip the 640 x 160 capillary line")
    # one small fixed case for a profiler
    p.add_argument("--profile-case", default=None,
                   choices=["probe", "capillary", "ensemble", "fine", "adjoint", "dynamic"])
    p.add_argument("--nx", type=int, default=8192)
    p.add_argument("--ny", type=int, default=1024)
    p.add_argument("--tiling", default=None, help="vec,ty of the fused kernel")
    p.add_argument("--groups", type=int, default=1)
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--case-steps", type=int, default=40)
    p.add_argument("--checkpoint-every", type=int, default=20)
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def workload(precision, seed=0):
    """the 640 x 160 coarse capillary"""
    from paper_1907_00080_gb300 import inputs
    return inputs.capillary(precision=precision, seed=seed, steps=200000, name="capillary_640x160")


def ensemble_workloads(precision, seed=0):
    """the 64-member ensemble (member i seeded seed + i)"""
    from paper_1907_00080_gb300 import inputs
    return inputs.capillary_ensemble(ENSEMBLE_N, seed=seed, precision=precision)


def cpu_model():
    """the host CPU's model name (lscpu, else /proc/cpuinfo)"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def ncu_traffic():
    """DRAM bytes per launch (read + write) of the current kernels, from the
    ncu summaries under profiles/: lines `traffic_per_launch: <key> <bytes>`"""
    out = {}
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return out
    for name in sorted(os.listdir(d)):
        if not name.endswith(".md"):
            continue
        with open(os.path.join(d, name)) as fh:
            for ln in fh:
                if ln.startswith("traffic_per_launch:"):
                    parts = ln.split()
                    if len(parts) >= 3:
                        out[parts[1]] = int(float(parts[2]))
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


# ------------------------------------------------------------------ reference arm
def cpu_oracle_mlups(wl, timesteps, threads=1):
    """Time the FP64 CPU oracle (as it stands) for `timesteps` steps, on one
    thread or, threads > 1, its OpenMP build with that many threads."""
    import oracle
    used = oracle.use_threads(threads)
    try:
        s = _oracle_sim(wl)
        s.step(1)
        t0 = time.perf_counter()
        s.step(timesteps)
        dt = time.perf_counter() - t0
        del s
    finally:
        oracle.use_threads(1)
    return wl.nx * wl.ny * timesteps / dt / 1e6, dt, used


def cpu_baseline(precision_note="FP64 C oracle"):
    """The oracle on member 0 of the ensemble: one thread (300 steps) and its
    OpenMP build on every host core (1500 steps); `value` is the all-core
    figure."""
    wl = ensemble_workloads("f64")[0]
    n1, n_all = 300, 1500
    m1, d1, _ = cpu_oracle_mlups(wl, n1, 1)
    cores = os.cpu_count() or 1
    ma, da, used = cpu_oracle_mlups(wl, n_all, cores)
    return {"value": ma, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": "%d time steps of ensemble member 0 (%dx%d, %d membranes, bonds), %s, OpenMP over nodes, "
                      "rows and vertices on %d threads, %.1f s" % (n_all, wl.nx, wl.ny, len(wl.membranes),
                                                                    precision_note, used, da),
            "cpu_model": cpu_model(), "flags": "gcc -O2 -ffp-contract=off -fopenmp",
            "single_thread": {"value": m1, "unit": UNIT, "cores": 1,
                              "sample": "%d time steps of the same member, one thread, %.1f s" % (n1, d1)}}


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (the job's time is its slowest
    rank's)."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    if args.profile_case:
        return profile_case_main(args)
    if args.impl == "reference":
        return reference_main(args)
    return lbib_main(args)


def reference_main(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    import oracle
    wl = ensemble_workloads("f64")[0]
    sample = 20
    cores = os.cpu_count() or 1
    used = oracle.use_threads(cores)
    s = _oracle_sim(wl)
    s.step(sample * args.warmup)
    t0 = time.perf_counter()
    s.step(sample * args.steps)
    dt = time.perf_counter() - t0
    del s
    oracle.use_threads(1)
    mlups = wl.nx * wl.ny * sample * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + "; FP64 CPU oracle on member 0 (%dx%d)" % (wl.nx, wl.ny),
                   "nx": wl.nx, "ny": wl.ny, "timesteps_per_step": sample},
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": "%d time steps per benchmark step of ensemble member 0, FP64 C oracle, OpenMP "
                                   "on %d threads" % (sample, used),
                         "cpu_model": cpu_model()},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _oracle_sim(wl):
    import oracle
    s = oracle.OracleSim(wl.nx, wl.ny, wl.tau, wl.body_force, wl.walls, init=wl.init)
    for m in wl.membranes:
        s.add_membrane(m.xy, m.ks, m.kb, m.ka, m.kind, m.ligands)
    b = wl.bonds
    s.set_receptors(wl.receptors, d_cut=b["d_cut"], y_eq=b["y_eq"], sigma=wl.sigma_lu,
                    kf_dt=b["kf_dt"], kr0_dt=b["kr0_dt"], beta_f=b["beta_f"], beta_r=b["beta_r"],
                    d_break=b["d_break"], seed=wl.seed, instance=wl.instance)
    s.set_repulsion(wl.d_rep)
    return s


def lbib_main(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1907_00080_gb300 import build, lbib, tuning
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    lbib.load()

    T = args.timesteps_per_step
    wls = ensemble_workloads(args.precision, seed=ENSEMBLE_N * rank)
    nodes = sum(wl.nx * wl.ny for wl in wls)
    markers = sum(wl.n_vertices for wl in wls)
    stream = torch.cuda.Stream()
    (tiling, groups), tuned = tuning.ensemble_shape(wls, cuda_stream=stream)
    ens = lbib.Ensemble(wls, cuda_stream=stream.cuda_stream, tiling=tiling)
    if ens.form != 1:
        raise RuntimeError("the benchmark ensemble did not take the batched form")
    ens.set_groups(groups)
    lps = ens.launches_per_step

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ens.step(T)
        ens.sync()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            starts[k].record(stream)
            ens.step(T)
            ends[k].record(stream)
        ens.sync()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clocks = clk.stop()
    ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    elapsed = ms / 1e3
    if dist is not None:
        elapsed = max_over_ranks(elapsed, dist, "cuda")
    value = nodes * T * args.steps * ws / elapsed / 1e6
    ens.close()

    # ---- the batched kernels timed alone on a scratch copy of the ensemble;
    # the top-level roofline is the kernel with the largest share
    pk, pk_kind = peaks()
    traffic = ncu_traffic()
    kernels = ensemble_kernels(lbib, torch, stream, wls, tiling, groups, args.precision, pk, traffic)
    top = max(kernels, key=lambda k: k["ms_per_launch"])
    roofline = dict(top)
    roofline["peak_kind"] = pk_kind + " (copy bandwidth, burst)"
    roofline["share_of_kernel_time"] = top["ms_per_launch"] / sum(k["ms_per_launch"] for k in kernels)
    roofline["note"] = ("dominant kernel of the ensemble's time step (all 64 members in one launch), timed alone "
                        "with CUDA events on a scratch copy; algorithmic bytes = 9 populations read + 9 written "
                        "per node (frac_with_ib also counts the IB coupling's bytes in the flagged force tiles: "
                        "force read, velocity written, other parity cleared); traffic from the ncu summary of "
                        "the same kernel under profiles/")

    probe = probe16 = None
    if not args.no_probe and rank == 0:
        probe = hbm_probe(lbib, torch, stream, args.precision, pk, pk_kind, traffic)
        # the FP16-storage form of the same probe (36 B/node; producer-warp schedule, 4 nodes per thread)
        probe16 = hbm_probe(lbib, torch, stream, "f16", pk, pk_kind, traffic, tiling=(4, 0))

    c2 = None
    if not args.no_c2 and rank == 0:
        c2 = capillary_line(lbib, torch, stream, args.precision, pk, traffic)

    forms = None
    if not args.no_forms and rank == 0:
        forms = {"ensemble": ensemble_form(lbib, torch, stream, wls, tiling, groups),
                 "precision": precision_forms(lbib, torch, stream),
                 "differentiation": differentiation_form(lbib, torch),
                 "couette_cell_free_layer": couette_form(lbib, torch, stream),
                 "dynamic_carriers": dynamic_form(lbib, torch, stream)}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = ensemble_e2e(lbib, torch, wls, tiling, groups, stream, T, max(2, min(args.steps, 4)))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": WORKLOAD, "members": len(wls), "nodes": nodes, "markers": markers,
                       "nx_range": [min(wl.nx for wl in wls), max(wl.nx for wl in wls)], "ny": wls[0].ny,
                       "timesteps_per_step": T, "tiling": list(tiling), "groups": groups,
                       "shape_from": "autotuner table" if tuned is None else "autotuned on this run",
                       "l2": "inputs larger than L2: 2 x 578 MB of populations (129 MB L2); no flush",
                       "parallelism": "one ensemble per GPU x%d" % ws},
            "roofline": roofline,
            "roofline_kernels": kernels,
            "roofline_hbm_probe": probe,
            "roofline_hbm_probe_f16": probe16,
            "capillary_640x160": c2,
            "forms": forms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": lps * T * args.steps,
            "kernels_per_timestep": lps,
            "clocks": clocks,
            "wall_s_timed_region": wall,
        }
        if tuned is not None:
            line["config"]["autotune_ms_per_step"] = {"%s/%d" % (t, g): v for (t, g), v in tuned.items()}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


KERNEL_NAMES = ("k_forces (forces, IB weights, spreading)", "k_lb_step / k_lb_stream (fused collide-stream)",
                "k_advance (interpolation, advance, bonds)")
ENSEMBLE_KERNEL_NAMES = ("k_forces_batch (forces, IB weights, spreading; all members)",
                         "k_lb_stream_ws_batch / k_lb_step_batch (fused collide-stream; all members)",
                         "k_advance_batch (interpolation, advance, bonds; all members)")


def ensemble_kernels(lbib, torch, stream, wls, tiling, groups, precision, pk, traffic):
    """The three batched kernels of the ensemble timed alone (200 back-to-back
    launches each, CUDA events on the stream; lbib_ensemble_profile_kernels on
    a scratch copy), with their algorithmic bytes per launch (the members'
    sums, as in alg_bytes_per_launch)."""
    scratch = lbib.Ensemble(wls, cuda_stream=stream.cuda_stream, tiling=tiling)
    scratch.set_groups(groups)
    with torch.cuda.stream(stream):
        scratch.step(4)
        scratch.sync()
        # the force tiles the fused kernel reads, from the markers' positions
        flagged = sum(flagged_nodes(wl, m.markers()) for wl, m in zip(wls, scratch.members))
        kms = lbib.lbib_ensemble_profile_kernels(scratch.ens, 200)
    scratch.close()
    alg = [0, 0, 0]
    for wl in wls:
        for k, b in enumerate(alg_bytes_per_launch(precision, wl)):
            alg[k] += b
    key = {0: "k_forces_batch", 1: "fused_batch", 2: "k_advance_batch"}
    out = []
    for k, (name, ms_k, b) in enumerate(zip(ENSEMBLE_KERNEL_NAMES, kms, alg)):
        gbs = b / (ms_k * 1e-3) / 1e9 if ms_k > 0 else 0.0
        out.append({"kernel": name, "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / pk["hbm_gbs"], "ms_per_launch": ms_k, "algorithmic_bytes_per_launch": b,
                    "traffic": traffic.get("%s:ensemble64_%s:%d,%d" % (key[k], precision, tiling[0], tiling[1]))})
        if k == 1 and ms_k > 0:
            # the same kernel with the bytes of its IB coupling counted
            nodes = sum(wl.nx * wl.ny for wl in wls)
            ib = flagged * ib_bytes_per_flagged_node(precision)
            out[-1].update(flagged_tile_fraction=flagged / nodes, ib_bytes_per_launch=ib,
                           achieved_with_ib=(b + ib) / (ms_k * 1e-3) / 1e9,
                           frac_with_ib=(b + ib) / (ms_k * 1e-3) / 1e9 / pk["hbm_gbs"])
    return out


def capillary_line(lbib, torch, stream, precision, pk, traffic, T=1000, steps=5, warmup=3):
    """The 640 x 160 coarse capillary alone (L2-resident, latency-bound): MLUPS
    over `steps` calls of T time steps (CUDA events; L2 flushed between
    calls) and its three kernels timed alone."""
    from paper_1907_00080_gb300 import tuning
    wl = workload(precision)
    tiling = tuning.bench_tiling(wl)
    sim = lbib.Simulation(wl, tiling=tiling, cuda_stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            sim.step(T)
        sim.sync()
        ms = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(T)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
    vec, ty = sim.tiling
    sim.close()
    del flush
    scratch = lbib.Simulation(wl, tiling=tiling, cuda_stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        scratch.step(4)
        scratch.sync()
        lbib.lbib_profile_kernels(scratch.ctx, 50)
        kms = lbib.lbib_profile_kernels(scratch.ctx, 500)
    scratch.close()
    alg = alg_bytes_per_launch(precision, wl)
    key = {0: "k_forces", 1: "fused", 2: "k_advance"}
    kernels = []
    for k, (name, ms_k, b) in enumerate(zip(KERNEL_NAMES, kms, alg)):
        gbs = b / (ms_k * 1e-3) / 1e9 if ms_k > 0 else 0.0
        kernels.append({"kernel": name, "ms_per_launch": ms_k, "algorithmic_bytes_per_launch": b,
                        "achieved_gbs": gbs, "frac": gbs / pk["hbm_gbs"],
                        "traffic": traffic.get("%s:capillary_640x160_%s" % (key[k], precision))})
    return {"workload": C2_WORKLOAD, "mlups": wl.nx * wl.ny * T * steps / (ms * 1e-3) / 1e6,
            "us_per_timestep": 1e3 * ms / (T * steps), "tiling": [vec, ty], "timesteps": T * steps,
            "l2": "flushed (256 MB write) between calls; within one the lattice (7.4 MB) is L2-resident",
            "kernels": kernels}


def ensemble_e2e(lbib, torch, wls, tiling, groups, stream, T, steps):
    """End to end through the public API with host buffers: per step, every
    member's populations (FP64) and markers go up from pinned host memory
    (lbib_ensemble_write_state), the ensemble advances T time steps, every
    member's markers come back (lbib_ensemble_read_markers); host wall clock."""
    ens = lbib.Ensemble(wls, cuda_stream=stream.cuda_stream, tiling=tiling)
    ens.set_groups(groups)
    with torch.cuda.stream(stream):
        ens.step(2)
        ens.sync()
        f_host, x_host, x_out = [], [], []
        for wl, m in zip(wls, ens.members):
            f = torch.empty((9, wl.ny, wl.nx), dtype=torch.float64, pin_memory=True).numpy()
            f[:] = m.populations()
            x = torch.empty((m.nv, 2), dtype=torch.float64, pin_memory=True).numpy()
            x[:] = m.markers()
            f_host.append(f)
            x_host.append(x)
            x_out.append(torch.empty((m.nv, 2), dtype=torch.float64, pin_memory=True).numpy())

        def one():
            # every member's populations and markers up in one call, the
            # steps, the status check, every member's markers back
            ens.write_state(f=f_host, xy=x_host)  # X^{n-1} = X^n from the same upload
            ens.step(T)
            ens.sync()
            ens.read_markers(x_out)

        one()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    ens.close()
    nodes = sum(wl.nx * wl.ny for wl in wls)
    h2d = sum(f.nbytes for f in f_host) + sum(x.nbytes for x in x_host)
    d2h = sum(x.nbytes for x in x_out)
    return {"value": nodes * T * steps / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps,
            "note": "host wall clock; each step uploads every member's populations + markers, advances %d time "
                    "steps, reads every member's markers back" % T}


def alg_bytes_per_launch(precision, wl):
    """Algorithmic bytes per launch of the three kernels of a time step.
    forces, per vertex: position 16, rest record (28 FP32 / 32 FP64), force
    2 values, 9 weights, stencil origin 8, 9 fixed-point spread
    read-modify-writes of 16 B (288).  fused, per node: 9 populations read +
    9 written.  advance, per vertex: 9 weights + stencil 8, 9 gathered
    velocities (2 values each), X^n and X^{n-1} read and written (64), U (2
    values)."""
    cs = 8 if precision == "f64" else 4
    rest = 32 if precision == "f64" else 28
    pop = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}[precision]
    nv = wl.n_vertices
    forces = nv * (16 + rest + 2 * cs + 9 * cs + 8 + 9 * 32)
    fused = pop * wl.nx * wl.ny
    advance = nv * (9 * cs + 8 + 18 * cs + 64 + 2 * cs)
    return forces, fused, advance


def flagged_nodes(wl, xy):
    """Nodes of the 32-node force tiles that the spreading of markers at xy
    (N, 2) flags: the tiles holding a node of some marker's 3 x 3 stencil
    (origin floor(x + 1/2), rows outside the walls dropped), as the force
    kernel flags them."""
    import numpy as np
    tx = (wl.nx + 31) // 32
    i0 = np.floor(xy[:, 0] + 0.5).astype(np.int64)
    j0 = np.floor(xy[:, 1] + 0.5).astype(np.int64)
    tiles = set()
    for dy in (-1, 0, 1):
        jj = j0 + dy
        ok = (jj >= 0) & (jj < wl.ny) if wl.walls else np.ones_like(jj, bool)
        jj = jj % wl.ny
        for dx in (-1, 0, 1):
            ii = (i0 + dx) % wl.nx
            tiles.update((jj[ok] * tx + ii[ok] // 32).tolist())
    # the last tile of a row is short when NX is not a multiple of 32
    last = wl.nx - 32 * (tx - 1)
    return sum(last if t % tx == tx - 1 else 32 for t in tiles)


def ib_bytes_per_flagged_node(precision):
    """Fused-kernel bytes of the IB coupling per node of a flagged force tile:
    the fixed-point force read (16), the velocity written for the
    interpolation (2 values of the compute type) and the other parity's force
    cleared (16; its tiles are the previous step's, about as many)."""
    cs = 8 if precision == "f64" else 4
    return 16 + 2 * cs + 16


def hbm_probe(lbib, torch, stream, precision, pk, pk_kind, traffic, tiling=None):
    """Fused kernel on an 8192 x 2048 lattice (1.2 GB of FP32 populations per
    buffer, far above L2) with the capillary's marker density scaled up."""
    from paper_1907_00080_gb300 import inputs
    nx, ny = 8192, 2048
    wl = inputs.probe_lattice(nx, ny, precision)  # 256 soft carriers of 50 markers
    sim = lbib.Simulation(wl, cuda_stream=stream.cuda_stream, tiling=tiling)
    vec, ty = sim.tiling
    with torch.cuda.stream(stream):
        sim.step(2)
        sim.sync()
        lbib.lbib_profile_fused(sim.ctx, 5)
        ms = lbib.lbib_profile_fused(sim.ctx, 40)
    sim.close()
    alg = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}[precision] * nx * ny
    gbs = alg / (ms * 1e-3) / 1e9
    # the 8192 x 1024 capture scaled by the nodes (traffic grows in proportion)
    t = traffic.get("fused:probe_8192x1024_%s:%d,%d" % (precision, vec, ty))
    return {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / pk["hbm_gbs"], "traffic": 2 * t if t else None, "nx": nx, "ny": ny,
            "tiling": [vec, ty], "ms_per_launch": ms, "algorithmic_bytes_per_launch": alg,
            "peak_kind": pk_kind + " (copy bandwidth, burst)", "mlups_fused_kernel": nx * ny / (ms * 1e-3) / 1e6}


def precision_forms(lbib, torch, stream, checkpoints=(1000, 10000), timed=2000):
    """Precision form: the fine capillary (2000 x 667, 4 red cells x 1700 + 3 rigid
    carriers x 210 markers released 1 lu from a wall, the paper's bond cut-off
    y_cr = 1.67 lu, so that bonds form) with populations stored in FP32, FP16 and
    BF16 (shifted: d_i 2^k) against the FP64 run from the same inputs.  Errors
    after each checkpoint (time steps): velocity L2 and Linf relative to the
    FP64 field, marker Linf in lattice units, bond count and the ligands whose
    bond differs from the FP64 run's; throughput over `timed` further steps
    (CUDA events on the stream)."""
    from paper_1907_00080_gb300 import inputs
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    res, ref = {}, {}
    for prec in ("f64", "f32", "f16", "bf16"):
        wl = inputs.fine_capillary_adhering(prec)
        sim = lbib.Simulation(wl, cuda_stream=stream.cuda_stream)
        r = {"tiling": list(sim.tiling), "storage_scale_exponent": int(lbib.lbib_storage_scale_exponent(sim.ctx))}
        done = 0
        with torch.cuda.stream(stream):
            for cp in checkpoints:
                sim.step(cp - done)
                done = cp
                sim.sync()
                _, ux, uy = sim.fields()
                x = sim.markers()
                bl = sim.bonds()
                nb = int((bl >= 0).sum())
                f = sim.populations()
                e = {"max_abs_deviation": float(np.max(np.abs(f - w))), "bonds": nb}
                if prec == "f64":
                    ref[cp] = (ux, uy, x, nb, bl)
                else:
                    rx = ref[cp]
                    du = np.hypot(ux - rx[0], uy - rx[1])
                    um = np.hypot(rx[0], rx[1])
                    e.update(u_err_linf=float(du.max() / um.max()),
                             u_err_l2=float(np.sqrt((du ** 2).sum() / (um ** 2).sum())),
                             marker_err_linf_lu=float(np.max(np.abs(x - rx[2]))), bond_count_diff=nb - rx[3],
                             ligands_with_other_bond=int((bl != rx[4]).sum()))
                r["after_%d_steps" % cp] = e
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(timed)
            e1.record(stream)
            sim.sync()
            ms = e0.elapsed_time(e1)
            # the fused kernel alone on this lattice (the three kernels timed
            # back to back, lbib_profile_kernels): its share of the roofline
            kms = lbib.lbib_profile_kernels(sim.ctx, 100)
        r["mlups"] = wl.nx * wl.ny * timed / (ms * 1e-3) / 1e6
        alg = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}[prec] * wl.nx * wl.ny
        r["fused_kernel"] = {"ms_per_launch": kms[1], "algorithmic_bytes": alg,
                             "achieved_gbs": alg / (kms[1] * 1e-3) / 1e9,
                             "frac_of_hbm": alg / (kms[1] * 1e-3) / 1e9 / peaks()[0]["hbm_gbs"],
                             "note": "two buffers of this lattice partly fit in the 129 MB L2"}
        res[prec] = r
        sim.close()
    base = res["f32"]["mlups"]
    for prec in ("f16", "bf16"):
        res[prec]["speedup_vs_f32"] = res[prec]["mlups"] / base
    return {"workload": "fine capillary 2000x667 (dx = 15 nm), 4 RBC x 1700 + 3 rigid carriers x 210 markers "
                        "released 1 lu from a wall, bond cut-off y_cr = 1.67 lu",
            "checkpoints": list(checkpoints), "timed_steps": timed, "results": res}


def couette_form(lbib, torch, stream, warm=2000, timed=4000):
    """The adhesion set-up of the cell-free layer (600 x 200 planar Couette
    flow, Re = 0.003, upper wall moving, receptors on the lower wall, one 1 um
    carrier released 1 lu above it), FP32 storage, rigid and soft carriers,
    sigma in {0.5, 1, 2}: throughput over `timed` steps after `warm` (CUDA
    events on the stream); at the end, from lbib_membrane_observables, the
    bonds n_L (and their ratio to the count after the warm-up), the rolling
    velocity over the wall speed, the lowest marker height and the region."""
    from paper_1907_00080_gb300 import inputs
    res = {}
    for carrier in ("rigid", "soft"):
        for sigma in (0.5, 1.0, 2.0):
            wl = inputs.couette_cfl_600x200("f32", sigma=sigma, carrier=carrier)
            sim = lbib.Simulation(wl, cuda_stream=stream.cuda_stream)
            with torch.cuda.stream(stream):
                sim.step(warm)
                sim.sync()
                o0 = sim.observables()[0]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(timed)
                e1.record(stream)
                sim.sync()
                ms = e0.elapsed_time(e1)
            o = sim.observables()[0]
            res["%s_sigma%g" % (carrier, sigma)] = {
                "mlups": wl.nx * wl.ny * timed / (ms * 1e-3) / 1e6, "bonds": int(o[5]),
                "n_L_over_n_L_after_warm": float(o[5] / o0[5]) if o0[5] > 0 else None,
                # mean centroid speed over the timed steps, over the wall speed
                "u_roll_over_u_wall": float((o[0] - o0[0]) / timed / wl.wall_velocity[1]),
                "carrier_min_height_lu": float(o[6]), "region": int(o[4]), "tiling": list(sim.tiling)}
            sim.close()
    return {"workload": "Couette 600x200 (dx = 15 nm, H_CFL = 3 um), Re = 0.003, one 1 um carrier x 210 markers, "
                        "FP32", "steps": warm + timed, "results": res}


def dynamic_form(lbib, torch, stream, warm=200, timed=4000, couette_warm=2000, couette_timed=4000):
    """The dynamic IB of Sec. 2.4 for the carriers (rigid: Newton-Euler; soft:
    Verlet; probe tractions and direct forcing) against their kinematic
    reading on the same workloads: the coarse 640 x 160 capillary in FP32 and
    FP64 (MLUPS over `timed` steps after `warm`, CUDA events on the stream, and
    the hydrodynamic-stress kernel's own time per launch), and the Couette
    cell-free-layer carrier at sigma = 1 (rolling velocity and bonds)."""
    from paper_1907_00080_gb300 import inputs, tuning
    cap = {}
    for prec in ("f32", "f64"):
        for model in ("kinematic", "dynamic"):
            wl = inputs.coarse_capillary_640x160(prec, carrier_model=model)
            sim = lbib.Simulation(wl, tiling=tuning.bench_tiling(wl), cuda_stream=stream.cuda_stream)
            with torch.cuda.stream(stream):
                sim.step(warm)
                sim.sync()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(timed)
                e1.record(stream)
                sim.sync()
                ms = e0.elapsed_time(e1)
                entry = {"mlups": wl.nx * wl.ny * timed / (ms * 1e-3) / 1e6, "us_per_step": 1e3 * ms / timed,
                         "kernels_per_step": sim.kernels_per_step}
                if model == "dynamic":
                    lbib.lbib_profile_hydro(sim.ctx, 20)
                    entry["k_hydro_us_per_launch"] = 1e3 * lbib.lbib_profile_hydro(sim.ctx, 500)
            cap["%s_%s" % (model, prec)] = entry
            sim.close()
    for prec in ("f32", "f64"):
        d, k = cap["dynamic_" + prec], cap["kinematic_" + prec]
        d["step_time_over_kinematic"] = d["us_per_step"] / k["us_per_step"]
    couette = {}
    for carrier in ("rigid", "soft"):
        wl = inputs.couette_cfl_600x200("f32", sigma=1.0, carrier=carrier, carrier_model="dynamic")
        sim = lbib.Simulation(wl, cuda_stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            sim.step(couette_warm)
            sim.sync()
            o0 = sim.observables()[0]
            sim.step(couette_timed)
            sim.sync()
        o = sim.observables()[0]
        couette["dynamic_%s_sigma1" % carrier] = {
            "bonds": int(o[5]), "n_L_over_n_L_after_warm": float(o[5] / o0[5]) if o0[5] > 0 else None,
            "u_roll_over_u_wall": float((o[0] - o0[0]) / couette_timed / wl.wall_velocity[1]),
            "carrier_min_height_lu": float(o[6])}
        sim.close()
    return {"workload": "capillary 640x160 (8 red cells, 4 carriers, 1 280 receptors), carriers kinematic "
                        "(rigid-projected / kinematic) vs dynamic (Newton-Euler / Verlet, rho_P/rho = 1.1); "
                        "Couette 600x200 one 1 um dynamic carrier, FP32",
            "capillary": cap, "couette_cell_free_layer": couette,
            "steps": {"capillary": warm + timed, "couette": couette_warm + couette_timed}}


def ensemble_form(lbib, torch, stream, wls, tiling, groups, steps=5000):
    """Ensemble form: the 64 coarse capillaries of the headline in the batched
    form (autotuned shape) against the same instances run one after another
    as plain single runs (each at its own default tiling), over `steps` time
    steps each.  MLUPS = all instances' nodes x steps / time (CUDA events on
    the stream)."""
    nodes = sum(wl.nx * wl.ny for wl in wls)

    def timed(run):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    with torch.cuda.stream(stream):
        ens = lbib.Ensemble(wls, cuda_stream=stream.cuda_stream, tiling=tiling)
        ens.set_groups(groups)
        ens.step(32)
        ens.sync()
        t_ens = timed(lambda: ens.step(steps))
        ens.sync()
        ens.close()
        sims = [lbib.Simulation(wl, cuda_stream=stream.cuda_stream) for wl in wls]
        for s_ in sims:
            s_.step(32)
        torch.cuda.synchronize()

        def sequential():
            for s_ in sims:
                s_.step(steps)

        t_seq = timed(sequential)
        for s_ in sims:
            s_.close()
    return {"workload": "%d coarse capillaries, NX %d-%d x NY 160, %d nodes, %d markers in all" % (
                len(wls), min(wl.nx for wl in wls), max(wl.nx for wl in wls), nodes,
                sum(wl.n_vertices for wl in wls)),
            "tiling": list(tiling), "groups": groups,
            "steps": steps, "ensemble_mlups": nodes * steps / t_ens / 1e6,
            "sequential_mlups": nodes * steps / t_seq / 1e6, "speedup_vs_sequential": t_seq / t_ens,
            "ensemble_ms_per_step": 1e3 * t_ens / steps, "sequential_ms_per_step": 1e3 * t_seq / steps}


def differentiation_form(lbib, torch, steps=5000, checkpoint_every=250):
    """Differentiation form: the 320 x 160 sensitivity case (2 red cells, a soft
    carrier released 1 lu above the wall), FP64: dJ/dp of the carrier's final
    height J1 and bond energy J2 with respect to (k_s, k_b, sigma, release
    height).  Reverse mode: one recorded run (checkpoints every 250 steps) and
    one backward sweep per observable, each giving all four derivatives; from
    an FP64 forward run and from an FP32 one (FP64 adjoint in both).
    Forward mode: four tangent runs.  Both timed against the plain FP64 solver
    over the same steps (host wall clock around synchronised calls)."""
    from paper_1907_00080_gb300 import sensitivity
    p0 = sensitivity.default_params()
    sensitivity.run(p0, 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, _ = sensitivity.run(p0, steps)
    t_primal = time.perf_counter() - t0
    t0 = time.perf_counter()
    rec = sensitivity.Recording(p0, steps, checkpoint_every=checkpoint_every)
    t_rec = time.perf_counter() - t0
    try:
        t0 = time.perf_counter()
        g1 = rec.gradient((1.0, 0.0))
        t_sweep = time.perf_counter() - t0
        g2 = rec.gradient((0.0, 1.0))
    finally:
        rec.close()
    jac_a = np.stack([g1, g2])
    # the same gradient from an FP32 forward run (FP64 adjoint and accumulation)
    sim32 = lbib.Simulation(sensitivity.make_workload(p0, steps, precision="f32"), precision="f32")
    sim32.step(10)
    sim32.sync()
    t0 = time.perf_counter()
    sim32.step(steps)
    sim32.sync()
    t_primal32 = time.perf_counter() - t0
    sim32.close()
    t0 = time.perf_counter()
    rec32 = sensitivity.Recording(p0, steps, checkpoint_every=checkpoint_every, precision="f32")
    t_rec32 = time.perf_counter() - t0
    try:
        t0 = time.perf_counter()
        h1 = rec32.gradient((1.0, 0.0))
        t_sweep32 = time.perf_counter() - t0
        h2 = rec32.gradient((0.0, 1.0))
    finally:
        rec32.close()
    jac32 = np.stack([h1, h2])
    rel32 = [float(np.max(np.abs(jac32[i] - jac_a[i]) / np.maximum(np.abs(jac_a[i]), 1e-300))) for i in range(2)]
    t0 = time.perf_counter()
    J2, jac, bonds = sensitivity.jacobian(p0, steps)
    t_jac = time.perf_counter() - t0
    rel = [float(np.max(np.abs(jac_a[i] - jac[i]) / np.maximum(np.abs(jac[i]), 1e-300))) for i in range(2)]
    return {"workload": "320x160, 2 RBC x 200 + 1 soft carrier x 50 markers, FP64", "steps": steps,
            "params": list(sensitivity.PARAMS), "J": [float(v) for v in J],
            "dJ_dp": [[float(v) for v in row] for row in jac_a], "bonds_at_end": int((bonds >= 0).sum()),
            "primal_ms_per_step": 1e3 * t_primal / steps,
            "adjoint": {"checkpoint_every": checkpoint_every, "record_ms_per_step": 1e3 * t_rec / steps,
                        "sweep_ms_per_step": 1e3 * t_sweep / steps,
                        "gradient_cost_vs_primal": (t_rec + t_sweep) / t_primal,
                        "max_rel_diff_vs_tangent": rel},
            "adjoint_fp32_forward": {"primal_ms_per_step": 1e3 * t_primal32 / steps,
                                     "record_ms_per_step": 1e3 * t_rec32 / steps,
                                     "sweep_ms_per_step": 1e3 * t_sweep32 / steps,
                                     "gradient_cost_vs_fp32_primal": (t_rec32 + t_sweep32) / t_primal32,
                                     "max_rel_diff_vs_fp64_adjoint": rel32},
            "tangent": {"jacobian_ms_per_step": 1e3 * t_jac / steps,
                        "cost_per_direction_vs_primal": t_jac / 4 / t_primal,
                        "gradient_cost_vs_primal": t_jac / 4 / t_primal * 4}}


# ------------------------------------------------------------------ profiler cases
ALG_BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}


def profile_case_main(args):
    """One small, fixed case for a profiler (ncu) or a quick timing; prints
    one JSON line.  probe: an nx x ny channel with soft carriers spread over
    it (inputs.probe_lattice), stepped twice, then --launches launches of the
    fused kernel alone (lbib_profile_fused).  capillary / fine / dynamic: the
    640 x 160 capillary, the 2000 x 667 fine capillary, or the capillary with
    dynamic carriers, stepped --case-steps time steps.  ensemble: the 64-member
    ensemble in the batched form (--tiling, --groups) stepped --case-steps
    time steps.  adjoint: the 320 x 160 sensitivity case (FP64) recorded for
    --case-steps steps with checkpoints every --checkpoint-every, then one
    backward sweep."""
    from paper_1907_00080_gb300 import build, inputs, lbib
    build.build()
    lbib.load()
    tiling = tuple(int(v) for v in args.tiling.split(",")) if args.tiling else None
    out = {"case": args.profile_case, "precision": args.precision}
    if args.profile_case == "probe":
        wl = inputs.probe_lattice(args.nx, args.ny, args.precision)
        sim = lbib.Simulation(wl, tiling=tiling)
        sim.step(2)
        sim.sync()
        ms = lbib.lbib_profile_fused(sim.ctx, args.launches)
        alg = ALG_BYTES_PER_NODE[args.precision] * wl.nx * wl.ny
        out.update(nx=wl.nx, ny=wl.ny, tiling=list(sim.tiling), launches=args.launches,
                   ms_per_launch=ms, algorithmic_bytes_per_launch=alg, gbs=alg / (ms * 1e-3) / 1e9)
        sim.close()
    elif args.profile_case == "ensemble":
        wls = ensemble_workloads(args.precision)
        ens = lbib.Ensemble(wls, tiling=tiling)
        if ens.form == 1:
            ens.set_groups(args.groups)
        ens.step(args.case_steps)
        ens.sync()
        out.update(members=len(wls), form=ens.form, groups=ens.groups, steps=args.case_steps,
                   tiling=list(tiling) if tiling else None)
        ens.close()
    elif args.profile_case == "adjoint":
        from paper_1907_00080_gb300 import sensitivity
        rec = sensitivity.Recording(sensitivity.default_params(), args.case_steps, args.checkpoint_every)
        try:
            g = rec.gradient((1.0, 1.0))
        finally:
            rec.close()
        out.update(precision="f64", steps=args.case_steps, checkpoint_every=args.checkpoint_every,
                   gradient=[float(v) for v in g])
    else:
        if args.profile_case == "fine":
            wl = inputs.fine_capillary_2000x667(args.precision)
        elif args.profile_case == "dynamic":
            wl = inputs.coarse_capillary_640x160(args.precision, carrier_model="dynamic")
        else:
            wl = inputs.coarse_capillary_640x160(args.precision)
        sim = lbib.Simulation(wl, tiling=tiling)
        sim.step(args.case_steps)
        sim.sync()
        out.update(nx=wl.nx, ny=wl.ny, steps=args.case_steps, tiling=list(sim.tiling))
        sim.close()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Shared test helpers: build the oracle twin of a workload and compare."""
import numpy as np

import oracle


def make_oracle(wl):
    s = oracle.OracleSim(wl.nx, wl.ny, wl.tau, wl.body_force, wl.walls, init=wl.init,
                         wall_velocity=wl.wall_velocity)
    for m in wl.membranes:
        k = s.add_membrane(m.xy, m.ks, m.kb, m.ka, m.kind, m.ligands)
        if m.kind in (2, 3):
            s.set_density(k, m.rho_p)
    if wl.receptors is not None and len(wl.receptors):
        b = wl.bonds
        s.set_receptors(wl.receptors, d_cut=b["d_cut"], y_eq=b["y_eq"], sigma=wl.sigma_lu,
                        kf_dt=b["kf_dt"], kr0_dt=b["kr0_dt"], beta_f=b["beta_f"], beta_r=b["beta_r"],
                        d_break=b["d_break"], seed=wl.seed, instance=wl.instance)
    s.set_repulsion(wl.d_rep)
    return s


def rel_err(a, b):
    """max |a - b| / max |b| (b the reference); 0 if both vanish"""
    d = np.max(np.abs(np.asarray(a) - np.asarray(b)))
    s = np.max(np.abs(np.asarray(b)))
    return 0.0 if d == 0 else d / (s if s > 0 else 1.0)


def dev_err(a, b, w):
    """error of populations measured on their deviation from the weights"""
    return rel_err(np.asarray(a) - w[:, None, None], np.asarray(b) - w[:, None, None])


W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def vel_err(ux, uy, ux0, uy0):
    """max componentwise velocity error over the reference speed scale"""
    d = max(np.max(np.abs(ux - ux0)), np.max(np.abs(uy - uy0)))
    s = max(np.max(np.abs(ux0)), np.max(np.abs(uy0)))
    return d / s


def f64_field_tol(u_scale):
    """FP64 field tolerance: 1e-12, or the plain-f oracle's own rounding floor
    (about 50 eps / u_scale relative, from O(1) population sums carrying an
    O(u) signal) when the flow is slow."""
    return max(1e-12, 50 * 2.22e-16 / u_scale)

"""Derivatives of carrier observables with respect to the carrier's stiffnesses,
the bond stiffness and its release height, through the reverse-mode adjoint
(lbib_adjoint_*: one backward sweep for the whole gradient) or the
forward-mode tangent (lbib_tangent_*: one run per parameter) of the CUDA time
step, behind a torch.autograd.Function.

Observables after T steps (lattice units):
  J1 = final height of the carrier's centroid above the lower wall (y = -1/2),
  J2 = elastic energy of the carrier's bonds, sum over bonds of
       sigma (d - y_eq)^2 / 2 (Eq. adhFor's spring).
Parameters p = (k_s, k_b, sigma, y_release) of the carrier (the last membrane
of the workload), all in lattice units.  The bond history of the run is held
fixed (bond events are discrete); dJ/dp is the derivative along that history.

This module only marshals: the state and its derivative are advanced by the
library's kernels; J1, J2 and their directional derivatives are short sums over
the final markers and bonds.
"""
from __future__ import annotations

import numpy as np

from paper_1907_00080_gb300 import inputs, lbib

PARAMS = ("k_s", "k_b", "sigma", "y_release")


def make_workload(p, steps, seed=0, bonds="default", precision="f64"):
    ks, kb, sigma, y0 = (float(v) for v in p)
    wl = inputs.adjoint_capillary_320x160(ks=ks, kb=kb, sigma_lu=sigma, release_y=y0, seed=seed, bonds=bonds,
                                          precision=precision)
    wl.steps = steps
    return wl


def observables(wl, xy, bonds):
    """J1, J2 and the pieces their derivatives need."""
    off = sum(len(m.xy) for m in wl.membranes[:-1])
    n = len(wl.membranes[-1].xy)
    car = xy[off:off + n]
    j1 = float(car[:, 1].mean() + 0.5)
    j2 = 0.0
    terms = []
    lig = wl.membranes[-1].ligands
    y_eq = wl.bonds["y_eq"]
    lig_base = sum(len(m.ligands) for m in wl.membranes[:-1])
    for q, e in enumerate(lig):
        r = int(bonds[lig_base + q])
        if r < 0:
            continue
        a, b = off + int(e), off + (int(e) + 1) % n
        c = 0.5 * (xy[a] + xy[b])
        d = wl.receptors[r] - c
        d[0] -= wl.nx * np.floor(d[0] / wl.nx + 0.5)
        dist = float(np.hypot(d[0], d[1]))
        j2 += 0.5 * wl.sigma_lu * (dist - y_eq) ** 2
        terms.append((a, b, d, dist))
    return j1, j2, (off, n, terms, y_eq)


def run(p, steps, seed=0, bonds="default"):
    """J = (J1, J2) of the FP64 solver after `steps` steps (no derivative)."""
    wl = make_workload(p, steps, seed, bonds)
    sim = lbib.Simulation(wl, precision="f64")
    sim.step(steps)
    j1, j2, _ = observables(wl, sim.markers(), sim.bonds())
    b = sim.bonds()
    sim.close()
    return np.array([j1, j2]), b


def jacobian(p, steps, seed=0, bonds="default"):
    """J (2,) and dJ/dp (2, 4) by four tangent runs (one per parameter)."""
    wl = make_workload(p, steps, seed, bonds)
    nm = len(wl.membranes)
    nv = wl.n_vertices
    jac = np.zeros((2, 4))
    J = None
    bond_hist = None
    for k in range(4):
        sim = lbib.Simulation(wl, precision="f64")
        t = lbib.lbib_tangent_create(sim.ctx)
        try:
            dks, dkb = np.zeros(nm), np.zeros(nm)
            dxy = np.zeros((nv, 2))
            dsig = 0.0
            if k == 0:
                dks[-1] = 1.0
            elif k == 1:
                dkb[-1] = 1.0
            elif k == 2:
                dsig = 1.0
            else:
                dxy[nv - len(wl.membranes[-1].xy):, 1] = 1.0
            lbib.lbib_tangent_seed(sim.ctx, t, dks, dkb, dsig, dxy, None)
            lbib.lbib_tangent_step(sim.ctx, t, steps)
            dX, _ = lbib.lbib_tangent_read(sim.ctx, t, nv)
            xy, bonds_f = sim.markers(), sim.bonds()
        finally:
            lbib.lbib_tangent_destroy(t)
            sim.close()
        j1, j2, _ = observables(wl, xy, bonds_f)
        if J is None:
            J, bond_hist = np.array([j1, j2]), bonds_f
        jac[:, k] = observable_directional(wl, xy, bonds_f, dX, dsig)
    return J, jac, bond_hist


def observable_directional(wl, xy, bonds, dX, dsigma):
    """(dJ1, dJ2) along a direction that moves the final markers by dX and
    the bond stiffness by dsigma."""
    _, _, (off, n, terms, y_eq) = observables(wl, xy, bonds)
    dj1 = float(dX[off:off + n, 1].mean())
    dj2 = 0.0
    for a, b, d, dist in terms:
        dc = 0.5 * (dX[a] + dX[b])
        ddist = -float(np.dot(d, dc)) / dist
        dj2 += wl.sigma_lu * (dist - y_eq) * ddist
        dj2 += dsigma * 0.5 * (dist - y_eq) ** 2
    return dj1, dj2


def observable_gradient(wl, xy, bonds, w):
    """dJ/dX^N (nv, 2) of J = w[0] J1 + w[1] J2 at the final markers, and the
    explicit dJ/dsigma of the bond energy."""
    _, _, (off, n, terms, y_eq) = observables(wl, xy, bonds)
    g = np.zeros((wl.n_vertices, 2))
    g[off:off + n, 1] += w[0] / n
    dsig = 0.0
    for a, b, d, dist in terms:
        gc = -w[1] * wl.sigma_lu * (dist - y_eq) / dist * d  # d J2 / d(ligand point)
        g[a] += 0.5 * gc
        g[b] += 0.5 * gc
        dsig += w[1] * 0.5 * (dist - y_eq) ** 2
    return g, dsig


class Recording:
    """One run of the sensitivity case, recorded for backward sweeps
    (checkpoints every `checkpoint_every` steps).  precision: the forward
    run's ("f64", or "f32" / "f16" / "bf16" storage with FP32 arithmetic); the
    adjoint and the gradients are FP64 in every case."""

    def __init__(self, p, steps, checkpoint_every=250, seed=0, bonds="default", precision="f64"):
        self.wl = make_workload(p, steps, seed, bonds, precision)
        self.sim = lbib.Simulation(self.wl, precision=precision)
        self.adj = None
        self.adj = lbib.lbib_adjoint_create(self.sim.ctx, checkpoint_every)
        lbib.lbib_adjoint_record(self.sim.ctx, self.adj, steps)
        self.xy, self.bonds = self.sim.markers(), self.sim.bonds()
        j1, j2, _ = observables(self.wl, self.xy, self.bonds)
        self.J = np.array([j1, j2])

    def gradient(self, w):
        """d(w . J)/dp (4,) from one backward sweep."""
        nv, nm = self.wl.n_vertices, len(self.wl.membranes)
        g, dsig = observable_gradient(self.wl, self.xy, self.bonds, w)
        lbib.lbib_adjoint_seed(self.sim.ctx, self.adj, g, None, None)
        lbib.lbib_adjoint_reverse(self.sim.ctx, self.adj)
        r = lbib.lbib_adjoint_read(self.sim.ctx, self.adj, nv, nm)
        nc = len(self.wl.membranes[-1].xy)
        # the release height moves X^0 and X^{-1} of every carrier vertex
        dy = float(r["xy"][nv - nc:, 1].sum() + r["xy_prev"][nv - nc:, 1].sum())
        return np.array([r["k_s"][-1], r["k_b"][-1], r["sigma"] + dsig, dy])

    def close(self):
        if self.adj is not None:
            lbib.lbib_adjoint_destroy(self.adj)
            self.adj = None
        if self.sim is not None:
            self.sim.close()
            self.sim = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adjoint_jacobian(p, steps, checkpoint_every=250, seed=0, bonds="default", precision="f64"):
    """J (2,) and dJ/dp (2, 4) by one recorded run and two backward sweeps."""
    rec = Recording(p, steps, checkpoint_every, seed, bonds, precision)
    try:
        jac = np.stack([rec.gradient((1.0, 0.0)), rec.gradient((0.0, 1.0))])
        return rec.J, jac, rec.bonds
    finally:
        rec.close()


def _torch_function():
    import torch

    class CarrierObservables(torch.autograd.Function):
        """J = (J1, J2)(p), p = (k_s, k_b, sigma, y_release) as a float64
        tensor.  mode "adjoint": forward records the FP64 run, backward seeds
        the adjoint with the incoming gradient and runs one backward sweep;
        mode "tangent": forward builds dJ/dp from four tangent runs, backward
        contracts the incoming gradient with it."""

        @staticmethod
        def forward(ctx, p, steps, seed=0, mode="adjoint", checkpoint_every=250, precision="f64"):
            pv = p.detach().cpu().numpy().astype(np.float64)
            ctx.rec = None
            if mode == "adjoint":
                ctx.rec = Recording(pv, int(steps), int(checkpoint_every), int(seed), precision=precision)
                J = ctx.rec.J
            elif mode == "tangent":
                J, jac, _ = jacobian(pv, int(steps), int(seed))
                ctx.save_for_backward(torch.as_tensor(jac, dtype=torch.float64))
            else:
                raise ValueError("mode must be 'adjoint' or 'tangent'")
            return torch.as_tensor(J, dtype=torch.float64, device=p.device)

        @staticmethod
        def backward(ctx, grad_out):
            w = grad_out.detach().to(torch.float64).cpu()
            if ctx.rec is not None:
                try:
                    g = torch.as_tensor(ctx.rec.gradient(w.numpy()), dtype=torch.float64)
                finally:
                    ctx.rec.close()
                    ctx.rec = None
            else:
                (jac,) = ctx.saved_tensors
                g = w @ jac
            return g.to(grad_out.device), None, None, None, None, None

    return CarrierObservables


def carrier_observables(p, steps, seed=0, mode="adjoint", checkpoint_every=250, precision="f64"):
    """torch entry point: J = carrier_observables(p, steps); J.backward(...).
    precision selects the forward run of the adjoint mode (the tangent mode is
    FP64)."""
    return _torch_function().apply(p, steps, seed, mode, checkpoint_every, precision)


def default_params(seed=0):
    wl = inputs.adjoint_capillary_320x160(seed=seed)
    car = wl.membranes[-1]
    return np.array([car.ks, car.kb, wl.sigma_lu, car.xy[:, 1].mean()])

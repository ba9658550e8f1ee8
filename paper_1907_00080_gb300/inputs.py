"""Seeded synthetic workloads for the LB-IB capillary problem.

This module only generates inputs (geometry, parameters in lattice units,
receptor arrays); it contains none of the time-step arithmetic, so the CUDA
path and the CPU oracle can both be fed from it without sharing any of the
method's code.  It imports nothing else from this package.

Paper set-up it follows (Coclite, arXiv 1907.00080, Sec. 3):
  * channel of height H, periodic in x, no-slip walls in y, Poiseuille drive
    with Re = u_max H / nu = 1e-2 and tau = 1 (nu = 1/6 lattice units);
  * red-cell rest contour, Eq. rbcShape;
  * capillary number Ca = rho nu u_max / k_s; bending E_b = k_b / (k_s r^2);
  * bond strength sigma in units rho nu^2 / H; ligand density rho_L = 0.5.
All randomness comes from numpy PCG64 with an explicit seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

NU_TAU1 = 1.0 / 6.0  # kinematic viscosity at tau = 1 in lattice units

# Bond-kinetics defaults (forward/reverse probabilities per step).  The paper
# gives only k_f / k_r0 = 8.5e3 (Sec. 3); the rest is this library's choice.
DEFAULT_BONDS = dict(d_cut=1.5, y_eq=0.75, kf_dt=1e-2, kr0_dt=1e-2 / 8.5e3,
                     beta_f=0.5, beta_r=2.0, d_break=3.0)
STRESS_BONDS = dict(d_cut=1.5, y_eq=0.75, kf_dt=0.05, kr0_dt=0.01,
                    beta_f=0.5, beta_r=2.0, d_break=3.0)


@dataclass
class Membrane:
    xy: np.ndarray            # (n, 2) CCW rest shape, unwrapped x
    ks: float
    kb: float
    ka: float
    kind: int = 0             # 0 kinematic, 1 rigid-projected, 2 dynamic, 3 dynamic rigid
    ligands: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    rho_p: float = 1.1        # particle / fluid density of a dynamic membrane (Sec. 3)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    tau: float = 1.0
    body_force: tuple = (0.0, 0.0)
    walls: int = 1
    init: str = "poiseuille"
    precision: str = "f32"
    membranes: List[Membrane] = field(default_factory=list)
    receptors: Optional[np.ndarray] = None    # (R, 2)
    bonds: dict = field(default_factory=lambda: dict(DEFAULT_BONDS))
    sigma_lu: float = 0.0
    seed: int = 0
    instance: int = 0
    d_rep: float = 2.0
    steps: int = 1000
    wall_velocity: tuple = (0.0, 0.0)         # x velocities of the lower and upper walls

    @property
    def n_vertices(self):
        return sum(len(m.xy) for m in self.membranes)

    @property
    def n_ligands(self):
        return sum(len(m.ligands) for m in self.membranes)


# ------------------------------------------------------------ parameter maps
def body_force_for(u_max: float, ny: int, nu: float = NU_TAU1) -> float:
    """Uniform body force giving a plane Poiseuille centreline speed u_max in a
    channel of height H = ny (walls half a node outside the fluid rows)."""
    return 8.0 * nu * u_max / float(ny) ** 2


def u_max_for_re(re: float, ny: int, nu: float = NU_TAU1) -> float:
    return re * nu / float(ny)


def sigma_lattice(sigma: float, ny: int, nu: float = NU_TAU1) -> float:
    """sigma given in units rho nu^2 / H (Sec. 2.2) -> lattice units."""
    return sigma * nu * nu / float(ny)


def ks_for_ca(ca: float, u_max: float, nu: float = NU_TAU1) -> float:
    """Ca = rho nu u_max / k_s (Sec. 3)."""
    return nu * u_max / ca


# ------------------------------------------------------------------ shapes
def circle(cx, cy, r, n, phase=0.5):
    """n vertices CCW on a circle, vertex k at angle 2 pi (k + phase) / n."""
    k = np.arange(n, dtype=np.float64)
    t = 2.0 * np.pi * (k + phase) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def _rbc_raw(alpha, q):
    x = alpha * np.sin(q)
    s = np.sin(q) ** 2
    y = 0.5 * alpha * (0.207 + 2.003 * s - 1.123 * s * s) * np.cos(q)
    return x, y


def rbc_contour(alpha: float, n: int, dense: int = 20000) -> np.ndarray:
    """Eq. rbcShape (a = 1, q in [-pi/2, 3pi/2]) resampled uniformly by arc
    length into n vertices, centred at the origin and oriented CCW."""
    q = np.linspace(-0.5 * np.pi, 1.5 * np.pi, dense, endpoint=False)
    x, y = _rbc_raw(alpha, q)
    pts = np.stack([x, y], axis=1)
    seg = np.linalg.norm(np.roll(pts, -1, axis=0) - pts, axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    total = s[-1]
    targets = np.arange(n) * total / n
    closed = np.concatenate([pts, pts[:1]], axis=0)
    xs = np.interp(targets, s, closed[:, 0])
    ys = np.interp(targets, s, closed[:, 1])
    out = np.stack([xs, ys], axis=1)
    if _signed_area(out) < 0:
        out = out[::-1].copy()
    return out - out.mean(axis=0)


def _signed_area(xy):
    x, y = xy[:, 0], xy[:, 1]
    return 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)


def _rotate(xy, ang):
    c, s = math.cos(ang), math.sin(ang)
    return xy @ np.array([[c, s], [-s, c]])


def _point_in_poly(px, py, poly, nx):
    # ray casting, with x taken at the periodic image closest to the polygon centre
    cx = poly[:, 0].mean()
    px = px - nx * math.floor((px - cx) / nx + 0.5)
    x1, y1 = poly[:, 0], poly[:, 1]
    x2, y2 = np.roll(x1, -1), np.roll(y1, -1)
    cross = (y1 > py) != (y2 > py)
    with np.errstate(divide="ignore", invalid="ignore"):
        xin = x1 + (py - y1) * (x2 - x1) / (y2 - y1)
    return bool(np.count_nonzero(cross & (px < xin)) % 2)


def place_membranes(shapes, nx, ny, rng, gap=2.0, wall_gap=2.0, y_range=None, max_tries=20000):
    """Random non-overlapping placement (uniform centre, uniform orientation).
    Vertices keep >= gap from every other membrane (periodic x) and >= wall_gap
    from the walls (at y = -1/2 and ny - 1/2)."""
    placed, centres, radii = [], [], []
    for k, shape in enumerate(shapes):
        ok = False
        for _ in range(max_tries):
            ang = rng.uniform(0.0, 2.0 * np.pi)
            xy = _rotate(shape, ang)
            ymin, ymax = xy[:, 1].min(), xy[:, 1].max()
            lo = -0.5 + wall_gap - ymin
            hi = ny - 0.5 - wall_gap - ymax
            if y_range is not None:
                lo, hi = max(lo, y_range[k][0]), min(hi, y_range[k][1])
            if hi <= lo:
                continue
            cx = rng.uniform(0.0, nx)
            cy = rng.uniform(lo, hi)
            cand = xy + np.array([cx, cy])
            c_n = cand.mean(axis=0)
            r_n = np.max(np.hypot(*(cand - c_n).T))
            bad = False
            for other, c_o, r_o in zip(placed, centres, radii):
                # bounding circles further apart than the gap: no contact possible
                dxc = c_n[0] - c_o[0]
                dxc -= nx * math.floor(dxc / nx + 0.5)
                if math.hypot(dxc, c_n[1] - c_o[1]) > r_n + r_o + gap:
                    continue
                # only vertices of `other` within r_n + gap of the candidate's
                # centre can be closer than gap to one of its vertices
                ox = other[:, 0] - c_n[0]
                ox -= nx * np.floor(ox / nx + 0.5)
                near = (np.abs(ox) <= r_n + gap) & (np.abs(other[:, 1] - c_n[1]) <= r_n + gap)
                if np.any(near):
                    d = cand[:, None, :] - other[near][None, :, :]
                    d[..., 0] -= nx * np.floor(d[..., 0] / nx + 0.5)
                    if np.min(np.hypot(d[..., 0], d[..., 1])) < gap:
                        bad = True
                        break
                if _point_in_poly(c_n[0], c_n[1], other, nx) or _point_in_poly(c_o[0], c_o[1], cand, nx):
                    bad = True
                    break
            if not bad:
                placed.append(cand)
                centres.append(c_n)
                radii.append(r_n)
                ok = True
                break
        if not ok:
            raise RuntimeError("could not place membrane %d" % k)
    return placed


def wall_receptors(nx, ny, lower=True, upper=True):
    """One receptor per wall node: (i, -1/2) on the lower wall and
    (i, ny - 1/2) on the upper wall, lower wall first, ascending i."""
    out = []
    i = np.arange(nx, dtype=np.float64)
    if lower:
        out.append(np.stack([i, np.full(nx, -0.5)], axis=1))
    if upper:
        out.append(np.stack([i, np.full(nx, ny - 0.5)], axis=1))
    return np.concatenate(out, axis=0) if out else np.zeros((0, 2))


# --------------------------------------------------------------- workloads
def capsule_128x32(precision="f64", bonds="default") -> Workload:
    """Plain FP64 case: 128x32 channel, u_max = 0.02, one circular capsule of
    radius 4 with 32 markers, k_s = 0.05, k_b = 0.005, area penalty 0.1, 32
    ligands, receptors on every lower-wall node, sigma = 1, cutoff 1.5."""
    nx, ny = 128, 32
    g = body_force_for(0.02, ny)
    mem = Membrane(xy=circle(32.0, 4.75, 4.0, 32), ks=0.05, kb=0.005, ka=0.1, kind=0,
                   ligands=np.arange(32, dtype=np.int32))
    wl = Workload(name="capsule_128x32", nx=nx, ny=ny, body_force=(g, 0.0), walls=1,
                  init="poiseuille", precision=precision, membranes=[mem],
                  receptors=wall_receptors(nx, ny, lower=True, upper=False),
                  sigma_lu=sigma_lattice(1.0, ny), seed=0, steps=1000)
    wl.bonds = dict(STRESS_BONDS if bonds == "stress" else DEFAULT_BONDS)
    return wl


def dynamic_carriers_128x48(precision="f64", bonds="stress") -> Workload:
    """Dynamic-IB case (Sec. 2.4): 128x48 channel, u_max = 0.02; a rigid
    dynamic carrier (radius 5, 32 markers, a ligand on every element) whose
    lowest vertex sits 1.27 lu above the lower wall, so that its probes and
    bonds reach the wall; a deformable dynamic carrier (radius 5, 32 markers,
    k_s = 5e-3, k_b = 5e-4) across the channel centre; a kinematic capsule
    (radius 4, 24 markers) between them; receptors on every lower-wall node."""
    nx, ny = 128, 48
    g = body_force_for(0.02, ny)
    mems = [
        Membrane(xy=circle(30.0, 5.75, 5.0, 32), ks=0.05, kb=0.005, ka=1.0, kind=3,
                 ligands=np.arange(32, dtype=np.int32)),
        Membrane(xy=circle(70.0, 24.3, 5.0, 32), ks=5e-3, kb=5e-4, ka=1.0, kind=2),
        Membrane(xy=circle(50.0, 14.0, 4.0, 24), ks=0.02, kb=0.002, ka=0.1, kind=0),
    ]
    wl = Workload(name="dynamic_carriers_128x48", nx=nx, ny=ny, body_force=(g, 0.0), walls=1,
                  init="poiseuille", precision=precision, membranes=mems,
                  receptors=wall_receptors(nx, ny, lower=True, upper=False),
                  sigma_lu=sigma_lattice(1.0, ny), seed=0, steps=1000)
    wl.bonds = dict(STRESS_BONDS if bonds == "stress" else DEFAULT_BONDS)
    return wl


def capillary(nx=640, ny=160, n_rbc=8, rbc_alpha=64.0, rbc_markers=200, n_carriers=4,
              carrier_radius=8.0, carrier_markers=50, ca_carrier=(0.0, 1e-2), sigma=1.0,
              re=1e-2, seed=0, precision="f32", steps=200000, name=None,
              bonds="default", release_y=None, carrier_model="kinematic", wall_gap=2.0) -> Workload:
    """Coarse capillary: 10x40 um at dx = 62.5 nm is a 160x640 lattice; 8
    biconcave red cells (8 um major axis -> alpha = 64 lu, 200 markers each),
    4 carriers of 1 um diameter (radius 8 lu, 50 markers), alternating rigid
    (Ca = 0) and soft (Ca = 1e-2) carriers, ligand density 0.5 (every other
    element), receptors on both walls, sigma = 1.  carrier_model "kinematic":
    rigid carriers rigid-projected, soft ones kinematic; "dynamic": the
    dynamic IB of Sec. 2.4 (rigid and deformable particles, rho_P / rho = 1.1)."""
    if carrier_model not in ("kinematic", "dynamic"):
        raise ValueError(carrier_model)
    dyn = carrier_model == "dynamic"
    rng = np.random.Generator(np.random.PCG64(seed))
    u_max = u_max_for_re(re, ny)
    g = body_force_for(u_max, ny)
    ks_rbc = ks_for_ca(1e-2, u_max)
    rbc = rbc_contour(rbc_alpha, rbc_markers)
    carrier = circle(0.0, 0.0, carrier_radius, carrier_markers)
    shapes = [rbc] * n_rbc + [carrier] * n_carriers
    y_range = None
    if release_y is not None:
        y_range = [(-1e9, 1e9)] * n_rbc + [(y - 1e-6, y + 1e-6) for y in release_y]
    placed = place_membranes(shapes, nx, ny, rng, y_range=y_range, wall_gap=wall_gap)
    mems = []
    for k in range(n_rbc):
        mems.append(Membrane(xy=placed[k], ks=ks_rbc, kb=0.0, ka=1.0, kind=0))
    lig = np.arange(0, carrier_markers, 2, dtype=np.int32)
    for c in range(n_carriers):
        ca = ca_carrier[c % len(ca_carrier)]
        if ca == 0.0:
            ks = ks_rbc
            kind = 3 if dyn else 1
        else:
            ks = ks_for_ca(ca, u_max)
            kind = 2 if dyn else 0
        kb = 0.05 * ks * carrier_radius ** 2
        mems.append(Membrane(xy=placed[n_rbc + c], ks=ks, kb=kb, ka=1.0, kind=kind, ligands=lig.copy()))
    wl = Workload(name=name or "capillary_%dx%d" % (nx, ny), nx=nx, ny=ny, body_force=(g, 0.0),
                  walls=1, init="poiseuille", precision=precision, membranes=mems,
                  receptors=wall_receptors(nx, ny), sigma_lu=sigma_lattice(sigma, ny),
                  seed=seed, steps=steps)
    if bonds == "physical":
        wl.bonds = physical_bonds(dx_nm=10000.0 / ny)
    else:
        wl.bonds = dict(STRESS_BONDS if bonds == "stress" else DEFAULT_BONDS)
    return wl


def physical_bonds(dx_nm: float) -> dict:
    """The paper's own cut-off y_cr = 25 nm (Sec. 2.2) in lattice units, with
    y_eq = y_cr / 2 and the default kinetics; only meaningful where the mesh
    resolves it (dx = 15 nm: 1.67 lu).  At dx = 62.5 nm it would be 0.4 lu,
    below the IB resolution, which is why the coarse mesh keeps 1.5 lu."""
    y_cr = 25.0 / dx_nm
    if y_cr < 1.0:
        raise ValueError("y_cr = 25 nm is %.2f lu on this mesh: below the IB resolution" % y_cr)
    return dict(DEFAULT_BONDS, d_cut=y_cr, y_eq=0.5 * y_cr, d_break=2.0 * y_cr)


def coarse_capillary_640x160(precision="f32", seed=0, steps=200000, carrier_model="kinematic") -> Workload:
    name = "capillary_640x160" + ("_dynamic" if carrier_model == "dynamic" else "")
    return capillary(precision=precision, seed=seed, steps=steps, name=name, carrier_model=carrier_model)


def fine_capillary_2000x667(precision="f32", sigma=1.0, carriers="rigid", seed=0, steps=20000,
                            bonds="default", release_y=None, wall_gap=2.0) -> Workload:
    """Fine mesh: 10 x 30 um at dx = 15 nm is a 667 x 2000 lattice; 4 red cells
    (8 um major axis -> alpha = 266.7 lu, 1700 markers each, about 19 % 2-D
    haematocrit), 3 carriers of 1 um diameter (radius 33.3 lu, 210 markers,
    105 ligands), all rigid (Ca = 0) or all soft (Ca = 1e-2), receptors on both
    walls, sigma in {0.5, 1, 2}.  bonds="physical" uses the paper's cut-off
    y_cr = 25 nm = 1.67 lu, which this mesh resolves.  release_y: the
    carriers' centre heights (3 values), else random."""
    nx, ny = 2000, 667
    ca = 0.0 if carriers == "rigid" else 1e-2
    return capillary(nx=nx, ny=ny, n_rbc=4, rbc_alpha=266.7, rbc_markers=1700, n_carriers=3,
                     carrier_radius=33.3, carrier_markers=210, ca_carrier=(ca,), sigma=sigma,
                     seed=seed, precision=precision, steps=steps, bonds=bonds, release_y=release_y,
                     wall_gap=wall_gap, name="fine_capillary_2000x667_%s_sigma%g" % (carriers, sigma))


def fine_capillary_adhering(precision="f32", sigma=1.0, carriers="rigid", seed=0) -> Workload:
    """The fine capillary with the paper's bond cut-off (y_cr = 1.67 lu) and
    its three carriers released 1 lu from a wall (two at the lower wall, one at
    the upper), so that bonds form from the first steps."""
    r, ny, gap = 33.3, 667, 1.0
    return fine_capillary_2000x667(precision, sigma=sigma, carriers=carriers, seed=seed, bonds="physical",
                                   release_y=(-0.5 + r + gap, -0.5 + r + gap, ny - 0.5 - r - gap), wall_gap=0.9)


def adjoint_capillary_320x160(ks=None, kb=None, sigma_lu=None, release_y=8.5, seed=0, precision="f64",
                              bonds="default") -> Workload:
    """Sensitivity case: 320 x 160 channel (Re = 1e-2), 2 red cells (200
    markers) and one soft carrier of radius 8 lu (50 markers, 25 ligands)
    whose centre starts at height release_y (8.5: its lowest vertex 1.0 lu
    above the lower wall at y = -1/2); receptors on both walls.  ks, kb and
    sigma_lu (lattice units) replace the carrier's stiffnesses and the bond
    stiffness when given.  The carrier is the last membrane."""
    nx, ny = 320, 160
    rng = np.random.Generator(np.random.PCG64(seed))
    u_max = u_max_for_re(1e-2, ny)
    ks_rbc = ks_for_ca(1e-2, u_max)
    rbcs = place_membranes([rbc_contour(64.0, 200)] * 2, nx, ny, rng)
    mems = [Membrane(xy=xy, ks=ks_rbc, kb=0.0, ka=1.0, kind=0) for xy in rbcs]
    # the carrier at height release_y (its lowest vertex exactly R below the
    # centre), at a random x at least 2 lu from the red cells
    for _ in range(20000):
        xy = circle(rng.uniform(0.0, nx), release_y, 8.0, 50)
        ok = True
        for other in rbcs:
            d = xy[:, None, :] - other[None, :, :]
            d[..., 0] -= nx * np.floor(d[..., 0] / nx + 0.5)
            if np.min(np.hypot(d[..., 0], d[..., 1])) < 2.0:
                ok = False
                break
        if ok:
            break
    ks_c = ks_for_ca(1e-2, u_max)
    mems.append(Membrane(xy=xy, ks=ks_c, kb=0.05 * ks_c * 64.0, ka=1.0, kind=0,
                         ligands=np.arange(0, 50, 2, dtype=np.int32)))
    wl = Workload(name="adjoint_capillary_320x160", nx=nx, ny=ny, body_force=(body_force_for(u_max, ny), 0.0),
                  walls=1, init="poiseuille", precision=precision, membranes=mems,
                  receptors=wall_receptors(nx, ny), sigma_lu=sigma_lattice(1.0, ny), seed=seed, steps=5000)
    wl.bonds = dict(STRESS_BONDS if bonds == "stress" else DEFAULT_BONDS)
    car = mems[-1]
    if ks is not None:
        car.ks = ks
    if kb is not None:
        car.kb = kb
    if sigma_lu is not None:
        wl.sigma_lu = sigma_lu
    return wl


def couette_cfl_600x200(precision="f32", sigma=1.0, carrier="rigid", gap=1.0, seed=0, steps=20000,
                        carrier_model="kinematic") -> Workload:
    """Adhesion in the cell-free layer (Sec. 4): planar Couette flow at
    Re = H_CFL u_w / nu = 0.003 in a channel of H_CFL = 3 um = 200 lu
    (dx = 15 nm) and length 3 H_CFL, periodic in x, the upper wall moving at
    u_w, the lower wall at rest and carrying the receptors (one per wall node).
    One 1 um carrier (radius 33.3 lu, 210 markers, a ligand on every other
    element) starts with its lowest marker `gap` lu above the lower wall at a
    random x; rigid (Ca = 0, rigid-projected) or soft (Ca = 1e-2 on the wall
    speed); with carrier_model "dynamic" the carrier follows the dynamic IB of
    Sec. 2.4 instead (rigid or deformable, rho_P / rho = 1.1).  Bonds use the
    physical cut-off y_cr = 25 nm = 1.67 lu and y_eq = y_cr / 2 (Sec. 2.2);
    sigma in units rho nu^2 / H_CFL."""
    if carrier_model not in ("kinematic", "dynamic"):
        raise ValueError(carrier_model)
    nx, ny = 600, 200
    rng = np.random.Generator(np.random.PCG64(seed))
    u_w = u_max_for_re(0.003, ny)
    r = 33.3
    xy = circle(rng.uniform(0.0, nx), -0.5 + gap + r, r, 210)
    xy[:, 1] += (-0.5 + gap) - xy[:, 1].min()
    dyn = carrier_model == "dynamic"
    if carrier == "rigid":
        ks, kind = ks_for_ca(1e-2, u_w), 3 if dyn else 1
    else:
        ks, kind = ks_for_ca(1e-2, u_w), 2 if dyn else 0
    mem = Membrane(xy=xy, ks=ks, kb=0.05 * ks * r * r, ka=1.0, kind=kind,
                   ligands=np.arange(0, 210, 2, dtype=np.int32))
    name = "couette_cfl_600x200_%s%s_sigma%g" % ("dynamic_" if dyn else "", carrier, sigma)
    wl = Workload(name=name, nx=nx, ny=ny, body_force=(0.0, 0.0),
                  walls=1, init="couette", precision=precision, membranes=[mem],
                  receptors=wall_receptors(nx, ny, lower=True, upper=False),
                  sigma_lu=sigma_lattice(sigma, ny), seed=seed, steps=steps, wall_velocity=(0.0, u_w))
    y_cr = 25.0 / 15.0
    wl.bonds = dict(DEFAULT_BONDS, d_cut=y_cr, y_eq=0.5 * y_cr)
    return wl


def capillary_ensemble(n=64, seed=0, precision="f32", l_min_um=32.0, l_max_um=64.0, dx_um=0.0625,
                       ny=160) -> List[Workload]:
    """Batched ensemble of coarse capillaries: instance i has length
    L_i ~ U[32, 64] um (NX_i = round(L_i / dx)), NY = 160, round(8 L_i / 40)
    red cells (the 640 x 160 density), 4 carriers released at heights drawn
    uniformly across the admissible width, Ca_i = (0, 1e-2)[i mod 2] (rigid or
    soft carriers), sigma_i = (0.5, 1, 2)[(i div 2) mod 3], seed_i = seed + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        L = rng.uniform(l_min_um, l_max_um)
        nx = int(round(L / dx_um))
        nx -= nx % 8  # whole 16-byte rows in every storage form
        n_rbc = int(round(8 * L / 40.0))
        r = 8.0
        release = list(rng.uniform(-0.5 + 2.0 + r, ny - 0.5 - 2.0 - r, size=4))
        ca = (0.0, 1e-2)[i % 2]
        sigma = (0.5, 1.0, 2.0)[(i // 2) % 3]
        out.append(capillary(nx=nx, ny=ny, n_rbc=n_rbc, ca_carrier=(ca,), sigma=sigma, seed=seed + i,
                             precision=precision, release_y=release,
                             name="capillary_%dx%d_i%d" % (nx, ny, i)))
    return out


def random_populations(nx, ny, base, seed=0, amp=1e-2):
    """Random positive populations base_i * (1 + amp * U(-1, 1)) per node; the
    caller supplies the nine base values (for unit parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.asarray(base, dtype=np.float64).reshape(9, 1, 1)
    return base * (1.0 + amp * rng.uniform(-1.0, 1.0, size=(9, ny, nx)))


def probe_lattice(nx, ny, precision="f32", n_carriers=None, seed=1) -> Workload:
    """Roofline probe of the fused kernel: an nx x ny channel (Poiseuille start
    at u_max = 1e-5) with soft circular carriers (R = 8, 50 markers) at seeded
    random positions, as many as give the 640 x 160 capillary's share of nodes
    under a marker stencil (256 on 8192 x 2048)."""
    wl = Workload(name="probe_%dx%d" % (nx, ny), nx=nx, ny=ny,
                  body_force=(body_force_for(1e-5, ny), 0.0), walls=1,
                  init="poiseuille", precision=precision, membranes=[], receptors=None)
    rng = np.random.Generator(np.random.PCG64(seed))
    if n_carriers is None:
        n_carriers = max(1, int(round(256 * nx * ny / (8192 * 2048))))
    for _ in range(n_carriers):
        cx, cy = rng.uniform(0, nx), rng.uniform(20, ny - 20)
        wl.membranes.append(Membrane(xy=circle(cx, cy, 8.0, 50), ks=1e-4, kb=0.0, ka=1.0))
    return wl

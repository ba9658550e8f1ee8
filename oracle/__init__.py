"""Plain FP64 CPU oracle of the LB-IB time step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: this package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference leg of
``bench.py``; the product library never imports, links or calls it.  It shares
no code with the CUDA path.  ``lbib_oracle.c`` holds all of the arithmetic and
cites the equation or section of the paper (arXiv 1907.00080) each step follows;
this module only builds it with gcc and marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbib_oracle.c")
_LIB = os.path.join(_HERE, "liblbib_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


_LIB_OMP = os.path.join(_HERE, "liblbib_oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) if stale; return the
    path.  openmp=True builds the OpenMP variant (the same source with its
    loop pragmas enabled; the loops it splits write disjoint elements, so it
    gives the same bits)."""
    out = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, *(["-fopenmp"] if openmp else []), _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


def use_threads(n: int) -> int:
    """Switch this process to the OpenMP build with n threads (n <= 1: back to
    the plain build).  Call before creating simulations: a simulation must be
    driven by the build that created it.  Returns the thread count in use."""
    global _lib
    with _lock:
        _lib = _load(build(openmp=n > 1))
    return int(_lib.orc_set_threads(int(n)))


_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_long
_U64 = ctypes.c_uint64
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_LP = ctypes.POINTER(ctypes.c_long)
_U64P = ctypes.POINTER(ctypes.c_uint64)

_SIGS = {
    "orc_create": (_P, [_I, _I, _D, _D, _D, _I]),
    "orc_destroy": (None, [_P]),
    "orc_set_populations": (None, [_P, _DP]),
    "orc_get_populations": (None, [_P, _DP]),
    "orc_get_fields": (None, [_P, _DP, _DP, _DP]),
    "orc_get_force_field": (None, [_P, _DP, _DP]),
    "orc_init_poiseuille": (None, [_P]),
    "orc_set_wall_velocity": (None, [_P, _D, _D]),
    "orc_init_couette": (None, [_P]),
    "orc_add_membrane": (_I, [_P, _DP, _I, _D, _D, _D, _I, _IP, _I]),
    "orc_set_receptors": (None, [_P, _DP, _I, _D, _D, _D, _D, _D, _D, _D, _D, _U64, _U64]),
    "orc_set_repulsion": (None, [_P, _D]),
    "orc_compute_forces": (None, [_P]),
    "orc_bonds_update": (None, [_P, _L]),
    "orc_step": (None, [_P, _L]),
    "orc_num_vertices": (_I, [_P]),
    "orc_num_ligands": (_I, [_P]),
    "orc_get_step": (_L, [_P]),
    "orc_get_markers": (None, [_P, _DP]),
    "orc_get_prev_markers": (None, [_P, _DP]),
    "orc_set_markers": (None, [_P, _DP, _DP]),
    "orc_get_forces": (None, [_P, _DP]),
    "orc_get_marker_velocity": (None, [_P, _DP]),
    "orc_get_bonds": (None, [_P, _IP]),
    "orc_set_bond": (None, [_P, _I, _I]),
    "orc_mass": (_D, [_P]),
    "orc_membrane_area": (_D, [_P, _I]),
    "orc_membrane_rest_area": (_D, [_P, _I]),
    "orc_philox4x64_10": (None, [_U64P, _U64P, _U64P]),
    "orc_uniform": (_D, [_U64, _U64, _L, _L, _L, _L]),
    "orc_equilibrium": (None, [_D, _D, _D, _DP]),
    "orc_guo_source": (None, [_D, _D, _D, _D, _D, _DP]),
    "orc_stream": (None, [_P, _DP, _DP]),
    "orc_moments": (None, [_P, _DP, _DP, _DP, _DP, _DP, _DP]),
    "orc_roma": (_D, [_D]),
    "orc_ib_weights": (None, [_P, _D, _D, _DP, _LP]),
    "orc_interp": (None, [_P, _DP, _DP, _I, _DP, _DP, _DP, _DP]),
    "orc_spread": (None, [_P, _I, _DP, _DP, _DP, _DP, _DP, _DP]),
    "orc_ring_area": (_D, [_I, _DP, _DP]),
    "orc_ring_rest": (None, [_I, _DP, _DP, _DP, _DP, _DP]),
    "orc_ring_forces": (None, [_I, _DP, _DP, _DP, _DP, _D, _D, _D, _D, _D, _I, _DP, _DP]),
    "orc_p_form": (_D, [_P, _D]),
    "orc_p_rupture": (_D, [_P, _D]),
    "orc_ring_mass_properties": (None, [_I, _DP, _DP, _DP, _DP, _DP, _DP]),
    "orc_mls_shape": (None, [_P, _D, _D, _DP, _LP]),
    "orc_mls_fit": (None, [_P, _D, _D, _DP, _DP]),
    "orc_hydro_element_forces": (None, [_P, _I, _DP]),
    "orc_compute_step_forces": (None, [_P]),
    "orc_particle_advance": (None, [_P, _L]),
    "orc_set_membrane_density": (None, [_P, _I, _D]),
    "orc_membrane_mass": (_D, [_P, _I]),
    "orc_membrane_inertia": (_D, [_P, _I]),
    "orc_set_forces": (None, [_P, _DP]),
    "orc_set_marker_velocity": (None, [_P, _DP]),
    "orc_get_particle_velocity": (None, [_P, _DP]),
    "orc_set_particle_velocity": (None, [_P, _DP]),
    "orc_get_hydro_forces": (None, [_P, _DP]),
    "orc_get_ib_forces": (None, [_P, _DP]),
    "orc_get_rigid_state": (None, [_P, _I, _DP]),
    "orc_set_rigid_state": (None, [_P, _I, _DP]),
    "orc_tangent_create": (_P, [_P]),
    "orc_tangent_destroy": (None, [_P]),
    "orc_tangent_seed": (None, [_P, _DP, _DP, _D, _DP, _DP, _DP]),
    "orc_tangent_step": (None, [_P, _L]),
    "orc_tangent_get": (None, [_P, _DP, _DP, _DP]),
    "orc_set_threads": (_I, [_I]),
}


def _load(path):
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- primitives
def roma(r: float) -> float:
    return lib().orc_roma(float(r))


def equilibrium(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_equilibrium(rho, ux, uy, _dp(out))
    return out


def guo_source(tau, ux, uy, gx, gy):
    out = np.zeros(9)
    lib().orc_guo_source(tau, ux, uy, gx, gy, _dp(out))
    return out


def philox4x64_10(counter, key):
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    o = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(c.ctypes.data_as(_U64P), k.ctypes.data_as(_U64P), o.ctypes.data_as(_U64P))
    return o


def uniform(seed, instance, step, lig, rec, tag):
    return lib().orc_uniform(seed, instance, step, lig, rec, tag)


def ring_area(xy):
    xy = _f64(xy).reshape(-1, 2)
    x, y = _f64(xy[:, 0]), _f64(xy[:, 1])
    return lib().orc_ring_area(len(x), _dp(x), _dp(y))


def ring_rest(xy):
    xy = _f64(xy).reshape(-1, 2)
    n = len(xy)
    x, y = _f64(xy[:, 0]), _f64(xy[:, 1])
    l0, th0, A0 = np.zeros(n), np.zeros(n), np.zeros(1)
    lib().orc_ring_rest(n, _dp(x), _dp(y), _dp(l0), _dp(th0), _dp(A0))
    return l0, th0, float(A0[0])


def ring_forces(xy, l0, th0, A0, ks, kb, ka, p_ref=1.0 / 3.0, which=7):
    xy = _f64(xy).reshape(-1, 2)
    n = len(xy)
    x, y = _f64(xy[:, 0]), _f64(xy[:, 1])
    fx, fy = np.zeros(n), np.zeros(n)
    lib().orc_ring_forces(n, _dp(x), _dp(y), _dp(_f64(l0)), _dp(_f64(th0)), A0, ks, kb, ka,
                          p_ref, which, _dp(fx), _dp(fy))
    return np.stack([fx, fy], axis=1)


def ring_mass_properties(xy):
    """(area, centroid relative to vertex 0, polar moment about the centroid)"""
    xy = _f64(xy).reshape(-1, 2)
    x, y = _f64(xy[:, 0]), _f64(xy[:, 1])
    o = np.zeros(4)
    lib().orc_ring_mass_properties(len(x), _dp(x), _dp(y), _dp(o[0:]), _dp(o[1:]), _dp(o[2:]), _dp(o[3:]))
    return float(o[0]), (float(o[1]), float(o[2])), float(o[3])


# ---------------------------------------------------------------- simulation
class OracleSim:
    """One oracle simulation (FP64, CPU).  walls=1: half-way bounce-back walls in
    y; walls=2: Zou-He known-velocity walls on the rows y = 0 and NY - 1."""

    def __init__(self, nx, ny, tau=1.0, body_force=(0.0, 0.0), walls=1, init="rest", wall_velocity=(0.0, 0.0)):
        self.nx, self.ny = int(nx), int(ny)
        self.walls = int(walls)
        self._s = lib().orc_create(self.nx, self.ny, float(tau), float(body_force[0]),
                                   float(body_force[1]), self.walls)
        self.nmem = 0
        self.mem_sizes = []
        lib().orc_set_wall_velocity(self._s, float(wall_velocity[0]), float(wall_velocity[1]))
        if init == "poiseuille":
            lib().orc_init_poiseuille(self._s)
        elif init == "couette":
            lib().orc_init_couette(self._s)
        elif init != "rest":
            raise ValueError(init)

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            lib().orc_destroy(s)
            self._s = None

    @property
    def N(self):
        return self.nx * self.ny

    # populations / fields
    def set_populations(self, f):
        f = _f64(f).reshape(9, self.ny, self.nx)
        lib().orc_set_populations(self._s, _dp(f))

    def populations(self):
        f = np.zeros((9, self.ny, self.nx))
        lib().orc_get_populations(self._s, _dp(f))
        return f

    def fields(self):
        r, a, b = (np.zeros((self.ny, self.nx)) for _ in range(3))
        lib().orc_get_fields(self._s, _dp(r), _dp(a), _dp(b))
        return r, a, b

    def force_field(self):
        a, b = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        lib().orc_get_force_field(self._s, _dp(a), _dp(b))
        return a, b

    def stream(self, fstar):
        fstar = _f64(fstar).reshape(9, self.ny, self.nx)
        out = np.zeros_like(fstar)
        lib().orc_stream(self._s, _dp(fstar), _dp(out))
        return out

    def moments(self, f, G=None):
        f = _f64(f).reshape(9, self.ny, self.nx)
        r, a, b = (np.zeros((self.ny, self.nx)) for _ in range(3))
        if G is None:
            lib().orc_moments(self._s, _dp(f), None, None, _dp(r), _dp(a), _dp(b))
        else:
            gx, gy = _f64(G[0]), _f64(G[1])
            lib().orc_moments(self._s, _dp(f), _dp(gx), _dp(gy), _dp(r), _dp(a), _dp(b))
        return r, a, b

    # membranes, receptors
    def add_membrane(self, xy, ks, kb, ka, kind=0, ligand_elems=None):
        xy = _f64(xy).reshape(-1, 2)
        lig = np.ascontiguousarray(ligand_elems if ligand_elems is not None else [], dtype=np.int32)
        m = lib().orc_add_membrane(self._s, _dp(xy), len(xy), ks, kb, ka, int(kind),
                                   lig.ctypes.data_as(_IP), len(lig))
        self.nmem += 1
        self.mem_sizes.append(len(xy))
        return m

    def set_receptors(self, xy, d_cut=1.5, y_eq=0.75, sigma=0.0, kf_dt=1e-2, kr0_dt=1e-2 / 8.5e3,
                      beta_f=0.5, beta_r=2.0, d_break=3.0, seed=0, instance=0):
        xy = _f64(xy).reshape(-1, 2)
        lib().orc_set_receptors(self._s, _dp(xy), len(xy), d_cut, y_eq, sigma, kf_dt, kr0_dt,
                                beta_f, beta_r, d_break, int(seed), int(instance))

    def set_repulsion(self, d_rep):
        lib().orc_set_repulsion(self._s, float(d_rep))

    # stepping
    def step(self, n=1):
        lib().orc_step(self._s, int(n))

    def compute_forces(self):
        lib().orc_compute_forces(self._s)

    def bonds_update(self, step):
        lib().orc_bonds_update(self._s, int(step))

    @property
    def step_count(self):
        return lib().orc_get_step(self._s)

    @property
    def nv(self):
        return lib().orc_num_vertices(self._s)

    @property
    def nlig(self):
        return lib().orc_num_ligands(self._s)

    def markers(self):
        xy = np.zeros((self.nv, 2))
        lib().orc_get_markers(self._s, _dp(xy))
        return xy

    def prev_markers(self):
        xy = np.zeros((self.nv, 2))
        lib().orc_get_prev_markers(self._s, _dp(xy))
        return xy

    def set_markers(self, xy, xy_prev=None):
        xy = _f64(xy).reshape(-1, 2)
        if xy_prev is None:
            lib().orc_set_markers(self._s, _dp(xy), None)
        else:
            lib().orc_set_markers(self._s, _dp(xy), _dp(_f64(xy_prev).reshape(-1, 2)))

    def forces(self):
        f = np.zeros((self.nv, 2))
        lib().orc_get_forces(self._s, _dp(f))
        return f

    def marker_velocity(self):
        u = np.zeros((self.nv, 2))
        lib().orc_get_marker_velocity(self._s, _dp(u))
        return u

    def bonds(self):
        b = np.zeros(self.nlig, dtype=np.int32)
        if self.nlig:
            lib().orc_get_bonds(self._s, b.ctypes.data_as(_IP))
        return b

    def set_bond(self, lig, rec):
        lib().orc_set_bond(self._s, int(lig), int(rec))

    def mass(self):
        return lib().orc_mass(self._s)

    def area(self, m):
        return lib().orc_membrane_area(self._s, int(m))

    def rest_area(self, m):
        return lib().orc_membrane_rest_area(self._s, int(m))

    def p_form(self, d):
        return lib().orc_p_form(self._s, float(d))

    def p_rupture(self, d):
        return lib().orc_p_rupture(self._s, float(d))

    # dynamic particles (kinds 2 and 3)
    def set_density(self, m, rho_p):
        lib().orc_set_membrane_density(self._s, int(m), float(rho_p))

    def mass_of(self, m):
        return lib().orc_membrane_mass(self._s, int(m))

    def inertia_of(self, m):
        return lib().orc_membrane_inertia(self._s, int(m))

    def mls_shape(self, x, y):
        phi = np.zeros((3, 9))
        idx = np.zeros(9, dtype=np.int64)
        lib().orc_mls_shape(self._s, float(x), float(y), _dp(phi), idx.ctypes.data_as(_LP))
        return phi, idx

    def mls_fit(self, x, y, g):
        g = _f64(g).reshape(self.ny, self.nx)
        out = np.zeros(3)
        lib().orc_mls_fit(self._s, float(x), float(y), _dp(g), _dp(out))
        return out

    def hydro_element_forces(self, m):
        fe = np.zeros((self.mem_sizes[m], 2))
        lib().orc_hydro_element_forces(self._s, int(m), _dp(fe))
        return fe

    def compute_step_forces(self):
        lib().orc_compute_step_forces(self._s)

    def particle_advance(self, step):
        lib().orc_particle_advance(self._s, int(step))

    def set_forces(self, fxy):
        lib().orc_set_forces(self._s, _dp(_f64(fxy).reshape(-1, 2)))

    def set_marker_velocity(self, uxy):
        lib().orc_set_marker_velocity(self._s, _dp(_f64(uxy).reshape(-1, 2)))

    def particle_velocity(self):
        v = np.zeros((self.nv, 2))
        lib().orc_get_particle_velocity(self._s, _dp(v))
        return v

    def set_particle_velocity(self, vxy):
        lib().orc_set_particle_velocity(self._s, _dp(_f64(vxy).reshape(-1, 2)))

    def hydro_forces(self):
        f = np.zeros((self.nv, 2))
        lib().orc_get_hydro_forces(self._s, _dp(f))
        return f

    def ib_forces(self):
        f = np.zeros((self.nv, 2))
        lib().orc_get_ib_forces(self._s, _dp(f))
        return f

    def set_rigid_state(self, m, state):
        """(u, v, u_prev, v_prev, omega, omega_prev); vertex velocities follow"""
        lib().orc_set_rigid_state(self._s, int(m), _dp(_f64(state)))

    def rigid_state(self, m):
        """(u, v, u_prev, v_prev, omega, omega_prev) of a rigid dynamic membrane"""
        o = np.zeros(6)
        lib().orc_get_rigid_state(self._s, int(m), _dp(o))
        return o

    # IB primitives on this lattice
    def ib_weights(self, x, y):
        w = np.zeros(9)
        idx = np.zeros(9, dtype=np.int64)
        lib().orc_ib_weights(self._s, float(x), float(y), _dp(w), idx.ctypes.data_as(_LP))
        return w, idx

    def interp(self, ux, uy, pts):
        pts = _f64(pts).reshape(-1, 2)
        px, py = _f64(pts[:, 0]), _f64(pts[:, 1])
        Ux, Uy = np.zeros(len(pts)), np.zeros(len(pts))
        lib().orc_interp(self._s, _dp(_f64(ux)), _dp(_f64(uy)), len(pts), _dp(px), _dp(py),
                         _dp(Ux), _dp(Uy))
        return np.stack([Ux, Uy], axis=1)

    def spread(self, pts, F):
        pts = _f64(pts).reshape(-1, 2)
        F = _f64(F).reshape(-1, 2)
        px, py = _f64(pts[:, 0]), _f64(pts[:, 1])
        fx, fy = _f64(F[:, 0]), _f64(F[:, 1])
        gx, gy = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        lib().orc_spread(self._s, len(pts), _dp(px), _dp(py), _dp(fx), _dp(fy), _dp(gx), _dp(gy))
        return gx, gy


# ---------------------------------------------------------------- tangent
class OracleTangent:
    """Forward-mode (dual-number) tangent of an OracleSim's trajectory along
    one direction of (k_s, k_b per membrane, sigma, X^n, X^{n-1}, f^n), with the
    primal's bond history.  ``step(n)`` advances the simulation and the
    tangent together (use it instead of ``sim.step``)."""

    def __init__(self, sim):
        self.sim = sim
        self._t = lib().orc_tangent_create(sim._s)
        if not self._t:
            raise ValueError("the oracle tangent needs kinematic membranes only (kind 0)")

    def __del__(self):
        t = getattr(self, "_t", None)
        if t:
            lib().orc_tangent_destroy(t)
            self._t = None

    def seed(self, dks=None, dkb=None, dsigma=0.0, dxy=None, dxy_prev=None, df=None):
        keep = [None if a is None else _f64(a) for a in (dks, dkb, dxy, dxy_prev, df)]
        ptrs = [None if a is None else _dp(a) for a in keep]
        lib().orc_tangent_seed(self._t, ptrs[0], ptrs[1], float(dsigma), ptrs[2], ptrs[3], ptrs[4])

    def step(self, n=1):
        lib().orc_tangent_step(self._t, int(n))

    def get(self):
        """(dX^n, dX^{n-1}) as (nv, 2) arrays and df^n as (9, ny, nx)."""
        nv = self.sim.nv
        dxy, dxp = np.zeros((nv, 2)), np.zeros((nv, 2))
        df = np.zeros((9, self.sim.ny, self.sim.nx))
        lib().orc_tangent_get(self._t, _dp(dxy), _dp(dxp), _dp(df))
        return dxy, dxp, df

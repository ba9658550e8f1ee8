"""Thin ctypes binding of the lbib C ABI (include/lbib.h).

Functions keep the C names and only marshal arguments: every step of the
time integration runs in the CUDA kernels of ``liblbib.so``.  A missing
library raises immediately; there is no CPU fallback.  Device pointers may be
passed as integers (e.g. ``torch.Tensor.data_ptr()``) with ``on_device=1``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbib.so")

# enums (mirror include/lbib.h)
LBIB_OK, LBIB_E_INVALID, LBIB_E_CUDA, LBIB_E_OOM, LBIB_E_TIMEOUT, LBIB_E_NONFINITE, LBIB_E_STATE = range(7)
LBIB_F64, LBIB_F32, LBIB_F32_STORE_F16, LBIB_F32_STORE_BF16 = range(4)
LBIB_WALLS_NONE, LBIB_WALLS_Y_BOUNCEBACK, LBIB_WALLS_ZOU_HE = 0, 1, 2
LBIB_INIT_REST, LBIB_INIT_POISEUILLE, LBIB_INIT_COUETTE = 0, 1, 2
LBIB_MEMBRANE_KINEMATIC, LBIB_MEMBRANE_RIGID_PROJECTED = 0, 1
LBIB_MEMBRANE_DYNAMIC, LBIB_MEMBRANE_DYNAMIC_RIGID = 2, 3

PRECISIONS = {"f64": LBIB_F64, "f32": LBIB_F32, "f16": LBIB_F32_STORE_F16, "bf16": LBIB_F32_STORE_BF16}
STATUS_NAMES = {0: "LBIB_OK", 1: "LBIB_E_INVALID", 2: "LBIB_E_CUDA", 3: "LBIB_E_OOM",
                4: "LBIB_E_TIMEOUT", 5: "LBIB_E_NONFINITE", 6: "LBIB_E_STATE"}


class lbib_lattice(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("prec", ctypes.c_int),
                ("init", ctypes.c_int)]


class lbib_bond_params(ctypes.Structure):
    _fields_ = [("d_cut", ctypes.c_double), ("y_eq", ctypes.c_double), ("sigma", ctypes.c_double),
                ("kf_dt", ctypes.c_double), ("kr0_dt", ctypes.c_double), ("beta_f", ctypes.c_double),
                ("beta_r", ctypes.c_double), ("d_break", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint64)]


class LbibError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_P = ctypes.c_void_p
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I = ctypes.c_int
_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "lbib_create": (_I, [ctypes.POINTER(lbib_lattice), _D, _DP, _I, _P, ctypes.POINTER(_P)]),
    "lbib_add_membrane": (_I, [_P, _DP, _I32, _D, _D, _D, _I, _I32P, _I32, _I32P]),
    "lbib_set_receptors": (_I, [_P, _DP, _I32, ctypes.POINTER(lbib_bond_params)]),
    "lbib_set_repulsion": (_I, [_P, _D]),
    "lbib_set_wall_velocity": (_I, [_P, _D, _D]),
    "lbib_membrane_observables": (_I, [_P, _DP]),
    "lbib_save": (_I, [_P, ctypes.c_char_p]),
    "lbib_load": (_I, [_P, ctypes.c_char_p]),
    "lbib_step": (_I, [_P, _I64]),
    "lbib_sync": (_I, [_P]),
    "lbib_step_count": (_I64, [_P]),
    "lbib_read_fields": (_I, [_P, _P, _P, _P, _I]),
    "lbib_read_populations": (_I, [_P, _P, _I]),
    "lbib_write_populations": (_I, [_P, _P, _I]),
    "lbib_read_markers": (_I, [_P, _I32, _DP]),
    "lbib_write_markers": (_I, [_P, _DP, _DP]),
    "lbib_read_marker_forces": (_I, [_P, _DP]),
    "lbib_read_marker_velocity": (_I, [_P, _DP]),
    "lbib_set_particle_density": (_I, [_P, _I32, _D]),
    "lbib_read_particle_velocity": (_I, [_P, _I32, _DP]),
    "lbib_read_bonds": (_I, [_P, _I32P, _I32P, _I32, _I32P]),
    "lbib_diagnostics": (_I, [_P, _DP, _DP]),
    "lbib_population_mass_noalloc": (_I, [_P, _I64, _P, _P]),
    "lbib_ensemble_create": (_I, [ctypes.POINTER(_P), _I32, _P, ctypes.POINTER(_P)]),
    "lbib_ensemble_step": (_I, [_P, _I64]),
    "lbib_ensemble_sync": (_I, [_P]),
    "lbib_ensemble_write_state": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _I32]),
    "lbib_ensemble_read_markers": (_I, [_P, ctypes.POINTER(_P)]),
    "lbib_ensemble_size": (_I32, [_P]),
    "lbib_ensemble_form": (_I32, [_P]),
    "lbib_ensemble_set_groups": (ctypes.c_int, [_P, _I32]),
    "lbib_ensemble_groups": (_I32, [_P]),
    "lbib_ensemble_profile_kernels": (ctypes.c_int, [_P, _I32, ctypes.POINTER(_D)]),
    "lbib_ensemble_launches_per_step": (_I32, [_P]),
    "lbib_ensemble_member": (_P, [_P, _I32]),
    "lbib_ensemble_last_error": (ctypes.c_char_p, [_P]),
    "lbib_ensemble_destroy": (None, [_P]),
    "lbib_slabs_create": (_I, [ctypes.POINTER(_P), _I32, ctypes.POINTER(_P)]),
    "lbib_slabs_step": (_I, [_P, _I64]),
    "lbib_slabs_sync": (_I, [_P]),
    "lbib_slabs_last_error": (ctypes.c_char_p, [_P]),
    "lbib_slabs_destroy": (None, [_P]),
    "lbib_slab_face": (_I, [_P, _I32, _I32, _P, _I32]),
    "lbib_storage_bytes": (_I32, [_P]),
    "lbib_tangent_create": (_I, [_P, ctypes.POINTER(_P)]),
    "lbib_tangent_seed": (_I, [_P, _DP, _DP, _D, _DP, _DP]),
    "lbib_tangent_step": (_I, [_P, _I64]),
    "lbib_tangent_read": (_I, [_P, _DP, _DP]),
    "lbib_tangent_destroy": (None, [_P]),
    "lbib_adjoint_create": (_I, [_P, _I32, ctypes.POINTER(_P)]),
    "lbib_adjoint_record": (_I, [_P, _I64]),
    "lbib_adjoint_seed": (_I, [_P, _DP, _DP, _DP]),
    "lbib_adjoint_reverse": (_I, [_P]),
    "lbib_adjoint_read": (_I, [_P, _DP, _DP, _DP, _DP, _DP, _DP]),
    "lbib_adjoint_recorded_steps": (_I64, [_P]),
    "lbib_adjoint_destroy": (None, [_P]),
    "lbib_set_tiling": (_I, [_P, _I32, _I32]),
    "lbib_get_tiling": (_I, [_P, _I32P, _I32P]),
    "lbib_profile_fused": (_I, [_P, _I32, _DP]),
    "lbib_profile_kernels": (_I, [_P, _I32, _DP]),
    "lbib_profile_hydro": (_I, [_P, _I32, _DP]),
    "lbib_kernels_per_step": (_I32, [_P]),
    "lbib_storage_scale_exponent": (_I32, [_P]),
    "lbib_last_error": (ctypes.c_char_p, [_P]),
    "lbib_destroy": (None, [_P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load liblbib.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("liblbib.so is not built: run __graft_entry__.build() "
                               "(or python -m paper_1907_00080_gb300.build)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, st):
    if st != LBIB_OK:
        msg = load().lbib_last_error(ctx).decode() if ctx else ""
        raise LbibError(st, msg)


def _dptr(a):
    return a.ctypes.data_as(_DP)


def _ptr(x):
    """host numpy array -> pointer; int -> device address; None -> NULL"""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    return x.ctypes.data_as(ctypes.c_void_p)


# ------------------------------------------------------------------ C names
def lbib_create(nx, ny, prec=LBIB_F32, init=LBIB_INIT_REST, tau=1.0, body_force=(0.0, 0.0),
                walls=LBIB_WALLS_Y_BOUNCEBACK, cuda_stream=None):
    lat = lbib_lattice(int(nx), int(ny), int(prec), int(init))
    bf = (ctypes.c_double * 2)(float(body_force[0]), float(body_force[1]))
    out = _P()
    st = load().lbib_create(ctypes.byref(lat), float(tau), bf, int(walls),
                            None if cuda_stream is None else ctypes.c_void_p(int(cuda_stream)),
                            ctypes.byref(out))
    if st != LBIB_OK:
        raise LbibError(st, "lbib_create(%d, %d) failed" % (nx, ny))
    return out


def lbib_add_membrane(ctx, xy, k_s, k_b, k_area, kind=LBIB_MEMBRANE_KINEMATIC, ligand_elems=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    lig = np.ascontiguousarray(ligand_elems if ligand_elems is not None else [], dtype=np.int32)
    mid = _I32()
    st = load().lbib_add_membrane(ctx, _dptr(xy), len(xy), float(k_s), float(k_b), float(k_area),
                                  int(kind), lig.ctypes.data_as(_I32P) if len(lig) else None,
                                  len(lig), ctypes.byref(mid))
    _check(ctx, st)
    return mid.value


def lbib_set_receptors(ctx, xy, d_cut=1.5, y_eq=0.75, sigma=0.0, kf_dt=1e-2, kr0_dt=1e-2 / 8.5e3,
                       beta_f=0.5, beta_r=2.0, d_break=3.0, seed=0, instance=0):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    p = lbib_bond_params(d_cut, y_eq, sigma, kf_dt, kr0_dt, beta_f, beta_r, d_break, int(seed), int(instance))
    _check(ctx, load().lbib_set_receptors(ctx, _dptr(xy), len(xy), ctypes.byref(p)))


def lbib_set_repulsion(ctx, d_rep):
    _check(ctx, load().lbib_set_repulsion(ctx, float(d_rep)))


def lbib_set_wall_velocity(ctx, u_bottom, u_top):
    _check(ctx, load().lbib_set_wall_velocity(ctx, float(u_bottom), float(u_top)))


def lbib_save(ctx, path):
    _check(ctx, load().lbib_save(ctx, os.fsencode(path)))


def lbib_load(ctx, path):
    _check(ctx, load().lbib_load(ctx, os.fsencode(path)))


OBSERVABLES = ("x_c", "y_c", "u_c", "v_c", "region", "bonds", "y_min", "y_max")


def lbib_membrane_observables(ctx, nmem):
    """(nmem, 8) array; columns as in OBSERVABLES"""
    out = np.zeros((max(nmem, 1), 8))
    _check(ctx, load().lbib_membrane_observables(ctx, _dptr(out)))
    return out[:nmem]


def lbib_step(ctx, n):
    _check(ctx, load().lbib_step(ctx, int(n)))


def lbib_sync(ctx):
    _check(ctx, load().lbib_sync(ctx))


def lbib_step_count(ctx):
    return load().lbib_step_count(ctx)


def lbib_read_fields(ctx, rho=None, ux=None, uy=None, on_device=0):
    _check(ctx, load().lbib_read_fields(ctx, _ptr(rho), _ptr(ux), _ptr(uy), int(on_device)))


def lbib_read_populations(ctx, f, on_device=0):
    _check(ctx, load().lbib_read_populations(ctx, _ptr(f), int(on_device)))


def lbib_write_populations(ctx, f, on_device=0):
    _check(ctx, load().lbib_write_populations(ctx, _ptr(f), int(on_device)))


def lbib_read_markers(ctx, membrane_id, xy):
    _check(ctx, load().lbib_read_markers(ctx, int(membrane_id), _dptr(xy)))


def lbib_write_markers(ctx, xy, xy_prev=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    xp = None if xy_prev is None else _dptr(np.ascontiguousarray(xy_prev, dtype=np.float64))
    _check(ctx, load().lbib_write_markers(ctx, _dptr(xy), xp))


def lbib_read_marker_forces(ctx, fxy):
    _check(ctx, load().lbib_read_marker_forces(ctx, _dptr(fxy)))


def lbib_read_marker_velocity(ctx, uxy):
    _check(ctx, load().lbib_read_marker_velocity(ctx, _dptr(uxy)))


def lbib_set_particle_density(ctx, membrane_id, rho_ratio):
    _check(ctx, load().lbib_set_particle_density(ctx, int(membrane_id), float(rho_ratio)))


def lbib_read_particle_velocity(ctx, membrane_id, uv):
    _check(ctx, load().lbib_read_particle_velocity(ctx, int(membrane_id), _dptr(uv)))


def lbib_read_bonds(ctx, cap):
    lig = np.zeros(max(cap, 1), dtype=np.int32)
    rec = np.zeros(max(cap, 1), dtype=np.int32)
    n = _I32()
    _check(ctx, load().lbib_read_bonds(ctx, lig.ctypes.data_as(_I32P), rec.ctypes.data_as(_I32P),
                                       int(cap), ctypes.byref(n)))
    k = min(n.value, cap)
    return lig[:k].copy(), rec[:k].copy(), n.value


def lbib_diagnostics(ctx, n_membranes=0):
    mass = np.zeros(1)
    areas = np.zeros(max(n_membranes, 1))
    _check(ctx, load().lbib_diagnostics(ctx, _dptr(mass), _dptr(areas) if n_membranes else None))
    return float(mass[0]), areas[:n_membranes]


def lbib_population_mass_noalloc(f_dev, n_nodes, mass_dev, stream=None):
    """Device addresses (ints) in, status out; enqueues only (no sync, no
    allocation).  Returns the lbib_status code (no context, no message)."""
    return load().lbib_population_mass_noalloc(ctypes.c_void_p(f_dev), int(n_nodes),
                                               ctypes.c_void_p(mass_dev),
                                               ctypes.c_void_p(stream) if stream else None)


def lbib_set_tiling(ctx, vec, ty):
    _check(ctx, load().lbib_set_tiling(ctx, int(vec), int(ty)))


def lbib_get_tiling(ctx):
    v, t = _I32(), _I32()
    _check(ctx, load().lbib_get_tiling(ctx, ctypes.byref(v), ctypes.byref(t)))
    return v.value, t.value


def lbib_profile_fused(ctx, reps):
    ms = np.zeros(1)
    _check(ctx, load().lbib_profile_fused(ctx, int(reps), _dptr(ms)))
    return float(ms[0])


def lbib_profile_hydro(ctx, reps):
    ms = np.zeros(1)
    _check(ctx, load().lbib_profile_hydro(ctx, int(reps), _dptr(ms)))
    return float(ms[0])


def lbib_profile_kernels(ctx, reps):
    """Mean ms per launch of (forces, fused collide-stream, advance)."""
    ms = np.zeros(3)
    _check(ctx, load().lbib_profile_kernels(ctx, int(reps), _dptr(ms)))
    return tuple(float(v) for v in ms)


def lbib_kernels_per_step(ctx):
    return load().lbib_kernels_per_step(ctx)


def lbib_storage_scale_exponent(ctx):
    return load().lbib_storage_scale_exponent(ctx)


def lbib_last_error(ctx):
    return load().lbib_last_error(ctx).decode()


def lbib_destroy(ctx):
    if ctx:
        load().lbib_destroy(ctx)


def _echeck(ens, st):
    if st != LBIB_OK:
        msg = load().lbib_ensemble_last_error(ens).decode() if ens else ""
        raise LbibError(st, msg)


def lbib_ensemble_create(ctxs, cuda_stream=None):
    arr = (_P * max(len(ctxs), 1))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    out = _P()
    st = load().lbib_ensemble_create(arr, len(ctxs), None if cuda_stream is None else _P(int(cuda_stream)),
                                     ctypes.byref(out))
    _echeck(None, st)
    return out


def lbib_ensemble_step(ens, n):
    _echeck(ens, load().lbib_ensemble_step(ens, int(n)))


def _ptr_table(arrays, n):
    """None -> NULL table; else a table of n pointers (None entries -> NULL)"""
    if arrays is None:
        return None
    if len(arrays) != n:
        raise ValueError("one entry per member")
    return (_P * n)(*[None if a is None else a.ctypes.data for a in arrays])


def lbib_ensemble_write_state(ens, n, f=None, xy=None, xy_prev=None):
    """f, xy, xy_prev: lists of n C-contiguous float64 host arrays (entries may
    be None) or None"""
    for arrs in (f, xy, xy_prev):
        for a in arrs or ():
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
                raise ValueError("C-contiguous float64 arrays")
    _echeck(ens, load().lbib_ensemble_write_state(ens, _ptr_table(f, n), _ptr_table(xy, n),
                                                  _ptr_table(xy_prev, n), 0))


def lbib_ensemble_read_markers(ens, xy):
    for a in xy:
        if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
            raise ValueError("C-contiguous float64 arrays")
    _echeck(ens, load().lbib_ensemble_read_markers(ens, _ptr_table(xy, len(xy))))


def lbib_ensemble_sync(ens):
    _echeck(ens, load().lbib_ensemble_sync(ens))


def lbib_ensemble_size(ens):
    return load().lbib_ensemble_size(ens)


def lbib_ensemble_form(ens):
    return load().lbib_ensemble_form(ens)


def lbib_ensemble_set_groups(ens, groups):
    _echeck(ens, load().lbib_ensemble_set_groups(ens, int(groups)))


def lbib_ensemble_groups(ens):
    return load().lbib_ensemble_groups(ens)


def lbib_ensemble_profile_kernels(ens, reps):
    """mean ms per launch of the batched force, fused and advance kernels
    (spends the ensemble: profile a scratch one)"""
    out = (_D * 3)()
    _echeck(ens, load().lbib_ensemble_profile_kernels(ens, int(reps), out))
    return list(out)


def lbib_ensemble_launches_per_step(ens):
    return load().lbib_ensemble_launches_per_step(ens)


def lbib_ensemble_member(ens, i):
    p = load().lbib_ensemble_member(ens, int(i))
    if not p:
        raise LbibError(LBIB_E_INVALID, "no member %d" % i)
    return _P(p)


def lbib_ensemble_last_error(ens):
    return load().lbib_ensemble_last_error(ens).decode()


def lbib_ensemble_destroy(ens):
    if ens:
        load().lbib_ensemble_destroy(ens)


def lbib_slabs_create(ctxs):
    arr = (_P * max(len(ctxs), 1))(*[c.value if isinstance(c, _P) else c for c in ctxs])
    out = _P()
    st = load().lbib_slabs_create(arr, len(ctxs), ctypes.byref(out))
    if st != LBIB_OK:
        msg = load().lbib_last_error(ctxs[0]).decode() if ctxs else ""
        raise LbibError(st, msg)
    return out


def _scheck(group, st):
    if st != LBIB_OK:
        raise LbibError(st, load().lbib_slabs_last_error(group).decode())


def lbib_slabs_step(group, n):
    _scheck(group, load().lbib_slabs_step(group, int(n)))


def lbib_slabs_sync(group):
    _scheck(group, load().lbib_slabs_sync(group))


def lbib_slabs_destroy(group):
    if group:
        load().lbib_slabs_destroy(group)


def lbib_slab_face(ctx, side, out, addr, on_device):
    """addr: host or device address of 3 x NY stored elements"""
    _check(ctx, load().lbib_slab_face(ctx, int(side), int(out), _P(int(addr)), int(on_device)))


def lbib_storage_bytes(ctx):
    return int(load().lbib_storage_bytes(ctx))


def lbib_tangent_create(ctx):
    out = _P()
    _check(ctx, load().lbib_tangent_create(ctx, ctypes.byref(out)))
    return out


def _dp_or_null(a):
    return None if a is None else _dptr(np.ascontiguousarray(a, dtype=np.float64))


def lbib_tangent_seed(ctx, t, dks=None, dkb=None, dsigma=0.0, dxy=None, dxy_prev=None):
    keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
            for a in (dks, dkb, dxy, dxy_prev)]
    ptrs = [None if a is None else _dptr(a) for a in keep]
    _check(ctx, load().lbib_tangent_seed(t, ptrs[0], ptrs[1], float(dsigma), ptrs[2], ptrs[3]))


def lbib_tangent_step(ctx, t, n):
    _check(ctx, load().lbib_tangent_step(t, int(n)))


def lbib_tangent_read(ctx, t, nv):
    dxy = np.zeros((nv, 2))
    dxp = np.zeros((nv, 2))
    _check(ctx, load().lbib_tangent_read(t, _dptr(dxy), _dptr(dxp)))
    return dxy, dxp


def lbib_tangent_destroy(t):
    if t:
        load().lbib_tangent_destroy(t)


def lbib_adjoint_create(ctx, checkpoint_every):
    out = _P()
    _check(ctx, load().lbib_adjoint_create(ctx, int(checkpoint_every), ctypes.byref(out)))
    return out


def lbib_adjoint_record(ctx, adj, n):
    _check(ctx, load().lbib_adjoint_record(adj, int(n)))


def lbib_adjoint_seed(ctx, adj, xy_bar=None, xy_prev_bar=None, f_bar=None):
    keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
            for a in (xy_bar, xy_prev_bar, f_bar)]
    ptrs = [None if a is None else _dptr(a) for a in keep]
    _check(ctx, load().lbib_adjoint_seed(adj, ptrs[0], ptrs[1], ptrs[2]))


def lbib_adjoint_reverse(ctx, adj):
    _check(ctx, load().lbib_adjoint_reverse(adj))


def lbib_adjoint_read(ctx, adj, nv, nmem, n_nodes=None):
    """Adjoints after the reverse sweep: dict of xy, xy_prev ([nv, 2]), k_s, k_b
    ([nmem]), sigma (float) and, when n_nodes is given, f ([9, n_nodes])."""
    xy = np.zeros((nv, 2))
    xyp = np.zeros((nv, 2))
    ks = np.zeros(max(nmem, 1))
    kb = np.zeros(max(nmem, 1))
    sg = np.zeros(1)
    f = None if n_nodes is None else np.zeros((9, n_nodes))
    _check(ctx, load().lbib_adjoint_read(adj, _dptr(xy), _dptr(xyp), _dptr(ks), _dptr(kb), _dptr(sg),
                                         None if f is None else _dptr(f)))
    return {"xy": xy, "xy_prev": xyp, "k_s": ks[:nmem], "k_b": kb[:nmem], "sigma": float(sg[0]), "f": f}


def lbib_adjoint_recorded_steps(adj):
    return load().lbib_adjoint_recorded_steps(adj)


def lbib_adjoint_destroy(adj):
    if adj:
        load().lbib_adjoint_destroy(adj)


# ------------------------------------------------------------------ convenience
class Simulation:
    """Owns one lbib context built from an ``inputs.Workload`` (marshalling only)."""

    def __init__(self, wl, precision=None, tiling=None, cuda_stream=None):
        prec = PRECISIONS[precision or wl.precision]
        init = {"poiseuille": LBIB_INIT_POISEUILLE, "couette": LBIB_INIT_COUETTE}.get(wl.init, LBIB_INIT_REST)
        self.wl = wl
        self.nx, self.ny = wl.nx, wl.ny
        self.ctx = lbib_create(wl.nx, wl.ny, prec, init, wl.tau, wl.body_force, wl.walls, cuda_stream)
        self.mem_sizes = []
        for k, m in enumerate(wl.membranes):
            lbib_add_membrane(self.ctx, m.xy, m.ks, m.kb, m.ka, m.kind, m.ligands)
            if m.kind in (LBIB_MEMBRANE_DYNAMIC, LBIB_MEMBRANE_DYNAMIC_RIGID):
                lbib_set_particle_density(self.ctx, k, m.rho_p)
            self.mem_sizes.append(len(m.xy))
        self.nv = sum(self.mem_sizes)
        self.nlig = wl.n_ligands
        if wl.receptors is not None and len(wl.receptors):
            b = wl.bonds
            lbib_set_receptors(self.ctx, wl.receptors, d_cut=b["d_cut"], y_eq=b["y_eq"],
                               sigma=wl.sigma_lu, kf_dt=b["kf_dt"], kr0_dt=b["kr0_dt"],
                               beta_f=b["beta_f"], beta_r=b["beta_r"], d_break=b["d_break"],
                               seed=wl.seed, instance=wl.instance)
        lbib_set_repulsion(self.ctx, wl.d_rep)
        if any(u != 0.0 for u in wl.wall_velocity):
            lbib_set_wall_velocity(self.ctx, *wl.wall_velocity)
        if tiling is not None:
            lbib_set_tiling(self.ctx, *tiling)

    def close(self):
        if self.ctx and not getattr(self, "owned_by_ensemble", False):
            lbib_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lbib_step(self.ctx, n)

    def sync(self):
        lbib_sync(self.ctx)

    def fields(self):
        r, a, b = (np.zeros((self.ny, self.nx)) for _ in range(3))
        lbib_read_fields(self.ctx, r, a, b)
        return r, a, b

    def populations(self):
        f = np.zeros((9, self.ny, self.nx))
        lbib_read_populations(self.ctx, f)
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        lbib_write_populations(self.ctx, f)

    def markers(self):
        xy = np.zeros((self.nv, 2))
        if self.nv:
            lbib_read_markers(self.ctx, -1, xy)
        return xy

    def forces(self):
        f = np.zeros((self.nv, 2))
        if self.nv:
            lbib_read_marker_forces(self.ctx, f)
        return f

    def marker_velocity(self):
        u = np.zeros((self.nv, 2))
        if self.nv:
            lbib_read_marker_velocity(self.ctx, u)
        return u

    def particle_velocity(self):
        """particle velocity of every vertex (zero on non-dynamic membranes),
        like the oracle's"""
        v = np.zeros((self.nv, 2))
        off = 0
        for k, m in enumerate(self.wl.membranes):
            n = len(m.xy)
            if m.kind in (LBIB_MEMBRANE_DYNAMIC, LBIB_MEMBRANE_DYNAMIC_RIGID):
                part = np.zeros((n, 2))
                lbib_read_particle_velocity(self.ctx, k, part)
                v[off:off + n] = part
            off += n
        return v

    def bonds(self):
        """bond_of_ligand array (-1 = free), like the oracle's"""
        lig, rec, n = lbib_read_bonds(self.ctx, self.nlig)
        out = -np.ones(self.nlig, dtype=np.int32)
        out[lig] = rec
        return out

    def diagnostics(self):
        return lbib_diagnostics(self.ctx, len(self.mem_sizes))

    def save(self, path):
        lbib_save(self.ctx, path)

    def load_state(self, path):
        lbib_load(self.ctx, path)

    def observables(self):
        """per-membrane observables (lbib_membrane_observables), (nmem, 8)"""
        return lbib_membrane_observables(self.ctx, len(self.mem_sizes))

    @property
    def tiling(self):
        return lbib_get_tiling(self.ctx)

    @property
    def kernels_per_step(self):
        return lbib_kernels_per_step(self.ctx)


class Ensemble:
    """Several workloads advanced together (lbib_ensemble_*); members keep the
    Simulation read-back methods.  Marshalling only."""

    def __init__(self, workloads, precision=None, cuda_stream=None, tiling=None):
        """tiling: (vec, ty) of the fused kernel for every member (row tiles,
        ty > 0, give the batched form); None keeps each member's default."""
        self.members = [Simulation(wl, precision=precision, tiling=tiling) for wl in workloads]
        self.ens = lbib_ensemble_create([m.ctx for m in self.members], cuda_stream)
        for m in self.members:
            m.owned_by_ensemble = True

    @property
    def form(self):
        """1: batched kernels over all members; 0: graph of member graphs"""
        return lbib_ensemble_form(self.ens)

    @property
    def launches_per_step(self):
        return lbib_ensemble_launches_per_step(self.ens)

    @property
    def groups(self):
        return lbib_ensemble_groups(self.ens)

    def set_groups(self, groups):
        lbib_ensemble_set_groups(self.ens, groups)

    def step(self, n=1):
        lbib_ensemble_step(self.ens, n)

    def sync(self):
        lbib_ensemble_sync(self.ens)

    def write_state(self, f=None, xy=None, xy_prev=None):
        """every member's populations (9, NY, NX) and markers (nv, 2) from host
        arrays in one call (lists with one entry per member, None to skip)"""
        lbib_ensemble_write_state(self.ens, len(self.members), f, xy, xy_prev)

    def read_markers(self, out):
        """every member's markers into the (nv, 2) float64 arrays of `out`"""
        lbib_ensemble_read_markers(self.ens, out)

    def close(self):
        if self.ens:
            lbib_ensemble_destroy(self.ens)
            self.ens = None
            for m in self.members:
                m.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Slabs:
    """A lattice-only workload split into x-slabs of the given interior widths
    (sum = NX), each a context with two ghost columns, advanced together with
    the halo exchange (lbib_slabs_*) on one shared CUDA stream.  f0 (9, NY, NX),
    optional, is the lattice's initial pre-collision state.  Marshalling only."""

    def __init__(self, wl, widths, precision=None, tiling=None, f0=None):
        import dataclasses

        import torch
        if wl.membranes:
            raise ValueError("slabs carry the lattice only")
        if sum(widths) != wl.nx:
            raise ValueError("the slab widths must add up to NX")
        self.widths = list(widths)
        self.stream = torch.cuda.Stream()
        self.sims = []
        x0 = 0
        for w in self.widths:
            sub = dataclasses.replace(wl, nx=w + 2, name="%s_slab%d" % (wl.name, len(self.sims)))
            sim = Simulation(sub, precision=precision, tiling=tiling, cuda_stream=self.stream.cuda_stream)
            if f0 is not None:
                cols = [(x0 - 1 + j) % wl.nx for j in range(w + 2)]
                sim.set_populations(np.asarray(f0)[:, :, cols])
            self.sims.append(sim)
            x0 += w
        self.group = lbib_slabs_create([s.ctx for s in self.sims])

    def step(self, n=1):
        lbib_slabs_step(self.group, n)

    def sync(self):
        lbib_slabs_sync(self.group)

    def populations(self):
        """(9, NY, NX): the interior columns of the slabs"""
        return np.concatenate([s.populations()[:, :, 1:-1] for s in self.sims], axis=2)

    def fields(self):
        parts = [s.fields() for s in self.sims]
        return tuple(np.concatenate([p[q][:, 1:-1] for p in parts], axis=1) for q in range(3))

    def close(self):
        if self.group:
            lbib_slabs_destroy(self.group)
            self.group = None
        for s in self.sims:
            s.close()
        self.sims = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""GPU parity of Zou and He's known-velocity walls (Sec. 2.1; walls on the
rows y = 0 and NY - 1) against the FP64 oracle, through the C ABI: lattice
start-up from random populations with a force and moving walls, the Couette
and Poiseuille closed forms reached from rest, both forms of the fused kernel
bitwise equal, a capsule adhering to a Zou-He wall, and the refusals.
Tolerances as in test_gpu_parity.py: FP64 1e-12 relative, FP32 1e-5 relative
(fields, populations) and 1e-5 lu (markers), bond sets bit-exact."""
import numpy as np
import pytest

from helpers import W9, dev_err, make_oracle, rel_err, vel_err
from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
ZH = 2


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def lb():
    from paper_1907_00080_gb300 import lbib
    return lbib


def zh_lattice(nx, ny, precision, tau=1.0, g=(0.0, 0.0), uw=(0.0, 0.0)):
    return inputs.Workload(name="zou_he", nx=nx, ny=ny, tau=tau, body_force=g, walls=ZH, init="rest",
                           precision=precision, membranes=[], receptors=None, wall_velocity=uw)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,tau", [(48, 16, 0.8), (130, 9, 1.0), (8, 5, 1.3)])
def test_random_start_with_force_and_moving_walls_matches_oracle(prec, nx, ny, tau):
    wl = zh_lattice(nx, ny, prec, tau=tau, g=(2e-5, -1e-5), uw=(0.003, -0.006))
    f0 = inputs.random_populations(nx, ny, W9, seed=nx + ny, amp=2e-2)
    s, r = lb().Simulation(wl), make_oracle(wl)
    s.set_populations(f0)
    r.set_populations(f0)
    for k in (1, 4, 20):
        s.step(k)
        r.step(k)
        assert dev_err(s.populations(), r.populations(), W9) < TOL[prec]
        rho, ux, uy = s.fields()
        rho0, ux0, uy0 = r.fields()
        assert vel_err(ux, uy, ux0, uy0) < TOL[prec]
        assert rel_err(rho, rho0) < TOL[prec]
    s.close()


@pytest.mark.parametrize("prec,tiling", [("f64", None), ("f32", None), ("f32", (2, 0)), ("f64", (1, 0))])
def test_couette_and_poiseuille_closed_forms_on_the_gpu(prec, tiling):
    """From rest: walls moving at -0.01 and 0.02 give the linear profile
    through the wall rows; a body force between resting walls gives the
    parabola G y (H - y) / (2 nu), H = NY - 1 (both exact steady states of the
    scheme), in both kernel forms."""
    tau, nx, ny = 1.0, 64, 17
    lbib = lb()
    s = lbib.Simulation(zh_lattice(nx, ny, prec, tau=tau, uw=(-0.01, 0.02)), tiling=tiling)
    s.step(6000)
    _, ux, uy = s.fields()
    u = -0.01 + 0.03 * np.arange(ny) / (ny - 1)
    tol = 1e-13 if prec == "f64" else 1e-6
    assert np.max(np.abs(ux - u[:, None])) < tol * 0.02 * 10
    s.close()
    G = 1e-6
    nu = (tau - 0.5) / 3
    s = lbib.Simulation(zh_lattice(nx, ny, prec, tau=tau, g=(G, 0.0)), tiling=tiling)
    s.step(6000)
    _, ux, _ = s.fields()
    y = np.arange(ny)
    u = G / (2 * nu) * y * (ny - 1 - y)
    tol = 1e-9 if prec == "f64" else 1e-5
    assert np.max(np.abs(ux - u[:, None])) / u.max() < tol
    s.close()


@pytest.mark.parametrize("prec,npt", [("f32", 2), ("f16", 4), ("f64", 1)])
def test_both_kernel_forms_agree_bitwise_with_zou_he_walls(prec, npt):
    nx, ny = 64, 20
    wl = zh_lattice(nx, ny, prec, tau=0.9, g=(1e-5, 0.0), uw=(0.002, 0.005))
    f0 = inputs.random_populations(nx, ny, W9, seed=3, amp=1e-2)
    a = lb().Simulation(wl, tiling=(2 if prec != "f64" else 1, 2))
    b = lb().Simulation(wl, tiling=(npt, 0))
    a.set_populations(f0)
    b.set_populations(f0)
    a.step(40)
    b.step(40)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def capsule_on_zou_he_wall(prec):
    """the 128 x 32 capsule case with the lower wall on the row y = 0: the
    capsule 1.25 lu above it, receptors on the wall row, a sheared flow from
    the upper wall"""
    wl = inputs.capsule_128x32(precision=prec, bonds="stress")
    wl.walls = ZH
    wl.init = "rest"
    wl.body_force = (0.0, 0.0)
    wl.wall_velocity = (0.0, 0.02)
    wl.membranes[0].xy = wl.membranes[0].xy + np.array([0.0, 0.5])
    wl.receptors = np.stack([np.arange(wl.nx, dtype=float), np.zeros(wl.nx)], axis=1)
    return wl


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_capsule_adhering_to_a_zou_he_wall_matches_oracle(prec):
    wl = capsule_on_zou_he_wall(prec)
    s, r = lb().Simulation(wl), make_oracle(wl)
    formed = 0
    for _ in range(6):
        s.step(50)
        r.step(50)
        b = s.bonds()
        assert np.array_equal(b, r.bonds())
        formed = max(formed, int((b >= 0).sum()))
    _, ux, uy = s.fields()
    _, ux0, uy0 = r.fields()
    assert vel_err(ux, uy, ux0, uy0) < TOL[prec]
    if prec == "f64":
        assert rel_err(s.markers(), r.markers()) < 1e-12
    else:
        assert np.max(np.abs(s.markers() - r.markers())) < 1e-5
    assert formed > 0
    s.close()


def test_zou_he_refusals():
    lbib = lb()
    # the Poiseuille and Couette starts belong to the half-way walls
    for init in ("poiseuille", "couette"):
        wl = zh_lattice(32, 8, "f64")
        wl.init = init
        with pytest.raises(lbib.LbibError):
            lbib.Simulation(wl)
    s = lbib.Simulation(zh_lattice(32, 12, "f64"))
    with pytest.raises(lbib.LbibError):
        lbib.lbib_add_membrane(s.ctx, inputs.circle(16, 6, 3, 20), 0.01, 0.0, 0.1, kind=2)
    s.close()

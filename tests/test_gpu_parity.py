"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.  Tolerances: FP64 1e-12 relative (fields and markers,
max-normalised), FP32 1e-5 relative for fields and 1e-5 lattice units for
markers; bond sets bit-exact."""
import numpy as np
import pytest

import oracle
from helpers import W9, dev_err, f64_field_tol, make_oracle, rel_err, vel_err
from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": dict(field=1e-12, marker_rel=1e-12, pop=1e-12),
       "f32": dict(field=1e-5, marker_abs=1e-5, pop=1e-5)}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def sim_of(wl, precision=None, tiling=None):
    from paper_1907_00080_gb300 import lbib
    return lbib.Simulation(wl, precision=precision, tiling=tiling)


def lattice_only(nx, ny, walls=1, tau=1.0, g=(0.0, 0.0), init="rest", precision="f64"):
    return inputs.Workload(name="lattice", nx=nx, ny=ny, tau=tau, body_force=g, walls=walls,
                           init=init, precision=precision, membranes=[], receptors=None)


def assert_markers(prec, got, ref):
    if prec == "f64":
        assert rel_err(got, ref) < TOL["f64"]["marker_rel"], rel_err(got, ref)
    else:
        assert np.max(np.abs(got - ref)) < TOL["f32"]["marker_abs"], np.max(np.abs(got - ref))


# ---------------------------------------------------------------- lattice only
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("walls", [1, 0])
@pytest.mark.parametrize("nx,ny", [(200, 37), (64, 6), (8, 5), (130, 16), (201, 9), (33, 7)])
def test_random_populations_stream_collide(prec, walls, nx, ny):
    wl = lattice_only(nx, ny, walls=walls, tau=0.8, g=(1e-5, -2e-6), precision=prec)
    f0 = inputs.random_populations(nx, ny, W9, seed=nx * ny + walls, amp=5e-2)
    s = sim_of(wl)
    r = make_oracle(wl)
    s.set_populations(f0)
    r.set_populations(f0)
    np.testing.assert_allclose(s.populations(), f0, rtol=0, atol=1e-15 if prec == "f64" else 1e-8)
    for k in (1, 4):
        s.step(k)
        r.step(k)
        assert dev_err(s.populations(), r.populations(), W9) < TOL[prec]["pop"]
        rho, ux, uy = s.fields()
        rho0, ux0, uy0 = r.fields()
        assert rel_err(rho - 1, rho0 - 1) < TOL[prec]["field"]
        assert rel_err(ux, ux0) < TOL[prec]["field"]
        assert rel_err(uy, uy0) < TOL[prec]["field"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_poiseuille_fixed_point_on_gpu(prec):
    nx, ny = 128, 32
    g = inputs.body_force_for(0.02, ny)
    wl = lattice_only(nx, ny, walls=1, g=(g, 0.0), init="poiseuille", precision=prec)
    s = sim_of(wl)
    r = make_oracle(wl)
    np.testing.assert_allclose(s.populations(), r.populations(), rtol=0, atol=1e-16 if prec == "f64" else 1e-8)
    s.step(1000)
    r.step(1000)
    _, ux, _ = s.fields()
    _, ux0, _ = r.fields()
    assert rel_err(ux, ux0) < TOL[prec]["field"]
    yy = np.arange(ny)
    closed = 3 * g * (yy + 0.5) * (ny - 0.5 - yy) + 0.25 * g
    # FP32 stores the deviations of f from w_i; u then carries ~1e-6 relative rounding
    assert np.max(np.abs(ux - closed[:, None])) / closed.max() < (1e-12 if prec == "f64" else 5e-6)


def test_tilings_agree_bitwise():
    wl = inputs.capsule_128x32(precision="f32", bonds="stress")
    from paper_1907_00080_gb300 import lbib
    outs = []
    for vec in (1, 2, 4):
        for ty in (1, 2, 4, 8):
            s = sim_of(wl, tiling=(vec, ty))
            s.step(50)
            outs.append((vec, ty, s.populations(), s.markers(), s.bonds()))
            s.close()
    for vec, ty, f, x, b in outs[1:]:
        assert np.array_equal(f, outs[0][2]), (vec, ty)
        assert np.array_equal(x, outs[0][3]), (vec, ty)
        assert np.array_equal(b, outs[0][4]), (vec, ty)


# persistent bulk-copy form of the fused kernel (tiling (npt, 0))
STREAM_FORMS = {"f64": [(1, 0), (2, 0)], "f32": [(1, 0), (2, 0), (4, 0)],
                "f16": [(2, 0), (4, 0), (8, 0)], "bf16": [(2, 0), (4, 0), (8, 0)]}


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("walls", [1, 0])
@pytest.mark.parametrize("nx,ny", [(200, 37), (8, 5), (1032, 9), (1024, 4)])
def test_persistent_form_matches_oracle(prec, walls, nx, ny):
    """Row segments of 256*npt nodes: single ragged segments (200, 8), a ragged
    last segment after whole ones (1032), whole segments only (1024)."""
    wl = lattice_only(nx, ny, walls=walls, tau=0.8, g=(1e-5, -2e-6), precision=prec)
    f0 = inputs.random_populations(nx, ny, W9, seed=nx * ny + walls + 7, amp=5e-2)
    r = make_oracle(wl)
    r.set_populations(f0)
    r.step(3)
    f_ref = r.populations()
    rho0, ux0, uy0 = r.fields()
    for tiling in STREAM_FORMS[prec]:
        s = sim_of(wl, tiling=tiling)
        assert s.tiling == tiling
        s.set_populations(f0)
        s.step(3)
        assert dev_err(s.populations(), f_ref, W9) < TOL[prec]["pop"], tiling
        rho, ux, uy = s.fields()
        assert rel_err(rho - 1, rho0 - 1) < TOL[prec]["field"], tiling
        assert rel_err(ux, ux0) < TOL[prec]["field"], tiling
        assert rel_err(uy, uy0) < TOL[prec]["field"], tiling
        s.close()


@pytest.mark.parametrize("prec,rowtile", [("f64", (2, 4)), ("f32", (4, 1)), ("f16", (8, 1)), ("bf16", (4, 2))])
def test_forms_agree_bitwise_capsule(prec, rowtile):
    wl = inputs.capsule_128x32(precision=prec, bonds="stress")
    outs = []
    for tiling in [rowtile] + STREAM_FORMS[prec]:
        s = sim_of(wl, tiling=tiling)
        s.step(60)
        rho, ux, uy = s.fields()
        outs.append((tiling, s.populations(), s.markers(), s.bonds(), ux))
        s.close()
    for tiling, f, x, b, ux in outs[1:]:
        assert np.array_equal(f, outs[0][1]), tiling
        assert np.array_equal(x, outs[0][2]), tiling
        assert np.array_equal(b, outs[0][3]), tiling
        assert np.array_equal(ux, outs[0][4]), tiling


def test_forms_agree_bitwise_capillary_640x160():
    wl = inputs.coarse_capillary_640x160(precision="f32")
    wl.bonds = dict(inputs.STRESS_BONDS)
    outs = []
    for tiling in [(1, 2), (2, 0), (4, 0)]:
        s = sim_of(wl, tiling=tiling)
        s.step(80)
        outs.append((tiling, s.populations(), s.markers(), s.bonds()))
        s.close()
    for tiling, f, x, b in outs[1:]:
        assert np.array_equal(f, outs[0][1]), tiling
        assert np.array_equal(x, outs[0][2]), tiling
        assert np.array_equal(b, outs[0][3]), tiling


def test_default_form_follows_lattice_size():
    small = sim_of(inputs.capsule_128x32("f32"))
    assert small.tiling[1] > 0
    big = sim_of(inputs.probe_lattice(2048, 1024, "f32"))
    assert big.tiling == (2, 0)
    big.step(2)
    _, ux, _ = big.fields()
    assert np.all(np.isfinite(ux))


def test_runs_are_deterministic():
    wl = inputs.capsule_128x32(precision="f64", bonds="stress")
    a, b = sim_of(wl), sim_of(wl)
    a.step(300)
    b.step(300)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.markers(), b.markers())
    assert np.array_equal(a.bonds(), b.bonds())


# ---------------------------------------------------------------- membranes
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_membrane_forces_match_oracle(prec):
    nx, ny = 96, 40
    wl = lattice_only(nx, ny, walls=1, g=(1e-6, 0.0), init="poiseuille", precision=prec)
    rng = np.random.Generator(np.random.PCG64(2))
    ring = inputs.circle(30.0, 12.0, 6.0, 40)
    rbc = inputs.rbc_contour(24.0, 120) + np.array([70.0, 25.0])
    wl.membranes = [inputs.Membrane(xy=ring, ks=0.05, kb=0.01, ka=0.3),
                    inputs.Membrane(xy=rbc, ks=0.02, kb=0.0, ka=1.0)]
    s, r = sim_of(wl), make_oracle(wl)
    # pre-stress both rings so that every force term is active
    xy = np.concatenate([ring, rbc]) + rng.normal(scale=0.15, size=(160, 2))
    from paper_1907_00080_gb300 import lbib
    lbib.lbib_write_markers(s.ctx, xy)
    r.set_markers(xy, xy)
    s.step(1)
    r.step(1)
    F, F0 = s.forces(), r.forces()
    assert rel_err(F, F0) < (1e-12 if prec == "f64" else 1e-5), rel_err(F, F0)
    assert rel_err(s.marker_velocity(), r.marker_velocity()) < TOL[prec]["field"]
    assert_markers(prec, s.markers(), r.markers())


def test_rest_shape_gives_exactly_zero_force():
    wl = inputs.capsule_128x32(precision="f32")
    wl.receptors = None
    wl.body_force = (0.0, 0.0)
    wl.init = "rest"
    s = sim_of(wl)
    s.step(1)
    assert np.all(s.forces() == 0.0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_repulsion_between_close_membranes(prec):
    nx, ny = 64, 32
    wl = lattice_only(nx, ny, walls=1, precision=prec)
    a = inputs.circle(20.0, 16.0, 4.0, 24)
    b = inputs.circle(29.4, 16.3, 4.0, 24)
    wl.membranes = [inputs.Membrane(xy=a, ks=0.0, kb=0.0, ka=0.0),
                    inputs.Membrane(xy=b, ks=0.0, kb=0.0, ka=0.0)]
    s, r = sim_of(wl), make_oracle(wl)
    s.step(1)
    r.step(1)
    F, F0 = s.forces(), r.forces()
    assert np.max(np.abs(F0)) > 0
    assert rel_err(F, F0) < (1e-12 if prec == "f64" else 1e-5)


def test_membrane_across_periodic_seam_and_near_wall():
    nx, ny = 64, 24
    g = inputs.body_force_for(0.02, ny)
    wl = lattice_only(nx, ny, walls=1, g=(g, 0.0), init="poiseuille", precision="f64")
    ring = inputs.circle(0.3, 3.2, 3.4, 30)  # straddles x = 0 and comes within 0.3 of the wall
    wl.membranes = [inputs.Membrane(xy=ring, ks=0.05, kb=0.005, ka=0.1, ligands=np.arange(30, dtype=np.int32))]
    wl.receptors = inputs.wall_receptors(nx, ny)
    wl.sigma_lu = 1e-3
    wl.bonds = dict(inputs.STRESS_BONDS)
    s, r = sim_of(wl), make_oracle(wl)
    for _ in range(6):
        s.step(50)
        r.step(50)
        assert np.array_equal(s.bonds(), r.bonds())
    assert rel_err(s.markers(), r.markers()) < 1e-12
    _, ux, uy = s.fields()
    _, ux0, uy0 = r.fields()
    assert vel_err(ux, uy, ux0, uy0) < 1e-12


# ---------------------------------------------------------------- end to end
@pytest.mark.parametrize("bonds", ["default", "stress"])
def test_capsule_128x32_fp64_1000_steps(bonds):
    wl = inputs.capsule_128x32(precision="f64", bonds=bonds)
    s, r = sim_of(wl), make_oracle(wl)
    m0 = s.diagnostics()[0]
    formed = 0
    for _ in range(10):
        s.step(100)
        r.step(100)
        b, b0 = s.bonds(), r.bonds()
        assert np.array_equal(b, b0)
        formed = max(formed, int((b >= 0).sum()))
    s.sync()
    rho, ux, uy = s.fields()
    rho0, ux0, uy0 = r.fields()
    assert vel_err(ux, uy, ux0, uy0) < 1e-12
    assert rel_err(rho, rho0) < 1e-12
    assert rel_err(s.markers(), r.markers()) < 1e-12
    assert rel_err(s.populations(), r.populations()) < 1e-12
    mass, areas = s.diagnostics()
    assert abs(mass - m0) / m0 < 1e-13
    assert abs(mass - r.mass()) / m0 < 1e-13
    assert abs(areas[0] - r.area(0)) / abs(r.area(0)) < 1e-12
    if bonds == "stress":
        assert formed > 0


def test_capsule_128x32_fp32_against_fp64_oracle():
    """FP32 storage and arithmetic against the FP64 oracle on the stiff capsule
    (k_s = 0.05, u_max = 0.02, stress kinetics): within 1e-5 (fields, relative
    to the speed scale) and 1e-5 lattice units (markers) after 100 and after
    1000 steps; bond sets bit-exact every 100 steps.  The FP32 collision
    carries the momentum without systematic rounding error; with the plain
    FP32 arithmetic the capsule drifted by 2e-4 lu over the 1000 steps."""
    wl = inputs.capsule_128x32(precision="f32", bonds="stress")
    s, r = sim_of(wl), make_oracle(wl)
    for k in range(10):
        s.step(100)
        r.step(100)
        assert np.array_equal(s.bonds(), r.bonds())
        if k in (0, 9):
            rho, ux, uy = s.fields()
            rho0, ux0, uy0 = r.fields()
            assert vel_err(ux, uy, ux0, uy0) < TOL["f32"]["field"]
            assert rel_err(rho, rho0) < TOL["f32"]["field"]
            assert np.max(np.abs(s.markers() - r.markers())) < TOL["f32"]["marker_abs"]


def test_coarse_capillary_640x160_fp32_1000_steps():
    """The coarse capillary in FP32 over 1000 steps against the oracle (stress
    kinetics on both walls): fields within 1e-5 of the speed scale, markers
    within 1e-5 lu, bond sets bit-exact every 100 steps."""
    from paper_1907_00080_gb300 import tuning
    wl = inputs.coarse_capillary_640x160(precision="f32")
    wl.bonds = dict(inputs.STRESS_BONDS)
    s = sim_of(wl, tiling=tuning.bench_tiling(wl))
    r = make_oracle(wl)
    for _ in range(10):
        s.step(100)
        r.step(100)
        assert np.array_equal(s.bonds(), r.bonds())
    rho, ux, uy = s.fields()
    rho0, ux0, uy0 = r.fields()
    assert vel_err(ux, uy, ux0, uy0) < TOL["f32"]["field"]
    assert rel_err(rho, rho0) < TOL["f32"]["field"]
    assert np.max(np.abs(s.markers() - r.markers())) < TOL["f32"]["marker_abs"]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_coarse_capillary_640x160(prec):
    """Full-size coarse capillary (8 red cells, 4 carriers, both walls with
    receptors) in the tiling the benchmark uses, 200 steps against the oracle."""
    from paper_1907_00080_gb300 import tuning
    wl = inputs.coarse_capillary_640x160(precision=prec)
    wl.bonds = dict(inputs.STRESS_BONDS)
    s = sim_of(wl, tiling=tuning.bench_tiling(wl))
    r = make_oracle(wl)
    for _ in range(4):
        s.step(50)
        r.step(50)
        assert np.array_equal(s.bonds(), r.bonds())
    rho, ux, uy = s.fields()
    rho0, ux0, uy0 = r.fields()
    # u_max ~ 1e-5 here: FP64 is held to the oracle's own rounding floor
    tol = f64_field_tol(np.max(np.abs(ux0))) if prec == "f64" else TOL["f32"]["field"]
    assert vel_err(ux, uy, ux0, uy0) < tol
    assert rel_err(rho, rho0) < TOL[prec]["field"]
    assert_markers(prec, s.markers(), r.markers())


def test_fields_unavailable_before_first_step_and_after_write():
    from paper_1907_00080_gb300 import lbib
    wl = lattice_only(32, 8)
    s = sim_of(wl)
    with pytest.raises(lbib.LbibError):
        s.fields()
    s.step(1)
    s.fields()
    s.set_populations(s.populations())
    with pytest.raises(lbib.LbibError):
        s.fields()


def test_invalid_arguments_are_rejected():
    from paper_1907_00080_gb300 import lbib
    with pytest.raises(lbib.LbibError):
        lbib.lbib_create(2, 8)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_create(32, 8, tau=0.5)
    ctx = lbib.lbib_create(32, 8)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_add_membrane(ctx, np.zeros((2, 2)), 0.1, 0.1, 0.1)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_set_tiling(ctx, 3, 1)
    lbib.lbib_step(ctx, 2)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_add_membrane(ctx, inputs.circle(5, 4, 2, 8), 0.1, 0.1, 0.1)
    lbib.lbib_destroy(ctx)

"""Pins of the oracle's full step orchestration (CPU only): the kinematic
advance against the printed BDF2 coefficients, the rigid projection, exact mass
conservation on the 128x32 capsule case with adhesion, and determinism."""
import json
import os

import numpy as np

import oracle
from paper_1907_00080_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def make(wl):
    s = oracle.OracleSim(wl.nx, wl.ny, wl.tau, wl.body_force, wl.walls, init=wl.init)
    for m in wl.membranes:
        s.add_membrane(m.xy, m.ks, m.kb, m.ka, m.kind, m.ligands)
    if wl.receptors is not None:
        b = wl.bonds
        s.set_receptors(wl.receptors, d_cut=b["d_cut"], y_eq=b["y_eq"], sigma=wl.sigma_lu,
                        kf_dt=b["kf_dt"], kr0_dt=b["kr0_dt"], beta_f=b["beta_f"],
                        beta_r=b["beta_r"], d_break=b["d_break"], seed=wl.seed,
                        instance=wl.instance)
    s.set_repulsion(wl.d_rep)
    return s


def test_advance_follows_eq_kinematicpos():
    wl = inputs.capsule_128x32()
    s = make(wl)
    x0 = s.markers()
    s.step(1)
    # first step: forward Euler with the interpolated velocity
    np.testing.assert_allclose(s.markers(), x0 + s.marker_velocity(), rtol=0, atol=1e-15)
    for _ in range(3):
        xn, xp = s.markers(), s.prev_markers()
        s.step(1)
        g = GOLD["kinematic_bdf2"]
        pred = g["c_prev"] * xn + g["c_prev2"] * xp + g["c_vel"] * s.marker_velocity()
        np.testing.assert_allclose(s.markers(), pred, rtol=0, atol=1e-13)


def test_marker_velocity_is_interpolated_fluid_velocity():
    wl = inputs.capsule_128x32()
    s = make(wl)
    x0 = s.markers()
    s.step(1)
    _, ux, uy = s.fields()
    U = s.interp(ux, uy, x0)
    np.testing.assert_allclose(s.marker_velocity(), U, rtol=0, atol=1e-17)
    # a capsule at rest shape in Poiseuille flow moves with the local flow speed
    assert np.all(s.marker_velocity()[:, 0] > 0)


def test_rigid_projection_gives_rigid_motion():
    nx, ny = 64, 32
    G = inputs.body_force_for(0.02, ny)
    s = oracle.OracleSim(nx, ny, 1.0, (G, 0.0), walls=1, init="poiseuille")
    ring = inputs.circle(20.0, 10.0, 5.0, 30)
    s.add_membrane(ring, ks=0.01, kb=0.001, ka=1.0, kind=1)
    s.step(1)
    d = s.markers() - ring  # Euler step: displacement = projected velocity
    c = ring.mean(axis=0)
    r = ring - c
    A = np.zeros((60, 3))
    A[0::2, 0] = 1
    A[1::2, 1] = 1
    A[0::2, 2] = -r[:, 1]
    A[1::2, 2] = r[:, 0]
    coef, res, *_ = np.linalg.lstsq(A, d.reshape(-1), rcond=None)
    assert np.max(np.abs(A @ coef - d.reshape(-1))) < 1e-14  # rounding of X1 - X0 at |X| ~ 20
    assert coef[2] < 0  # shear below the centreline spins the body clockwise
    # pairwise distances are preserved to first order (rigid velocity field)
    dist0 = np.hypot(*(ring[0] - ring[15]))
    dist1 = np.hypot(*(s.markers()[0] - s.markers()[15]))
    assert abs(dist1 - dist0) < 1e-6


def test_capsule_case_mass_and_bonds():
    wl = inputs.capsule_128x32(bonds="stress")
    s = make(wl)
    m0 = s.mass()
    nb = []
    for _ in range(10):
        s.step(100)
        nb.append(int((s.bonds() >= 0).sum()))
    assert abs(s.mass() - m0) / m0 < 1e-13
    assert max(nb) > 0  # bonds do form in the stress kinetics
    A = s.area(0)
    assert abs(A / s.rest_area(0) - 1) < 0.05


def test_oracle_is_deterministic():
    wl = inputs.capsule_128x32(bonds="stress")
    a, b = make(wl), make(wl)
    a.step(200)
    b.step(200)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.markers(), b.markers())
    assert np.array_equal(a.bonds(), b.bonds())


def test_repulsion_pushes_close_membranes_apart():
    nx, ny = 64, 32
    s = oracle.OracleSim(nx, ny, 1.0, (0.0, 0.0), walls=1)
    a = inputs.circle(20.0, 16.0, 4.0, 24)
    b = inputs.circle(29.5, 16.0, 4.0, 24)  # gap 1.5 < d_rep = 2
    s.add_membrane(a, 0.0, 0.0, 0.0)
    s.add_membrane(b, 0.0, 0.0, 0.0)
    s.compute_forces()
    F = s.forces()
    # the facing vertices are pushed inward, i.e. away from the other body
    ia = np.argmax(a[:, 0])
    ib = np.argmin(b[:, 0])
    assert F[ia, 0] < 0 and F[24 + ib, 0] > 0
    c0 = GOLD["repulsion"]["prefactor"]
    d = np.hypot(*(a[ia] - b[ib]))
    assert abs(F[ia, 0]) >= c0 * d ** -2.5 * 0.99
    far = np.hypot(a[:, 0] - 25.0, a[:, 1] - 16.0) > 4.0
    assert np.all(F[:24][far] == 0.0)


def test_whole_step_carries_a_relaxed_capsule_with_a_uniform_flow():
    """A closed-form check of the whole step's orchestration (forces ->
    spreading -> collision -> interpolation -> BDF2): both walls moving at U
    keep the fluid uniform (tau = 1 Couette state of equal wall speeds), the
    capsule at its rest shape feels no force, the interpolated velocity of a
    uniform field is U (partition of unity of the shape functions, near the
    walls too), and Euler then BDF2 give X^n = X^0 + n U exactly."""
    import oracle
    U = 0.013
    s = oracle.OracleSim(64, 16, tau=1.0, walls=1, init="couette", wall_velocity=(U, U))
    ring = np.stack([20.0 + 3.0 * np.cos(2 * np.pi * (np.arange(24) + 0.5) / 24),
                     3.3 + 3.0 * np.sin(2 * np.pi * (np.arange(24) + 0.5) / 24)], axis=1)
    s.add_membrane(ring, 0.05, 0.005, 0.1)
    x0 = s.markers()
    s.step(40)
    x = s.markers()
    np.testing.assert_allclose(x[:, 0], x0[:, 0] + 40 * U, rtol=0, atol=1e-12)
    np.testing.assert_allclose(x[:, 1], x0[:, 1], rtol=0, atol=1e-13)
    rho, ux, uy = s.fields()
    np.testing.assert_allclose(ux, U, rtol=0, atol=1e-15)
    np.testing.assert_allclose(uy, 0.0, rtol=0, atol=1e-15)
    np.testing.assert_allclose(s.forces(), 0.0, rtol=0, atol=1e-13)  # the rest shape, translated


def test_openmp_build_gives_the_same_bits():
    """The oracle's OpenMP build (loop pragmas over nodes, rows and vertices,
    each writing its own elements) reproduces the plain build bit for bit:
    the coarse-capillary set-up on a 160 x 48 lattice with two red cells and
    a carrier near each other (repulsion), stress bond kinetics, 30 steps."""
    import oracle
    from helpers import make_oracle
    from paper_1907_00080_gb300 import inputs
    wl = inputs.capillary(nx=160, ny=48, n_rbc=2, rbc_alpha=16.0, rbc_markers=60, n_carriers=1,
                          carrier_radius=5.0, carrier_markers=30, precision="f64", seed=5)
    wl.bonds = dict(inputs.STRESS_BONDS)
    try:
        a = make_oracle(wl)
        a.step(30)
        ref = (a.populations(), a.markers(), a.bonds(), a.forces())
        del a
        assert oracle.use_threads(4) == 4
        b = make_oracle(wl)
        b.step(30)
        got = (b.populations(), b.markers(), b.bonds(), b.forces())
        del b
    finally:
        oracle.use_threads(1)
    for x, y in zip(got, ref):
        np.testing.assert_array_equal(x, y)

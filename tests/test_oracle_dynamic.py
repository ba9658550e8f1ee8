"""Pins of the oracle's dynamic IB for particles (Sec. 2.4), CPU only.

Each part is checked against a fact of geometry or mechanics, not against its
own formula:
  - polygon mass properties: closed forms for a rectangle, a triangle and the
    regular N-gon (J = A R^2 (2 + cos(2 pi / N)) / 6);
  - the MLS fit reproduces linear fields (value and gradient), also where a
    wall row drops out; its value row equals the Roma interpolation inside;
  - Eq. hydroForP: a linear pressure field gives, per element,
    -(g . q_l) n_l l_l at the probe q_l = c_l + 1.2 n_l, and in total
    -(A + 0.6 N s) g on a regular N-gon (side s);
  - Eq. hydroForNu: a linear velocity field u = u_0 + B x gives, per element,
    nu (B + B^T) n_l l_l, and no net force or moment;
  - the forcing term: in a uniform flow u_0 a particle at rest exerts
    -2 dV_v u_0 per vertex (-2 u_0 times the perimeter in total) and none when
    it moves with the flow;
  - Eqs. linearVelRig / angularVelRig: under a constant force or moment the
    printed second-order update gives u_k = k F / m and omega_k = k M / I
    exactly (it is exact for linear growth), the body stays rigid and turns
    by sum omega_k;
  - Eq. verletVel: the backward difference is exact for quadratic paths.
"""
import numpy as np
import pytest

import oracle
from paper_1907_00080_gb300 import inputs

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def feq(rho, ux, uy):
    """D2Q9 equilibrium of given node fields (Eq. feq), written out here."""
    eu = EX[:, None, None] * ux[None] + EY[:, None, None] * uy[None]
    uu = ux * ux + uy * uy
    return W9[:, None, None] * rho[None] * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * uu[None])


def grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def ngon(cx, cy, R, n):
    return inputs.circle(cx, cy, R, n)


def normals(xy):
    """outward unit normals, lengths and centroids of the elements of a CCW ring"""
    e = np.roll(xy, -1, axis=0) - xy
    L = np.hypot(e[:, 0], e[:, 1])
    n = np.stack([e[:, 1], -e[:, 0]], axis=1) / L[:, None]
    c = 0.5 * (xy + np.roll(xy, -1, axis=0))
    return n, L, c


# ---------------------------------------------------------------- geometry
def test_mass_properties_closed_forms():
    a, b = 3.0, 1.5
    rect = np.array([[10, 20], [10 + a, 20], [10 + a, 20 + b], [10, 20 + b]], dtype=float)
    A, (cx, cy), J = oracle.ring_mass_properties(rect)
    assert A == pytest.approx(a * b, rel=1e-15)
    assert (cx, cy) == pytest.approx((a / 2, b / 2), rel=1e-15)
    assert J == pytest.approx(a * b * (a * a + b * b) / 12, rel=1e-14)
    # right triangle with legs p, q: polar moment about its centroid p q (p^2 + q^2) / 36
    p, q = 2.0, 5.0
    tri = np.array([[1, 1], [1 + p, 1], [1, 1 + q]], dtype=float)
    A, (cx, cy), J = oracle.ring_mass_properties(tri)
    assert A == pytest.approx(p * q / 2, rel=1e-15)
    assert (cx, cy) == pytest.approx((p / 3, q / 3), rel=1e-14)
    assert J == pytest.approx(p * q * (p * p + q * q) / 36, rel=1e-13)
    for n in (3, 7, 50, 210):
        R = 8.0
        xy = ngon(40.3, 17.9, R, n)
        al = 2 * np.pi / n
        A, (cx, cy), J = oracle.ring_mass_properties(xy)
        A_ex = n * R * R * np.sin(al) / 2
        assert A == pytest.approx(A_ex, rel=1e-13)
        assert (xy[0, 0] + cx, xy[0, 1] + cy) == pytest.approx((40.3, 17.9), abs=1e-12)
        assert J == pytest.approx(A_ex * R * R * (2 + np.cos(al)) / 6, rel=1e-12)


def test_mass_and_inertia_follow_the_density():
    s = oracle.OracleSim(48, 32, 1.0, walls=1)
    xy = ngon(24.0, 16.0, 6.0, 40)
    m = s.add_membrane(xy, 1e-3, 0.0, 1.0, kind=3)
    A, _, J = oracle.ring_mass_properties(xy)
    assert s.mass_of(m) == pytest.approx(1.1 * A, rel=1e-14)  # rho_P / rho = 1.1 by default
    assert s.inertia_of(m) == pytest.approx(1.1 * J, rel=1e-14)
    s.set_density(m, 2.5)
    assert s.mass_of(m) == pytest.approx(2.5 * A, rel=1e-14)


# ---------------------------------------------------------------- MLS fit
@pytest.mark.parametrize("walls", [1, 0])
def test_mls_fit_reproduces_linear_fields(walls):
    nx, ny = 40, 24
    s = oracle.OracleSim(nx, ny, 1.0, walls=walls)
    x, y = grid(nx, ny)
    rng = np.random.default_rng(3)
    a0, bx, by = 0.7, -0.31, 0.45
    g = a0 + bx * x + by * y
    pts = np.column_stack([rng.uniform(3, nx - 4, 60), rng.uniform(2, ny - 3, 60)])
    if walls:
        # near the walls one stencil row falls outside and the 3x3 system is solved
        near = np.column_stack([rng.uniform(3, nx - 4, 40),
                                np.concatenate([rng.uniform(-0.45, 0.49, 20), rng.uniform(ny - 1.49, ny - 0.55, 20)])])
        pts = np.vstack([pts, near])
    for px, py in pts:
        val, gx, gy = s.mls_fit(px, py, g)
        assert val == pytest.approx(a0 + bx * px + by * py, abs=1e-13)
        assert gx == pytest.approx(bx, abs=1e-12)
        assert gy == pytest.approx(by, abs=1e-12)


def test_mls_value_row_is_the_roma_interpolation_inside():
    s = oracle.OracleSim(32, 20, 1.0, walls=1)
    rng = np.random.default_rng(5)
    for px, py in np.column_stack([rng.uniform(3, 28, 30), rng.uniform(2, 17, 30)]):
        phi, idx = s.mls_shape(px, py)
        w, idx2 = s.ib_weights(px, py)
        np.testing.assert_array_equal(idx, idx2)
        np.testing.assert_allclose(phi[0], w, rtol=0, atol=1e-15)


def test_mls_fit_outside_the_fluid():
    s = oracle.OracleSim(32, 20, 1.0, walls=1)
    x, y = grid(32, 20)
    c = np.full((20, 32), 0.125)
    # one fluid row left: the gradient is undetermined; constant value, zero gradient
    val, gx, gy = s.mls_fit(10.3, -0.9, c + 0.0 * x)
    assert (val, gx, gy) == pytest.approx((0.125, 0.0, 0.0), abs=1e-16)
    # no fluid node in reach: all zero
    assert np.all(s.mls_fit(10.3, -2.6, c) == 0.0)


# ---------------------------------------------------------------- hydrodynamic stresses
def dynamic_ring(nx=64, ny=48, tau=1.0, walls=1, R=6.0, n=40, kind=2, gbody=(0.0, 0.0)):
    s = oracle.OracleSim(nx, ny, tau, gbody, walls=walls)
    xy = ngon(nx / 2 + 0.37, ny / 2 - 0.21, R, n)
    m = s.add_membrane(xy, 1e-3, 1e-4, 1.0, kind=kind)
    return s, m, xy


def test_pressure_force_closed_form():
    s, m, xy = dynamic_ring()
    x, y = grid(s.nx, s.ny)
    g = np.array([2.0e-4, -1.3e-4])
    p0 = 1.0e-5
    rho = 1.0 + 3.0 * (p0 + g[0] * x + g[1] * y)  # p = (rho - 1) / 3 = p0 + g . x, u = 0
    s.set_populations(W9[:, None, None] * rho[None])
    fe = s.hydro_element_forces(m)
    n, L, c = normals(xy)
    q = c + 1.2 * n
    p_q = p0 + q @ g
    np.testing.assert_allclose(fe, -(p_q * L)[:, None] * n, rtol=0, atol=1e-15)
    A = oracle.ring_area(xy)
    N, side = len(xy), L.mean()
    np.testing.assert_allclose(fe.sum(0), -(A + 0.6 * N * side) * g, rtol=1e-9, atol=0)


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_viscous_force_closed_form(tau):
    s, m, xy = dynamic_ring(tau=tau)
    x, y = grid(s.nx, s.ny)
    u0 = np.array([3e-3, -1e-3])
    B = np.array([[2.0e-4, -3.1e-4], [1.7e-4, -0.6e-4]])
    ux = u0[0] + B[0, 0] * x + B[0, 1] * y
    uy = u0[1] + B[1, 0] * x + B[1, 1] * y
    s.set_populations(feq(np.ones_like(x), ux, uy))
    fe = s.hydro_element_forces(m)
    nu = (tau - 0.5) / 3.0
    n, L, c = normals(xy)
    expect = nu * (n @ (B + B.T).T) * L[:, None]
    np.testing.assert_allclose(fe, expect, rtol=0, atol=1e-14 * np.abs(expect).max() * 1e3)
    assert np.abs(fe.sum(0)).max() < 1e-12 * np.abs(expect).max() * len(xy)
    r = c - xy.mean(0)
    torque = np.sum(r[:, 0] * fe[:, 1] - r[:, 1] * fe[:, 0])
    assert abs(torque) < 1e-12 * np.abs(expect).max() * len(xy) * 10


def test_vertex_hydro_force_is_half_of_each_adjacent_element():
    s, m, xy = dynamic_ring(tau=0.9, kind=2)
    x, y = grid(s.nx, s.ny)
    rng = np.random.default_rng(11)
    ux = 1e-3 * np.sin(2 * np.pi * x / s.nx) * (1 + 0.1 * y / s.ny)
    uy = 1e-3 * np.cos(2 * np.pi * y / s.ny)
    rho = 1.0 + 1e-4 * rng.standard_normal(x.shape)
    s.set_populations(feq(rho, ux, uy))
    fe = s.hydro_element_forces(m)
    s.compute_step_forces()
    h = s.hydro_forces()
    np.testing.assert_allclose(h, 0.5 * (fe + np.roll(fe, 1, axis=0)), rtol=0, atol=1e-18)
    # the total force of a dynamic membrane holds the hydrodynamic part
    s2, _, _ = dynamic_ring(tau=0.9, kind=0)
    s2.set_populations(feq(rho, ux, uy))
    s2.compute_forces()
    np.testing.assert_allclose(s.forces(), s2.forces() + h, rtol=0, atol=1e-18)


# ---------------------------------------------------------------- forcing term
@pytest.mark.parametrize("kind", [2, 3])
def test_forcing_term_in_uniform_flow(kind):
    s, m, xy = dynamic_ring(walls=0, kind=kind)
    u0 = np.array([2.5e-3, -1.5e-3])
    ones = np.ones((s.ny, s.nx))
    s.set_populations(feq(ones, u0[0] * ones, u0[1] * ones))
    s.compute_step_forces()
    n, L, c = normals(xy)
    dV = 0.5 * (L + np.roll(L, 1))
    np.testing.assert_allclose(s.ib_forces(), -2.0 * dV[:, None] * u0[None], rtol=1e-13)
    np.testing.assert_allclose(s.ib_forces().sum(0), -2.0 * L.sum() * u0, rtol=1e-13)
    assert np.abs(s.hydro_forces()).max() < 1e-16
    # moving with the flow: nothing to correct (rounding of the interpolation only)
    s.set_particle_velocity(np.tile(u0, (len(xy), 1)))
    s.compute_step_forces()
    assert np.abs(s.ib_forces()).max() < 1e-16


def test_forcing_term_is_what_the_fluid_receives():
    """One step in a periodic box: the fluid's momentum changes by the body
    force plus the particle's forcing terms (spreading keeps the sum)."""
    s, m, xy = dynamic_ring(walls=0, kind=2, gbody=(1e-6, 0.0))
    ones = np.ones((s.ny, s.nx))
    u0 = np.array([2e-3, 0.0])
    s.set_populations(feq(ones, u0[0] * ones, u0[1] * ones))
    f0 = s.populations()
    j0 = np.array([(f0 * EX[:, None, None]).sum(), (f0 * EY[:, None, None]).sum()])
    s.step(1)
    f1 = s.populations()
    j1 = np.array([(f1 * EX[:, None, None]).sum(), (f1 * EY[:, None, None]).sum()])
    total = s.nx * s.ny * np.array([1e-6, 0.0]) + s.ib_forces().sum(0)
    np.testing.assert_allclose(j1 - j0, total, rtol=1e-9, atol=1e-12)  # sums of ~3000 O(1e-3) terms


# ---------------------------------------------------------------- Newton
def test_rigid_constant_force_gives_linear_velocity():
    s, m, xy = dynamic_ring(kind=3)
    s.set_density(m, 1.7)
    f0 = np.array([3e-5, -1e-5])
    K = 12
    c0 = xy.mean(0)
    for k in range(K):
        s.set_forces(np.tile(f0, (len(xy), 1)))
        s.particle_advance(k)
        st = s.rigid_state(m)
        a = len(xy) * f0 / s.mass_of(m)
        np.testing.assert_allclose(st[:2], (k + 1) * a, rtol=1e-12)
        assert abs(st[4]) < 1e-18
    xyK = s.markers()
    np.testing.assert_allclose(xyK.mean(0) - c0, a * K * (K + 1) / 2, rtol=1e-10)
    np.testing.assert_allclose(xyK - xyK.mean(0), xy - c0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(s.particle_velocity(), np.tile(K * a, (len(xy), 1)), rtol=1e-12)


def test_rigid_constant_moment_gives_linear_spin():
    R, n = 6.0, 40
    s, m, xy = dynamic_ring(kind=3, R=R, n=n)
    f0 = 2e-5
    K = 10
    c0 = np.array([s.nx / 2 + 0.37, s.ny / 2 - 0.21])
    al = 2 * np.pi / n
    A = n * R * R * np.sin(al) / 2
    I = 1.1 * A * R * R * (2 + np.cos(al)) / 6
    M = n * f0 * R
    turned = 0.0
    for k in range(K):
        r = s.markers() - c0
        t = np.stack([-r[:, 1], r[:, 0]], axis=1) / np.hypot(r[:, 0], r[:, 1])[:, None]
        s.set_forces(f0 * t)
        s.particle_advance(k)
        om = s.rigid_state(m)[4]
        assert om == pytest.approx((k + 1) * M / I, rel=1e-11)
        turned += om
    r = s.markers() - c0
    np.testing.assert_allclose(np.hypot(r[:, 0], r[:, 1]), R, rtol=1e-12)
    ang = np.arctan2(r[:, 1], r[:, 0]) - np.arctan2(xy[:, 1] - c0[1], xy[:, 0] - c0[0])
    ang = (ang + np.pi) % (2 * np.pi) - np.pi
    np.testing.assert_allclose(ang, turned, rtol=1e-10)
    V = s.particle_velocity()
    np.testing.assert_allclose(V, om * np.stack([-r[:, 1], r[:, 0]], axis=1), rtol=0, atol=1e-15)


def test_soft_velocity_is_exact_for_quadratic_paths():
    s, m, xy = dynamic_ring(kind=2, n=30)
    nv = len(xy)
    c = np.array([1e-4, -2e-4])
    f = np.array([4e-5, 1e-5])
    mv = 1.1 * oracle.ring_area(xy) / nv
    h = 0.5 * f / mv
    K = 9
    for k in range(K):
        s.set_marker_velocity(np.tile(k * c, (nv, 1)))
        s.set_forces(np.tile(f, (nv, 1)))
        s.particle_advance(k)
        V = s.particle_velocity()
        # path x^k = x^0 + c k (k - 1) / 2 + h k; its derivative at k + 1 is c (k + 1/2) + h
        want = h if k == 0 else c * (k + 0.5) + h
        np.testing.assert_allclose(V, np.tile(want, (nv, 1)), rtol=1e-9, atol=1e-17)
    np.testing.assert_allclose(s.markers() - xy, np.tile(c * K * (K - 1) / 2 + h * K, (nv, 1)), rtol=1e-10)


@pytest.mark.parametrize("walls", [0, 1])
def test_drag_opposes_the_motion_of_a_rigid_particle(walls):
    """In a fluid at rest the probe tractions and the forcing term must slow a
    rigid particle down.  Its spin decays monotonically and does not reverse.
    Its translation stays below the initial speed and does not reverse: the
    fluid only ever receives energy from the particle.  It need not decay
    monotonically, since the fluid first entrained by the forcing term pushes
    back."""
    s, m, xy = dynamic_ring(nx=64, ny=64, walls=walls, R=8.0, n=50, kind=3)
    s.set_rigid_state(m, [0.0, 0.0, 0.0, 0.0, 1e-4, 1e-4])
    last = 1e-4
    for _ in range(6):
        s.step(50)
        om = s.rigid_state(m)[4]
        assert 0.0 < om < last
        last = om
    s, m, xy = dynamic_ring(nx=64, ny=64, walls=walls, R=8.0, n=50, kind=3)
    s.set_rigid_state(m, [1e-3, 0.0, 1e-3, 0.0, 0.0, 0.0])
    for _ in range(8):
        s.step(25)
        u = s.rigid_state(m)[0]
        assert 0.0 < u < 1e-3
    assert u < 0.5e-3


# ---------------------------------------------------------------- free disc in shear
def _disc_in_couette(offset, steps, N=64, R=6.0, nv=40, uw=0.01):
    """A free, neutrally buoyant rigid disc (rho_P = rho) released at rest in
    the planar Couette flow of walls moving at -uw and +uw (shear rate
    2 uw / N).  Returns the rigid state (u, v, u', v', omega, omega'), the
    centroid and the shear rate."""
    s = oracle.OracleSim(N, N, tau=1.0, walls=1, init="couette", wall_velocity=(-uw, uw))
    cx, cy = N / 2, (N - 1) / 2.0 + offset
    m = s.add_membrane(ngon(cx, cy, R, nv), 0.0, 0.0, 0.0, 3, None)
    s.set_density(m, 1.0)
    s.step(steps)
    return s.rigid_state(m), s.markers().mean(axis=0) - np.array([cx, cy]), 2 * uw / N


def test_free_rigid_disc_on_the_centreline_spins_at_half_the_shear_rate():
    """Eqs. linearVelRig / angularVelRig with the stresses of Eqs. hydroForP /
    hydroForNu: a torque-free, force-free disc in simple shear u = g (y - y_c)
    turns with the local fluid rotation, omega = -g / 2 (half the vorticity),
    and, on the centreline, does not translate (the flow is point-symmetric
    about its centre).  Measured 0.994 g / 2 after 3000 steps (the walls are
    5 radii away)."""
    st, drift, g = _disc_in_couette(0.0, 3000)
    assert st[4] / (-g / 2) == pytest.approx(1.0, abs=0.02)
    assert abs(st[0]) < 1e-12 and abs(st[1]) < 1e-12
    assert np.max(np.abs(drift)) < 1e-10


def test_free_rigid_disc_off_the_centreline_moves_with_the_flow():
    """Off the centreline the disc is carried by the flow at its height, in
    the flow's direction, and still turns at about -g / 2; the mirror position
    (the flow's point symmetry) gives the opposite velocity and the same spin.
    The bound on the speed is 10 %: the explicit coupling lets the disc run
    ahead of the undisturbed profile (measured +7.7 % at R = 6 lu, +2.4 % at
    R = 10 lu, after 3000 and 6000 steps)."""
    up, dp, g = _disc_in_couette(8.0, 3000)
    um, dm, _ = _disc_in_couette(-8.0, 3000)
    u_local = g * (8.0 + dp[1])
    assert up[0] > 0 and um[0] < 0
    assert up[0] / u_local == pytest.approx(1.0, abs=0.10)
    assert up[0] == pytest.approx(-um[0], rel=1e-6)
    assert up[4] == pytest.approx(um[4], rel=1e-6)
    assert up[4] / (-g / 2) == pytest.approx(1.0, abs=0.05)
    assert abs(up[1]) < 0.05 * abs(up[0])

"""Pins of the oracle's lattice-Boltzmann part (CPU only).

Each test checks the oracle against something fixed outside it: the paper's
printed constants, moment identities the equilibrium must satisfy, the exact
discrete Poiseuille fixed point, the linear-mode eigenvalue of the LB operator,
the continuum viscosity, and exact conservation laws.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1907_00080_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))

# velocity set evaluated from the printed formula of Eq. GaussHermite
E_PAPER = np.array(
    [[0, 0]]
    + [[round(math.cos((i - 1) * math.pi / 2)), round(math.sin((i - 1) * math.pi / 2))] for i in range(1, 5)]
    + [[round(math.sqrt(2) * math.cos((2 * i - 9) * math.pi / 4)),
        round(math.sqrt(2) * math.sin((2 * i - 9) * math.pi / 4))] for i in range(5, 9)],
    dtype=np.float64,
)
W_PAPER = np.array([GOLD["d2q9_weights"]["w0"]] + [GOLD["d2q9_weights"]["w_axis"]] * 4
                   + [GOLD["d2q9_weights"]["w_diag"]] * 4)


def test_equilibrium_rest_is_paper_weights():
    feq = oracle.equilibrium(1.0, 0.0, 0.0)
    np.testing.assert_allclose(feq, W_PAPER, rtol=0, atol=1e-16)


def test_equilibrium_velocity_order_matches_eq_gausshermite():
    # first-order response in u recovers e_i: feq_i(u) - w_i = w_i e_i.u / c_s^2 + O(u^2)
    d = 1e-7
    cs2 = GOLD["cs2"]["value"]
    ex = (oracle.equilibrium(1.0, d, 0.0) - oracle.equilibrium(1.0, -d, 0.0)) / (2 * d) * cs2 / W_PAPER
    ey = (oracle.equilibrium(1.0, 0.0, d) - oracle.equilibrium(1.0, 0.0, -d)) / (2 * d) * cs2 / W_PAPER
    np.testing.assert_allclose(ex, E_PAPER[:, 0], atol=1e-8)
    np.testing.assert_allclose(ey, E_PAPER[:, 1], atol=1e-8)


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.03, 0.02, -0.01), (0.97, -0.05, 0.04)])
def test_equilibrium_hermite_moments(rho, ux, uy):
    # Gauss-Hermite quadrature conditions: sum feq = rho, sum feq e = rho u,
    # sum feq e e = rho (c_s^2 I + u u)
    feq = oracle.equilibrium(rho, ux, uy)
    e = E_PAPER
    cs2 = GOLD["cs2"]["value"]
    u = np.array([ux, uy])
    assert abs(feq.sum() - rho) < 1e-15
    np.testing.assert_allclose(feq @ e, rho * u, atol=1e-16)
    P = np.einsum("i,ia,ib->ab", feq, e, e)
    np.testing.assert_allclose(P, rho * (cs2 * np.eye(2) + np.outer(u, u)), atol=1e-15)


@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_guo_source_moments(tau):
    # Guo forcing: sum F = 0, sum F e = (1 - 1/2tau) G, sum F e e = (1 - 1/2tau)(u G + G u)
    u = np.array([0.03, -0.02])
    G = np.array([1e-3, 2e-3])
    F = oracle.guo_source(tau, u[0], u[1], G[0], G[1])
    pre = 1 - 1 / (2 * tau)
    e = E_PAPER
    assert abs(F.sum()) < 1e-18
    np.testing.assert_allclose(F @ e, pre * G, atol=1e-18)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", F, e, e),
                               pre * (np.outer(u, G) + np.outer(G, u)), atol=1e-18)


def poiseuille_closed_form(ny, G):
    # exact discrete fixed point for tau = 1, half-way bounce-back, body force G:
    # bulk second difference -G/nu, wall row 3 u(0) - u(1) = 5 G (derived from
    # the streamed moments of feq + Guo source), solved by a parabola + slip G/4
    nu = 1.0 / 6.0
    y = np.arange(ny, dtype=np.float64)
    return G / (2 * nu) * (y + 0.5) * (ny - 0.5 - y) + 0.25 * G


def test_poiseuille_fixed_point_one_stream():
    nx, ny, G = 4, 32, 2.6041666666666667e-05
    s = oracle.OracleSim(nx, ny, 1.0, (G, 0.0), walls=1)
    u = poiseuille_closed_form(ny, G)
    fstar = np.zeros((9, ny, nx))
    for y in range(ny):
        col = oracle.equilibrium(1.0, u[y], 0.0) + oracle.guo_source(1.0, u[y], 0.0, G, 0.0)
        fstar[:, y, :] = col[:, None]
    f = s.stream(fstar)
    rho, ux, uy = s.moments(f)
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-14)
    # relative to the centreline speed (the wall rows carry the smallest u)
    assert np.max(np.abs(ux - u[:, None])) / u.max() < 1e-14
    assert np.max(np.abs(uy)) < 1e-15  # rounding of O(1) population sums


def test_poiseuille_fixed_point_is_stationary_1000_steps():
    nx, ny = 8, 32
    G = inputs.body_force_for(0.02, ny)
    s = oracle.OracleSim(nx, ny, 1.0, (G, 0.0), walls=1, init="poiseuille")
    f0 = s.populations()
    s.step(1000)
    f1 = s.populations()
    assert np.max(np.abs(f1 - f0)) / np.max(np.abs(f0)) < 1e-13
    rho, ux, uy = s.fields()
    u = poiseuille_closed_form(ny, G)
    assert np.max(np.abs(ux - u[:, None])) / u.max() < 1e-13
    np.testing.assert_allclose(rho, 1.0, atol=1e-13)
    # centreline speed of the continuum profile the drive was sized for
    assert abs(u.max() / 0.02 - 1.0) < 1e-2


def test_poiseuille_reached_from_rest():
    nx, ny = 2, 16
    G = 1e-5
    s = oracle.OracleSim(nx, ny, 1.0, (G, 0.0), walls=1, init="rest")
    s.step(12000)
    _, ux, _ = s.fields()
    u = poiseuille_closed_form(ny, G)
    assert np.max(np.abs(ux[:, 0] - u)) / u.max() < 1e-10


def _shear_mode(N, tau):
    """Eigen-decomposition of the linear LB operator M(k) = diag(e^{-i k.e})(I - w(I - Wm)),
    Wm_ij = w_i (1 + e_i.e_j / c_s^2), k = (0, 2 pi / N): return the eigenvalue and
    eigenvector of the shear mode (largest x-momentum content)."""
    k = np.array([0.0, 2 * np.pi / N])
    e, w = E_PAPER, W_PAPER
    Wm = w[:, None] * (1 + 3 * e @ e.T)
    om = 1.0 / tau
    M = np.diag(np.exp(-1j * (e @ k))) @ (np.eye(9) - om * (np.eye(9) - Wm))
    lam, V = np.linalg.eig(M)
    jx = np.abs(e[:, 0] @ V) / np.linalg.norm(V, axis=0)
    m = int(np.argmax(jx))
    return lam[m], V[:, m]


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_shear_wave_decays_with_linear_operator_eigenvalue(tau):
    # the part of the response odd in the amplitude (runs at +amp and -amp) is
    # governed by the linear operator alone: quadratic terms of feq cancel
    N, amp, steps = 32, 1e-5, 60
    lam, v = _shear_mode(N, tau)
    assert abs(lam.imag) < 1e-12
    lam = lam.real
    y = np.arange(N)
    mode = np.real(v[:, None] * np.exp(1j * 2 * np.pi * y / N)[None, :])  # (9, N)
    mode = mode / np.max(np.abs(mode))
    out = []
    for a in (amp, -amp):
        s = oracle.OracleSim(2, N, tau, (0.0, 0.0), walls=0)
        s.set_populations(W_PAPER[:, None, None] + a * mode[:, :, None] * np.ones((1, 1, 2)))
        s.step(steps)
        out.append(s.populations())
    odd = 0.5 * (out[0] - out[1])
    expect = amp * lam ** steps * mode[:, :, None]
    assert np.max(np.abs(odd - expect)) / (amp * lam ** steps) < 1e-9


def test_shear_wave_decay_closed_form_tau1():
    # at tau = 1 the post-collision state is feq, and the x-momentum of a shear
    # wave u_x = A sin(k y) obeys u(y) <- 2/3 u(y) + 1/6 (u(y-1) + u(y+1)), so its
    # amplitude decays by exactly (2 + cos k)/3 per step; against the continuum
    # exp(-nu k^2) the relative error is O(k^4) (ratio 16 per halving of k)
    errs = []
    nu = GOLD["viscosity_tau"]["nu"]
    for N in (16, 32, 64):
        y = np.arange(N)
        k = 2 * np.pi / N
        amps = []
        for a in (1e-6, -1e-6):
            s = oracle.OracleSim(1, N, 1.0, (0.0, 0.0), walls=0)
            u = a * np.sin(k * y)
            f0 = np.stack([oracle.equilibrium(1.0, ui, 0.0) for ui in u], axis=1)[:, :, None]
            s.set_populations(f0)
            s.step(1)
            a0 = np.sum(s.populations()[:, :, 0] * E_PAPER[:, 0:1] * np.sin(k * y)[None, :])
            s.step(50)
            a1 = np.sum(s.populations()[:, :, 0] * E_PAPER[:, 0:1] * np.sin(k * y)[None, :])
            amps.append((a0, a1))
        a0 = 0.5 * (amps[0][0] - amps[1][0])
        a1 = 0.5 * (amps[0][1] - amps[1][1])
        lam = (a1 / a0) ** (1.0 / 50)
        assert abs(lam / ((2 + math.cos(k)) / 3) - 1.0) < 1e-9
        rate = -math.log(lam)
        errs.append(abs(rate / (nu * k * k) - 1.0))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14 < r1 < 18 and 14 < r2 < 18, errs


def test_mass_conserved_with_walls_and_ib_forces():
    nx, ny = 24, 16
    G = 1e-5
    s = oracle.OracleSim(nx, ny, 1.0, (G, 0.0), walls=1, init="poiseuille")
    ring = inputs.circle(10.0, 8.0, 4.0, 24)
    ring[3] += [0.4, 0.2]  # pre-stressed, so forces are non-zero
    m = s.add_membrane(ring, ks=0.05, kb=0.005, ka=0.1)
    m0 = s.mass()
    s.step(1000)
    assert abs(s.mass() - m0) / m0 < 1e-13
    assert m == 0


def test_momentum_budget_periodic_box():
    # P^{n+1} - P^n = N G_body + sum_v F_v   (periodic in x and y)
    nx, ny = 16, 12
    G = np.array([2e-6, -1e-6])
    s = oracle.OracleSim(nx, ny, 1.0, tuple(G), walls=0)
    base = inputs.random_populations(nx, ny, W_PAPER, seed=3, amp=1e-3)
    s.set_populations(base)
    ring = inputs.circle(7.3, 5.9, 3.0, 18)
    ring[2] += [0.3, -0.2]
    ring[9] += [-0.1, 0.25]
    s.add_membrane(ring, ks=0.05, kb=0.01, ka=0.2)
    P0 = np.einsum("iyx,ia->a", s.populations(), E_PAPER)
    s.step(1)
    P1 = np.einsum("iyx,ia->a", s.populations(), E_PAPER)
    F = s.forces().sum(axis=0)
    assert np.max(np.abs(F)) < 1e-15  # internal forces sum to zero
    budget = nx * ny * G + s.forces().sum(axis=0)
    # rounding of ~2000 O(0.1) populations per step bounds the residual near 1e-14
    np.testing.assert_allclose(P1 - P0, budget, rtol=0, atol=1e-13)
    # with a single external point force the budget must see it exactly
    gx, gy = s.force_field()
    np.testing.assert_allclose([gx.sum(), gy.sum()], budget, rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- moving walls
def couette_profile(ny, u_bot, u_top):
    """planar Couette flow between walls at y = -1/2 and y = NY - 1/2"""
    y = np.arange(ny, dtype=np.float64)
    return u_bot + (u_top - u_bot) * (y + 0.5) / ny


def test_couette_state_is_the_tau1_fixed_point():
    """tau = 1: the Couette initial state (post-collision feq of the linear
    profile) is reproduced by every step (moving-wall bounce-back at both
    walls), with rho = 1 and u = the closed-form profile."""
    import oracle
    nx, ny = 12, 8
    s = oracle.OracleSim(nx, ny, tau=1.0, walls=1, init="couette", wall_velocity=(-0.004, 0.01))
    f0 = s.populations()
    s.step(200)
    np.testing.assert_allclose(s.populations(), f0, rtol=0, atol=1e-15)
    rho, ux, uy = s.fields()
    np.testing.assert_allclose(rho, 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(ux, np.broadcast_to(couette_profile(ny, -0.004, 0.01)[:, None], (ny, nx)),
                               rtol=0, atol=1e-15)
    np.testing.assert_allclose(uy, 0.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.8, 1.3])
def test_couette_from_rest_reaches_the_linear_profile(tau):
    """From rest, the flow driven by the moving walls relaxes to the linear
    profile with the walls exactly half-way (exact for a linear profile at any
    tau with this bounce-back)."""
    import oracle
    nx, ny = 4, 6
    s = oracle.OracleSim(nx, ny, tau=tau, walls=1, init="rest", wall_velocity=(-0.005, 0.01))
    m0 = s.mass()
    s.step(20000)
    rho, ux, uy = s.fields()
    np.testing.assert_allclose(ux, np.broadcast_to(couette_profile(ny, -0.005, 0.01)[:, None], (ny, nx)),
                               rtol=0, atol=1e-13)
    np.testing.assert_allclose(uy, 0.0, rtol=0, atol=1e-14)
    assert abs(s.mass() - m0) <= 1e-12 * m0


def test_walls_moving_together_carry_the_fluid_along():
    """Both walls at the same velocity U: the fluid reaches the uniform flow U
    (a Galilean check of the momentum term's sign and size)."""
    import oracle
    s = oracle.OracleSim(4, 5, tau=1.0, walls=1, init="rest", wall_velocity=(0.02, 0.02))
    s.step(5000)
    rho, ux, uy = s.fields()
    np.testing.assert_allclose(ux, 0.02, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- Zou-He walls
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.3])
def test_zou_he_couette_from_rest_is_the_linear_profile(tau):
    """Sec. 2.1 (Zou and He's known-velocity walls on the wall rows y = 0 and
    y = NY - 1): planar Couette flow between walls moving at u_b and u_t,
    started from rest, reaches u(y) = u_b + (u_t - u_b) y / (NY - 1) with
    rho = 1 at any tau (the linear profile is the scheme's exact steady
    state)."""
    nx, ny, ub, ut = 8, 17, -0.01, 0.02
    s = oracle.OracleSim(nx, ny, tau=tau, walls=2, init="rest", wall_velocity=(ub, ut))
    s.step(20000)
    rho, ux, uy = s.fields()
    u = ub + (ut - ub) * np.arange(ny) / (ny - 1)
    assert np.max(np.abs(ux - u[:, None])) < 1e-13
    assert np.max(np.abs(uy)) < 1e-14
    assert np.max(np.abs(rho - 1.0)) < 1e-11


@pytest.mark.parametrize("tau", [1.0, 1.3])
def test_zou_he_poiseuille_from_rest_is_the_parabola(tau):
    """A uniform body force G between resting Zou-He walls (the channel of
    height H = NY - 1 between the wall rows) reaches the plane Poiseuille
    profile u(y) = G y (H - y) / (2 nu), zero on the wall rows: the known
    velocity includes the Guo half-force, so the wall rows carry no slip."""
    nx, ny, G = 4, 17, 1e-6
    nu = (tau - 0.5) / 3.0
    s = oracle.OracleSim(nx, ny, tau=tau, body_force=(G, 0.0), walls=2, init="rest")
    s.step(30000)
    _, ux, _ = s.fields()
    y = np.arange(ny)
    u = G / (2 * nu) * y * (ny - 1 - y)
    assert np.max(np.abs(ux - u[:, None])) / u.max() < 1e-9
    assert np.max(np.abs(ux[[0, -1]])) < 1e-15


def test_zou_he_rows_take_the_wall_velocity_every_step():
    """From a random state with a force field, every collision on the wall rows
    sees exactly the wall velocity (the condition's definition), while mass
    elsewhere is untouched by it."""
    nx, ny = 12, 9
    s = oracle.OracleSim(nx, ny, tau=0.9, body_force=(3e-5, -2e-5), walls=2, init="rest",
                         wall_velocity=(0.004, -0.007))
    rng = np.random.default_rng(3)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    s.set_populations(w[:, None, None] * (1 + 0.05 * rng.uniform(-1, 1, (9, ny, nx))))
    for _ in range(3):
        s.step(1)
        _, ux, uy = s.fields()
        assert np.max(np.abs(ux[0] - 0.004)) < 1e-15 and np.max(np.abs(ux[-1] + 0.007)) < 1e-15
        assert np.max(np.abs(uy[[0, -1]])) < 1e-16

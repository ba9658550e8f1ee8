"""Pins of the oracle's membrane mechanics (CPU only): zero force at the rest
shape, force balance of each contribution, regular-polygon geometry, the
turning-angle theorem, gradient consistency of the stretching and area terms,
and area restoration under the penalty."""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00080_gb300 import inputs


def shapes():
    return {
        "circle32": inputs.circle(5.0, 3.0, 4.0, 32),
        "rbc200": inputs.rbc_contour(64.0, 200) + np.array([100.0, 40.0]),
        "carrier50": inputs.circle(-3.0, 7.0, 8.0, 50),
    }


@pytest.mark.parametrize("name", ["circle32", "rbc200", "carrier50"])
def test_rest_shape_has_exactly_zero_force(name):
    xy = shapes()[name]
    l0, th0, A0 = oracle.ring_rest(xy)
    F = oracle.ring_forces(xy, l0, th0, A0, ks=0.05, kb=0.005, ka=0.1)
    assert np.all(F == 0.0)


@pytest.mark.parametrize("which", [1, 2, 4, 7])
def test_forces_sum_to_zero(which):
    rng = np.random.Generator(np.random.PCG64(which))
    for xy in shapes().values():
        l0, th0, A0 = oracle.ring_rest(xy)
        pert = xy + rng.normal(scale=0.2, size=xy.shape)
        F = oracle.ring_forces(pert, l0, th0, A0, ks=0.05, kb=0.005, ka=0.1, which=which)
        scale = np.max(np.abs(F))
        assert scale > 0
        assert np.max(np.abs(F.sum(axis=0))) < 1e-13 * scale * len(xy)


@pytest.mark.parametrize("n", [3, 4, 7, 32, 50, 200])
def test_regular_polygon_area_and_angle(n):
    R = 2.5
    xy = inputs.circle(1.0, -2.0, R, n)
    l0, th0, A0 = oracle.ring_rest(xy)
    assert abs(A0 - 0.5 * n * R * R * math.sin(2 * math.pi / n)) < 1e-13 * A0
    np.testing.assert_allclose(th0, 2 * math.pi / n, rtol=1e-12)
    np.testing.assert_allclose(l0, 2 * R * math.sin(math.pi / n), rtol=1e-13)


def test_turning_angles_sum_to_two_pi():
    # any simple CCW polygon turns through exactly 2 pi
    for xy in shapes().values():
        _, th0, _ = oracle.ring_rest(xy)
        assert abs(th0.sum() - 2 * math.pi) < 1e-12


def _energy_stretch(xy, l0, ks):
    d = xy - np.roll(xy, -1, axis=0)
    return 0.5 * ks * np.sum((np.hypot(d[:, 0], d[:, 1]) - l0) ** 2)


def test_stretch_force_is_minus_gradient_of_potential():
    # Eq. strainPot: V = 1/2 k_s (l - l0)^2 per element; Eq. strainFor must be -grad V
    rng = np.random.Generator(np.random.PCG64(3))
    xy0 = inputs.circle(0.0, 0.0, 3.0, 12)
    l0, th0, A0 = oracle.ring_rest(xy0)
    xy = xy0 + rng.normal(scale=0.3, size=xy0.shape)
    F = oracle.ring_forces(xy, l0, th0, A0, ks=0.07, kb=0.0, ka=0.0, which=1)
    h = 1e-6
    for v in range(len(xy)):
        for c in range(2):
            p, m = xy.copy(), xy.copy()
            p[v, c] += h
            m[v, c] -= h
            g = (_energy_stretch(p, l0, 0.07) - _energy_stretch(m, l0, 0.07)) / (2 * h)
            assert abs(F[v, c] + g) < 1e-8


def test_area_force_is_along_area_gradient():
    # Eq. areaFor summed to vertices equals k_a p_ref (1 - A/A0) dA/dx_v
    rng = np.random.Generator(np.random.PCG64(4))
    xy0 = inputs.circle(0.0, 0.0, 3.0, 16)
    l0, th0, A0 = oracle.ring_rest(xy0)
    xy = 0.97 * xy0 + rng.normal(scale=0.05, size=xy0.shape)
    ka, pref = 0.3, 1.0 / 3.0
    F = oracle.ring_forces(xy, l0, th0, A0, ks=0.0, kb=0.0, ka=ka, p_ref=pref, which=4)
    A = oracle.ring_area(xy)
    h = 1e-6
    for v in range(len(xy)):
        for c in range(2):
            p, m = xy.copy(), xy.copy()
            p[v, c] += h
            m[v, c] -= h
            dA = (oracle.ring_area(p) - oracle.ring_area(m)) / (2 * h)
            assert abs(F[v, c] - ka * pref * (1 - A / A0) * dA) < 1e-9
    # compressed ring -> forces point outward
    c = xy.mean(axis=0)
    assert np.sum((F * (xy - c)).sum(axis=1) > 0) == len(xy)


def test_bending_restores_a_bump():
    xy0 = inputs.circle(0.0, 0.0, 4.0, 24)
    l0, th0, A0 = oracle.ring_rest(xy0)
    xy = xy0.copy()
    xy[5] *= 1.05  # push one vertex outward
    F = oracle.ring_forces(xy, l0, th0, A0, ks=0.0, kb=0.01, ka=0.0, which=2)
    out = xy[5] / np.linalg.norm(xy[5])
    assert F[5] @ out < 0          # bumped vertex pulled back in
    assert F[4] @ out > 0 and F[6] @ out > 0  # neighbours pushed out
    # split of the neighbour forces follows the element lengths
    l_left = np.linalg.norm(xy[5] - xy[4])
    l_right = np.linalg.norm(xy[6] - xy[5])
    ratio = np.linalg.norm(F[4]) / np.linalg.norm(F[6])
    assert abs(ratio - l_left / l_right) < 1e-12
    # rigid motions and uniform scaling leave angles (hence bending) unchanged
    c, s_ = math.cos(0.7), math.sin(0.7)
    moved = 1.3 * xy0 @ np.array([[c, s_], [-s_, c]]) + np.array([10.0, -4.0])
    Fm = oracle.ring_forces(moved, l0, th0, A0, ks=0.0, kb=0.01, ka=0.0, which=2)
    assert np.max(np.abs(Fm)) < 1e-15


def test_area_penalty_restores_area():
    xy0 = inputs.rbc_contour(20.0, 80)
    l0, th0, A0 = oracle.ring_rest(xy0)
    xy = xy0 * math.sqrt(0.95)  # 5 % area loss
    prev = abs(oracle.ring_area(xy) / A0 - 1)
    for it in range(400):
        F = oracle.ring_forces(xy, l0, th0, A0, ks=0.0, kb=0.0, ka=1.0, which=4)
        xy = xy + 0.5 * F
        err = abs(oracle.ring_area(xy) / A0 - 1)
        assert err <= prev + 1e-15
        prev = err
    assert prev < 1e-8


def test_rbc_contour_matches_eq_rbcshape():
    # every resampled vertex lies on the printed parametric curve
    alpha = 64.0
    xy = inputs.rbc_contour(alpha, 200)
    q = np.linspace(-0.5 * np.pi, 1.5 * np.pi, 400001)
    x = alpha * np.sin(q)
    s = np.sin(q) ** 2
    y = 0.5 * alpha * (0.207 + 2.003 * s - 1.123 * s * s) * np.cos(q)
    curve = np.stack([x, y], axis=1)
    curve -= curve.mean(axis=0) * 0  # raw curve is symmetric about the origin
    for p in xy[::7]:
        assert np.min(np.hypot(curve[:, 0] - p[0], curve[:, 1] - p[1])) < 2e-3
    assert inputs._signed_area(xy) > 0


def test_bending_regular_ngon_against_flat_rest_angles():
    """Eq. bendFor on a regular N-gon with rest angles 0 (a straight rest
    shape): every vertex turns by theta = 2 pi / N.  Vertex v gets
    -k_b theta n_v from its own term and k_b theta / 2 n_{v -+ 1} from each
    neighbour's (equal elements), and n_{v -+ 1} is n_v turned by -+ 2 pi / N,
    so F_v = k_b theta (cos(2 pi / N) - 1) n_v, whatever the radius."""
    kb = 0.013
    for N in (7, 12, 50):
        for R in (3.0, 11.5):
            xy = inputs.circle(2.0, -1.0, R, N)
            l0, _, A0 = oracle.ring_rest(xy)
            F = oracle.ring_forces(xy, l0, np.zeros(N), A0, ks=0.0, kb=kb, ka=0.0, which=2)
            theta = 2 * math.pi / N
            # outward vertex normal of a regular polygon: the radial direction
            n = (xy - np.array([2.0, -1.0])) / R
            expect = kb * theta * (math.cos(theta) - 1.0) * n
            np.testing.assert_allclose(F, expect, rtol=0, atol=1e-14 * kb)


def test_bending_split_follows_unequal_element_lengths():
    """One bent vertex between elements of unequal length (l_L = 1, l_R = 3),
    every other vertex at its rest angle: the vertex gets -k_b (theta -
    theta_0) n_v, its left neighbour l_L / (l_L + l_R) of the opposite and the
    right one l_R / (l_L + l_R).  n_v is the unit vector normal to the sum of
    the two unit edge vectors, pointing out of the ring."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0 + 3.0 * math.cos(0.4), 3.0 * math.sin(0.4)],
                   [-0.5, 3.5]])
    n = len(xy)
    l0, th0, A0 = oracle.ring_rest(xy)
    v, dth, kb = 1, 0.05, 0.02
    th0 = th0.copy()
    th0[v] -= dth  # only vertex 1 is away from its rest angle, by dth
    F = oracle.ring_forces(xy, l0, th0, A0, ks=0.0, kb=kb, ka=0.0, which=2)
    eL = xy[1] - xy[0]
    eR = xy[2] - xy[1]
    lL, lR = np.linalg.norm(eL), np.linalg.norm(eR)
    assert (lL, lR) == pytest.approx((1.0, 3.0), rel=1e-15)
    t = eL / lL + eR / lR
    nv = np.array([t[1], -t[0]]) / np.linalg.norm(t)
    assert nv @ (xy[1] - xy.mean(axis=0)) > 0  # outward
    np.testing.assert_allclose(F[1], -kb * dth * nv, rtol=0, atol=1e-16)
    np.testing.assert_allclose(F[0], kb * dth * lL / (lL + lR) * nv, rtol=0, atol=1e-16)
    np.testing.assert_allclose(F[2], kb * dth * lR / (lL + lR) * nv, rtol=0, atol=1e-16)
    assert np.all(F[3] == 0.0)
    assert np.linalg.norm(F[2]) / np.linalg.norm(F[0]) == pytest.approx(3.0, rel=1e-13)

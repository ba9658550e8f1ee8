"""Pins of the oracle's immersed-boundary exchange (CPU only): Roma kernel
moments, MLS consistency near walls, interior equivalence to the Roma weights,
and exact adjointness of interpolation and spreading by brute-force sums."""
import numpy as np
import pytest

import oracle


def test_roma_kernel_discrete_moments():
    # Roma, Peskin & Berger: sum_k phi(r-k) = 1, sum_k (r-k) phi(r-k) = 0,
    # sum_k phi(r-k)^2 = 1/2 for every shift r
    rng = np.random.Generator(np.random.PCG64(11))
    for r in np.concatenate([rng.uniform(-0.5, 0.5, 200), [0.0, 0.5, -0.5, 0.25]]):
        ks = np.arange(-3, 4)
        ph = np.array([oracle.roma(r - k) for k in ks])
        assert abs(ph.sum() - 1.0) < 1e-15
        assert abs(((r - ks) * ph).sum()) < 1e-15
        assert abs((ph ** 2).sum() - 0.5) < 1e-15
    assert oracle.roma(1.5) == 0.0 and oracle.roma(-1.6) == 0.0
    assert abs(oracle.roma(0.0) - 2.0 / 3.0) < 1e-16


def test_interior_weights_are_roma_products_and_consistent():
    s = oracle.OracleSim(16, 12, walls=1)
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(50):
        x, y = rng.uniform(0, 16), rng.uniform(2.0, 9.0)
        w, idx = s.ib_weights(x, y)
        assert np.all(idx >= 0)
        i0, j0 = np.floor(x + 0.5), np.floor(y + 0.5)
        k = 0
        for b in (-1, 0, 1):
            for a in (-1, 0, 1):
                assert w[k] == oracle.roma(i0 + a - x) * oracle.roma(j0 + b - y)
                assert idx[k] == int((j0 + b) % 12) * 16 + int((i0 + a) % 16)
                k += 1
        assert abs(w.sum() - 1.0) < 1e-15


@pytest.mark.parametrize("y", [-0.45, -0.2, 0.0, 0.3, 0.49, 0.51, 10.7, 11.2, 11.45])
def test_mls_near_wall_reproduces_linear_fields(y):
    # walls at y = -1/2 and 11.5; out-of-fluid nodes dropped, MLS with a linear
    # basis must interpolate any linear field exactly
    nx, ny = 16, 12
    s = oracle.OracleSim(nx, ny, walls=1)
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    for x in (3.3, 7.5, 0.2, 15.8):
        for a, b, c in [(1.0, 0.0, 0.0), (0.3, 0.7, -0.2), (-0.1, 0.0, 1.3)]:
            # a linear field seen through periodic x stays linear only away from
            # the seam: use the unwrapped node coordinate of each stencil node
            w, idx = s.ib_weights(x, y)
            i0, j0 = np.floor(x + 0.5), np.floor(y + 0.5)
            val = 0.0
            k = 0
            for bb in (-1, 0, 1):
                for aa in (-1, 0, 1):
                    if idx[k] >= 0:
                        val += w[k] * (a + b * (i0 + aa) + c * (j0 + bb))
                    k += 1
            assert abs(val - (a + b * x + c * y)) < 1e-13
        w, idx = s.ib_weights(x, y)
        assert np.all(idx[w != 0] >= 0)


def test_interp_spread_adjoint_brute_force():
    # <u, S F> = <I u, F> summed explicitly over every node and marker
    nx, ny = 8, 6
    s = oracle.OracleSim(nx, ny, walls=1)
    rng = np.random.Generator(np.random.PCG64(7))
    pts = np.stack([rng.uniform(-3, 11, 14), rng.uniform(-0.45, 5.45, 14)], axis=1)
    pts[0] = [0.1, -0.4]   # near the lower wall and the periodic seam
    pts[1] = [7.9, 5.4]    # near the upper wall
    ux, uy = rng.normal(size=(ny, nx)), rng.normal(size=(ny, nx))
    F = rng.normal(size=(len(pts), 2))
    U = s.interp(ux, uy, pts)
    gx, gy = s.spread(pts, F)
    lhs = 0.0
    for j in range(ny):
        for i in range(nx):
            lhs += ux[j, i] * gx[j, i] + uy[j, i] * gy[j, i]
    rhs = 0.0
    for v in range(len(pts)):
        rhs += U[v, 0] * F[v, 0] + U[v, 1] * F[v, 1]
    assert abs(lhs - rhs) < 1e-14 * max(1.0, abs(lhs))


def test_spread_conserves_total_force():
    nx, ny = 10, 8
    s = oracle.OracleSim(nx, ny, walls=1)
    rng = np.random.Generator(np.random.PCG64(9))
    pts = np.stack([rng.uniform(0, 10, 20), rng.uniform(-0.45, 7.45, 20)], axis=1)
    F = rng.normal(size=(20, 2))
    gx, gy = s.spread(pts, F)
    np.testing.assert_allclose([gx.sum(), gy.sum()], F.sum(axis=0), atol=1e-14)


def test_periodic_y_stencil_wraps():
    s = oracle.OracleSim(8, 6, walls=0)
    w, idx = s.ib_weights(0.2, 5.7)
    assert np.all(idx >= 0)
    assert abs(w.sum() - 1.0) < 1e-15
    rows = sorted(set(int(i) // 8 for i in idx))
    assert rows == [0, 1, 5]  # nearest row 6 wraps to 0: rows 5, 6->0, 7->1

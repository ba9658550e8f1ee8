"""Pins of the oracle's adhesion model and random stream (CPU only): Philox
against numpy's independent Philox4x64-10, uniformity of the draws, the bond
spring as the gradient of its energy, bond-formation and rupture statistics on
a fixed geometry, and the lowest-ligand-wins rule."""
import math

import numpy as np
import pytest

import oracle
from paper_1907_00080_gb300 import inputs


def test_philox_matches_numpy_bit_generator():
    # numpy's Philox (4x64, 10 rounds) increments its 256-bit counter before
    # each block, so state counter c yields Philox(c + 1, key)
    rng = np.random.Generator(np.random.PCG64(1))
    for _ in range(200):
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        ctr[0] = ctr[0] | np.uint64(1)  # avoid the carry case in the +1
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        bg = np.random.Philox(counter=ctr - np.array([1, 0, 0, 0], dtype=np.uint64), key=key)
        ref = bg.random_raw(4)
        out = oracle.philox4x64_10(ctr, key)
        assert np.array_equal(out, ref)


def test_uniform_draws_are_uniform():
    n = 40000
    u = np.array([oracle.uniform(0, 0, s, l, 3, 0) for s in range(200) for l in range(n // 200)])
    assert u.min() >= 0.0 and u.max() < 1.0
    counts, _ = np.histogram(u, bins=50, range=(0, 1))
    exp = n / 50
    chi2 = np.sum((counts - exp) ** 2 / exp)
    assert chi2 < 100  # 49 dof: P(chi2 > 100) < 3e-5
    # tags and receptors give independent streams
    a = np.array([oracle.uniform(0, 0, 5, l, 3, 0) for l in range(2000)])
    b = np.array([oracle.uniform(0, 0, 5, l, 3, 1) for l in range(2000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.1


def _strip(K, spacing=2.0, y_lig=0.5, height=5.0):
    # a long thin ring whose bottom elements sit just above the lower wall:
    # bottom vertices at x = 0, spacing, ..., top edge returning at y = height
    bottom = [[k * spacing, y_lig] for k in range(K + 1)]
    top = [[k * spacing, height] for k in range(K, -1, -1)]
    return np.array(bottom + top, dtype=float)


def test_bond_spring_is_minus_gradient_of_energy():
    # Eq. adhFor: spring of stiffness sigma and rest length y_eq between the
    # ligand point (element centroid) and the receptor, split half/half
    nx, ny = 64, 16
    s = oracle.OracleSim(nx, ny, walls=1)
    xy = _strip(3)
    s.add_membrane(xy, ks=0.0, kb=0.0, ka=0.0, ligand_elems=[1])
    rec = np.array([[3.4, -0.5]])
    sigma, y_eq = 0.2, 0.75
    s.set_receptors(rec, sigma=sigma, y_eq=y_eq)
    s.set_bond(0, 0)
    s.compute_forces()
    F = s.forces()

    def energy(p):
        c = 0.5 * (p[1] + p[2])
        d = np.hypot(*(rec[0] - c))
        return 0.5 * sigma * (d - y_eq) ** 2

    h = 1e-6
    for v in range(len(xy)):
        for c in range(2):
            p, m = xy.copy(), xy.copy()
            p[v, c] += h
            m[v, c] -= h
            g = (energy(p) - energy(m)) / (2 * h)
            assert abs(F[v, c] + g) < 1e-9
    assert np.all(F[[0, 3, 4, 5, 6, 7], :] == 0.0)
    np.testing.assert_array_equal(F[1], F[2])


def test_bond_spring_uses_periodic_minimum_image():
    nx, ny = 32, 8
    s = oracle.OracleSim(nx, ny, walls=1)
    xy = _strip(2, spacing=1.0)
    s.add_membrane(xy, ks=0.0, kb=0.0, ka=0.0, ligand_elems=[0])
    s.set_receptors(np.array([[31.5, -0.5]]), sigma=0.1, y_eq=0.75)  # across the seam
    s.set_bond(0, 0)
    s.compute_forces()
    F = s.forces()
    assert F[0, 0] < 0 and F[0, 1] < 0  # pulled toward x = -0.5 (the image of 31.5)


def test_formation_statistics_fixed_geometry():
    # no rupture (k_r0 = 0): each ligand binds at its own receptor with
    # probability P_f per step, so after n steps the bonded fraction is
    # 1 - (1 - P_f)^n (binomial, 4 sigma)
    K, nsteps = 1500, 12
    nx, ny = 2 * K + 8, 12
    s = oracle.OracleSim(nx, ny, walls=1)
    s.add_membrane(_strip(K), ks=0.0, kb=0.0, ka=0.0, ligand_elems=np.arange(K))
    rec = np.array([[2 * k + 1.0, -0.5] for k in range(K)])
    s.set_receptors(rec, kf_dt=0.05, kr0_dt=0.0, seed=123, d_break=100.0)
    d = 1.0
    pf = s.p_form(d)
    for n in range(nsteps):
        s.bonds_update(n)
    b = s.bonds()
    frac = np.mean(b >= 0)
    p = 1 - (1 - pf) ** nsteps
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / K)
    assert np.all(b[b >= 0] == np.arange(K)[b >= 0])  # each binds its own receptor


def test_rupture_statistics_fixed_geometry():
    K, nsteps = 1500, 10
    nx, ny = 2 * K + 8, 12
    s = oracle.OracleSim(nx, ny, walls=1)
    s.add_membrane(_strip(K), ks=0.0, kb=0.0, ka=0.0, ligand_elems=np.arange(K))
    rec = np.array([[2 * k + 1.0, -0.5] for k in range(K)])
    s.set_receptors(rec, kf_dt=0.0, kr0_dt=0.02, seed=7, d_break=100.0)
    for k in range(K):
        s.set_bond(k, k)
    pr = s.p_rupture(1.0)
    assert 0.02 < pr < 0.05
    for n in range(nsteps):
        s.bonds_update(n)
    frac = np.mean(s.bonds() >= 0)
    p = (1 - pr) ** nsteps
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / K)


def test_bond_breaks_beyond_break_length_and_cutoff_blocks_formation():
    nx, ny = 32, 12
    s = oracle.OracleSim(nx, ny, walls=1)
    xy = _strip(2, y_lig=4.0, height=8.0)
    s.add_membrane(xy, ks=0.0, kb=0.0, ka=0.0, ligand_elems=[0, 1])
    s.set_receptors(np.array([[1.0, -0.5], [3.0, -0.5]]), kf_dt=50.0, kr0_dt=0.0, d_break=3.0)
    s.set_bond(0, 0)
    s.bonds_update(0)
    # distance 4.5 >= d_break: ruptured; 4.5 >= d_cut: no formation
    assert np.all(s.bonds() == -1)


def test_lowest_ligand_wins_a_contested_receptor():
    nx, ny = 32, 12
    s = oracle.OracleSim(nx, ny, walls=1)
    xy = _strip(2, spacing=1.0)  # ligand points at x = 0.5 and 1.5, y = 0.5
    s.add_membrane(xy, ks=0.0, kb=0.0, ka=0.0, ligand_elems=[0, 1])
    s.set_receptors(np.array([[1.0, -0.5]]), kf_dt=50.0, kr0_dt=0.0)
    assert s.p_form(math.hypot(0.5, 1.0)) > 1 - 1e-12
    s.bonds_update(0)
    assert list(s.bonds()) == [0, -1]


def test_just_ruptured_receptor_is_not_rebound_in_the_same_step():
    nx, ny = 32, 12
    s = oracle.OracleSim(nx, ny, walls=1)
    xy = _strip(2, spacing=1.0)
    s.add_membrane(xy, ks=0.0, kb=0.0, ka=0.0, ligand_elems=[0, 1])
    s.set_receptors(np.array([[1.0, -0.5]]), kf_dt=50.0, kr0_dt=50.0)
    s.set_bond(1, 0)
    s.bonds_update(0)
    assert list(s.bonds()) == [-1, -1]
    s.bonds_update(1)
    assert (s.bonds() >= 0).sum() <= 1


def test_physical_cutoff_where_the_mesh_resolves_it():
    """The paper's y_cr = 25 nm (Sec. 2.2) in lattice units: 1.67 lu at
    dx = 15 nm (fine mesh), refused at dx = 62.5 nm (0.4 lu, below the IB
    resolution); y_eq = y_cr / 2."""
    from paper_1907_00080_gb300 import inputs
    b = inputs.physical_bonds(15.0)
    assert b["d_cut"] == pytest.approx(25.0 / 15.0, rel=1e-15)
    assert b["y_eq"] == pytest.approx(12.5 / 15.0, rel=1e-15)
    assert b["d_break"] == pytest.approx(50.0 / 15.0, rel=1e-15)
    with pytest.raises(ValueError):
        inputs.physical_bonds(62.5)
    wl = inputs.fine_capillary_2000x667("f32", bonds="physical")
    assert wl.bonds["d_cut"] == pytest.approx(25.0 / (10000.0 / 667), rel=1e-12)  # dx = 10 um / 667


def _kinetics(y_eq=0.75, kf_dt=0.01, kr0_dt=0.004, beta_f=0.5, beta_r=2.0):
    s = oracle.OracleSim(16, 8, walls=1)
    s.add_membrane(_strip(2), ks=0.0, kb=0.0, ka=0.0, ligand_elems=[0])
    s.set_receptors(np.array([[1.0, -0.5]]), y_eq=y_eq, d_cut=2 * y_eq, kf_dt=kf_dt, kr0_dt=kr0_dt,
                    beta_f=beta_f, beta_r=beta_r)
    return s


def test_bond_probabilities_at_the_equilibrium_length():
    """Sec. 2.2 (wall-particle interaction): at the equilibrium bond length the
    spring is unloaded, so formation and rupture run at their unloaded rates:
    per step P_f = 1 - exp(-k_f dt) and P_r = 1 - exp(-k_r0 dt) (a Poisson event
    at that rate within one step)."""
    for y_eq, kf, kr in ((0.75, 0.01, 0.01 / 8.5e3), (0.8333, 0.05, 0.01), (1.3, 0.3, 0.2)):
        s = _kinetics(y_eq=y_eq, kf_dt=kf, kr0_dt=kr)
        assert s.p_form(y_eq) == pytest.approx(-math.expm1(-kf), rel=1e-14)
        assert s.p_rupture(y_eq) == pytest.approx(-math.expm1(-kr), rel=1e-14)
    # the paper's only number: k_f / k_r0 = 8.5e3 gives that ratio of the
    # unloaded per-step probabilities in the small-rate limit
    s = _kinetics(kf_dt=1e-6, kr0_dt=1e-6 / 8.5e3)
    assert s.p_form(0.75) / s.p_rupture(0.75) == pytest.approx(8.5e3, rel=1e-5)


def test_bond_probabilities_symmetric_and_monotone_in_the_stretch():
    """Formation slows and rupture speeds up as the bond is stretched or
    compressed away from y_eq, symmetrically in d - y_eq."""
    y_eq = 0.75
    s = _kinetics(y_eq=y_eq, kf_dt=0.05, kr0_dt=0.01)
    dev = np.linspace(0.0, 0.7, 36)
    pf_plus = np.array([s.p_form(y_eq + e) for e in dev])
    pf_minus = np.array([s.p_form(y_eq - e) for e in dev])
    pr_plus = np.array([s.p_rupture(y_eq + e) for e in dev])
    pr_minus = np.array([s.p_rupture(y_eq - e) for e in dev])
    np.testing.assert_allclose(pf_plus, pf_minus, rtol=1e-13)
    np.testing.assert_allclose(pr_plus, pr_minus, rtol=1e-13)
    assert np.all(np.diff(pf_plus) < 0) and np.all(np.diff(pr_plus) > 0)
    assert np.all((pf_plus > 0) & (pf_plus < 1) & (pr_plus > 0) & (pr_plus < 1))


def test_bond_probabilities_scale_with_the_relative_stretch():
    """The rates depend on the stretch only through z = (d - y_eq) / y_eq with
    a Gaussian factor: -log(1 - P) = k dt exp(-+beta z^2).  Fitting a
    parabola in z to log(-log(1 - P)) recovers log(k dt) as its constant and
    -beta_f (formation) or +beta_r (rupture) as its curvature, for two
    different y_eq; the two lengths give the same P at the same z."""
    kf, kr, bf, br = 0.05, 0.01, 0.5, 2.0
    z = np.linspace(-0.9, 0.9, 41)
    curves = []
    for y_eq in (0.75, 1.9):
        s = _kinetics(y_eq=y_eq, kf_dt=kf, kr0_dt=kr, beta_f=bf, beta_r=br)
        pf = np.array([s.p_form(y_eq * (1 + q)) for q in z])
        pr = np.array([s.p_rupture(y_eq * (1 + q)) for q in z])
        cf = np.polyfit(z, np.log(-np.log1p(-pf)), 2)
        cr = np.polyfit(z, np.log(-np.log1p(-pr)), 2)
        assert cf[0] == pytest.approx(-bf, rel=1e-9) and abs(cf[1]) < 1e-9
        assert cf[2] == pytest.approx(math.log(kf), rel=1e-9)
        assert cr[0] == pytest.approx(br, rel=1e-9) and abs(cr[1]) < 1e-9
        assert cr[2] == pytest.approx(math.log(kr), rel=1e-9)
        curves.append((pf, pr))
    np.testing.assert_allclose(curves[0][0], curves[1][0], rtol=1e-12)
    np.testing.assert_allclose(curves[0][1], curves[1][1], rtol=1e-12)

"""GPU tests of the reverse-mode adjoint of the FP64 time step (lbib_adjoint_*).

The adjoint is the transpose of the forward-mode tangent along the same bond
history, so for any tangent direction v and any adjoint seed w
    <w, J v> = <J^T w, v>
must hold to FP64 rounding over a whole trajectory (the dot-product test).
Further checks: gradients of the carrier observables against the tangent
Jacobian and against central differences of the FP64 solver, independence from
the checkpoint interval (ragged last segments), the adjoint of the populations
against central differences, the state the context is left in, the autograd
backward, and the error paths."""
import numpy as np
import pytest

from paper_1907_00080_gb300 import inputs, sensitivity

pytestmark = pytest.mark.gpu

STEPS = 200


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


def tangent_run(wl, steps, dks, dkb, dsig, dxy):
    L = lb()
    sim = L.Simulation(wl, precision="f64")
    t = L.lbib_tangent_create(sim.ctx)
    try:
        L.lbib_tangent_seed(sim.ctx, t, dks, dkb, dsig, dxy, None)
        L.lbib_tangent_step(sim.ctx, t, steps)
        return L.lbib_tangent_read(sim.ctx, t, wl.n_vertices)
    finally:
        L.lbib_tangent_destroy(t)
        sim.close()


def adjoint_run(wl, steps, K, xb, xpb, f_bar=None, want_f=False):
    L = lb()
    sim = L.Simulation(wl, precision="f64")
    adj = L.lbib_adjoint_create(sim.ctx, K)
    try:
        L.lbib_adjoint_record(sim.ctx, adj, steps)
        L.lbib_adjoint_seed(sim.ctx, adj, xb, xpb, f_bar)
        L.lbib_adjoint_reverse(sim.ctx, adj)
        n_nodes = wl.nx * wl.ny if want_f else None
        return L.lbib_adjoint_read(sim.ctx, adj, wl.n_vertices, len(wl.membranes), n_nodes)
    finally:
        L.lbib_adjoint_destroy(adj)
        sim.close()


def dot_identity(wl, steps, K, seed):
    """Both sides of <w, J v> = <J^T w, v> for random v and w, and the sum of
    the absolute values of the terms (the scale of the rounding)."""
    rng = np.random.default_rng(seed)
    nm, nv = len(wl.membranes), wl.n_vertices
    dks, dkb = rng.standard_normal(nm), rng.standard_normal(nm)
    dsig = float(rng.standard_normal())
    dxy = rng.standard_normal((nv, 2))
    xb, xpb = rng.standard_normal((nv, 2)), rng.standard_normal((nv, 2))
    dX, dXp = tangent_run(wl, steps, dks, dkb, dsig, dxy)
    r = adjoint_run(wl, steps, K, xb, xpb)
    lhs_terms = np.concatenate([(xb * dX).ravel(), (xpb * dXp).ravel()])
    # the tangent seeds dX^{-1} = dX^0 (dxy_prev NULL)
    rhs_terms = np.concatenate([r["k_s"] * dks, r["k_b"] * dkb, [r["sigma"] * dsig],
                                (r["xy"] * dxy).ravel(), (r["xy_prev"] * dxy).ravel()])
    scale = np.abs(lhs_terms).sum() + np.abs(rhs_terms).sum()
    return lhs_terms.sum(), rhs_terms.sum(), scale


@pytest.mark.parametrize("steps,K", [(37, 8), (16, 16), (1, 4)])
def test_dot_product_sensitivity_case(steps, K):
    """Two red cells and a soft carrier with bonds forming on the lower wall
    (every force term: stretch, bend, area, repulsion, bonds)."""
    wl = sensitivity.make_workload(sensitivity.default_params(), steps)
    lhs, rhs, scale = dot_identity(wl, steps, K, seed=steps)
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)


def test_dot_product_capsule_periodic_bounce_back():
    """The 128 x 32 capsule (walls, body force, every element a ligand)."""
    wl = inputs.capsule_128x32("f64")
    lhs, rhs, scale = dot_identity(wl, 25, 7, seed=3)
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)


@pytest.fixture(scope="module")
def jacobians():
    p0 = sensitivity.default_params()
    Jt, jac_t, bt = sensitivity.jacobian(p0, STEPS)
    Ja, jac_a, ba = sensitivity.adjoint_jacobian(p0, STEPS, checkpoint_every=64)
    return p0, Jt, jac_t, bt, Ja, jac_a, ba


def test_adjoint_gradient_matches_tangent_jacobian(jacobians):
    p0, Jt, jac_t, bt, Ja, jac_a, ba = jacobians
    np.testing.assert_array_equal(Ja, Jt)
    np.testing.assert_array_equal(ba, bt)
    assert (ba >= 0).sum() > 0
    for i in range(2):
        for k in range(4):
            assert abs(jac_a[i, k] - jac_t[i, k]) <= 1e-9 * abs(jac_t[i, k]) + 1e-12 * np.abs(jac_t[i]).max(), \
                (i, sensitivity.PARAMS[k], jac_a[i, k], jac_t[i, k])


@pytest.mark.parametrize("k", [2, 3])
def test_adjoint_gradient_matches_central_differences(jacobians, k):
    """sigma and the release height against central differences of the FP64
    solver with the same bond history."""
    p0, _, _, bonds, J, jac, _ = jacobians
    h = 1e-4 if k == 3 else 1e-4 * abs(p0[k])
    pp, pm = p0.copy(), p0.copy()
    pp[k] += h
    pm[k] -= h
    Jp, bp = sensitivity.run(pp, STEPS)
    Jm, bm = sensitivity.run(pm, STEPS)
    assert np.array_equal(bp, bonds) and np.array_equal(bm, bonds)
    fd = (Jp - Jm) / (2 * h)
    for i in range(2):
        tol = 1e-6 * abs(fd[i]) + 1e-13 * abs(J[i]) / h
        assert abs(jac[i, k] - fd[i]) <= tol, (sensitivity.PARAMS[k], i, jac[i, k], fd[i])


@pytest.mark.parametrize("prec,rel", [("f32", 1e-3), ("f16", 1e-2), ("bf16", 5e-2)])
def test_reduced_precision_forward_run(jacobians, prec, rel):
    """The adjoint of a forward run in FP32 arithmetic (populations stored in
    FP32, FP16 or BF16), gradients accumulated in FP64: against the FP64 run's
    adjoint, within the stated relative bound (measured at 200 steps: 1.2e-4
    FP32, 8e-5 FP16, 3.6e-3 BF16, the largest on dJ1/dk_s, a derivative of
    1e-4 of the others' size)."""
    p0, _, _, _, Ja, jac_a, ba = jacobians
    J, jac, b = sensitivity.adjoint_jacobian(p0, STEPS, checkpoint_every=64, precision=prec)
    np.testing.assert_array_equal(b, ba)
    for i in range(2):
        for k in range(4):
            assert abs(jac[i, k] - jac_a[i, k]) <= rel * abs(jac_a[i, k]) + 1e-12 * np.abs(jac_a[i]).max(), \
                (prec, i, sensitivity.PARAMS[k], jac[i, k], jac_a[i, k])


def test_checkpoint_interval_does_not_change_the_gradient():
    p0 = sensitivity.default_params()
    steps = 60
    grads = []
    for K in (1, 7, 60, 100):
        rec = sensitivity.Recording(p0, steps, checkpoint_every=K)
        try:
            grads.append(rec.gradient((1.0, 3.0)))
        finally:
            rec.close()
    for g in grads[1:]:
        np.testing.assert_allclose(g, grads[0], rtol=1e-11, atol=1e-14 * np.abs(grads[0]).max())


def test_population_adjoint_matches_central_differences():
    """J = <c, f^N> over a patch of nodes; dJ/df^0 along a direction on a
    nearby patch, against central differences of the FP64 solver."""
    L = lb()
    steps = 12
    wl = inputs.capsule_128x32("f64")
    N = wl.nx * wl.ny
    rng = np.random.default_rng(11)
    c = np.zeros((9, wl.ny, wl.nx))
    c[:, 2:8, 26:34] = rng.standard_normal((9, 6, 8))
    delta = np.zeros((9, wl.ny, wl.nx))
    delta[:, 3:7, 28:33] = rng.standard_normal((9, 4, 5)) * 1e-3
    r = adjoint_run(wl, steps, 5, None, None, f_bar=c.reshape(9, N), want_f=True)
    pred = float((r["f"] * delta.reshape(9, N)).sum())

    def J(sign, h):
        sim = L.Simulation(wl, precision="f64")
        try:
            f0 = sim.populations()
            sim.set_populations(f0 + sign * h * delta)
            sim.step(steps)
            return float((c * sim.populations()).sum())
        finally:
            sim.close()

    h = 1e-3
    fd = (J(1, h) - J(-1, h)) / (2 * h)
    assert abs(pred) > 1e-6
    assert abs(pred - fd) <= 1e-6 * abs(fd), (pred, fd)


def test_population_adjoint_one_step_matches_oracle_differences():
    """Lattice only (no markers), one step: the adjoint seeded with a one-hot at
    population 2 of node x of f^1 is nonzero only at the nine populations of
    f^0 at x - e_2 (the node it is pulled from), and there equals the central
    difference of the oracle's step (the collision's Jacobian row)."""
    from helpers import make_oracle
    L = lb()
    wl = inputs.capsule_128x32("f64")
    wl.membranes = []
    wl.receptors = np.zeros((0, 2))
    N = wl.nx * wl.ny
    node = 5 * wl.nx + 17
    e = np.zeros((9, N))
    e[2, node] = 1.0
    sim = L.Simulation(wl, precision="f64")
    f0 = sim.populations()
    adj = L.lbib_adjoint_create(sim.ctx, 3)
    try:
        L.lbib_adjoint_record(sim.ctx, adj, 1)
        L.lbib_adjoint_seed(sim.ctx, adj, None, None, e)
        L.lbib_adjoint_reverse(sim.ctx, adj)
        r = L.lbib_adjoint_read(sim.ctx, adj, 0, 0, N)
    finally:
        L.lbib_adjoint_destroy(adj)
        sim.close()
    src = node - wl.nx
    nz = np.argwhere(r["f"] != 0.0)
    assert set(map(tuple, nz)) <= {(i, src) for i in range(9)}
    orc = make_oracle(wl)
    h = 1e-6
    for i in range(9):
        vals = []
        for sgn in (1, -1):
            f = f0.reshape(9, N).copy()
            f[i, src] += sgn * h
            orc.set_populations(f.reshape(9, wl.ny, wl.nx))
            orc.step(1)
            vals.append(orc.populations().reshape(9, N)[2, node])
            orc = make_oracle(wl)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(r["f"][i, src] - fd) <= 1e-8, (i, r["f"][i, src], fd)


def test_context_is_left_at_the_recorded_end_state():
    L = lb()
    p0 = sensitivity.default_params()
    steps = 40
    wl = sensitivity.make_workload(p0, steps)
    ref = L.Simulation(wl, precision="f64")
    ref.step(steps + 10)
    x_ref, b_ref, f_ref = ref.markers(), ref.bonds(), ref.populations()
    ref.close()
    sim = L.Simulation(wl, precision="f64")
    adj = L.lbib_adjoint_create(sim.ctx, 9)
    try:
        L.lbib_adjoint_record(sim.ctx, adj, steps)
        assert L.lbib_adjoint_recorded_steps(adj) == steps
        x_end = sim.markers()
        L.lbib_adjoint_seed(sim.ctx, adj, np.ones((wl.n_vertices, 2)), None, None)
        L.lbib_adjoint_reverse(sim.ctx, adj)
        np.testing.assert_array_equal(sim.markers(), x_end)
        sim.step(10)
        np.testing.assert_array_equal(sim.markers(), x_ref)
        np.testing.assert_array_equal(sim.bonds(), b_ref)
        np.testing.assert_array_equal(sim.populations(), f_ref)
    finally:
        L.lbib_adjoint_destroy(adj)
        sim.close()


def test_autograd_backward_runs_the_adjoint(jacobians):
    import torch
    p0, _, _, _, Ja, jac_a, _ = jacobians
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    out = sensitivity.carrier_observables(p, STEPS, mode="adjoint", checkpoint_every=64)
    np.testing.assert_array_equal(out.detach().numpy(), Ja)
    (out[0] + 2.0 * out[1]).backward()
    ref = jac_a[0] + 2.0 * jac_a[1]
    np.testing.assert_allclose(p.grad.numpy(), ref, rtol=1e-11, atol=1e-14 * np.abs(ref).max())


def test_error_paths():
    L = lb()
    wl_rigid = inputs.capsule_128x32("f64")
    wl_rigid.membranes[0].kind = 1
    sr = L.Simulation(wl_rigid)
    try:
        with pytest.raises(L.LbibError) as ei:
            L.lbib_adjoint_create(sr.ctx, 4)
        assert ei.value.status == L.LBIB_E_INVALID
    finally:
        sr.close()
    wl = inputs.capsule_128x32("f64")
    sim = L.Simulation(wl, precision="f64")
    try:
        with pytest.raises(L.LbibError) as ei:
            L.lbib_adjoint_create(sim.ctx, 0)
        assert ei.value.status == L.LBIB_E_INVALID
        adj = L.lbib_adjoint_create(sim.ctx, 4)
        try:
            assert L.lbib_adjoint_recorded_steps(adj) == 0
            with pytest.raises(L.LbibError) as ei:
                L.lbib_adjoint_seed(sim.ctx, adj)
            assert ei.value.status == L.LBIB_E_STATE
            with pytest.raises(L.LbibError) as ei:
                L.lbib_adjoint_reverse(sim.ctx, adj)
            assert ei.value.status == L.LBIB_E_STATE
            with pytest.raises(L.LbibError) as ei:
                L.lbib_adjoint_record(sim.ctx, adj, 0)
            assert ei.value.status == L.LBIB_E_INVALID
            L.lbib_adjoint_record(sim.ctx, adj, 3)
            L.lbib_adjoint_seed(sim.ctx, adj)
            L.lbib_adjoint_reverse(sim.ctx, adj)
            with pytest.raises(L.LbibError) as ei:  # a second sweep needs a new seed
                L.lbib_adjoint_reverse(sim.ctx, adj)
            assert ei.value.status == L.LBIB_E_STATE
        finally:
            L.lbib_adjoint_destroy(adj)
    finally:
        sim.close()


def test_derivatives_match_the_oracle_tangent():
    """The oracle's own forward-mode tangent (dual numbers in the plain C
    oracle, pinned to the oracle's central differences in
    test_oracle_tangent.py) on the sensitivity case: the GPU tangent's marker
    derivatives along a random direction of every parameter and marker, and
    the adjoint's dJ/dp for the four carrier parameters."""
    import oracle
    from helpers import make_oracle
    L = lb()
    steps = 60
    p0 = sensitivity.default_params()
    wl = sensitivity.make_workload(p0, steps)
    nm, nv = len(wl.membranes), wl.n_vertices
    nc = len(wl.membranes[-1].xy)

    def oracle_run(dks, dkb, dsig, dxy):
        s = make_oracle(wl)
        t = oracle.OracleTangent(s)
        t.seed(dks, dkb, dsig, dxy, None)
        t.step(steps)
        dX, _, _ = t.get()
        return dX, s.markers(), s.bonds()

    rng = np.random.default_rng(21)
    dks, dkb = rng.standard_normal(nm) * 1e-3, rng.standard_normal(nm) * 1e-3
    dsig = float(rng.standard_normal()) * 1e-4
    dxy = rng.standard_normal((nv, 2))
    dX_o, _, bonds_o = oracle_run(dks, dkb, dsig, dxy)
    dX_g, _ = tangent_run(wl, steps, dks, dkb, dsig, dxy)
    assert np.abs(dX_g - dX_o).max() <= 1e-8 * np.abs(dX_o).max(), np.abs(dX_g - dX_o).max()

    jac_o = np.zeros((2, 4))
    for k in range(4):
        a, b = np.zeros(nm), np.zeros(nm)
        s_ = 0.0
        d = np.zeros((nv, 2))
        if k == 0:
            a[-1] = 1.0
        elif k == 1:
            b[-1] = 1.0
        elif k == 2:
            s_ = 1.0
        else:
            d[nv - nc:, 1] = 1.0
        dX, xy, bo = oracle_run(a, b, s_, d)
        jac_o[:, k] = sensitivity.observable_directional(wl, xy, bo, dX, s_)
    J, jac_a, bonds = sensitivity.adjoint_jacobian(p0, steps, checkpoint_every=16)
    np.testing.assert_array_equal(bonds, bonds_o)
    for i in range(2):
        for k in range(4):
            assert abs(jac_a[i, k] - jac_o[i, k]) <= 1e-8 * abs(jac_o[i, k]) + 1e-11 * np.abs(jac_o[i]).max(), \
                (i, sensitivity.PARAMS[k], jac_a[i, k], jac_o[i, k])


def test_sensitivity_case_fp32_forward_5000_steps_matches_central_differences():
    """The differentiation form as specified: the 320 x 160 sensitivity case,
    FP32 forward run over 5000 steps with checkpoints every 250, FP64 adjoint
    and gradient accumulation.  All eight derivatives dJ_i/dp_k against central
    differences of the FP64 solver with h = 1e-4 (relative for k_s, k_b and
    sigma, lattice units for the release height), along the same bond history,
    within 1e-3 relative (plus 1e-6 of the row's largest entry)."""
    p0 = sensitivity.default_params()
    steps = 5000
    J, jac, bonds = sensitivity.adjoint_jacobian(p0, steps, checkpoint_every=250, precision="f32")
    assert (bonds >= 0).sum() > 0
    for k in range(4):
        h = 1e-4 if k == 3 else 1e-4 * abs(p0[k])
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        Jp, bp = sensitivity.run(pp, steps)
        Jm, bm = sensitivity.run(pm, steps)
        assert np.array_equal(bp, bonds) and np.array_equal(bm, bonds), sensitivity.PARAMS[k]
        fd = (Jp - Jm) / (2 * h)
        for i in range(2):
            tol = 1e-3 * abs(fd[i]) + 1e-6 * np.abs(jac[i]).max()
            assert abs(jac[i, k] - fd[i]) <= tol, (sensitivity.PARAMS[k], i, jac[i, k], fd[i])

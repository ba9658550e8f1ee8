"""GPU tests of the differentiation form: forward-mode tangent of the FP64 time
step (lbib_tangent_*) for the carrier observables J1 (centroid height above
the lower wall) and J2 (bond elastic energy) with respect to the carrier's
k_s, k_b, the bond stiffness sigma and the release height, on the 320 x 160
capillary with 2 red cells and a soft carrier released 1 lu above the wall.

Checks: against central finite differences of the FP64 CUDA solver (bond
history identical in the perturbed runs), against central differences of the
FP64 oracle, and the torch.autograd.Function's backward."""
import numpy as np
import pytest

from helpers import make_oracle
from paper_1907_00080_gb300 import sensitivity

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


@pytest.fixture(scope="module")
def tangent():
    p0 = sensitivity.default_params()
    J, jac, bonds = sensitivity.jacobian(p0, STEPS)
    return p0, J, jac, bonds


def fd_step(p0, k):
    return 1e-4 if k == 3 else 1e-4 * abs(p0[k])


def test_bonds_form_in_the_window(tangent):
    _, J, _, bonds = tangent
    assert (bonds >= 0).sum() > 0 and J[1] > 0


def fd_noise(J, h):
    """FP64 trajectories of perturbed runs differ by rounding at about 1e-13
    relative after a few hundred steps: the noise floor of a central difference."""
    return 1e-13 * abs(J) / h


@pytest.mark.parametrize("k", [2, 3])
def test_tangent_matches_central_differences(tangent, k):
    """sigma and the release height, on the observables themselves (k_s and k_b
    move J1, J2 by less than the FP64 rounding of the trajectory in this window:
    see the deformed-carrier test)."""
    p0, J, jac, bonds = tangent
    h = fd_step(p0, k)
    pp, pm = p0.copy(), p0.copy()
    pp[k] += h
    pm[k] -= h
    Jp, bp = sensitivity.run(pp, STEPS)
    Jm, bm = sensitivity.run(pm, STEPS)
    assert np.array_equal(bp, bonds) and np.array_equal(bm, bonds)  # same bond history at the end
    fd = (Jp - Jm) / (2 * h)
    for i in range(2):
        tol = 1e-6 * abs(fd[i]) + fd_noise(J[i], h)
        assert abs(jac[i, k] - fd[i]) <= tol, (sensitivity.PARAMS[k], i, jac[i, k], fd[i])


def deformed_carrier(p, steps):
    """The sensitivity case with the carrier's initial shape stretched 5 % along
    x (rest shape unchanged): its elastic recoil makes every marker position
    depend strongly on k_s and k_b."""
    wl = sensitivity.make_workload(p, steps)
    car = wl.membranes[-1]
    c = car.xy.mean(axis=0)
    x0 = np.concatenate([m.xy for m in wl.membranes])
    x0[-len(car.xy):] = c + (car.xy - c) * np.array([1.05, 1 / 1.05])
    return wl, x0


@pytest.mark.parametrize("k", [0, 1])
def test_tangent_of_positions_deformed_carrier(k):
    from paper_1907_00080_gb300 import lbib
    steps = 100
    p0 = sensitivity.default_params()
    wl, x0 = deformed_carrier(p0, steps)
    nm, nv = len(wl.membranes), wl.n_vertices
    s = lbib.Simulation(wl, precision="f64")
    lbib.lbib_write_markers(s.ctx, x0, x0)
    t = lbib.lbib_tangent_create(s.ctx)
    d = np.zeros(nm)
    d[-1] = 1.0
    lbib.lbib_tangent_seed(s.ctx, t, d if k == 0 else None, d if k == 1 else None, 0.0, None, None)
    lbib.lbib_tangent_step(s.ctx, t, steps)
    dX, _ = lbib.lbib_tangent_read(s.ctx, t, nv)
    lbib.lbib_tangent_destroy(t)
    s.close()

    def primal(p):
        w, x = deformed_carrier(p, steps)
        q = lbib.Simulation(w, precision="f64")
        lbib.lbib_write_markers(q.ctx, x, x)
        q.step(steps)
        out = q.markers()
        q.close()
        return out

    h = 1e-3 * p0[k]  # large enough to clear the FP64 noise of the trajectories
    pp, pm = p0.copy(), p0.copy()
    pp[k] += h
    pm[k] -= h
    fd = (primal(pp) - primal(pm)) / (2 * h)
    assert np.abs(fd).max() > 0.1
    assert np.abs(dX - fd).max() <= 2e-5 * np.abs(fd).max(), np.abs(dX - fd).max() / np.abs(fd).max()


def test_tangent_matches_oracle_differences():
    """The oracle (plain FP64 C) differentiated by central differences over 60
    steps, for the release height and sigma."""
    steps = 60
    p0 = sensitivity.default_params()
    _, jac, _ = sensitivity.jacobian(p0, steps)
    for k in (3, 2):
        h = fd_step(p0, k)
        vals = []
        for sgn in (1, -1):
            p = p0.copy()
            p[k] += sgn * h
            wl = sensitivity.make_workload(p, steps)
            r = make_oracle(wl)
            r.step(steps)
            j1, j2, _ = sensitivity.observables(wl, r.markers(), r.bonds())
            vals.append(np.array([j1, j2]))
        fd = (vals[0] - vals[1]) / (2 * h)
        for i in range(2):
            tol = 1e-6 * abs(fd[i]) + fd_noise(vals[0][i], h)
            assert abs(jac[i, k] - fd[i]) <= tol, (k, i, jac[i, k], fd[i])


def test_autograd_function_backward(tangent):
    import torch
    p0, J, jac, _ = tangent
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    out = sensitivity.carrier_observables(p, STEPS, mode="tangent")
    np.testing.assert_allclose(out.detach().numpy(), J, rtol=0, atol=0)
    (out[0] + 2.0 * out[1]).backward()
    np.testing.assert_allclose(p.grad.numpy(), jac[0] + 2.0 * jac[1], rtol=1e-14, atol=0)

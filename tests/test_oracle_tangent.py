"""Pins of the oracle's forward-mode tangent (oracle.OracleTangent, dual
numbers in lbib_oracle.c) against central differences of the oracle's own
primal step: the tangent of every marker position after a few steps, for each
kind of direction (k_s, k_b, sigma, the initial markers, the populations).

The cases are built so that every branch of the step carries derivative:
  - a capsule stretched 5 % (rest shape unchanged) whose lowest marker sits
    0.3 lu above the lower wall (MLS re-solve with a dropped stencil row), with
    one bond set from step 0 (the bond spring), under the Poiseuille flow;
  - two capsules 1.5 lu apart (repulsion, d_rep = 2).
The bond history of the perturbed runs is checked to equal the unperturbed
one, so the differences see the same event path as the tangent."""
import numpy as np
import pytest

import oracle
from helpers import make_oracle
from paper_1907_00080_gb300 import inputs

STEPS = 20


def near_wall_case():
    """Stretched capsule near the wall with a bond at its lowest element."""
    wl = inputs.capsule_128x32("f64")
    m = wl.membranes[0]
    c = m.xy.mean(axis=0)
    x0 = c + (m.xy - c) * np.array([1.05, 1.0 / 1.05])
    x0[:, 1] += 0.3 - x0[:, 1].min()
    return wl, x0


def two_capsules_case():
    wl = inputs.capsule_128x32("f64")
    a = inputs.circle(40.0, 14.0, 4.0, 32)
    b = inputs.circle(49.5, 14.0, 4.0, 32)
    wl.membranes = [inputs.Membrane(xy=a, ks=0.05, kb=0.005, ka=0.1),
                    inputs.Membrane(xy=b, ks=0.05, kb=0.005, ka=0.1)]
    wl.receptors = np.zeros((0, 2))
    x0 = np.concatenate([a, b])
    return wl, x0


def build(wl, x0, ks_scale=None, kb_scale=None, sigma=None, bond=True):
    """Oracle run of the case, the rest shape from wl, initial markers x0."""
    w = inputs.Workload(**{k: getattr(wl, k) for k in wl.__dataclass_fields__})
    w.membranes = [inputs.Membrane(xy=m.xy, ks=m.ks * (ks_scale[i] if ks_scale is not None else 1.0),
                                   kb=m.kb * (kb_scale[i] if kb_scale is not None else 1.0), ka=m.ka,
                                   kind=m.kind, ligands=m.ligands) for i, m in enumerate(wl.membranes)]
    if sigma is not None:
        w.sigma_lu = sigma
    s = make_oracle(w)
    s.set_markers(x0, x0)
    if bond and s.nlig:
        # bond the ligand on the lowest element to the receptor below it
        e = int(np.argmin(x0[:, 1] + np.roll(x0[:, 1], -1)))
        cx = 0.5 * (x0[e, 0] + x0[(e + 1) % len(x0), 0])
        r = int(np.argmin(np.abs(w.receptors[:, 0] - cx)))
        s.set_bond(e, r)
    return s


def central(run, h):
    (xp, bp), (xm, bm) = run(h), run(-h)
    assert np.array_equal(bp, bm)
    return (xp - xm) / (2 * h)


def tangent(wl, x0, **seed):
    s = build(wl, x0)
    t = oracle.OracleTangent(s)
    t.seed(**seed)
    t.step(STEPS)
    dX, dXp, df = t.get()
    return dX, s.bonds()


def check(dX, fd, rel=2e-6):
    scale = np.abs(fd).max()
    assert scale > 0
    err = np.abs(dX - fd).max()
    assert err <= rel * scale + 1e-10, (err, scale)


@pytest.mark.parametrize("which", ["k_s", "k_b"])
def test_tangent_stiffness_near_wall(which):
    wl, x0 = near_wall_case()
    d = np.ones(1)
    dX, b0 = tangent(wl, x0, **({"dks": d} if which == "k_s" else {"dkb": d}))
    k = wl.membranes[0].ks if which == "k_s" else wl.membranes[0].kb
    h = 1e-3 * k

    def run(eps):
        sc = np.array([1.0 + eps / k])
        s = build(wl, x0, ks_scale=sc if which == "k_s" else None, kb_scale=sc if which == "k_b" else None)
        s.step(STEPS)
        return s.markers(), s.bonds()

    fd = central(run, h)
    assert np.array_equal(run(0.0)[1], b0)
    check(dX, fd)


def test_tangent_sigma_with_a_bond():
    wl, x0 = near_wall_case()
    dX, b0 = tangent(wl, x0, dsigma=1.0)
    assert (b0 >= 0).any()
    h = 1e-2 * wl.sigma_lu  # the response is nearly linear in sigma; smaller h sinks into rounding

    def run(eps):
        s = build(wl, x0, sigma=wl.sigma_lu + eps)
        s.step(STEPS)
        return s.markers(), s.bonds()

    check(dX, central(run, h))


@pytest.mark.parametrize("case", ["near_wall", "two_capsules"])
def test_tangent_initial_markers(case):
    wl, x0 = near_wall_case() if case == "near_wall" else two_capsules_case()
    rng = np.random.default_rng(4)
    v = rng.standard_normal(x0.shape)
    dX, _ = tangent(wl, x0, dxy=v)
    h = 1e-5

    def run(eps):
        s = build(wl, x0 + eps * v)
        s.step(STEPS)
        return s.markers(), s.bonds()

    check(dX, central(run, h))


def test_repulsion_is_active_in_the_two_capsule_case():
    wl, x0 = two_capsules_case()
    s = build(wl, x0)
    s.compute_forces()
    f_rep = s.forces()
    wl2, _ = two_capsules_case()
    far = x0.copy()
    far[32:, 0] += 20.0
    s2 = build(wl2, far)
    s2.compute_forces()
    # the facing vertices feel the repulsion only in the close placement
    assert np.abs(f_rep[:32] - s2.forces()[:32]).max() > 1e-6


def test_tangent_populations():
    wl, x0 = near_wall_case()
    rng = np.random.default_rng(9)
    df = np.zeros((9, wl.ny, wl.nx))
    df[:, 2:9, 28:37] = rng.standard_normal((9, 7, 9)) * 1e-3
    dX, _ = tangent(wl, x0, df=df)
    s0 = build(wl, x0)
    f0 = s0.populations()
    h = 1e-3

    def run(eps):
        s = build(wl, x0)
        s.set_populations(f0 + eps * df)
        s.step(STEPS)
        return s.markers(), s.bonds()

    check(dX, central(run, h), rel=1e-5)


def test_zero_direction_gives_zero_tangent_and_the_primal_is_unchanged():
    wl, x0 = near_wall_case()
    s = build(wl, x0)
    t = oracle.OracleTangent(s)
    t.seed()
    t.step(5)
    dX, dXp, df = t.get()
    assert not dX.any() and not dXp.any() and not df.any()
    s2 = build(wl, x0)
    s2.step(5)
    np.testing.assert_array_equal(s.markers(), s2.markers())
    np.testing.assert_array_equal(s.populations(), s2.populations())


def test_rigid_membranes_are_refused():
    wl = inputs.capsule_128x32("f64")
    wl.membranes[0].kind = 1
    s = make_oracle(wl)
    with pytest.raises(ValueError):
        oracle.OracleTangent(s)

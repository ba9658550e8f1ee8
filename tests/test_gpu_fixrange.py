"""Range of the fixed-point accumulators (GPU, through the C ABI).

The spread IB force is accumulated per node as 64-bit integers scaled by
2^52, and the repulsion magnitudes per vertex as integers scaled by 2^60.  A
contribution at or beyond its bound (64 lu of force per vertex and node; a
repulsion of 1 per vertex and segment, which Eq. repFor reaches at 9.4e-3 lu,
i.e. overlapping membranes), or one that is not finite, is clamped and
reported: lbib_sync returns LBIB_E_NONFINITE and the context is poisoned.
Close membranes inside the range still match the oracle.
"""
import numpy as np
import pytest

from helpers import make_oracle
from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu

E_NONFINITE, E_STATE = 5, 6


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def two_rings(gap, precision):
    """Two rings of radius 4 (32 vertices, vertex 0 of each on the +x axis)
    whose nearest vertices (vertex 0 of the left ring, vertex 16 of the right
    one) are `gap` apart on a horizontal line; fluid at rest."""
    R = 4.0
    a = inputs.circle(20.0, 16.0, R, 32, phase=0.0)
    b = inputs.circle(20.0 + 2 * R + gap, 16.0, R, 32, phase=0.0)
    mem = [inputs.Membrane(xy=xy, ks=1e-3, kb=0.0, ka=0.1) for xy in (a, b)]
    return inputs.Workload(name="rings", nx=64, ny=32, init="rest", precision=precision, membranes=mem)


def expect_nonfinite(wl):
    from paper_1907_00080_gb300 import lbib
    s = lbib.Simulation(wl)
    s.step(1)
    with pytest.raises(lbib.LbibError) as e:
        s.sync()
    assert e.value.status == E_NONFINITE
    assert "fixed-point" in str(e.value)
    with pytest.raises(lbib.LbibError) as e:
        s.step(1)  # poisoned
    assert e.value.status == E_STATE
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("gap", [1e-3, 0.0])
def test_overlapping_membranes_are_reported(prec, gap):
    # 1e-3 lu: Eq. repFor gives 8.8e-6 * 1e-3^-2.5 = 280; coincident: infinite
    expect_nonfinite(two_rings(gap, prec))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_close_membranes_inside_the_range_match_the_oracle(prec):
    # 0.05 lu: repulsion 0.016 per vertex, well inside the accumulator's range
    from paper_1907_00080_gb300 import lbib
    wl = two_rings(0.05, prec)
    s, r = lbib.Simulation(wl), make_oracle(wl)
    s.step(3)
    s.sync()
    r.step(3)
    F, F0 = s.forces(), r.forces()
    tol = 1e-12 if prec == "f64" else 1e-5
    assert np.max(np.abs(F - F0)) <= tol * np.max(np.abs(F0))
    assert np.max(np.abs(F0)) > 1e-3  # the repulsion dominates
    s.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spread_force_beyond_the_range_is_reported(prec):
    # a ring of 32 vertices stretched by 10 % with k_s = 1e6: each element
    # pulls with k_s dl = 7.8e4 lu, about 1.5e4 lu of net force per vertex,
    # so w F reaches thousands of lu at the nearest nodes
    xy = inputs.circle(32.0, 16.0, 4.0, 32)
    wl = inputs.Workload(name="stiff", nx=64, ny=32, init="rest", precision=prec,
                         membranes=[inputs.Membrane(xy=xy, ks=1e6, kb=0.0, ka=0.0)])
    from paper_1907_00080_gb300 import lbib
    s = lbib.Simulation(wl)
    lbib.lbib_write_markers(s.ctx, 1.1 * (xy - [32.0, 16.0]) + [32.0, 16.0])
    s.step(1)
    with pytest.raises(lbib.LbibError) as e:
        s.sync()
    assert e.value.status == E_NONFINITE
    s.close()

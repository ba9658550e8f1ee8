"""GPU test of lbib_membrane_observables (the per-membrane quantities of the
margination and adhesion studies, Sec. 4) against their definitions evaluated
on the FP64 oracle's state after the same steps: centroid, centroid velocity
(X^n - X^{n-1}), channel region, bonds, lowest and highest vertex."""
import numpy as np
import pytest

from helpers import make_oracle
from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def reference(wl, x, xp, bonds):
    """The definitions, from the oracle's markers and bonds."""
    out = []
    off, loff = 0, 0
    for m in wl.membranes:
        n, nl = len(m.xy), len(m.ligands)
        X, Xp = x[off:off + n], xp[off:off + n]
        yc = X[:, 1].mean()
        h = (yc + 0.5) / wl.ny
        region = 0.0 if 0.3 <= h <= 0.7 else (1.0 if 0.2 <= h <= 0.8 else 2.0)
        out.append([X[:, 0].mean(), yc, (X[:, 0] - Xp[:, 0]).mean(), (X[:, 1] - Xp[:, 1]).mean(), region,
                    float((bonds[loff:loff + nl] >= 0).sum()), X[:, 1].min() + 0.5, X[:, 1].max() + 0.5])
        off += n
        loff += nl
    return np.array(out)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_observables_match_their_definitions_on_the_oracle_state(prec):
    from paper_1907_00080_gb300 import lbib
    wl = inputs.coarse_capillary_640x160(prec)
    s = lbib.Simulation(wl)
    r = make_oracle(wl)
    s.step(120)
    r.step(120)
    got = s.observables()
    ref = reference(wl, r.markers(), r.prev_markers(), r.bonds())
    assert got.shape == (len(wl.membranes), 8)
    np.testing.assert_array_equal(got[:, 4], ref[:, 4])
    np.testing.assert_array_equal(got[:, 5], ref[:, 5])
    pos_tol = 1e-10 if prec == "f64" else 1e-5
    for c in (0, 1, 6, 7):
        np.testing.assert_allclose(got[:, c], ref[:, c], rtol=0, atol=pos_tol)
    vel_tol = 1e-14 if prec == "f64" else 1e-5 * 1e-2
    for c in (2, 3):
        np.testing.assert_allclose(got[:, c], ref[:, c], rtol=0, atol=max(vel_tol, 1e-8 * np.abs(ref[:, c]).max()))
    assert set(np.unique(got[:, 4])) <= {0.0, 1.0, 2.0}
    s.close()


def test_adhering_carrier_in_couette_flow():
    """In the Couette set-up the carrier holds bonds, sits in the lower
    cell-free layer and moves downstream."""
    from paper_1907_00080_gb300 import lbib
    wl = inputs.couette_cfl_600x200("f64", sigma=1.0, carrier="soft")
    s = lbib.Simulation(wl)
    s.step(1500)
    o = s.observables()[0]
    assert o[4] == 2.0 and o[5] > 0 and o[2] > 0.0 and o[6] > 0.0
    s.close()

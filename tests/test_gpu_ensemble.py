"""GPU tests of the ensemble form (lbib_ensemble_*): independent capillaries of
different lengths advanced by one graph launch per chunk of steps.  Every
member must compute exactly what it computes alone (same kernels, same
inputs: bitwise), and a member must match the oracle like any single run."""
import numpy as np
import pytest

from helpers import f64_field_tol, make_oracle, rel_err, vel_err
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


def small_ensemble(n, precision, seed=3):
    wls = inputs.capillary_ensemble(n, seed=seed, precision=precision, l_min_um=16.0, l_max_um=24.0)
    for wl in wls:
        wl.bonds = dict(inputs.STRESS_BONDS)
    return wls


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_ensemble_members_match_single_runs_bitwise(precision):
    from paper_1907_00080_gb300 import lbib
    wls = small_ensemble(4, precision)
    assert len({wl.nx for wl in wls}) > 1  # channels of different lengths
    ens = lbib.Ensemble(wls)
    ens.step(37)  # two chunks of 16 and five single steps
    ens.step(21)
    ens.sync()
    for wl, m in zip(wls, ens.members):
        s = lbib.Simulation(wl)
        s.step(58)
        assert np.array_equal(m.populations(), s.populations()), wl.name
        assert np.array_equal(m.markers(), s.markers()), wl.name
        assert np.array_equal(m.bonds(), s.bonds()), wl.name
        _, ux, _ = m.fields()
        _, ux1, _ = s.fields()
        assert np.array_equal(ux, ux1)
        assert lbib.lbib_step_count(m.ctx) == 58
        s.close()
    ens.close()


def test_ensemble_member_matches_oracle():
    from paper_1907_00080_gb300 import lbib
    wls = small_ensemble(2, "f64", seed=5)
    ens = lbib.Ensemble(wls)
    ens.step(30)
    ens.sync()
    for wl, m in zip(wls, ens.members):
        r = make_oracle(wl)
        r.step(30)
        _, ux, uy = m.fields()
        _, ux0, uy0 = r.fields()
        assert vel_err(ux, uy, ux0, uy0) < f64_field_tol(np.max(np.abs(ux0)))
        assert rel_err(m.markers(), r.markers()) < 1e-12
        assert np.array_equal(m.bonds(), r.bonds())
    ens.close()


def test_ensemble_rejects_bad_members():
    from paper_1907_00080_gb300 import lbib
    a = lbib.Simulation(inputs.capsule_128x32("f32"))
    with pytest.raises(lbib.LbibError):
        lbib.lbib_ensemble_create([a.ctx, a.ctx])
    with pytest.raises(lbib.LbibError):
        lbib.lbib_ensemble_create([])
    a.close()

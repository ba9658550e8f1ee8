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


@pytest.mark.parametrize("precision,tiling,groups", [("f32", (1, 4), 1), ("f64", (1, 2), 2), ("f16", (2, 2), 1),
                                                    ("f32", (4, 1), 3), ("f32", (2, 2), 5),
                                                    ("f32", (2, 0), 1), ("f32", (1, 0), 2), ("f64", (1, 0), 1),
                                                    ("f16", (4, 0), 2), ("bf16", (2, 0), 1)])
def test_batched_ensemble_matches_single_runs_bitwise(precision, tiling, groups):
    """Members sharing the precision and the fused kernel's form and shape
    (row tiles (vec, ty), or the persistent form (npt, 0)) run in the batched
    form (three launches per time step for each group of members); each member
    still computes bit for bit what it computes alone with that tiling, over
    chunks of 16 steps and single steps, with stress kinetics (bonds form and
    break), whatever the grouping."""
    from paper_1907_00080_gb300 import lbib
    wls = small_ensemble(5, precision, seed=11)
    assert len({wl.nx for wl in wls}) > 1
    ens = lbib.Ensemble(wls, tiling=tiling)
    assert ens.form == 1
    assert ens.groups == 1 and ens.launches_per_step == 3
    ens.set_groups(groups)
    assert ens.groups == groups and ens.launches_per_step == 3 * groups
    ens.step(35)
    ens.step(16)
    ens.sync()
    for wl, m in zip(wls, ens.members):
        s = lbib.Simulation(wl, tiling=tiling)
        s.step(51)
        assert np.array_equal(m.populations(), s.populations()), wl.name
        assert np.array_equal(m.markers(), s.markers()), wl.name
        assert np.array_equal(m.bonds(), s.bonds()), wl.name
        _, ux, _ = m.fields()
        _, ux1, _ = s.fields()
        assert np.array_equal(ux, ux1)
        assert lbib.lbib_step_count(m.ctx) == 51
        s.close()
    ens.close()


def test_batched_ensemble_member_matches_oracle_and_other_forms_fall_back():
    """A batched member against the oracle (FP64, 40 steps); members with
    different tile shapes run as a graph of member graphs, with the same
    results."""
    from paper_1907_00080_gb300 import lbib
    wls = small_ensemble(3, "f64", seed=7)
    ens = lbib.Ensemble(wls, tiling=(1, 4))
    assert ens.form == 1
    ens.step(40)
    ens.sync()
    wl, m = wls[1], ens.members[1]
    r = make_oracle(wl)
    r.step(40)
    _, ux, uy = m.fields()
    _, ux0, uy0 = r.fields()
    assert vel_err(ux, uy, ux0, uy0) < f64_field_tol(np.max(np.abs(ux0)))
    assert rel_err(m.markers(), r.markers()) < 1e-12
    assert np.array_equal(m.bonds(), r.bonds())
    # mixed tilings: graph of member graphs, same bits as the batched run
    members = [lbib.Simulation(w, tiling=t) for w, t in zip(wls, [(1, 4), (1, 2), (1, 4)])]
    e2 = lbib.lbib_ensemble_create([s.ctx for s in members])
    for s in members:
        s.owned_by_ensemble = True
    assert lbib.lbib_ensemble_form(e2) == 0
    lbib.lbib_ensemble_step(e2, 40)
    lbib.lbib_ensemble_sync(e2)
    for k in (0, 2):
        assert np.array_equal(members[k].markers(), ens.members[k].markers())
        assert np.array_equal(members[k].populations(), ens.members[k].populations())
    lbib.lbib_ensemble_destroy(e2)
    for s in members:
        s.ctx = None
    ens.close()


def test_ensemble_groups_are_refused_outside_their_range():
    from paper_1907_00080_gb300 import lbib
    wls = small_ensemble(3, "f32", seed=2)
    ens = lbib.Ensemble(wls, tiling=(1, 4))
    for bad in (0, 4):
        with pytest.raises(lbib.LbibError):
            ens.set_groups(bad)
    ens.close()
    members = [lbib.Simulation(w, tiling=t) for w, t in zip(wls, [(1, 4), (1, 2), (1, 4)])]
    e2 = lbib.lbib_ensemble_create([s.ctx for s in members])
    for s in members:
        s.owned_by_ensemble = True
    with pytest.raises(lbib.LbibError):
        lbib.lbib_ensemble_set_groups(e2, 1)
    assert lbib.lbib_ensemble_groups(e2) == 0
    lbib.lbib_ensemble_destroy(e2)
    for s in members:
        s.ctx = None


def test_benchmark_ensemble_takes_its_tuned_shape():
    """The 64-member ensemble of the benchmark: the shape stored by the
    autotuner (or tuned on the spot) gives the batched form, and the ensemble
    steps with it."""
    from paper_1907_00080_gb300 import lbib, tuning
    wls = inputs.capillary_ensemble(64, seed=0, precision="f32")
    (tiling, groups), tuned = tuning.ensemble_shape(wls)
    if tuned is None:
        assert tuning.ENSEMBLE_TABLE[tuning.ensemble_key(wls)] == (tiling, groups)
    else:
        assert (tiling, groups) == min(tuned, key=tuned.get)
    ens = lbib.Ensemble(wls, tiling=tiling)
    assert ens.form == 1
    ens.set_groups(groups)
    assert ens.groups == groups and ens.launches_per_step == 3 * groups
    ens.step(20)
    ens.sync()
    for m in ens.members[:3]:
        assert lbib.lbib_step_count(m.ctx) == 20
        assert lbib.lbib_get_tiling(m.ctx) == tuple(tiling)
    ens.close()


def test_benchmark_ensemble_members_match_the_oracle():
    """The full 64-member ensemble (8.03 M nodes, 138,600 markers) in the shape
    the benchmark times: after 40 steps, the shortest, a middle and the longest
    member against the oracle at the FP32 bounds (velocity within 1e-5 of the
    speed scale, markers within 1e-5 lu, bond sets bit-exact)."""
    from paper_1907_00080_gb300 import lbib, tuning
    wls = inputs.capillary_ensemble(64, seed=0, precision="f32")
    (tiling, groups), _ = tuning.ensemble_shape(wls)
    ens = lbib.Ensemble(wls, tiling=tiling)
    assert ens.form == 1
    ens.set_groups(groups)
    ens.step(40)
    ens.sync()
    order = np.argsort([wl.nx for wl in wls])
    for i in (order[0], order[len(order) // 2], order[-1]):
        wl, m = wls[i], ens.members[i]
        r = make_oracle(wl)
        r.step(40)
        _, ux, uy = m.fields()
        _, ux0, uy0 = r.fields()
        assert vel_err(ux, uy, ux0, uy0) < 1e-5, (wl.name, vel_err(ux, uy, ux0, uy0))
        assert np.max(np.abs(m.markers() - r.markers())) < 1e-5
        assert np.array_equal(m.bonds(), r.bonds())
    ens.close()


def test_ensemble_state_calls_match_the_member_calls():
    """lbib_ensemble_write_state / lbib_ensemble_read_markers (all members, one
    wait) give the same bits as the per-member write and read calls."""
    from paper_1907_00080_gb300 import lbib
    wls = small_ensemble(3, "f32", seed=13)
    runs = []
    for batched_io in (False, True):
        ens = lbib.Ensemble(wls, tiling=(1, 0))
        ens.step(5)
        ens.sync()
        f = [np.ascontiguousarray(m.populations() * (1 + 1e-3 * k)) for k, m in enumerate(ens.members)]
        x = [np.ascontiguousarray(m.markers() + 0.01 * (k + 1)) for k, m in enumerate(ens.members)]
        if batched_io:
            ens.write_state(f=f, xy=x, xy_prev=x)
        else:
            for m, fk, xk in zip(ens.members, f, x):
                lbib.lbib_write_populations(m.ctx, fk)
                lbib.lbib_write_markers(m.ctx, xk, xk)
        ens.step(7)
        ens.sync()
        out = [np.zeros((m.nv, 2)) for m in ens.members]
        if batched_io:
            ens.read_markers(out)
        else:
            for m, o in zip(ens.members, out):
                lbib.lbib_read_markers(m.ctx, -1, o)
        runs.append((out, [m.populations() for m in ens.members]))
        ens.close()
    for a, b in zip(runs[0][0], runs[1][0]):
        assert np.array_equal(a, b)
    for a, b in zip(runs[0][1], runs[1][1]):
        assert np.array_equal(a, b)

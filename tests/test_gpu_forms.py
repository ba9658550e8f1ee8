"""GPU tests of the precision form: populations stored as shifted deviations
(d_i 2^k) in FP16 or BF16 with FP32 arithmetic, on the fine capillary
(2000 x 667 at dx = 15 nm, 4 red cells x 1700 markers, 3 carriers x 210).

The FP64 GPU run is first tied to the oracle on this workload; the 16-bit and
FP32 storage forms are then measured against that FP64 run.  16-bit storage
is not expected to match FP64 to a parity tolerance: the bounds below state
its error (about 4x the values measured on a GB300: FP32 1.8e-5, FP16 2.5e-4,
BF16 2.1e-3 relative Linf velocity after 1000 steps; markers 1.8e-8, 6.1e-7,
5.1e-6 lattice units)."""
import numpy as np
import pytest

from helpers import f64_field_tol, make_oracle, rel_err, vel_err
from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu

# stated error after 1000 steps against FP64: velocity (Linf and L2, relative
# to the FP64 field) and marker positions (Linf, lattice units)
BOUNDS = {"f32": dict(u_linf=1e-4, u_l2=5e-5, x=1e-7),
          "f16": dict(u_linf=1e-3, u_l2=5e-4, x=3e-6),
          "bf16": dict(u_linf=1e-2, u_l2=5e-3, x=2e-5)}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def test_fine_capillary_fp64_matches_oracle():
    from paper_1907_00080_gb300 import lbib
    wl = inputs.fine_capillary_2000x667("f64", bonds="stress")
    s, r = lbib.Simulation(wl), make_oracle(wl)
    s.step(10)
    r.step(10)
    _, ux, uy = s.fields()
    _, ux0, uy0 = r.fields()
    assert vel_err(ux, uy, ux0, uy0) < f64_field_tol(np.max(np.abs(ux0)))
    assert rel_err(s.markers(), r.markers()) < 1e-12
    assert np.array_equal(s.bonds(), r.bonds())
    s.close()


@pytest.fixture(scope="module")
def fine_runs():
    """1000 steps of the fine capillary in every storage form."""
    from paper_1907_00080_gb300 import lbib
    out = {}
    for prec in ("f64", "f32", "f16", "bf16"):
        s = lbib.Simulation(inputs.fine_capillary_2000x667(prec))
        s.step(1000)
        _, ux, uy = s.fields()
        mass, areas = s.diagnostics()
        out[prec] = dict(ux=ux, uy=uy, x=s.markers(), bonds=s.bonds(), mass=mass, areas=areas,
                         k=lbib.lbib_storage_scale_exponent(s.ctx), f=s.populations())
        s.close()
    return out


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_storage_form_error_against_fp64(fine_runs, prec):
    ref, got = fine_runs["f64"], fine_runs[prec]
    du = np.hypot(got["ux"] - ref["ux"], got["uy"] - ref["uy"])
    um = np.hypot(ref["ux"], ref["uy"])
    b = BOUNDS[prec]
    assert du.max() / um.max() < b["u_linf"], du.max() / um.max()
    assert np.sqrt((du ** 2).sum() / (um ** 2).sum()) < b["u_l2"]
    assert np.max(np.abs(got["x"] - ref["x"])) < b["x"]
    assert np.array_equal(got["bonds"], ref["bonds"])
    # the invariants stay FP64 reductions: mass to the storage rounding, areas
    assert abs(got["mass"] - ref["mass"]) / ref["mass"] < (1e-6 if prec == "f32" else 1e-4)
    np.testing.assert_allclose(got["areas"], ref["areas"], rtol=1e-6)


def test_fp16_scale_keeps_headroom(fine_runs):
    """FP16 stores d_i 2^k with k chosen from the Poiseuille peak deviation
    w_1 3 u_max = u_max / 3 (so that it sits near 2^12): the largest stored
    value must stay well inside the FP16 range (65504) and above its normal
    range (6.1e-5)."""
    r = fine_runs["f16"]
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    dmax = np.max(np.abs(r["f"] - w))
    scaled = dmax * 2.0 ** r["k"]
    assert 2 ** 10 < scaled < 2 ** 14
    assert np.all(np.isfinite(r["f"]))


@pytest.fixture(scope="module")
def adhering_runs():
    """1000 steps of the fine capillary with its carriers released 1 lu from a
    wall and the paper's bond cut-off, in every storage form."""
    from paper_1907_00080_gb300 import lbib
    out = {}
    for prec in ("f64", "f32", "f16", "bf16"):
        s = lbib.Simulation(inputs.fine_capillary_adhering(prec))
        s.step(1000)
        out[prec] = dict(x=s.markers(), bonds=s.bonds())
        s.close()
    return out


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_storage_forms_keep_the_bonds(adhering_runs, prec):
    """Bonds form in 1000 steps; FP32 storage keeps the FP64 run's bond set
    (its bond decisions fall back to FP64 near ties), the 16-bit forms differ
    from it on at most 5 % of the bonded ligands (measured: see the bench's
    precision form)."""
    ref, got = adhering_runs["f64"], adhering_runs[prec]
    nb = int((ref["bonds"] >= 0).sum())
    assert nb >= 10
    diff = int((got["bonds"] != ref["bonds"]).sum())
    print("bonds", nb, "ligands with another bond", diff, "marker err", np.max(np.abs(got["x"] - ref["x"])))
    if prec == "f32":
        assert diff == 0
    else:
        assert diff <= 0.05 * nb

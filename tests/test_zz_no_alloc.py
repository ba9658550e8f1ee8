"""GPU test of lbib_population_mass_noalloc, the allocation-free mass reduction
(a library service with no counterpart in the paper).  It must agree with the
mass that lbib_diagnostics reports for the same populations, on two calls in a
row, both after the rest of the suite and alone in a fresh process.  Collected
last on purpose (file name)."""
import os
import subprocess
import sys

import pytest

from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REL_TOL = 1e-12  # FP64 sums of the same values in two orders


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def check_against_diagnostics(wl, precision, steps=12):
    """Step the workload, read its populations into a device buffer, and compare
    two consecutive allocation-free mass calls with lbib_diagnostics."""
    import torch
    from paper_1907_00080_gb300 import lbib
    sim = lbib.Simulation(wl, precision=precision)
    try:
        sim.step(steps)
        mass_ref, _ = lbib.lbib_diagnostics(sim.ctx)
        n_nodes = wl.nx * wl.ny
        f = torch.empty(9 * n_nodes, dtype=torch.float64, device="cuda")
        lbib.lbib_read_populations(sim.ctx, f.data_ptr(), on_device=1)
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        torch.cuda.synchronize()
        for k in range(2):
            st = lbib.lbib_population_mass_noalloc(f.data_ptr(), n_nodes, out[k:].data_ptr(), stream)
            assert st == lbib.LBIB_OK, st
        torch.cuda.synchronize()
        m = out.cpu().numpy()
        for v in m:
            assert abs(v - mass_ref) <= REL_TOL * abs(mass_ref), (v, mass_ref)
        assert m[0] == m[1]  # fixed summation order
        return m, mass_ref
    finally:
        sim.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_mass_matches_diagnostics_capsule(precision):
    check_against_diagnostics(inputs.capsule_128x32(precision), precision)


def test_noalloc_mass_matches_diagnostics_capillary_640x160():
    check_against_diagnostics(inputs.coarse_capillary_640x160("f32"), "f32", steps=20)


def test_noalloc_mass_edges_and_errors():
    import torch
    from paper_1907_00080_gb300 import lbib
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    # n_nodes = 0 gives 0
    assert lbib.lbib_population_mass_noalloc(0, 0, out.data_ptr()) == lbib.LBIB_OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # a ragged size over several blocks of the first kernel, against an exact
    # integer sum (values are small integers, so every order is exact)
    n_nodes = 16384 * 3 // 9 + 5
    vals = torch.arange(9 * n_nodes, dtype=torch.float64, device="cuda").remainder_(17.0)
    assert lbib.lbib_population_mass_noalloc(vals.data_ptr(), n_nodes, out.data_ptr()) == lbib.LBIB_OK
    torch.cuda.synchronize()
    assert out.item() == float(vals.sum().item())
    # rejected without a launch: NULL output, negative or too large n_nodes,
    # host memory, misaligned pointer
    assert lbib.lbib_population_mass_noalloc(vals.data_ptr(), n_nodes, 0) == lbib.LBIB_E_INVALID
    assert lbib.lbib_population_mass_noalloc(vals.data_ptr(), -1, out.data_ptr()) == lbib.LBIB_E_INVALID
    assert lbib.lbib_population_mass_noalloc(vals.data_ptr(), 7456541, out.data_ptr()) == lbib.LBIB_E_INVALID
    host = torch.zeros(9, dtype=torch.float64)
    assert lbib.lbib_population_mass_noalloc(host.data_ptr(), 1, out.data_ptr()) == lbib.LBIB_E_INVALID
    assert lbib.lbib_population_mass_noalloc(vals.data_ptr() + 4, 1, out.data_ptr()) == lbib.LBIB_E_INVALID
    torch.cuda.synchronize()
    assert out.item() == float(vals.sum().item())  # untouched by the rejected calls


def test_noalloc_mass_in_a_fresh_process():
    code = ("import sys; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
            "import test_zz_no_alloc as t\n"
            "from paper_1907_00080_gb300 import inputs, lbib\n"
            "lbib.load()\n"
            "m, ref = t.check_against_diagnostics(inputs.capsule_128x32('f64'), 'f64')\n"
            "print('fresh-process mass', m[0], m[1], ref)\n") % (ROOT, os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process mass" in r.stdout

"""GPU edge cases of size: lattices whose population buffers hold more than
2^31 values (64-bit indexing in every kernel) and lattices taller than one
launch grid's 65535 rows, checked through a property that holds at any size:
with tau = 1 the discrete Poiseuille state is a fixed point, so after a few
steps the velocity equals its closed form u(y) = G/(2 nu)(y + 1/2)(NY - 1/2 - y)
+ G/4 (sampled rows, including the last ones, read on the device)."""
import numpy as np
import pytest

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


def poiseuille(nx, ny, prec):
    g = inputs.body_force_for(0.02, ny)
    wl = inputs.Workload(name="poiseuille", nx=nx, ny=ny, body_force=(g, 0.0), walls=1, init="poiseuille",
                         precision=prec, membranes=[], receptors=None)
    return wl, g


def check_profile(sim, nx, ny, g, rows, tol):
    """u_x of the sampled rows (every x) against the closed form, read into a
    device buffer (the full field does not go through the host)."""
    import torch
    from paper_1907_00080_gb300 import lbib
    ux = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    lbib.lbib_read_fields(sim.ctx, None, ux.data_ptr(), None, on_device=1)
    torch.cuda.synchronize()
    nu = 1.0 / 6.0
    for y in rows:
        ref = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y) + 0.25 * g
        got = ux[y].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * 0.02, (y, np.max(np.abs(got - ref)))


@pytest.mark.parametrize("prec,tiling,tol", [("f32", None, 1e-5), ("f32", (4, 1), 1e-5), ("f16", None, 2e-3)])
def test_buffers_beyond_2_pow_31_values(prec, tiling, tol):
    """16384 x 16384: 9 N = 2.4e9 populations per buffer (9.7 GB in FP32)."""
    from paper_1907_00080_gb300 import lbib
    nx = ny = 16384
    wl, g = poiseuille(nx, ny, prec)
    sim = lbib.Simulation(wl, tiling=tiling)
    sim.step(3)
    check_profile(sim, nx, ny, g, [0, 1, ny // 2, ny - 2, ny - 1], tol)
    sim.close()


def test_lattice_taller_than_one_grid():
    """8 x 70000: the row-tile form takes more rows per block so that the grid
    stays within 65535 blocks; a shape that cannot is refused."""
    from paper_1907_00080_gb300 import lbib
    nx, ny = 8, 70000
    wl, g = poiseuille(nx, ny, "f32")
    sim = lbib.Simulation(wl)
    with pytest.raises(lbib.LbibError) as ei:
        lbib.lbib_set_tiling(sim.ctx, 1, 1)
    assert ei.value.status == lbib.LBIB_E_INVALID
    sim.step(3)
    assert sim.tiling[1] >= 2
    check_profile(sim, nx, ny, g, [0, ny // 2, ny - 1], 1e-5)
    sim.close()

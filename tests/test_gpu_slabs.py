"""GPU tests of the x-slab decomposition of one lattice (lbib_slabs_*): the
lattice split into sub-domains with two ghost columns each, advanced on one
GPU with the halo exchange after every step, reproduces the undivided
lattice's populations bit for bit (random initial populations, walls and
periodic y, body force, moving walls, all precisions, both kernel forms, even
and uneven slabs); mismatched slabs are refused."""
import numpy as np
import pytest

from helpers import W9
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


def lb():
    from paper_1907_00080_gb300 import lbib
    return lbib


def lattice(nx, ny, prec, walls=1, tau=0.8, uw=(0.0, 0.0)):
    # 16-bit storage picks its scale from the body force, whose y part counts
    # the lattice's width: the slabs (narrower) would get another scale, so the
    # 16-bit cases drive along x only
    g = (2e-6, -5e-7) if prec in ("f64", "f32") else (2e-6, 0.0)
    return inputs.Workload(name="lat", nx=nx, ny=ny, tau=tau, body_force=g, walls=walls,
                           init="rest", precision=prec, membranes=[], receptors=None, wall_velocity=uw)


def compare(wl, widths, prec, tiling=None, steps=(1, 36), seed=1):
    L = lb()
    # 16-bit storage: deviations within the range its scale leaves (the
    # scale follows the body force)
    amp = 3e-2 if prec in ("f64", "f32") else 1e-4
    f0 = inputs.random_populations(wl.nx, wl.ny, W9, seed=seed, amp=amp)
    whole = L.Simulation(wl, precision=prec)
    whole.set_populations(f0)
    parts = L.Slabs(wl, widths, precision=prec, tiling=tiling, f0=f0)
    np.testing.assert_array_equal(parts.populations(), whole.populations())
    for k in steps:
        whole.step(k)
        parts.step(k)
        np.testing.assert_array_equal(parts.populations(), whole.populations())
    rho, ux, uy = parts.fields()
    rho0, ux0, uy0 = whole.fields()
    np.testing.assert_array_equal(ux, ux0)
    parts.close()
    whole.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("walls", [1, 0])
def test_three_even_slabs_match_the_whole_lattice(prec, walls):
    compare(lattice(90, 20, prec, walls=walls), [30, 30, 30], prec)


def test_uneven_slabs_and_the_persistent_form():
    """Slab widths 30, 34, 26 (ghosts included: 32, 36, 28, multiples of the
    16-byte halo) in the persistent bulk-copy form of the fused kernel."""
    compare(lattice(90, 24, "f32"), [30, 34, 26], "f32", tiling=(2, 0))


def test_slabs_with_moving_walls():
    compare(lattice(96, 16, "f64", tau=1.0, uw=(-0.003, 0.01)), [24, 40, 32], "f64")


def test_many_narrow_slabs():
    compare(lattice(64, 12, "f32"), [4] * 16, "f32", steps=(1, 20))


def test_mismatched_slabs_are_refused():
    import torch
    L = lb()
    st = torch.cuda.Stream()
    a = L.Simulation(lattice(12, 8, "f32"), cuda_stream=st.cuda_stream)
    b = L.Simulation(lattice(12, 10, "f32"), cuda_stream=st.cuda_stream)  # other rows
    c = L.Simulation(lattice(12, 8, "f32"))  # its own stream
    wl_m = lattice(40, 16, "f32")
    wl_m.membranes = [inputs.Membrane(xy=inputs.circle(20.0, 8.0, 4.0, 24), ks=0.05, kb=0.0, ka=0.1)]
    d = L.Simulation(wl_m, cuda_stream=st.cuda_stream)
    for pair in ([a, b], [a, c], [a, d], [a]):
        with pytest.raises(L.LbibError) as ei:
            L.lbib_slabs_create([s.ctx for s in pair])
        assert ei.value.status == L.LBIB_E_INVALID
    for s in (a, b, c, d):
        s.close()

"""GPU tests of the tile-shape autotuner: it times every candidate shape of the
fused kernel through the C ABI and returns one of them, and the shape it
returns gives the same bits as the library's default shape."""
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


@pytest.mark.parametrize("precision", ["f32", "f16"])
def test_autotune_times_every_candidate(precision):
    from paper_1907_00080_gb300 import lbib, tuning
    wl = inputs.capsule_128x32(precision)
    best, res = tuning.autotune(lambda t: lbib.Simulation(wl, tiling=t), precision, wl.nx, steps=16, reps=1)
    assert set(res) == set(tuning.candidates(precision, wl.nx))
    assert best in res and all(v > 0 for v in res.values())
    # the chosen shape computes what the default shape computes
    a, b = lbib.Simulation(wl, tiling=best), lbib.Simulation(wl)
    a.step(20)
    b.step(20)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.markers(), b.markers())
    a.close()
    b.close()

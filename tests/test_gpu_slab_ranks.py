"""GPU tests of the one-slab-per-rank decomposition: two or three processes,
each holding one x-slab context (all on cuda:0 here: one GPU per test run;
their kernels never wait on one another, the halo goes through the host over
gloo after every step), reproduce the undivided lattice's populations bit for
bit; the face copies are refused on contexts with membranes."""
import os
import socket
import sys

import numpy as np
import pytest

from helpers import W9
from paper_1907_00080_gb300 import inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_00080_gb300 import build, lbib
    build.build()
    lbib.load()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def lattice(nx, ny, prec, walls=1):
    # 16-bit storage picks its scale from the body force, whose y part counts
    # the lattice's width: the 16-bit cases drive along x only
    g = (2e-6, -5e-7) if prec in ("f64", "f32") else (2e-6, 0.0)
    return inputs.Workload(name="lat", nx=nx, ny=ny, tau=0.8, body_force=g, walls=walls,
                           init="rest", precision=prec, membranes=[], receptors=None)


def initial(wl, prec, seed=3):
    amp = 3e-2 if prec in ("f64", "f32") else 1e-4
    return inputs.random_populations(wl.nx, wl.ny, W9, seed=seed, amp=amp)


def _rank(rank, world, port, wl, prec, steps, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1907_00080_gb300 import lbib
    from paper_1907_00080_gb300.slab_ranks import RankSlab
    lbib.load()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rs = RankSlab(wl, rank, world, precision=prec, f0=initial(wl, prec))
        rs.step(steps)
        q.put((rank, rs.interior()))
        rs.close()
    finally:
        dist.destroy_process_group()


def run_ranks(wl, prec, world, steps):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, wl, prec, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return np.concatenate([got[r] for r in range(world)], axis=2)


@pytest.mark.parametrize("prec,walls,world,nx", [("f32", 1, 2, 96), ("f64", 0, 3, 101),
                                                 ("f16", 1, 2, 128), ("bf16", 1, 3, 132)])
def test_ranks_match_the_undivided_lattice(prec, walls, world, nx):
    from paper_1907_00080_gb300 import lbib
    wl = lattice(nx, 40, prec, walls)
    steps = 37
    whole = lbib.Simulation(wl, precision=prec)
    whole.set_populations(initial(wl, prec))
    whole.step(steps)
    ref = whole.populations()
    whole.close()
    np.testing.assert_array_equal(run_ranks(wl, prec, world, steps), ref)


def test_faces_refused_with_membranes():
    from paper_1907_00080_gb300 import lbib
    wl = inputs.capillary(precision="f32")
    s = lbib.Simulation(wl)
    import torch
    buf = torch.empty(3 * wl.ny * 4, dtype=torch.uint8)
    with pytest.raises(lbib.LbibError):
        lbib.lbib_slab_face(s.ctx, 0, 1, buf.data_ptr(), 0)
    s.close()

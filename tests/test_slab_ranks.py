"""CPU checks of the one-slab-per-rank decomposition (gloo, world sizes 1 to
3): the ring delivers each face to the right ghost column, and a lattice step
with the fused kernel's storage convention (the buffer holds post-collision
populations, a step pulls f_i(x - c_i) and collides) run as slabs on separate
ranks equals the undivided run bit for bit.  The step here is a numpy
stand-in for the device slab; the device path is checked in
test_gpu_slab_ranks.py."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
PLUS, MINUS = [1, 5, 8], [3, 6, 7]


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpySlab:
    """D2Q9 BGK with a constant body-force source, periodic in x and y: the
    same post-collision storage as the device slab (a step is pull, then
    collide), arithmetic identical node by node wherever the node sits."""
    elem_bytes = 8

    def __init__(self, f, tau=0.8, g=1e-5):
        self.f, self.tau, self.g = f.copy(), tau, g

    def step(self, n=1):
        for _ in range(n):
            p = np.stack([np.roll(np.roll(self.f[i], cy, axis=0), cx, axis=1) for i, (cx, cy) in enumerate(C)])
            rho = p.sum(axis=0)
            ux = sum(p[i] * C[i][0] for i in range(9)) / rho
            uy = sum(p[i] * C[i][1] for i in range(9)) / rho
            for i, (cx, cy) in enumerate(C):
                cu = 3 * (cx * ux + cy * uy)
                feq = W[i] * rho * (1 + cu + 0.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
                p[i] += -(p[i] - feq) / self.tau + 3 * W[i] * cx * self.g
            self.f = p

    def face(self, side, out, buf):
        dirs = MINUS if (side == 0) == (out == 1) else PLUS
        nx = self.f.shape[2]
        col = (1 if side == 0 else nx - 2) if out else (0 if side == 0 else nx - 1)
        a = buf.numpy().view(np.float64).reshape(3, -1)
        if out:
            a[:] = self.f[dirs, :, col]
        else:
            self.f[dirs, :, col] = a

    def interior(self):
        return self.f[:, :, 1:-1].copy()


def initial(nx, ny, seed=5):
    rng = np.random.default_rng(seed)
    return W[:, None, None] * (1 + 0.05 * rng.standard_normal((9, ny, nx)))


def slab_of(f0, rank, world):
    from paper_1907_00080_gb300.slab_ranks import slab_widths
    nx = f0.shape[2]
    widths = slab_widths(nx, world)
    x0, w = sum(widths[:rank]), widths[rank]
    return NumpySlab(f0[:, :, [(x0 - 1 + j) % nx for j in range(w + 2)]])


def lattice_wl(nx, ny):
    from paper_1907_00080_gb300.inputs import Workload
    return Workload(name="numpy_ring", nx=nx, ny=ny, precision="f64", tau=0.8, body_force=(1e-5, 0.0),
                    walls=0, membranes=[])


def _rank(rank, world, port, nx, ny, steps, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1907_00080_gb300.slab_ranks import HaloRing, RankSlab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        # the ring alone: rank-coded faces reach the right ghost columns
        ring = HaloRing(rank, world)
        left = torch.full((6,), 10 * rank + 1, dtype=torch.uint8)
        right = torch.full((6,), 10 * rank + 2, dtype=torch.uint8)
        in_l, in_r = ring.exchange(left, right)
        faces = (int(in_l[0]), int(in_r[0]))
        rs = RankSlab(lattice_wl(nx, ny), rank, world, slab=slab_of(initial(nx, ny), rank, world))
        rs.step(steps)
        q.put((rank, faces, rs.x0, rs.interior()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nx", [(2, 24), (3, 25)])
def test_ranks_match_undivided(world, nx):
    import torch.multiprocessing as mp
    from paper_1907_00080_gb300.slab_ranks import slab_widths
    ny, steps = 9, 30
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, nx, ny, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, faces, x0, f = q.get(timeout=180)
        got[r] = (faces, x0, f)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        # left ghost from the left neighbour's right face, right ghost from the right's left face
        assert got[r][0] == (10 * ((r - 1) % world) + 2, 10 * ((r + 1) % world) + 1)
    ref = NumpySlab(initial(nx, ny))
    ref.step(steps)
    whole = np.concatenate([got[r][2] for r in range(world)], axis=2)
    widths = slab_widths(nx, world)
    assert [got[r][1] for r in range(world)] == [sum(widths[:r]) for r in range(world)]
    assert np.array_equal(whole, ref.f)


def test_single_rank_wraps_onto_itself():
    from paper_1907_00080_gb300.slab_ranks import RankSlab
    nx, ny = 12, 7
    rs = RankSlab(lattice_wl(nx, ny), 0, 1, slab=slab_of(initial(nx, ny), 0, 1))
    rs.step(20)
    ref = NumpySlab(initial(nx, ny))
    ref.step(20)
    assert np.array_equal(rs.interior(), ref.f)


def test_widths_and_refusals():
    from paper_1907_00080_gb300.slab_ranks import slab_widths
    assert slab_widths(10, 3) == [4, 3, 3]
    assert slab_widths(8, 8) == [1] * 8
    with pytest.raises(ValueError):
        slab_widths(3, 4)


def test_stepping_without_the_exchange_breaks_the_match():
    """The stand-in is sensitive to the halo: slabs stepped with stale ghost
    columns drift from the undivided run, so the match above is not vacuous."""
    nx, ny = 24, 9
    f0 = initial(nx, ny)
    parts = [slab_of(f0, r, 2) for r in range(2)]
    for p in parts:
        p.step(10)
    ref = NumpySlab(f0)
    ref.step(10)
    assert not np.array_equal(np.concatenate([p.interior() for p in parts], axis=2), ref.f)

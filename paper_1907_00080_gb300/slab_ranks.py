"""One x-slab of the lattice per process (rank), the halo moved between ranks
by the host over torch.distributed after every step.

The lattice-only step (Sec. 2.1: BGK collision with the Guo force, pull
streaming) needs, at the two edge columns of a slab, post-collision values
that only the neighbouring slabs hold: the three populations moving in +x
(1, 5, 8) of the left neighbour's last interior column and the three moving
in -x (3, 6, 7) of the right neighbour's first.  Each slab is a context of
width W + 2 whose columns 0 and W + 1 are ghosts.  After each step a rank
copies its two leaving faces out of the device (lbib_slab_face), sends them to
its neighbours, receives the two entering faces and writes them into its
ghost columns before the next step.  The ring is periodic in x (rank 0's left
neighbour is the last rank), as the undivided lattice is.  The exchange is a
point-to-point send and receive per face (no collective); with one rank the
faces wrap onto the rank itself.

Only the lattice is decomposed: membranes couple to every node their kernel
support touches, and a membrane crossing a slab edge would need its markers'
forces and velocities summed across ranks, which this module does not do
(contexts with membranes are refused by lbib_slab_face).

Marshalling and transport only: the step and the face copies run in the
library's kernels and copies.
"""
import dataclasses

import numpy as np

from . import lbib

# point-to-point tags: faces moving to the right neighbour / to the left
TAG_RIGHTWARD, TAG_LEFTWARD = 0x1B1, 0x1B2


def slab_widths(nx, world):
    """Near-equal interior widths adding up to nx (the first nx % world
    slabs one column wider)."""
    if world < 1 or nx < world:
        raise ValueError("need at least one column per rank")
    q, r = divmod(nx, world)
    return [q + (1 if k < r else 0) for k in range(world)]


class HaloRing:
    """Moves faces around a periodic ring of ranks over the default
    torch.distributed process group (host tensors: gloo)."""

    def __init__(self, rank, world):
        self.rank, self.world = rank, world
        self.left, self.right = (rank - 1) % world, (rank + 1) % world

    def exchange(self, out_left, out_right):
        """out_left / out_right: this rank's leaving faces (to the left / right
        neighbour).  Returns (in_left, in_right): the faces entering its left
        ghost column (the left neighbour's right face) and its right ghost
        column (the right neighbour's left face)."""
        if self.world == 1:
            return out_right.clone(), out_left.clone()
        import torch.distributed as dist
        in_left, in_right = out_right.new_empty(out_right.shape), out_left.new_empty(out_left.shape)
        reqs = [dist.isend(out_right, self.right, tag=TAG_RIGHTWARD),
                dist.isend(out_left, self.left, tag=TAG_LEFTWARD),
                dist.irecv(in_left, self.left, tag=TAG_RIGHTWARD),
                dist.irecv(in_right, self.right, tag=TAG_LEFTWARD)]
        for r in reqs:
            r.wait()
        return in_left, in_right


class DeviceSlab:
    """A slab context on this rank's GPU: step and face copies through the
    C-ABI.  Face buffers are host tensors of 3 x NY stored elements."""

    def __init__(self, wl, precision=None, tiling=None, f0=None):
        self.sim = lbib.Simulation(wl, precision=precision, tiling=tiling)
        if f0 is not None:
            self.sim.set_populations(f0)
        self.ny = wl.ny
        self.elem_bytes = lbib.lbib_storage_bytes(self.sim.ctx)

    def step(self, n=1):
        self.sim.step(n)

    def face(self, side, out, buf):
        lbib.lbib_slab_face(self.sim.ctx, side, out, buf.data_ptr(), 0)

    def interior(self):
        return self.sim.populations()[:, :, 1:-1]

    def close(self):
        self.sim.close()


class RankSlab:
    """This rank's slab of a lattice-only workload ``wl`` split over ``world``
    ranks along x.  f0 (9, NY, NX), optional: the undivided lattice's initial
    populations (each rank takes its columns and the two beside them).
    ``slab`` replaces the device slab (an object with step, face, interior and
    elem_bytes); ``ring`` the transport."""

    def __init__(self, wl, rank, world, precision=None, tiling=None, f0=None, ring=None, slab=None):
        if wl.membranes:
            raise ValueError("slabs carry the lattice only")
        widths = slab_widths(wl.nx, world)
        self.rank, self.world = rank, world
        self.x0, self.width = sum(widths[:rank]), widths[rank]
        self.ring = ring or HaloRing(rank, world)
        if slab is None:
            sub = dataclasses.replace(wl, nx=self.width + 2, name="%s_rank%d" % (wl.name, rank))
            cols = None
            if f0 is not None:
                cols = np.asarray(f0)[:, :, [(self.x0 - 1 + j) % wl.nx for j in range(self.width + 2)]]
            slab = DeviceSlab(sub, precision=precision, tiling=tiling, f0=cols)
        self.slab = slab
        import torch
        nbytes = 3 * wl.ny * slab.elem_bytes
        pin = isinstance(slab, DeviceSlab)
        self.out = [torch.empty(nbytes, dtype=torch.uint8, pin_memory=pin) for _ in range(2)]
        self.steps = 0

    def step(self, n=1):
        for _ in range(int(n)):
            self.slab.step(1)
            self.slab.face(0, 1, self.out[0])
            self.slab.face(1, 1, self.out[1])
            in_left, in_right = self.ring.exchange(self.out[0], self.out[1])
            self.slab.face(0, 0, in_left)
            self.slab.face(1, 0, in_right)
            self.steps += 1

    def interior(self):
        """(9, NY, W): this rank's columns x0 .. x0 + W - 1"""
        return self.slab.interior()

    def close(self):
        close = getattr(self.slab, "close", None)
        if close:
            close()

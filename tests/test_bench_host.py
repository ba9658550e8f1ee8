"""CPU checks of bench.py's roofline bookkeeping: every DRAM-traffic key the
JSON line looks up has a line in the ncu summaries under profiles/, each of
those summaries states the ncu command it came from, and the count of nodes in
flagged force tiles equals a brute-force count on small lattices."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1907_00080_gb300 import inputs, tuning  # noqa: E402


def test_traffic_lines_for_every_reported_kernel():
    t = bench.ncu_traffic()
    wls = inputs.capillary_ensemble(64)
    (vec, ty), _groups = tuning.ENSEMBLE_TABLE[tuning.ensemble_key(wls)]
    for k in ("k_forces_batch", "fused_batch", "k_advance_batch"):
        assert "%s:ensemble64_f32:%d,%d" % (k, vec, ty) in t, k
    for k in ("k_forces", "fused", "k_advance"):
        assert "%s:capillary_640x160_f32" % k in t, k
    # the probes: FP32 in the library's default form for 8192 x 2048, FP16 at (4, 0)
    assert "fused:probe_8192x1024_f32:2,0" in t
    assert "fused:probe_8192x1024_f16:4,0" in t
    # per launch: more than the flags and less than a few times the populations
    for key, v in t.items():
        assert 1e5 < v < 2e9, key


def test_each_traffic_summary_states_its_command():
    d = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name)) as fh:
            text = fh.read()
        if "traffic_per_launch:" in text:
            assert "ncu --clock-control none" in text, name


def brute_flagged(nx, ny, walls, xy, tile_w):
    """nodes of the tiles that hold a node of some marker's 3 x 3 stencil,
    one node and one marker at a time"""
    tiles = set()
    for x, y in xy:
        i0, j0 = int(np.floor(x + 0.5)), int(np.floor(y + 0.5))
        for dy in (-1, 0, 1):
            j = j0 + dy
            if walls and not 0 <= j < ny:
                continue
            j %= ny
            for dx in (-1, 0, 1):
                i = (i0 + dx) % nx
                tiles.add((j, i // tile_w))
    flagged = 0
    for j in range(ny):
        for i in range(nx):
            if (j, i // tile_w) in tiles:
                flagged += 1
    return flagged


@pytest.mark.parametrize("nx,ny,walls", [(70, 9, 1), (64, 8, 0), (33, 5, 1)])
def test_flagged_nodes_match_brute_force(nx, ny, walls):
    rng = np.random.default_rng(nx + ny)
    # markers anywhere, at the periodic ends and next to (or on) the walls
    xy = np.column_stack([rng.uniform(-0.5, nx - 0.5, 40), rng.uniform(-0.5, ny - 0.5, 40)])
    xy = np.vstack([xy, [[0.1, 0.2], [nx - 0.6, ny - 0.6], [nx / 2, 0.0], [31.6, ny / 2]]])
    wl = inputs.Workload(name="flag", nx=nx, ny=ny, walls=walls)
    # the fused kernels' force tiles are 32 nodes of one row
    assert bench.flagged_nodes(wl, xy) == brute_flagged(nx, ny, walls, xy, 32)

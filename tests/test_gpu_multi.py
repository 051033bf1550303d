"""GPU parity of batched multi-source BFS (64-bit lane masks) against the oracle.

Every lane's level row must equal the oracle's levels for its root bit-exactly;
parent rows (minimum-id parent mode) must equal the oracle's min_parent.
"""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = pytest.mark.gpu


def _run(bfs, g, roots, want_parent=False, opts=None):
    import torch
    k = len(roots)
    level = torch.empty(k * g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(k * g.n, dtype=torch.int32, device="cuda") if want_parent else None
    g.run_multi(roots, level, parent=parent, opts=opts)
    g.sync()
    lv = level.cpu().numpy().reshape(k, g.n)
    pa = parent.cpu().numpy().reshape(k, g.n) if want_parent else None
    return lv, pa


@pytest.mark.parametrize("scale", [10, 14])
def test_multi_64_lanes_all_modes(gpu_lib, scale):
    bfs = gpu_lib
    w = workloads.RMAT[scale]
    e = w.edges()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    roots = w.roots(e, 64).tolist()
    want = np.stack([oracle.levels(ref, r) for r in roots])
    for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY):
        lv, _ = _run(bfs, g, roots, opts=bfs.options(mode=mode))
        assert np.array_equal(lv, want), mode


def test_multi_uneven_lane_counts_and_repeats(gpu_lib):
    bfs = gpu_lib
    e = graphgen.erdos_renyi(5000, 12000, seed=4)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    base = graphgen.pick_roots(e, 50, 2).tolist()
    for roots in ([base[0]], base[:3], base + base[:30] + [base[7]] * 20):   # 1, 3, 101 lanes (two launches)
        lv, _ = _run(bfs, g, roots)
        for i, r in enumerate(roots):
            assert np.array_equal(lv[i], oracle.levels(ref, r)), (len(roots), i)


def test_multi_parents_min_id(gpu_lib):
    bfs = gpu_lib
    w = workloads.RMAT[12]
    e = w.edges()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    roots = w.roots(e, 20).tolist()
    lv, pa = _run(bfs, g, roots, want_parent=True)
    for i, r in enumerate(roots):
        want = oracle.levels(ref, r)
        assert np.array_equal(lv[i], want)
        assert np.array_equal(pa[i], oracle.min_parent(ref, want))


def test_multi_small_shapes(gpu_lib):
    bfs = gpu_lib
    shapes = [graphgen.path(300), graphgen.star(200), graphgen.complete(30), graphgen.random_small(90, 80, 5)]
    u, offs = graphgen.disjoint_union(shapes + [graphgen.from_pairs(4, [(1, 1)])])
    ref = oracle.build_csr(u.n, u.src, u.dst)
    g = bfs.Graph.from_edges(u.src, u.dst, u.n)
    roots = [0, 150, 299, int(offs[1]), int(offs[2]) + 5, int(offs[3]), int(offs[4]) + 1, int(offs[4]) + 3]
    lv, _ = _run(bfs, g, roots)
    for i, r in enumerate(roots):
        assert np.array_equal(lv[i], oracle.levels(ref, r))


def test_multi_torus_high_diameter(gpu_lib):
    bfs = gpu_lib
    side = 128
    e = graphgen.torus(side, seed=3000)
    inv = graphgen.torus_coordinates(side, seed=3000)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    x, y = inv % side, inv // side
    roots = [0, 5, 999, side * side - 1]
    lv, _ = _run(bfs, g, roots)
    for i, r in enumerate(roots):
        dx = np.abs(x - x[r])
        dy = np.abs(y - y[r])
        assert np.array_equal(lv[i], np.minimum(dx, side - dx) + np.minimum(dy, side - dy))


def test_multi_hub_first_rows(gpu_lib):
    """Bottom-up pulls over hub-first rows give the same level rows (64 lanes, all
    direction modes)."""
    bfs = gpu_lib
    w = workloads.RMAT[14]
    e = w.edges()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    roots = w.roots(e, 64).tolist()
    want = np.stack([oracle.levels(ref, r) for r in roots])
    for mode in (bfs.MODE_DO, bfs.MODE_BU_ONLY):
        lv, _ = _run(bfs, g, roots, opts=bfs.options(mode=mode, bu_rows=bfs.BU_ROWS_HUB_FIRST))
        assert np.array_equal(lv, want), mode


def test_multi_deep_levels_past_byte_staging(gpu_lib):
    """Levels are staged one byte per (lane, vertex) up to depth 253 and written
    to the int32 rows directly beyond; a 700-vertex path crosses that boundary
    from several roots at once (min-id parents too)."""
    bfs = gpu_lib
    e = graphgen.path(700)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    roots = [0, 350, 699, 1, 698, 200]
    lv, pa = _run(bfs, g, roots, want_parent=True)
    for i, r in enumerate(roots):
        want = oracle.levels(ref, r)
        assert np.array_equal(lv[i], want), r
        assert np.array_equal(pa[i], oracle.min_parent(ref, want)), r

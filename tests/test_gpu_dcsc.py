"""The device-built DCSC tiles equal the oracle's DCSC definition, array for array."""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["rmat12", "rmat16", "er_ragged", "small"])
def test_dcsc_layout_matches_oracle(gpu_lib, which):
    bfs = gpu_lib
    if which == "rmat12":
        e = workloads.RMAT[12].edges()
    elif which == "rmat16":
        e = workloads.RMAT[16].edges()
    elif which == "er_ragged":
        e = graphgen.erdos_renyi(100_003, 400_000, seed=3)
    else:
        e, _ = graphgen.disjoint_union([graphgen.path(40), graphgen.star(30), graphgen.from_pairs(5, [(1, 1)])])
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, dcsc=True)
    p, B, tp, jc, cp, ir = g.dcsc_host()
    assert B % 32 == 0 and p * B >= e.n and (p - 1) * B < e.n
    wtp, wjc, wcp, wir = oracle.dcsc_tiles(e.n, ref.offsets, ref.cols, B, B)
    assert np.array_equal(tp, wtp)
    assert np.array_equal(jc, wjc)
    assert np.array_equal(cp, wcp)
    assert np.array_equal(ir, wir)


def _case(bfs, e):
    import torch
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, dcsc=True)
    lv = torch.empty(e.n, dtype=torch.int32, device="cuda")
    pa = torch.empty(e.n, dtype=torch.int32, device="cuda")
    return ref, g, lv, pa


@pytest.mark.parametrize("which", ["rmat12", "rmat15", "er_ragged", "small", "torus"])
def test_dcsc_search_levels_all_modes(gpu_lib, which):
    bfs = gpu_lib
    if which == "rmat12":
        e = workloads.RMAT[12].edges()
    elif which == "rmat15":
        e = workloads.RMAT[15].edges()
    elif which == "er_ragged":
        e = graphgen.erdos_renyi(100_003, 400_000, seed=3)
    elif which == "torus":
        e = graphgen.torus(96, seed=3000)
    else:
        e, _ = graphgen.disjoint_union([graphgen.path(40), graphgen.star(30), graphgen.from_pairs(5, [(1, 1)])])
    ref, g, lv, pa = _case(bfs, e)
    labels = oracle.components(ref)
    roots = graphgen.pick_roots(e, 6, 21).tolist() + [e.n - 1]
    for root in roots:
        want = oracle.levels(ref, root)
        for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY, bfs.MODE_RANDOM):
            info = g.run(root, parent=pa, level=lv, opts=bfs.options(mode=mode, layout=bfs.LAYOUT_DCSC_TILED, seed=5),
                         stats=True, record_levels=4096)
            got = lv.cpu().numpy()
            assert np.array_equal(got, want), (which, root, mode)
            assert oracle.certify(ref, root, got, pa.cpu().numpy(), labels) == (0, -1), (which, root, mode)
            assert info["num_levels"] == int(want.max()) + 1


def test_dcsc_schedule_and_min_parent(gpu_lib):
    """Per-level direction/frontier counters equal the oracle's schedule; with minimum-id
    parents the tile walk runs in block order, so bottom-up examinations equal the serial
    early-exit count too."""
    bfs = gpu_lib
    w = workloads.RMAT[14]
    e = w.edges()
    ref, g, lv, pa = _case(bfs, e)
    for root in w.roots(e, 5).tolist():
        want = oracle.levels(ref, root)
        pmin = oracle.min_parent(ref, want)
        for mode, omode in ((bfs.MODE_DO, oracle.MODE_DO), (bfs.MODE_BU_ONLY, oracle.MODE_BU)):
            info = g.run(root, parent=pa, level=lv, stats=True, record_levels=4096,
                         opts=bfs.options(mode=mode, layout=bfs.LAYOUT_DCSC_TILED, parent_mode=bfs.PARENT_MIN_ID))
            assert np.array_equal(lv.cpu().numpy(), want)
            assert np.array_equal(pa.cpu().numpy(), pmin)
            s = oracle.do_schedule(ref, want, omode)
            rec = info["records"]
            for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
                assert np.array_equal(rec[:, col], getattr(s, name)), (root, mode, name)


def test_dcsc_multiroot_union(gpu_lib):
    bfs = gpu_lib
    parts = [graphgen.rmat(sc, seed=600 + sc) for sc in (7, 10, 9)]
    u, offs = graphgen.disjoint_union(parts)
    ref, g, lv, pa = _case(bfs, u)
    roots = [int(offs[i]) + int(graphgen.pick_roots(p, 1, i)[0]) for i, p in enumerate(parts)]
    g.run_multiroot(roots, parent=pa, level=lv, opts=bfs.options(layout=bfs.LAYOUT_DCSC_TILED))
    got = lv.cpu().numpy()
    for i, p in enumerate(parts):
        pr = oracle.build_csr(p.n, p.src, p.dst)
        assert np.array_equal(got[offs[i]:offs[i + 1]], oracle.levels(pr, roots[i] - int(offs[i])))

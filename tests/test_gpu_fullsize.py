"""Full-size parity, in the launch configuration bench.py times (direction-optimizing,
CSR, alpha 14, beta 24, one persistent launch per search).

* R-MAT scale 26 (built with the hub-first row copy, as bench.py builds it): the
  device CSR equals the oracle's bit for bit; sampled hub-first rows equal the oracle's
  definition; levels of sampled
  roots equal the oracle's serial Algorithm 1; every sampled root's levels and parents
  pass the oracle's certificate (a property that proves level = hop distance at any
  size); the per-level counters equal the oracle's direction-optimizing schedule.
* 4096 x 4096 torus: levels of 8 roots equal the closed form (4097 levels each).
* 64-lane multi-source at R-MAT scale 22 (the batched configuration): sampled lane rows
  equal the oracle; every row passes the level-only certificate.

The oracle needs minutes of host time here (numpy sort of 2.1e9 keys, serial BFS);
sample sizes are chosen to keep the file within about ten minutes on the GPU host.
"""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def rmat26(gpu_lib):
    bfs = gpu_lib
    w = workloads.RMAT[26]
    e = w.edges()
    roots = w.roots(e, 64).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    del e
    yield w, g, ref, roots
    g.close()


def test_rmat26_csr_bit_exact(rmat26):
    _, g, ref, _ = rmat26
    assert g.nnz == ref.nnz
    off, cols = g.csr_host()
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(cols, ref.cols)


def test_rmat26_levels_parents_schedule(gpu_lib, rmat26):
    import torch
    bfs = gpu_lib
    _, g, ref, roots = rmat26
    labels = oracle.components(ref)
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    opts = bfs.options(mode=bfs.MODE_DO, alpha=14, beta=24)
    for i, root in enumerate(roots[:6]):
        info = g.run(root, parent=parent, level=level, opts=opts, stats=True, record_levels=4096)
        lv = level.cpu().numpy()
        pa = parent.cpu().numpy()
        assert oracle.certify(ref, root, lv, pa, labels) == (0, -1), root
        if i < 2:
            want = oracle.levels(ref, root)
            assert np.array_equal(lv, want), root
            s = oracle.do_schedule(ref, want, oracle.MODE_DO, 14, 24)
            rec = info["records"]
            for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
                assert np.array_equal(rec[:, col], getattr(s, name)), (root, name)


def test_rmat26_hub_first_rows_and_searches(gpu_lib, rmat26):
    """The bench's configuration (bottom-up over hub-first rows): sampled rows of the
    device's reordered copy equal the oracle's definition; sampled roots' levels equal
    the oracle's and pass the certificate with their parents."""
    import torch
    bfs = gpu_lib
    _, g, ref, roots = rmat26
    hf = g.hub_first_host()
    deg = np.diff(ref.offsets)
    rng = np.random.default_rng(2626)
    for u in rng.choice(np.flatnonzero(deg > 0), 2000, replace=False).tolist() + [int(np.argmax(deg))]:
        row = ref.cols[ref.offsets[u]:ref.offsets[u + 1]]
        want = row[np.lexsort((row, -deg[row]))]
        assert np.array_equal(hf[ref.offsets[u]:ref.offsets[u + 1]], want), u
    del hf
    labels = oracle.components(ref)
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    opts = bfs.options(mode=bfs.MODE_DO, alpha=14, beta=24, bu_rows=bfs.BU_ROWS_HUB_FIRST)
    for i, root in enumerate(roots[:4]):
        g.run(root, parent=parent, level=level, opts=opts)
        lv = level.cpu().numpy()
        assert oracle.certify(ref, root, lv, parent.cpu().numpy(), labels) == (0, -1), root
        if i < 1:
            assert np.array_equal(lv, oracle.levels(ref, root)), root


def test_torus4096_closed_form(gpu_lib):
    import torch
    bfs = gpu_lib
    side = 4096
    w = workloads.TORUS4096
    e = w.edges()
    inv = graphgen.torus_coordinates(side, seed=w.graph_seed)
    roots = w.roots(e, 8).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    del e
    x, y = inv % side, inv // side
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for root in roots:
        info = g.run(root, level=level, stats=True)
        dx = np.abs(x - x[root])
        dy = np.abs(y - y[root])
        want = np.minimum(dx, side - dx) + np.minimum(dy, side - dy)
        assert np.array_equal(level.cpu().numpy(), want), root
        assert info["num_levels"] == side + 1
    g.close()


def test_multi64_rmat22(gpu_lib):
    import torch
    bfs = gpu_lib
    w = workloads.RMAT[22]
    e = w.edges()
    roots = w.roots(e, 64).tolist()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    del e
    lv = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
    g.run_multi(roots, lv)
    g.sync()
    rows = lv.cpu().numpy().reshape(64, g.n)
    labels = oracle.components(ref)
    for i, r in enumerate(roots):
        assert oracle.certify(ref, r, rows[i], None, labels) == (0, -1), i
        if i % 8 == 0:
            assert np.array_equal(rows[i], oracle.levels(ref, r)), i
    g.close()

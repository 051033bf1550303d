"""Full-size parity, in the launch configuration bench.py times (direction-optimizing,
CSR, alpha 14, beta 24, one persistent launch per search, bottom-up over the hub-first
rows unless stated).

* R-MAT scale 26 (built with the hub-first row copy, as bench.py builds it): the
  device CSR equals the oracle's bit for bit; the first-neighbour plane equals the
  oracle's hub-first rows (first id, degree flag) for every vertex; all 64 bench roots
  pass the oracle's certificate with their parents (a property that proves level =
  hop distance at any size), 4 of them equal the oracle's serial Algorithm 1 bit for
  bit, and for 2 the per-level counters equal the oracle's direction-optimizing
  schedule over the hub-first rows; over the id-ordered rows 4 roots are certified
  and 2 compared with the oracle's levels and schedule.
* Erdos-Renyi n = 2^26, E[deg] = 16: 16 roots certified, 4 bit-exact.
* R-MAT scale 24 with DCSC column-block tiles: 2 roots bit-exact in each of the
  direction-optimizing, top-down-only and bottom-up-only modes.
* 4096 x 4096 torus: levels of 8 roots equal the closed form (4097 levels each).
* 64-lane multi-source at R-MAT scale 22 (the batched configuration): sampled lane rows
  equal the oracle; every row passes the level-only certificate.

The oracle needs minutes of host time here (numpy sort of 2.1e9 keys, serial BFS);
certificates and serial searches of different roots run on host threads (the C
oracle releases the interpreter lock), so the file stays within about ten minutes.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

THREADS = min(16, os.cpu_count() or 1)


def _parallel(fn, items):
    with cf.ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(fn, items))


def _search_and_certify(bfs, g, ref, labels, roots, opts, exact=(), batch=8):
    """Run every root on the GPU (outputs copied to host in batches), certify all of
    them on host threads and compare the roots in `exact` with oracle.levels."""
    import torch
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    def check(t):
        root, lv, pa = t
        cert = oracle.certify(ref, root, lv, pa, labels)
        same = np.array_equal(lv, oracle.levels(ref, root)) if root in exact else True
        return cert, same

    for b0 in range(0, len(roots), batch):
        got = []
        for root in roots[b0:b0 + batch]:
            g.run(root, parent=parent, level=level, opts=opts)
            got.append((root, level.cpu().numpy(), parent.cpu().numpy()))
        for (root, _, _), (cert, same) in zip(got, _parallel(check, got)):
            assert cert == (0, -1), (root, cert)
            assert same, root


@pytest.fixture(scope="module")
def rmat26(gpu_lib):
    bfs = gpu_lib
    w = workloads.RMAT[26]
    e = w.edges()
    roots = w.roots(e, 64).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    del e
    labels = oracle.components(ref)
    yield w, g, ref, roots, labels
    g.close()


def test_rmat26_csr_bit_exact(rmat26):
    _, g, ref, _, _ = rmat26
    assert g.nnz == ref.nnz
    off, cols = g.csr_host()
    assert np.array_equal(off, ref.offsets)
    assert np.array_equal(cols, ref.cols)


def test_rmat26_levels_parents_schedule(gpu_lib, rmat26):
    """Bottom-up over the id-ordered rows (the paper's order)."""
    import torch
    bfs = gpu_lib
    _, g, ref, roots, labels = rmat26
    opts = bfs.options(mode=bfs.MODE_DO, alpha=14, beta=24)
    _search_and_certify(bfs, g, ref, labels, roots[:4], opts)
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for root in roots[:2]:
        info = g.run(root, level=level, opts=opts, stats=True, record_levels=4096)
        want = oracle.levels(ref, root)
        assert np.array_equal(level.cpu().numpy(), want), root
        s = oracle.do_schedule(ref, want, oracle.MODE_DO, 14, 24)
        rec = info["records"]
        for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
            assert np.array_equal(rec[:, col], getattr(s, name)), (root, name)


def test_rmat26_hub_first_all_bench_roots(gpu_lib, rmat26):
    """The bench's configuration (bottom-up over hub-first rows): the device's
    reordered rows (sampled) and its first-neighbour plane (every vertex) equal the
    oracle's definition; all 64 bench roots are certified, 4 bit-exact; for 2 the
    per-level counters equal the oracle's schedule over the oracle's hub-first rows."""
    import torch
    bfs = gpu_lib
    _, g, ref, roots, labels = rmat26
    hub = oracle.hub_first_rows(ref)
    deg = np.diff(ref.offsets)
    hf = g.hub_first_host()
    rng = np.random.default_rng(2626)
    for u in rng.choice(np.flatnonzero(deg > 0), 2000, replace=False).tolist() + [int(np.argmax(deg))]:
        assert np.array_equal(hf[ref.offsets[u]:ref.offsets[u + 1]], hub.cols[ref.offsets[u]:ref.offsets[u + 1]]), u
    del hf
    first, _ = g.bu_planes_host()
    want = np.zeros(g.n, np.uint32)
    has = deg > 0
    want[has] = hub.cols[ref.offsets[:-1][has]].astype(np.uint32) | np.where(deg[has] >= 2, 1 << 31, 0).astype(np.uint32)
    assert np.array_equal(first.view(np.uint32), want)
    del first, want
    opts = bfs.options(mode=bfs.MODE_DO, alpha=14, beta=24, bu_rows=bfs.BU_ROWS_HUB_FIRST)
    _search_and_certify(bfs, g, ref, labels, roots, opts, exact=set(roots[:4]))
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for root in roots[:2]:
        info = g.run(root, level=level, opts=opts, stats=True, record_levels=4096)
        lv = level.cpu().numpy()
        s = oracle.do_schedule(hub, lv, oracle.MODE_DO, 14, 24)
        rec = info["records"]
        for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
            assert np.array_equal(rec[:, col], getattr(s, name)), (root, name)


def test_er26_bench_configuration(gpu_lib):
    """Erdos-Renyi n = 2^26 with expected degree 16 (configuration 3), as bench.py
    builds and searches it: 16 seeded roots certified, 4 bit-exact."""
    bfs = gpu_lib
    w = workloads.Workload("er", 26)
    e = w.edges()
    roots = w.roots(e, 16).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    del e
    labels = oracle.components(ref)
    opts = bfs.options(mode=bfs.MODE_DO, alpha=14, beta=24, bu_rows=bfs.BU_ROWS_HUB_FIRST)
    _search_and_certify(bfs, g, ref, labels, roots, opts, exact=set(roots[:4]))
    g.close()


def test_dcsc_rmat24_all_modes(gpu_lib):
    """Column-block DCSC tiles at R-MAT scale 24 (configuration 2): 2 seeded roots
    bit-exact with the oracle in each direction mode, parents certified."""
    import torch
    bfs = gpu_lib
    w = workloads.RMAT[24]
    e = w.edges()
    roots = w.roots(e, 2).tolist()
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, dcsc=True)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    del e
    labels = oracle.components(ref)
    want = dict(zip(roots, _parallel(lambda r: oracle.levels(ref, r), roots)))
    level = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY):
        got = []
        for root in roots:
            g.run(root, parent=parent, level=level, opts=bfs.options(mode=mode, layout=bfs.LAYOUT_DCSC_TILED))
            got.append((root, level.cpu().numpy(), parent.cpu().numpy()))
        for root, lv, _ in got:
            assert np.array_equal(lv, want[root]), (root, mode)
        res = _parallel(lambda t: oracle.certify(ref, t[0], t[1], t[2], labels), got)
        assert all(r == (0, -1) for r in res), (mode, res)
    g.close()


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

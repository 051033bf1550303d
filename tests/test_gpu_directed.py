"""Directed graphs on the GPU against the oracle: the device's out-edge CSR and its
transpose equal the oracle's bit for bit; levels are bit-exact (every direction mode,
plain and minimum-id parents); parents pass the certificate along directed edges (a
parent must have an edge *to* its child); the per-level counters equal the oracle's
directed schedule (m_f over out-degrees, m_u over in-degrees, bottom-up examinations
over the in-edge rows)."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def _cases():
    return [graphgen.random_small(2, 1, 1), graphgen.random_small(40, 90, 3), graphgen.random_small(300, 700, 5),
            graphgen.from_pairs(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 4), (5, 3), (0, 1)]),
            graphgen.rmat(12, seed=1212), graphgen.rmat(16, seed=1616), graphgen.erdos_renyi(100_003, 400_000, seed=9)]


@pytest.mark.parametrize("gi", range(7))
def test_directed_graph_parity(gpu_lib, gi):
    import torch
    bfs = gpu_lib
    e = _cases()[gi]
    out, inn = oracle.build_digraph(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, directed=True)
    off, cols = g.csr_host()
    assert np.array_equal(off, out.offsets) and np.array_equal(cols, out.cols)
    toff, tcols = g.transpose_host()
    assert np.array_equal(toff, inn.offsets) and np.array_equal(tcols, inn.cols)
    level = torch.empty(e.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(e.n, dtype=torch.int32, device="cuda")
    odeg, ideg = out.degree(), inn.degree()
    roots = sorted({0, e.n - 1, int(np.argmax(odeg)), int(np.argmax(ideg))})
    modes = {bfs.MODE_DO: oracle.MODE_DO, bfs.MODE_TD_ONLY: oracle.MODE_TD, bfs.MODE_BU_ONLY: oracle.MODE_BU}
    for root in roots:
        _, want, _ = oracle.bfs_topdown(out, root)
        reached = oracle.reach(out, root)
        for mode, omode in modes.items():
            info = g.run(root, parent=parent, level=level, opts=bfs.options(mode=mode), stats=True,
                         record_levels=4096)
            lv, pa = level.cpu().numpy(), parent.cpu().numpy()
            assert np.array_equal(lv, want), (e.name, root, mode)
            assert oracle.certify_dir(out, root, lv, pa, reached) == (0, -1), (e.name, root, mode)
            s = oracle.do_schedule_dir(out, inn, want, omode, 14, 24)
            for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
                assert np.array_equal(info["records"][:, col], getattr(s, name)), (e.name, root, mode, name)
        g.run(root, parent=parent, level=level, opts=bfs.options(parent_mode=bfs.PARENT_MIN_ID))
        pa = parent.cpu().numpy()
        # minimum-id parents: the smallest u with u -> v one level closer
        for v in np.flatnonzero(want > 0)[:2000].tolist():
            preds = inn.cols[inn.offsets[v]:inn.offsets[v + 1]]
            assert pa[v] == preds[want[preds] == want[v] - 1].min(), (e.name, root, v)
    g.close()


def test_directed_graph_refusals(gpu_lib):
    bfs = gpu_lib
    e = graphgen.random_small(50, 100, 2)
    with pytest.raises(bfs.BfsError) as ex:
        bfs.Graph.from_edges(e.src, e.dst, e.n, directed=True, hub_first=True)
    assert ex.value.status == 7
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, directed=True)
    import torch
    lv = torch.empty(2 * e.n, dtype=torch.int32, device="cuda")
    with pytest.raises(bfs.BfsError) as ex:
        g.run_multi([0, 1], lv)
    assert ex.value.status == 7
    srv = bfs.Server(hbm_budget_bytes=1 << 28)
    with pytest.raises(bfs.BfsError):
        srv.add_graph(g)
    srv.close()
    u = bfs.Graph.from_edges(e.src, e.dst, e.n)
    with pytest.raises(bfs.BfsError) as ex:
        u.transpose_host()
    assert ex.value.status == 1
    u.close()
    g.close()

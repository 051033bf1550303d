"""The continuous-batching server: every query's levels equal the oracle's and are the
same whether the query ran alone or in a mix with others on several resident graphs."""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = pytest.mark.gpu


def _graphs(bfs):
    out = []
    for e in (workloads.RMAT[12].edges(), workloads.RMAT[15].edges(), graphgen.torus(64, seed=3000),
              graphgen.erdos_renyi(3001, 9000, seed=8)):
        out.append((e, oracle.build_csr(e.n, e.src, e.dst), bfs.Graph.from_edges(e.src, e.dst, e.n)))
    return out


def test_server_mix_equals_alone_and_oracle(gpu_lib):
    bfs = gpu_lib
    gs = _graphs(bfs)
    srv = bfs.Server(hbm_budget_bytes=4 << 30, max_lanes=64)
    slots = [srv.add_graph(g) for _, _, g in gs]
    rng = np.random.default_rng(11)
    queries = []
    for q in range(300):
        i = int(rng.integers(0, len(gs)))
        e = gs[i][0]
        root = int(graphgen.pick_roots(e, 40, 77 + i)[int(rng.integers(0, 40))])
        queries.append((i, root))
    # alone: one at a time
    alone = {}
    for i, root in queries[:12]:
        out = np.empty(gs[i][0].n, np.int32)
        t = srv.submit(slots[i], root, out)
        assert srv.wait(t, 60000)
        alone[(i, root)] = out
    # mix: all at once
    outs = []
    for i, root in queries:
        out = np.empty(gs[i][0].n, np.int32)
        outs.append((i, root, out, srv.submit(slots[i], root, out)))
    for i, root, out, t in outs:
        assert srv.wait(t, 120000)
        assert np.array_equal(out, oracle.levels(gs[i][1], root)), (i, root)
        if (i, root) in alone:
            assert np.array_equal(out, alone[(i, root)])
        assert srv.latency_us(t) > 0
    st = srv.stats()
    assert st["completed"] == len(queries) + 12
    assert st["lanes_filled"] > st["launches"]       # levels were shared by several queries
    srv.close()


def test_server_budget_limits_lanes(gpu_lib):
    bfs = gpu_lib
    e = workloads.RMAT[12].edges()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    with pytest.raises(bfs.BfsError):
        bfs.Server(hbm_budget_bytes=1024).add_graph(g)
    # masks (24n) plus room for two level rows (4n each)
    srv = bfs.Server(hbm_budget_bytes=24 * e.n + 8 * e.n + (1 << 20) * 8, max_lanes=64)
    slot = srv.add_graph(g)
    roots = graphgen.pick_roots(e, 30, 5).tolist()
    outs = [(r, np.empty(e.n, np.int32)) for r in roots]
    ts = [srv.submit(slot, r, o) for r, o in outs]
    for (r, o), t in zip(outs, ts):
        assert srv.wait(t, 60000)
        assert np.array_equal(o, oracle.levels(ref, r))
    with pytest.raises(bfs.BfsError):
        srv.submit(slot, e.n, np.empty(e.n, np.int32))
    with pytest.raises(bfs.BfsError):
        srv.submit(7, 0, np.empty(e.n, np.int32))
    with pytest.raises(bfs.BfsError):
        srv.poll(123456789)
    srv.close()


def test_server_deep_graph_runs_concurrent_searches(gpu_lib):
    """A graph of large diameter (256 x 256 torus: 257 levels) is served by concurrent
    single-source searches instead of lanes; mixed with an R-MAT slot, every result
    still equals the oracle / the torus closed form, alone and in a burst."""
    bfs = gpu_lib
    side = 256
    et = graphgen.torus(side, seed=3000)
    inv = graphgen.torus_coordinates(side, seed=3000)
    x, y = inv % side, inv // side
    er = workloads.RMAT[12].edges()
    rref = oracle.build_csr(er.n, er.src, er.dst)
    gt = bfs.Graph.from_edges(et.src, et.dst, et.n)
    gr = bfs.Graph.from_edges(er.src, er.dst, er.n)
    srv = bfs.Server(hbm_budget_bytes=4 << 30, max_lanes=64)
    st_, sr_ = srv.add_graph(gt), srv.add_graph(gr)
    rng = np.random.default_rng(21)
    troots = rng.integers(0, et.n, 40).tolist()
    rroots = graphgen.pick_roots(er, 40, 9).tolist()
    outs = []
    for a, b in zip(troots, rroots):
        ot, orr = np.empty(et.n, np.int32), np.empty(er.n, np.int32)
        outs.append(("t", a, ot, srv.submit(st_, a, ot)))
        outs.append(("r", b, orr, srv.submit(sr_, b, orr)))
    for kind, root, out, t in outs:
        assert srv.wait(t, 120000)
        if kind == "t":
            dx, dy = np.abs(x - x[root]), np.abs(y - y[root])
            want = np.minimum(dx, side - dx) + np.minimum(dy, side - dy)
        else:
            want = oracle.levels(rref, root)
        assert np.array_equal(out, want), (kind, root)
    srv.close()
    gt.close()
    gr.close()


def test_server_allocator_hook(gpu_lib):
    """bfs_server_create_ex: every device buffer the server owns comes from the
    caller's allocator (here PyTorch's caching allocator, with the calls counted),
    is returned by destroy, and queries still equal the oracle."""
    import ctypes
    import torch
    bfs = gpu_lib
    L = bfs._lib
    calls = {"alloc": 0, "free": 0, "live": {}}

    def _alloc(nbytes, stream, ctx):
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0))
        calls["alloc"] += 1
        calls["live"][p] = nbytes
        return p

    def _free(ptr, nbytes, stream, ctx):
        calls["free"] += 1
        calls["live"].pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    class Hook:
        pass

    hook = Hook()
    hook.cb = (L.ALLOC_FN(_alloc), L.FREE_FN(_free))
    hook.struct = L.Allocator(hook.cb[0], hook.cb[1], None)
    e = workloads.RMAT[13].edges()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    srv = bfs.Server(hbm_budget_bytes=2 << 30, max_lanes=64, allocator=hook)
    slot = srv.add_graph(g)
    assert calls["alloc"] > 0
    roots = graphgen.pick_roots(e, 40, 5).tolist()
    outs = [(r, np.empty(e.n, np.int32)) for r in roots]
    tickets = [srv.submit(slot, r, o) for r, o in outs]
    for (r, o), t in zip(outs, tickets):
        assert srv.wait(t, 60000)
        assert np.array_equal(o, oracle.levels(ref, r)), r
    srv.close()
    assert calls["free"] == calls["alloc"] and not calls["live"]
    with pytest.raises(bfs.BfsError):
        bad = Hook()
        bad.struct = L.Allocator(hook.cb[0], L.FREE_FN(0), None)
        bfs.Server(hbm_budget_bytes=1 << 30, allocator=bad)
    g.close()

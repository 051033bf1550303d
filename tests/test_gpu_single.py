"""GPU parity of the single-source / multi-root search against the CPU oracle.

Levels are compared element by element (bit-exact: integer output, zero
tolerance).  Parents are legitimately non-unique, so they are checked by the
oracle's certificate (valid BFS tree of the oracle's own graph), and bit-exact
against the oracle in BFS_PARENT_MIN_ID mode.  The per-level device counters
(direction, frontier sizes, bottom-up examination counts) must equal the
oracle's direction-optimizing schedule exactly.
"""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = pytest.mark.gpu

MODES = None


def _modes(bfs):
    return {"do": bfs.MODE_DO, "td": bfs.MODE_TD_ONLY, "bu": bfs.MODE_BU_ONLY, "random": bfs.MODE_RANDOM}


class Case:
    def __init__(self, bfs, e, dcsc=False):
        import torch
        self.e = e
        self.ref = oracle.build_csr(e.n, e.src, e.dst)
        self.g = bfs.Graph.from_edges(e.src, e.dst, e.n, dcsc=dcsc)
        self.labels = oracle.components(self.ref)
        self.level = torch.empty(e.n, dtype=torch.int32, device="cuda")
        self.parent = torch.empty(e.n, dtype=torch.int32, device="cuda")

    def run(self, root, opts=None, stats=False):
        info = self.g.run(root, parent=self.parent, level=self.level, opts=opts, stats=stats, record_levels=1 << 14)
        return self.level.cpu().numpy(), self.parent.cpu().numpy(), info


def _check_csr(case):
    off, cols = case.g.csr_host()
    assert case.g.nnz == case.ref.nnz
    assert np.array_equal(off, case.ref.offsets)
    assert np.array_equal(cols, case.ref.cols)


def _small_graphs():
    gs = [graphgen.random_small(n, m, s) for n, m, s in
          [(1, 0, 0), (2, 1, 1), (5, 3, 2), (33, 20, 5), (64, 300, 7), (100, 90, 8), (257, 600, 11)]]
    gs += [graphgen.path(70), graphgen.cycle(65), graphgen.star(100), graphgen.complete(40)]
    u, _ = graphgen.disjoint_union([graphgen.path(5), graphgen.complete(4), graphgen.from_pairs(3, [(0, 0)])])
    gs.append(u)
    return gs


@pytest.mark.parametrize("gi", range(12))
def test_small_graphs_every_root_every_mode(gpu_lib, gi):
    bfs = gpu_lib
    case = Case(bfs, _small_graphs()[gi])
    _check_csr(case)
    for root in range(case.e.n):
        want = oracle.levels(case.ref, root)
        for name, mode in _modes(bfs).items():
            lv, pa, _ = case.run(root, bfs.options(mode=mode, seed=root * 7 + 1))
            assert np.array_equal(lv, want), (case.e.name, root, name)
            assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), (case.e.name, root, name)


@pytest.mark.parametrize("scale", [12, 16])
def test_rmat_levels_parents_all_modes(gpu_lib, scale):
    bfs = gpu_lib
    w = workloads.RMAT[scale]
    e = w.edges()
    case = Case(bfs, e)
    _check_csr(case)
    for root in w.roots(e, 16).tolist():
        want = oracle.levels(case.ref, root)
        for name, mode in _modes(bfs).items():
            lv, pa, info = case.run(root, bfs.options(mode=mode, seed=root), stats=True)
            assert np.array_equal(lv, want), (scale, root, name)
            assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), (scale, root, name)
            assert info["num_levels"] == int(want.max()) + 1
            assert info["reached"] == int((want >= 0).sum())


def test_ragged_er_spans_many_tiles(gpu_lib):
    bfs = gpu_lib
    n = 100_003   # not a multiple of 32: ragged last bitmap word
    e = graphgen.erdos_renyi(n, 8 * n, seed=77)
    case = Case(bfs, e)
    _check_csr(case)
    for root in graphgen.pick_roots(e, 4, 5).tolist():
        want = oracle.levels(case.ref, root)
        for mode in (bfs.MODE_DO, bfs.MODE_BU_ONLY, bfs.MODE_TD_ONLY):
            lv, pa, _ = case.run(root, bfs.options(mode=mode))
            assert np.array_equal(lv, want)
            assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1)


@pytest.mark.parametrize("scale", [12, 16])
def test_level_records_match_oracle_schedule(gpu_lib, scale):
    """Device per-level counters == the oracle's direction-optimizing schedule, for DO/TD/BU."""
    bfs = gpu_lib
    w = workloads.RMAT[scale]
    e = w.edges()
    case = Case(bfs, e)
    for root in w.roots(e, 6).tolist():
        want = oracle.levels(case.ref, root)
        for mode, omode in ((bfs.MODE_DO, oracle.MODE_DO), (bfs.MODE_TD_ONLY, oracle.MODE_TD),
                            (bfs.MODE_BU_ONLY, oracle.MODE_BU)):
            for alpha, beta in ((14, 24), (2, 100)):
                _, _, info = case.run(root, bfs.options(mode=mode, alpha=alpha, beta=beta), stats=True)
                s = oracle.do_schedule(case.ref, want, omode, alpha, beta)
                rec = info["records"]
                assert rec.shape[0] == s.num_levels
                got = {k: rec[:, i] for i, k in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"])}
                for k in ["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]:
                    assert np.array_equal(got[k], getattr(s, k)), (scale, root, mode, alpha, k)


def test_min_id_parents_bit_exact(gpu_lib):
    bfs = gpu_lib
    w = workloads.RMAT[14]
    e = w.edges()
    case = Case(bfs, e)
    for root in w.roots(e, 6).tolist():
        want = oracle.levels(case.ref, root)
        pmin = oracle.min_parent(case.ref, want)
        for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY, bfs.MODE_RANDOM):
            opts = bfs.options(mode=mode, parent_mode=bfs.PARENT_MIN_ID, seed=3)
            lv, pa, _ = case.run(root, opts)
            assert np.array_equal(lv, want)
            assert np.array_equal(pa, pmin), (root, mode)
            # parent only: the library keeps the levels it needs privately
            case.parent.fill_(-7)
            case.g.run(root, parent=case.parent, opts=opts)
            assert np.array_equal(case.parent.cpu().numpy(), pmin), (root, mode, "parent only")


def test_torus_closed_form(gpu_lib):
    bfs = gpu_lib
    side = 256
    e = graphgen.torus(side, seed=3000)
    inv = graphgen.torus_coordinates(side, seed=3000)
    case = Case(bfs, e)
    x, y = inv % side, inv // side
    for root in [0, 12345, side * side - 1]:
        lv, pa, info = case.run(root, stats=True)
        dx = np.abs(x - x[root])
        dy = np.abs(y - y[root])
        want = np.minimum(dx, side - dx) + np.minimum(dy, side - dy)
        assert np.array_equal(lv, want)
        assert info["num_levels"] == side + 1
        assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1)


def test_path_bottom_up_only_same_level_discovery(gpu_lib):
    """Bottom-up must test the *current* frontier: on a path every level finds one vertex."""
    bfs = gpu_lib
    n = 3000
    case = Case(bfs, graphgen.path(n))
    for root in (0, 1234, n - 1):
        lv, pa, info = case.run(root, bfs.options(mode=bfs.MODE_BU_ONLY), stats=True)
        assert np.array_equal(lv, np.abs(np.arange(n) - root))
        assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1)


def test_hub_first_rows_and_searches(gpu_lib):
    """BFS_FLAG_BUILD_HUB_FIRST: the device's reordered rows equal the oracle's
    hub_first() bit for bit, and so do the row heads (degree + first 7 ids of each
    reordered row); searches scanning them bottom-up give exact levels,
    valid parents, and per-level counters equal to the oracle's schedule over the
    hub-first rows; the option is refused where it cannot apply."""
    bfs = gpu_lib
    graphs = [workloads.RMAT[14].edges(), graphgen.random_small(257, 600, 11), graphgen.torus(64, seed=3000),
              graphgen.erdos_renyi(100_003, 800_000, seed=5), graphgen.path(700), graphgen.star(600, center=17)]
    modes = {bfs.MODE_DO: oracle.MODE_DO, bfs.MODE_TD_ONLY: oracle.MODE_TD, bfs.MODE_BU_ONLY: oracle.MODE_BU}
    for e in graphs:
        case = Case(bfs, e)
        g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
        h = oracle.hub_first(case.ref)
        assert np.array_equal(g.hub_first_host(), h.cols), e.name
        # row heads: [deg(u), the first min(deg, 7) ids of u's hub-first row, 0 after them]
        deg = np.diff(case.ref.offsets)
        want = np.zeros((e.n, 8), np.int32)
        want[:, 0] = deg
        for t in range(7):
            has = deg > t
            want[has, 1 + t] = h.cols[case.ref.offsets[:-1][has] + t]
        assert np.array_equal(g.row_heads_host(), want), e.name
        # the plane a bottom-up sweep streams (first id of each hub-first row, bit 31
        # set for two or more neighbours, 0 for degree 0) and the degree clamped to a byte
        first, deg8 = g.bu_planes_host()
        assert np.array_equal(first.view(np.uint32), want[:, 1].astype(np.uint32) | np.where(deg >= 2, 1 << 31, 0)
                              .astype(np.uint32)), e.name
        assert np.array_equal(deg8, np.minimum(deg, 255).astype(np.uint8)), e.name
        case.g.close()
        case.g = g
        deg = np.diff(case.ref.offsets)
        roots = [int(v) for v in np.flatnonzero(deg > 0)[[0, -1]]] + [int(np.argmax(deg))]
        for root in roots:
            want = oracle.levels(case.ref, root)
            for mode, omode in modes.items():
                opts = bfs.options(mode=mode, bu_rows=bfs.BU_ROWS_HUB_FIRST)
                lv, pa, info = case.run(root, opts, stats=True)
                assert np.array_equal(lv, want), (e.name, root, mode)
                assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), (e.name, root, mode)
                s = oracle.do_schedule(h, want, omode, 14, 24)
                rec = info["records"]
                for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
                    assert np.array_equal(rec[:, col], getattr(s, name)), (e.name, root, mode, name)
    plain = Case(bfs, graphgen.path(40))
    with pytest.raises(bfs.BfsError) as ex:
        plain.run(0, bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST))
    assert ex.value.status == 7          # BFS_ERR_UNSUPPORTED: graph built without the flag
    with pytest.raises(bfs.BfsError) as ex:
        plain.g.row_heads_host()
    assert ex.value.status == 1          # BFS_ERR_INVALID: no row heads without the flag
    g = bfs.Graph.from_edges(plain.e.src, plain.e.dst, plain.e.n, hub_first=True)
    with pytest.raises(bfs.BfsError) as ex:
        g.run(0, parent=plain.parent, opts=bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST,
                                                        parent_mode=bfs.PARENT_MIN_ID))
    assert ex.value.status == 1          # BFS_ERR_INVALID: minimum-id parents need id order
    g.close()


def test_deep_levels_and_partial_outputs(gpu_lib):
    """Depths past 253 (levels are staged one byte per vertex up to depth 253,
    written directly beyond it), with both outputs, level only and parent only, in
    every direction mode and both parent modes; a level-only run followed by a
    parent-only one must not leave stale values."""
    import torch
    bfs = gpu_lib
    n = 700
    case = Case(bfs, graphgen.path(n))
    lv_only = torch.empty(n, dtype=torch.int32, device="cuda")
    pa_only = torch.empty(n, dtype=torch.int32, device="cuda")
    for root in (0, 350, n - 1):
        want = np.abs(np.arange(n) - root)
        pwant = np.where(np.arange(n) < root, np.arange(n) + 1, np.arange(n) - 1)
        pwant[root] = root
        for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY):
            for pm in (bfs.PARENT_ANY, bfs.PARENT_MIN_ID):
                opts = bfs.options(mode=mode, parent_mode=pm)
                lv, pa, info = case.run(root, opts, stats=True)
                assert np.array_equal(lv, want), (root, mode, pm)
                assert np.array_equal(pa, pwant), (root, mode, pm)
                assert info["num_levels"] == want.max() + 1
                lv_only.fill_(-7)
                case.g.run(root, level=lv_only, opts=opts)
                assert np.array_equal(lv_only.cpu().numpy(), want), (root, mode, pm)
                pa_only.fill_(-7)
                case.g.run(root, parent=pa_only, opts=opts)
                assert np.array_equal(pa_only.cpu().numpy(), pwant), (root, mode, pm)
    # the same over the hub-first rows (first-probe sweep, final whole-sector pass),
    # and with outputs that are 4- but not 16-byte aligned (the pass's scalar path)
    g = bfs.Graph.from_edges(case.e.src, case.e.dst, n, hub_first=True)
    buf = torch.empty(2 * n + 8, dtype=torch.int32, device="cuda")
    for root in (0, 350, n - 1):
        want = np.abs(np.arange(n) - root)
        pwant = np.where(np.arange(n) < root, np.arange(n) + 1, np.arange(n) - 1)
        pwant[root] = root
        for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY):
            opts = bfs.options(mode=mode, bu_rows=bfs.BU_ROWS_HUB_FIRST)
            for lv_t, pa_t in ((case.level, case.parent), (buf[1:n + 1], buf[n + 3:2 * n + 3])):
                lv_t.fill_(-7)
                pa_t.fill_(-7)
                g.run(root, parent=pa_t, level=lv_t, opts=opts)
                assert np.array_equal(lv_t.cpu().numpy(), want), (root, mode)
                assert np.array_equal(pa_t.cpu().numpy(), pwant), (root, mode)
            lv_only.fill_(-7)
            g.run(root, level=lv_only, opts=opts)
            assert np.array_equal(lv_only.cpu().numpy(), want), (root, mode)
            pa_only.fill_(-7)
            g.run(root, parent=pa_only, opts=opts)
            assert np.array_equal(pa_only.cpu().numpy(), pwant), (root, mode)
    g.close()


def test_degree_zero_root_and_empty_graph(gpu_lib):
    bfs = gpu_lib
    e = graphgen.from_pairs(70, [(0, 1), (1, 2), (5, 5), (40, 41)])
    case = Case(bfs, e)
    for root in (5, 69, 0, 40):
        want = oracle.levels(case.ref, root)
        for mode in (bfs.MODE_DO, bfs.MODE_BU_ONLY, bfs.MODE_TD_ONLY):
            lv, pa, info = case.run(root, bfs.options(mode=mode), stats=True)
            assert np.array_equal(lv, want)
            assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1)
    empty = Case(bfs, graphgen.from_pairs(10, []))
    lv, pa, info = empty.run(3, stats=True)
    assert lv.tolist() == [-1, -1, -1, 0, -1, -1, -1, -1, -1, -1] and pa[3] == 3 and info["num_levels"] == 1


def test_outputs_optional(gpu_lib):
    import torch
    bfs = gpu_lib
    w = workloads.RMAT[12]
    e = w.edges()
    case = Case(bfs, e)
    root = int(w.roots(e, 1)[0])
    want = oracle.levels(case.ref, root)
    lv = torch.empty(e.n, dtype=torch.int32, device="cuda")
    case.g.run(root, level=lv)
    assert np.array_equal(lv.cpu().numpy(), want)
    pa = torch.empty(e.n, dtype=torch.int32, device="cuda")
    case.g.run(root, parent=pa)
    pa = pa.cpu().numpy()
    assert np.array_equal(pa >= 0, want >= 0)
    info = case.g.run(root, stats=True)
    assert info["reached"] == int((want >= 0).sum())


def test_multiroot_disjoint_union_equals_parts(gpu_lib):
    """An uneven batch of graphs as one search over their disjoint union."""
    bfs = gpu_lib
    parts = [graphgen.rmat(s, seed=500 + s) for s in (6, 9, 11, 12, 8, 10)]
    u, offs = graphgen.disjoint_union(parts)
    roots = [int(offs[i]) + int(graphgen.pick_roots(p, 1, 9 + i)[0]) for i, p in enumerate(parts)]
    case = Case(bfs, u)
    for mode in (bfs.MODE_DO, bfs.MODE_TD_ONLY, bfs.MODE_BU_ONLY):
        case.g.run_multiroot(roots, parent=case.parent, level=case.level, opts=bfs.options(mode=mode))
        lv = case.level.cpu().numpy()
        pa = case.parent.cpu().numpy()
        for i, p in enumerate(parts):
            pr = oracle.build_csr(p.n, p.src, p.dst)
            want = oracle.levels(pr, roots[i] - int(offs[i]))
            assert np.array_equal(lv[offs[i]:offs[i + 1]], want), (i, mode)
        for i in range(len(parts)):
            assert pa[roots[i]] == roots[i]


def test_multiroot_nearest_root_distance(gpu_lib):
    """Roots in one component: level = distance to the nearest root (oracle on a super-root graph)."""
    bfs = gpu_lib
    e = graphgen.rmat(11, seed=42)
    roots = graphgen.pick_roots(e, 5, 3).tolist()
    case = Case(bfs, e)
    case.g.run_multiroot(roots + roots[:2], parent=case.parent, level=case.level)
    lv = case.level.cpu().numpy()
    sup = e.n
    aug = graphgen.EdgeList(e.n + 1, np.concatenate([e.src, np.full(len(roots), sup, np.int32)]),
                            np.concatenate([e.dst, np.array(roots, np.int32)]))
    ref = oracle.build_csr(aug.n, aug.src, aug.dst)
    d = oracle.levels(ref, sup)[: e.n]
    want = np.where(d >= 1, d - 1, -1)
    assert np.array_equal(lv, want)


def test_invalid_arguments(gpu_lib):
    import torch
    bfs = gpu_lib
    e = graphgen.rmat(8, seed=1)
    case = Case(bfs, e)
    with pytest.raises(bfs.BfsError) as ex:
        case.g.run(e.n)
    assert ex.value.status == 1
    with pytest.raises(bfs.BfsError) as ex:
        case.g.run(-1)
    assert ex.value.status == 1
    with pytest.raises(bfs.BfsError):
        case.g.run(0, parent=case.parent, opts=bfs.options(parent_mode=7))
    with pytest.raises(bfs.BfsError):
        bfs.Graph.from_edges(np.array([0, 5], np.int32), np.array([1, 300], np.int32), 10)
    # CSR validation
    ref = oracle.build_csr(e.n, e.src, e.dst)
    g2 = bfs.Graph.from_csr(ref.offsets, ref.cols, e.n, check_symmetry=True)
    off, cols = g2.csr_host()
    assert np.array_equal(off, ref.offsets) and np.array_equal(cols, ref.cols)
    bad = ref.cols.copy()
    row = int(np.argmax(np.diff(ref.offsets)))
    s = int(ref.offsets[row])
    bad[s], bad[s + 1] = bad[s + 1], bad[s]
    with pytest.raises(bfs.BfsError):
        bfs.Graph.from_csr(ref.offsets, bad, e.n)
    bad = ref.cols.copy()
    bad[s] = row
    with pytest.raises(bfs.BfsError):
        bfs.Graph.from_csr(ref.offsets, bad, e.n)
    # directed (asymmetric) CSR: rejected only when asked to check
    off = np.array([0, 1, 1], np.int64)
    cols = np.array([1], np.int32)
    bfs.Graph.from_csr(off, cols, 2).close()
    with pytest.raises(bfs.BfsError):
        bfs.Graph.from_csr(off, cols, 2, check_symmetry=True)


def test_barrier_timeout_returns_error_and_recovers(gpu_lib):
    """A grid barrier that waits for an arrival that never comes gives up after timeout_ms,
    reports BFS_ERR_TIMEOUT, and the next search on the same graph is correct."""
    bfs = gpu_lib
    w = workloads.RMAT[10]
    e = w.edges()
    case = Case(bfs, e)
    root = int(w.roots(e, 1)[0])
    L = bfs._lib
    L.check(L.load().bfs_debug_set_barrier_extra(case.g.handle, 1), "debug_set_barrier_extra")
    with pytest.raises(bfs.BfsError) as ex:
        case.run(root, bfs.options(timeout_ms=200), stats=True)
    assert ex.value.status == 4
    L.check(L.load().bfs_debug_set_barrier_extra(case.g.handle, 0), "debug_set_barrier_extra")
    lv, pa, _ = case.run(root, stats=True)
    assert np.array_equal(lv, oracle.levels(case.ref, root))


def test_streams_and_repeat(gpu_lib):
    import torch
    bfs = gpu_lib
    w = workloads.RMAT[13]
    e = w.edges()
    case = Case(bfs, e)
    roots = w.roots(e, 8).tolist()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.empty(e.n, dtype=torch.int32, device="cuda") for _ in roots]
    for i, r in enumerate(roots):
        case.g.run(r, level=outs[i], stream=s1 if i % 2 else s2)
    case.g.sync(s1)
    case.g.sync(s2)
    torch.cuda.synchronize()
    for i, r in enumerate(roots):
        assert np.array_equal(outs[i].cpu().numpy(), oracle.levels(case.ref, r))


def test_autotune_picks_a_grid_point_and_levels_do_not_change(gpu_lib, tmp_path, monkeypatch):
    bfs = gpu_lib
    from paper_1705_04590_gb300 import autotune
    w = workloads.RMAT[14]
    e = w.edges()
    case = Case(bfs, e)
    roots = w.roots(e, 4).tolist()
    best, ms = autotune.autotune(case.g, roots)
    assert best.alpha in (6, 14, 24, 32, 96) and best.beta in (12, 24, 64, 128)
    assert best.td_big_degree in (64, 96, 256) and best.td_chunk in (0, 128, 256, 512, 1024)
    assert best.ctas_per_sm in (0, 1) and best.cluster_size in (0, 1, 8, 16)
    assert ms > 0
    monkeypatch.setenv("BFS_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    o1 = autotune.tuned_options(case.g, roots)
    o2 = autotune.tuned_options(case.g, roots)        # served from the cache file
    knobs = ("alpha", "beta", "td_big_degree", "td_chunk", "ctas_per_sm", "cluster_size")
    assert [getattr(o1, k) for k in knobs] == [getattr(o2, k) for k in knobs]
    for root in roots:
        lv, pa, _ = case.run(root, o1)
        assert np.array_equal(lv, oracle.levels(case.ref, root))
        assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1)


def test_edges64_entry_point(gpu_lib):
    """bfs_graph_create_from_edges64 (64-bit endpoint arrays, host and device): the CSR
    equals the oracle's bit for bit and searches are exact; an endpoint outside
    [0, n) is refused."""
    import torch
    bfs = gpu_lib
    e = graphgen.random_small(5000, 40000, 3)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    s64, d64 = e.src.astype(np.int64), e.dst.astype(np.int64)
    for src, dst in ((s64, d64), (torch.from_numpy(s64).cuda(), torch.from_numpy(d64).cuda())):
        g = bfs.Graph.from_edges(src, dst, e.n, hub_first=True)
        off, cols = g.csr_host()
        assert np.array_equal(off, ref.offsets) and np.array_equal(cols, ref.cols)
        lv = torch.empty(e.n, dtype=torch.int32, device="cuda")
        root = int(np.argmax(ref.degree()))
        g.run(root, level=lv, opts=bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST))
        assert np.array_equal(lv.cpu().numpy(), oracle.levels(ref, root))
        g.close()
    bad = s64.copy()
    bad[77] = e.n
    with pytest.raises(bfs.BfsError) as ex:
        bfs.Graph.from_edges(bad, d64, e.n)
    assert ex.value.status == 1


def test_launch_knobs_keep_levels_exact(gpu_lib):
    """The tuning knobs (top-down chunk size, CTAs per SM, hub cut-off) change the
    work split only: levels bit-exact, parents certified, per-level counters equal
    to the oracle's schedule; out-of-range values are refused."""
    bfs = gpu_lib
    w = workloads.RMAT[16]
    e = w.edges()
    case = Case(bfs, e)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    h = oracle.hub_first(case.ref)
    for root in w.roots(e, 2).tolist():
        want = oracle.levels(case.ref, root)
        for kw in (dict(td_chunk=64), dict(td_chunk=4096, td_big_degree=64), dict(ctas_per_sm=1),
                   dict(ctas_per_sm=1, td_chunk=128, bu_rows=bfs.BU_ROWS_HUB_FIRST)):
            hub = kw.get("bu_rows") == bfs.BU_ROWS_HUB_FIRST
            case.g, keep = (g, case.g) if hub else (case.g, None)
            lv, pa, info = case.run(root, bfs.options(**kw), stats=True)
            if keep is not None:
                case.g = keep
            assert np.array_equal(lv, want), (root, kw)
            assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), (root, kw)
            s = oracle.do_schedule(h if hub else case.ref, want, oracle.MODE_DO, 14, 24)
            for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
                assert np.array_equal(info["records"][:, col], getattr(s, name)), (root, kw, name)
    for kw in (dict(td_chunk=32), dict(td_chunk=5000), dict(ctas_per_sm=-1)):
        with pytest.raises(bfs.BfsError) as ex:
            case.run(0, bfs.options(**kw))
        assert ex.value.status == 1
    g.close()


def test_powerlaw_graph_bench_configuration(gpu_lib):
    """The Twitter-sized workload's generator (power-law expected degrees, exponent 2.1,
    rank offset 50) at 1/32 of its size (1.92 M vertices, 45.9 M edges), searched as
    bench.py searches it: levels bit-exact for 3 roots, parents certified, per-level
    counters equal to the oracle's schedule over the hub-first rows."""
    import torch
    bfs = gpu_lib
    e = graphgen.powerlaw(61_500_000 // 32, 1_470_000_000 // 32, 2.1, 50.0, seed=4000)
    ref = oracle.build_csr(e.n, e.src, e.dst)
    labels = oracle.components(ref)
    h = oracle.hub_first_rows(ref)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n, hub_first=True)
    level = torch.empty(e.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(e.n, dtype=torch.int32, device="cuda")
    opts = bfs.options(bu_rows=bfs.BU_ROWS_HUB_FIRST)
    for root in graphgen.pick_roots(e, 3, 4001).tolist():
        info = g.run(root, parent=parent, level=level, opts=opts, stats=True, record_levels=256)
        lv, pa = level.cpu().numpy(), parent.cpu().numpy()
        want = oracle.levels(ref, root)
        assert np.array_equal(lv, want), root
        assert oracle.certify(ref, root, lv, pa, labels) == (0, -1), root
        s = oracle.do_schedule(h, want, oracle.MODE_DO, 14, 24)
        for col, name in enumerate(["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]):
            assert np.array_equal(info["records"][:, col], getattr(s, name)), (root, name)
    g.close()

"""Pins of the CPU oracle against things other than itself (CPU only).

* Figure 3 fixture (hand-derived, tests/golden/fig3.txt)
* brute-force unit-weight relaxation on tiny graphs
* networkx shortest paths / components (an independent library), where installed
* closed forms: path, star, complete graph, torus
* Algorithm 1 and Algorithm 2 give the same levels (direction invariance)
* planted mistakes are rejected by the certificate
* the direction-optimizing schedule against hand-derived cases and a literal
  Python walk of Algorithm 2 on tiny graphs
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from tests.golden import fixtures


def csr(g):
    return oracle.build_csr(g.n, g.src, g.dst)


# ------------------------------------------------------------------ CSR build

def _set_csr(n, src, dst):
    adj = [set() for _ in range(n)]
    for u, v in zip(src.tolist(), dst.tolist()):
        if u != v:
            adj[u].add(v)
            adj[v].add(u)
    return [sorted(a) for a in adj]


@pytest.mark.parametrize("seed", range(6))
def test_build_csr_matches_set_definition(seed):
    g = graphgen.random_small(40, 120, seed)
    c = csr(g)
    want = _set_csr(g.n, g.src, g.dst)
    assert c.offsets[0] == 0 and len(c.offsets) == g.n + 1
    for v in range(g.n):
        assert c.cols[c.offsets[v]:c.offsets[v + 1]].tolist() == want[v]


def test_build_csr_fig3():
    f = fixtures.fig3()
    pairs = [(r, c) for r, cs in f["rows"].items() for c in cs]
    g = graphgen.from_pairs(6, pairs)
    c = csr(g)
    edges = {(u, int(v)) for u in range(6) for v in c.cols[c.offsets[u]:c.offsets[u + 1]]}
    tree = {(0, 1), (0, 3), (1, 4), (2, 3), (2, 5)}
    assert edges == tree | {(b, a) for a, b in tree}


def test_build_csr_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([0, 5], np.int32), np.array([1, 1], np.int32))


# ------------------------------------------------------------------ BFS pins

def test_fig3_levels_and_parents():
    f = fixtures.fig3()
    pairs = [(r, c) for r, cs in f["rows"].items() for c in cs]
    c = csr(graphgen.from_pairs(6, pairs))
    for fn in (oracle.bfs_topdown, oracle.bfs_bottomup):
        parent, level, L = fn(c, f["root"])
        assert level.tolist() == f["level"]
        assert parent.tolist() == f["parent"]
        assert L == 4


def _tiny_graphs():
    gs = [graphgen.random_small(n, m, s) for n, m, s in
          [(1, 0, 0), (2, 1, 1), (5, 3, 2), (16, 10, 3), (16, 40, 4), (33, 20, 5), (64, 64, 6), (64, 300, 7),
           (100, 90, 8), (128, 128, 9), (200, 400, 10), (256, 256, 11)]]
    gs += [graphgen.path(17), graphgen.cycle(12), graphgen.star(20), graphgen.complete(9)]
    two, _ = graphgen.disjoint_union([graphgen.path(5), graphgen.complete(4), graphgen.from_pairs(3, [])])
    gs.append(two)
    return gs


@pytest.mark.parametrize("gi", range(17))
def test_topdown_matches_brute_force(gi):
    g = _tiny_graphs()[gi]
    c = csr(g)
    for root in range(g.n):
        bf = oracle.brute_force_levels(g.n, g.src, g.dst, root)
        p, lv, L = oracle.bfs_topdown(c, root)
        assert np.array_equal(lv, bf), (g.name, root)
        assert L == bf.max() + 1
        assert oracle.certify(c, root, lv, p) == (0, -1)


@pytest.mark.parametrize("gi", range(17))
def test_bottomup_equals_topdown(gi):
    g = _tiny_graphs()[gi]
    c = csr(g)
    for root in range(0, g.n, max(1, g.n // 13)):
        _, l1, L1 = oracle.bfs_topdown(c, root)
        p2, l2, L2 = oracle.bfs_bottomup(c, root)
        assert np.array_equal(l1, l2) and L1 == L2
        # in-order early exit over sorted rows yields the minimum-id parent
        assert np.array_equal(p2, oracle.min_parent(c, l2))


def test_against_networkx():
    nx = pytest.importorskip("networkx")
    g = graphgen.rmat(10, seed=1010)
    c = csr(g)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from((u, v) for u, v in zip(g.src.tolist(), g.dst.tolist()) if u != v)
    for root in graphgen.pick_roots(g, 4, 99).tolist():
        lv = oracle.levels(c, root)
        d = nx.single_source_shortest_path_length(G, root)
        want = np.full(g.n, -1, np.int32)
        for k, v in d.items():
            want[k] = v
        assert np.array_equal(lv, want)
    lab = oracle.components(c)
    comps = list(nx.connected_components(G))
    assert len(set(lab.tolist())) == len(comps)
    for comp in comps:
        assert len({int(lab[v]) for v in comp}) == 1
        assert int(lab[next(iter(comp))]) == min(comp)


def test_closed_forms_path_star_complete():
    n = 50
    c = csr(graphgen.path(n))
    for r in (0, 17, 49):
        assert np.array_equal(oracle.levels(c, r), np.abs(np.arange(n) - r))
    c = csr(graphgen.star(30, center=4))
    lv = oracle.levels(c, 4)
    assert lv[4] == 0 and np.all(np.delete(lv, 4) == 1)
    lv = oracle.levels(c, 7)
    assert lv[7] == 0 and lv[4] == 1 and np.all(np.delete(lv, [4, 7]) == 2)
    c = csr(graphgen.complete(12))
    lv = oracle.levels(c, 3)
    assert lv[3] == 0 and np.all(np.delete(lv, 3) == 1)


@pytest.mark.parametrize("side", [5, 16, 33])
def test_torus_closed_form(side):
    g = graphgen.torus(side, seed=3000)
    inv = graphgen.torus_coordinates(side, seed=3000)
    c = csr(g)
    x, y = inv % side, inv // side
    for root in [0, 7, side * side - 1]:
        lv = oracle.levels(c, root)
        dx = np.abs(x - x[root])
        dy = np.abs(y - y[root])
        want = np.minimum(dx, side - dx) + np.minimum(dy, side - dy)
        assert np.array_equal(lv, want)
        assert lv.max() == 2 * (side // 2)


def test_isolated_root_and_degree_zero():
    g = graphgen.from_pairs(5, [(0, 1), (1, 2), (3, 3)])
    c = csr(g)
    p, lv, L = oracle.bfs_topdown(c, 3)          # only a self-loop: degree 0
    assert lv.tolist() == [-1, -1, -1, 0, -1] and p.tolist() == [-1, -1, -1, 3, -1] and L == 1
    p, lv, L = oracle.bfs_topdown(c, 4)
    assert lv.tolist() == [-1, -1, -1, -1, 0] and L == 1


# ------------------------------------------------------------------ certificate

def test_certificate_rejects_planted_mistakes():
    g = graphgen.rmat(9, seed=1009)
    c = csr(g)
    root = int(graphgen.pick_roots(g, 1, 5)[0])
    p, lv, _ = oracle.bfs_topdown(c, root)
    lab = oracle.components(c)
    assert oracle.certify(c, root, lv, p, lab) == (0, -1)
    reached = np.flatnonzero((lv > 1))
    v = int(reached[0])
    # level off by one
    bad = lv.copy(); bad[v] += 1
    assert oracle.certify(c, root, bad, p, lab)[0] in (2, 3)
    # all levels shifted by +1 except root: parent levels break
    bad = np.where(lv > 0, lv + 1, lv).astype(np.int32)
    assert oracle.certify(c, root, bad, p, lab)[0] in (2, 3)
    assert oracle.certify(c, root, bad, None, lab)[0] == 3
    # parent that is not a neighbour
    badp = p.copy(); badp[v] = root
    if not np.any(c.cols[c.offsets[root]:c.offsets[root + 1]] == v):
        assert oracle.certify(c, root, lv, badp, lab) == (2, v)
    # parent at the same level
    same = [int(u) for u in c.cols[c.offsets[v]:c.offsets[v + 1]] if lv[u] == lv[v]]
    if same:
        badp = p.copy(); badp[v] = same[0]
        assert oracle.certify(c, root, lv, badp, lab) == (2, v)
    # a reached vertex reported unreachable
    bad = lv.copy(); bad[v] = -1
    badp = p.copy(); badp[v] = -1
    assert oracle.certify(c, root, bad, badp, lab)[0] in (4, 5)
    # wrong root
    bad = lv.copy(); bad[root] = 1
    assert oracle.certify(c, root, bad, p, lab)[0] == 1
    # an unreachable vertex (other component) reported at some level
    unreached = np.flatnonzero(lv < 0)
    if unreached.size:
        bad = lv.copy(); bad[unreached[0]] = 3
        assert oracle.certify(c, root, bad, None, lab)[0] in (3, 4, 5)


# ------------------------------------------------------------------ DO schedule

def _alg2_walk(c, level, d):
    """Literal Algorithm 2 step at level d in Python: for each unvisited vertex
    with neighbours, count neighbour examinations up to the first one in the
    frontier (inclusive)."""
    scanned = examined = 0
    for u in range(c.n):
        if 0 <= level[u] <= d:
            continue
        row = c.cols[c.offsets[u]:c.offsets[u + 1]].tolist()
        if not row:
            continue
        scanned += 1
        for k, v in enumerate(row):
            examined += 1
            if level[v] == d:
                break
    return scanned, examined


def test_schedule_star_hand_derived():
    n = 100
    c = csr(graphgen.star(n, center=0))
    s = oracle.do_schedule(c, oracle.levels(c, 0))
    # level 0: m_f = 99, m_u = 99 -> 99*14 > 99 -> bottom-up; level 1: n_f = 99, 99*24 >= 100 stays
    assert s.dir.tolist() == [1, 1]
    assert s.nf.tolist() == [1, 99] and s.mf.tolist() == [99, 99]
    assert s.scanned.tolist() == [99, 0] and s.examined.tolist() == [99, 0]
    s = oracle.do_schedule(c, oracle.levels(c, 5))
    # level 0 (leaf 5): m_f = 1, m_u = 197 -> top-down; level 1 (centre): 99*14 > 98 -> bottom-up
    assert s.dir.tolist() == [0, 1, 1]
    assert s.nf.tolist() == [1, 1, 98] and s.mf.tolist() == [1, 99, 98]
    assert s.nnext.tolist() == [1, 98, 0]


def test_schedule_path_switches_back():
    n = 100
    c = csr(graphgen.path(n))
    s = oracle.do_schedule(c, oracle.levels(c, 0))
    # level d frontier {d}: m_f = 2, m_u = 197 - 2d; bottom-up from d = 85, then n_f*24 < 100
    # sends it back to top-down on the next level, alternating.
    assert s.dir[:85].tolist() == [0] * 85
    assert s.dir[85] == 1 and s.dir[86] == 0 and s.dir[87] == 1
    td = oracle.do_schedule(c, oracle.levels(c, 0), mode=oracle.MODE_TD)
    assert td.dir.tolist() == [0] * n
    bu = oracle.do_schedule(c, oracle.levels(c, 0), mode=oracle.MODE_BU)
    assert bu.dir.tolist() == [1] * n


@pytest.mark.parametrize("seed", range(4))
def test_schedule_counts_match_literal_walk(seed):
    g = graphgen.rmat(8, seed=300 + seed)
    c = csr(g)
    root = int(graphgen.pick_roots(g, 1, seed)[0])
    lv = oracle.levels(c, root)
    s = oracle.do_schedule(c, lv, mode=oracle.MODE_BU)
    deg = np.diff(c.offsets)
    for d in range(s.num_levels):
        assert s.nf[d] == np.sum(lv == d)
        assert s.mf[d] == deg[lv == d].sum()
        assert s.nnext[d] == np.sum(lv == d + 1)
        assert (s.scanned[d], s.examined[d]) == _alg2_walk(c, lv, d)
    sd = oracle.do_schedule(c, lv, mode=oracle.MODE_DO)
    # re-derive each direction from the rule with m_u recomputed from scratch
    cur = 0
    for d in range(sd.num_levels):
        m_u = deg[(lv > d) | (lv < 0)].sum()
        if cur == 0 and sd.mf[d] * 14 > m_u:
            cur = 1
        elif cur == 1 and sd.nf[d] * 24 < c.n:
            cur = 0
        assert sd.dir[d] == cur


# ------------------------------------------------------------------ DCSC definition

def _fig3_csr():
    f = fixtures.fig3()
    off = np.zeros(7, np.int64)
    cols = []
    for r in range(6):
        cols += sorted(f["rows"][r])
        off[r + 1] = len(cols)
    return f, off, np.array(cols, np.int64)


def test_dcsc_fig3_whole_matrix():
    """Figure 3's matrix as one tile: JC/CP/IR exactly as derived by hand."""
    f, off, cols = _fig3_csr()
    tp, JC, CP, IR = oracle.dcsc_tiles(6, off, cols, 6, 6)
    assert tp.tolist() == [0, len(f["jc"])]
    assert JC.tolist() == f["jc"] and CP.tolist() == f["cp"] and IR.tolist() == f["ir"]


def test_dcsc_fig3_two_thread_row_split():
    """The row split of the multithreaded 2D layout (rows 0-2 and 3-5, one DCSC each)."""
    f, off, cols = _fig3_csr()
    tp, JC, CP, IR = oracle.dcsc_tiles(6, off, cols, 3, 6)
    for i, (jc, cp, ir) in enumerate(f["split"]):
        a, b = tp[i], tp[i + 1]
        assert JC[a:b].tolist() == jc
        assert (CP[a:b + 1] - CP[a]).tolist() == cp
        assert (IR[CP[a]:CP[b]] + 3 * i).tolist() == ir


def test_dcsc_round_trip_random():
    """Expanding every tile's DCSC gives back exactly the CSR's nonzeros."""
    g = graphgen.random_small(50, 200, 9)
    c = csr(g)
    for rb, cb in ((7, 7), (5, 13), (50, 50), (64, 3)):
        tp, JC, CP, IR = oracle.dcsc_tiles(c.n, c.offsets, c.cols, rb, cb)
        ncb = (c.n + cb - 1) // cb
        got = set()
        for t in range(len(tp) - 1):
            i, j = divmod(t, ncb)
            for x in range(tp[t], tp[t + 1]):
                for e in range(CP[x], CP[x + 1]):
                    got.add((i * rb + int(IR[e]), j * cb + int(JC[x])))
        want = {(u, int(v)) for u in range(c.n) for v in c.cols[c.offsets[u]:c.offsets[u + 1]]}
        assert got == want
        assert np.all(np.diff(CP) > 0)


def test_certificate_without_parents_needs_predecessors():
    """Level-only certification: levels that are too small pass the edge-span and
    component checks, so the certificate must also find a predecessor one level
    closer for every reached vertex."""
    g = graphgen.rmat(9, seed=1009)
    c = csr(g)
    root = int(graphgen.pick_roots(g, 1, 5)[0])
    lv = oracle.levels(c, root)
    lab = oracle.components(c)
    assert oracle.certify(c, root, lv, None, lab) == (0, -1)
    flat = np.where(lv > 0, 1, lv).astype(np.int32)       # every reached vertex at level 1
    assert (lv > 1).any()
    assert oracle.certify(c, root, flat, None, lab)[0] == 2
    zero = lv.copy()
    zero[np.flatnonzero(lv == 1)[0]] = 0                   # a second vertex at level 0
    assert oracle.certify(c, root, zero, None, lab)[0] == 2


# ------------------------------------------------------------------ hub-first row order

@pytest.mark.parametrize("seed", range(3))
def test_hub_first_rows_match_definition(seed):
    """Each row of hub_first() is the same neighbour set, in the order given by a
    plain Python sort on (-degree, id) of the set-built adjacency."""
    g = graphgen.rmat(9, seed=700 + seed)
    c = csr(g)
    h = oracle.hub_first(c)
    adj = _set_csr(g.n, g.src, g.dst)
    deg = [len(a) for a in adj]
    assert np.array_equal(h.offsets, c.offsets)
    for u in range(g.n):
        want = sorted(adj[u], key=lambda v: (-deg[v], v))
        assert h.cols[h.offsets[u]:h.offsets[u + 1]].tolist() == want


@pytest.mark.parametrize("seed", range(3))
def test_hub_first_rows_in_c_match_definition(seed):
    """hub_first_rows (row by row in C: insertion sort for rows of <= 32, merge
    sort above) gives every row in the order of a plain Python sort on (-degree,
    id) of the set-built adjacency, and equals the lexsort hub_first() on larger
    graphs whose hub rows take the merge-sort branch."""
    g = graphgen.rmat(9, seed=700 + seed)
    c = csr(g)
    h = oracle.hub_first_rows(c)
    adj = _set_csr(g.n, g.src, g.dst)
    deg = [len(a) for a in adj]
    assert np.array_equal(h.offsets, c.offsets)
    assert max(deg) > 32
    for u in range(g.n):
        want = sorted(adj[u], key=lambda v: (-deg[v], v))
        assert h.cols[h.offsets[u]:h.offsets[u + 1]].tolist() == want
    for e in (graphgen.rmat(13, seed=90 + seed), graphgen.star(300, center=7 + seed), graphgen.from_pairs(5, [])):
        c = csr(e)
        assert np.array_equal(oracle.hub_first_rows(c).cols, oracle.hub_first(c).cols)


@pytest.mark.parametrize("seed", range(3))
def test_hub_first_schedule_counts_follow_row_order(seed):
    """Levels do not depend on the row order; the bottom-up examination counts of
    the schedule equal a literal walk of Algorithm 2 over the hub-first rows; and
    in that order each searcher stops at its frontier neighbour of highest degree."""
    g = graphgen.rmat(8, seed=310 + seed)
    c = csr(g)
    h = oracle.hub_first(c)
    root = int(graphgen.pick_roots(g, 1, seed)[0])
    lv = oracle.levels(c, root)
    assert np.array_equal(oracle.levels(h, root), lv)
    s = oracle.do_schedule(h, lv, mode=oracle.MODE_BU)
    for d in range(s.num_levels):
        assert (s.scanned[d], s.examined[d]) == _alg2_walk(h, lv, d)
    # a vertex reached at level d+1 examines, in hub-first order, up to and
    # including its first level-d neighbour of highest degree
    deg = np.diff(c.offsets)
    for d in range(s.num_levels):
        total = 0
        for u in np.flatnonzero((lv > d) | (lv < 0)):
            row = h.cols[h.offsets[u]:h.offsets[u + 1]]
            hits = np.flatnonzero(lv[row] == d)
            total += int(hits[0]) + 1 if hits.size else row.size
            if hits.size:
                assert deg[row[hits[0]]] == deg[row[lv[row] == d]].max()
        assert total == s.examined[d]


# ------------------------------------------------------------------ directed graphs

def _digraphs():
    gs = [graphgen.random_small(n, m, s) for n, m, s in [(2, 1, 1), (9, 20, 2), (40, 90, 3), (64, 300, 4),
                                                         (130, 260, 5)]]
    gs.append(graphgen.from_pairs(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 4), (5, 3), (1, 1), (0, 1)]))
    gs.append(graphgen.rmat(8, seed=91))
    return gs


@pytest.mark.parametrize("gi", range(7))
def test_directed_bfs_matches_brute_force_networkx_and_bottom_up(gi):
    """Directed graphs: Algorithm 1 over the out-edge CSR gives the brute-force
    directed distances and networkx's directed shortest-path lengths from every root;
    Algorithm 2 over the transpose gives the same levels; both outputs pass the
    directed certificate; the reached set equals networkx's descendants."""
    nx = pytest.importorskip("networkx")
    e = _digraphs()[gi]
    out, inn = oracle.build_digraph(e.n, e.src, e.dst)
    G = nx.DiGraph()
    G.add_nodes_from(range(e.n))
    G.add_edges_from((int(u), int(v)) for u, v in zip(e.src, e.dst) if u != v)
    for root in range(e.n):
        want = oracle.brute_force_levels(e.n, e.src, e.dst, root, directed=True)
        nxd = nx.single_source_shortest_path_length(G, root)
        assert np.array_equal(want, np.array([nxd.get(v, -1) for v in range(e.n)], np.int32))
        pa, lv, _ = oracle.bfs_topdown(out, root)
        assert np.array_equal(lv, want), root
        pb, lb, _ = oracle.bfs_bottomup(inn, root)
        assert np.array_equal(lb, want), root
        rch = oracle.reach(out, root)
        assert set(np.flatnonzero(rch).tolist()) == {root} | set(nx.descendants(G, root))
        assert oracle.certify_dir(out, root, lv, pa, rch) == (0, -1)
        assert oracle.certify_dir(out, root, lb, pb, rch) == (0, -1)
        assert oracle.certify_dir(out, root, lv, None, rch) == (0, -1)


def test_build_digraph_is_the_set_definition():
    e = graphgen.random_small(70, 400, 9)
    out, inn = oracle.build_digraph(e.n, e.src, e.dst)
    succ = [set() for _ in range(e.n)]
    pred = [set() for _ in range(e.n)]
    for u, v in zip(e.src.tolist(), e.dst.tolist()):
        if u != v:
            succ[u].add(v)
            pred[v].add(u)
    for u in range(e.n):
        assert out.cols[out.offsets[u]:out.offsets[u + 1]].tolist() == sorted(succ[u])
        assert inn.cols[inn.offsets[u]:inn.offsets[u + 1]].tolist() == sorted(pred[u])


def test_certify_dir_rejects_planted_mistakes():
    """Each planted mistake fails the directed certificate with its code; the
    reversed-parent case is one an undirected checker would accept."""
    e = graphgen.from_pairs(6, [(0, 1), (1, 2), (2, 3), (4, 0), (3, 5)])
    out, _ = oracle.build_digraph(e.n, e.src, e.dst)
    root = 0
    pa, lv, _ = oracle.bfs_topdown(out, root)
    assert lv.tolist() == [0, 1, 2, 3, -1, 4]
    assert oracle.certify_dir(out, root, lv, pa) == (0, -1)
    bad = lv.copy(); bad[2] = 3; bad[3] = 4; bad[5] = 5           # 1 -> 2 spans two levels
    assert oracle.certify_dir(out, root, bad, None)[0] in (2, 3)
    bad = lv.copy(); bad[4] = 1                                     # 4 is not reachable from 0
    assert oracle.certify_dir(out, root, bad, None) == (5, 4)
    bad = lv.copy(); bad[5] = -1                                    # 5 is reachable
    assert oracle.certify_dir(out, root, bad, None)[0] in (3, 5)
    # 0 -> 1, 0 -> 2, 1 -> 3, 3 -> 2: vertex 3 (level 2) has parent 1; vertex 2 is also one
    # level closer and joined to 3, but by 3 -> 2 only, so it is not a parent of 3
    e = graphgen.from_pairs(4, [(0, 1), (0, 2), (1, 3), (3, 2)])
    out, _ = oracle.build_digraph(e.n, e.src, e.dst)
    pa, lv, _ = oracle.bfs_topdown(out, 0)
    assert lv.tolist() == [0, 1, 1, 2] and pa[3] == 1
    wrong = pa.copy(); wrong[3] = 2
    assert oracle.certify_dir(out, 0, lv, wrong) == (2, 3)
    und = oracle.build_csr(e.n, e.src, e.dst)
    assert oracle.certify(und, 0, lv, wrong) == (0, -1)            # the undirected reading accepts it


@pytest.mark.parametrize("seed", range(3))
def test_directed_schedule_counts(seed):
    """do_schedule_dir: on an undirected graph it is do_schedule; on a directed one its
    bottom-up examination counts equal a literal Algorithm 2 walk over the in-rows,
    m_f sums out-degrees of the frontier, and the direction sequence follows the rule
    with m_u = in-degree sum of the vertices not yet reached, recomputed from scratch."""
    g = graphgen.rmat(9, seed=500 + seed)
    c = csr(g)
    root = int(graphgen.pick_roots(g, 1, seed)[0])
    lv = oracle.levels(c, root)
    for mode in (oracle.MODE_DO, oracle.MODE_BU):
        a = oracle.do_schedule(c, lv, mode)
        b = oracle.do_schedule_dir(c, c, lv, mode)
        for name in ("dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"):
            assert np.array_equal(getattr(a, name), getattr(b, name)), name
    out, inn = oracle.build_digraph(g.n, g.src, g.dst)
    pa, lv, _ = oracle.bfs_topdown(out, root)
    odeg, ideg = out.degree(), inn.degree()
    s = oracle.do_schedule_dir(out, inn, lv, oracle.MODE_BU)
    for d in range(s.num_levels):
        assert (s.scanned[d], s.examined[d]) == _alg2_walk(inn, lv, d)
        assert s.mf[d] == odeg[lv == d].sum() and s.nf[d] == (lv == d).sum()
    s = oracle.do_schedule_dir(out, inn, lv, oracle.MODE_DO, 14, 24)
    cur = 0
    for d in range(s.num_levels):
        unreached = (lv < 0) | (lv > d)
        m_u = int(ideg[unreached].sum())
        n_f, m_f = int((lv == d).sum()), int(odeg[lv == d].sum())
        if cur == 0 and m_f * 14 > m_u:
            cur = 1
        elif cur == 1 and n_f * 24 < g.n:
            cur = 0
        assert s.dir[d] == cur, d

"""Cluster levels: top-down levels with a small frontier run by thread-block
cluster 0 alone (frontier in distributed shared memory, one hardware cluster
barrier per level) while the rest of the grid waits.

Whatever the cluster size, levels must equal the oracle's (or the torus's
closed form) element by element, parents must pass the oracle's certificate,
MIN_ID parents must equal the oracle's, and the per-level counters must equal
the oracle's direction-optimizing schedule.  The hand-over cases are covered:
a frontier that outgrows a CTA's shared memory (entries spill to the global
queue), a vertex above the degree cap, the direction rule turning to
bottom-up, several roots, and a long path (thousands of cluster levels).
"""
import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 2, 4, 8, 16]
REC = ["dir", "nf", "mf", "nnext", "mnext", "scanned", "examined"]


class Case:
    def __init__(self, bfs, e):
        import torch
        self.e = e
        self.ref = oracle.build_csr(e.n, e.src, e.dst)
        self.g = bfs.Graph.from_edges(e.src, e.dst, e.n)
        self.labels = oracle.components(self.ref)
        self.level = torch.empty(e.n, dtype=torch.int32, device="cuda")
        self.parent = torch.empty(e.n, dtype=torch.int32, device="cuda")

    def run(self, root, opts):
        info = self.g.run(root, parent=self.parent, level=self.level, opts=opts, stats=True, record_levels=1 << 17)
        return self.level.cpu().numpy(), self.parent.cpu().numpy(), info


def _schedule_equal(info, s, tag):
    rec = info["records"]
    assert rec.shape[0] == s.num_levels, tag
    for i, k in enumerate(REC):
        assert np.array_equal(rec[:, i], getattr(s, k)), (tag, k)


def _cluster_levels(info) -> int:
    return int((info["records"][:, 8] == -1).sum())


def test_torus_every_cluster_size(gpu_lib):
    bfs = gpu_lib
    side = 256
    e = graphgen.torus(side, seed=3001)
    inv = graphgen.torus_coordinates(side, seed=3001)
    x, y = inv % side, inv // side
    case = Case(bfs, e)
    for root in graphgen.pick_roots(e, 2, 9).tolist():
        dx, dy = np.abs(x - x[root]), np.abs(y - y[root])
        want = np.minimum(dx, side - dx) + np.minimum(dy, side - dy)
        for mode, omode in ((bfs.MODE_DO, oracle.MODE_DO), (bfs.MODE_TD_ONLY, oracle.MODE_TD)):
            s = oracle.do_schedule(case.ref, want, omode, 14, 24)
            for c in SIZES:
                lv, pa, info = case.run(root, bfs.options(mode=mode, cluster_size=c))
                tag = (root, mode, c)
                assert np.array_equal(lv, want), tag
                assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), tag
                _schedule_equal(info, s, tag)
                nclu = _cluster_levels(info)
                if c == 1:
                    assert nclu == 0, tag
                else:
                    # maximum degree 4: automatic picks clusters of 16; every level is small
                    assert nclu >= side // 2, (tag, nclu)


@pytest.mark.parametrize("scale", [12, 16])
def test_rmat_forced_clusters(gpu_lib, scale):
    """R-MAT with clusters forced: cluster levels at the ends of the search, the grid
    (and bottom-up) in the middle; hand-overs at heavy vertices and at the switch."""
    bfs = gpu_lib
    w = workloads.RMAT[scale]
    e = w.edges()
    case = Case(bfs, e)
    total = 0
    for root in w.roots(e, 6).tolist():
        want = oracle.levels(case.ref, root)
        pmin = oracle.min_parent(case.ref, want)
        for mode, omode in ((bfs.MODE_DO, oracle.MODE_DO), (bfs.MODE_TD_ONLY, oracle.MODE_TD)):
            for alpha, beta in ((14, 24), (2, 100)):
                s = oracle.do_schedule(case.ref, want, omode, alpha, beta)
                for c in (8, 16):
                    tag = (scale, root, mode, alpha, c)
                    lv, pa, info = case.run(root, bfs.options(mode=mode, alpha=alpha, beta=beta, cluster_size=c))
                    assert np.array_equal(lv, want), tag
                    assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), tag
                    _schedule_equal(info, s, tag)
                    total += _cluster_levels(info)
        lv, pa, _ = case.run(root, bfs.options(parent_mode=bfs.PARENT_MIN_ID, cluster_size=16))
        assert np.array_equal(lv, want)
        assert np.array_equal(pa, pmin), root
    assert total > 0


@pytest.mark.parametrize("hubs,c", [(320, 16), (160, 8)])
def test_spill_past_shared_memory(gpu_lib, hubs, c):
    """Hubs of degree 128 under one root: the cluster level that expands them
    finds 127 leaves per hub, more than a CTA's shared-memory buffer holds for
    the CTAs that took 32 hubs; the surplus goes to the global queue and the
    grid takes the next level."""
    bfs = gpu_lib
    leaves = 127
    n = 1 + hubs + hubs * leaves
    h = np.arange(1, hubs + 1, dtype=np.int32)
    src = np.concatenate([np.zeros(hubs, np.int32), np.repeat(h, leaves)])
    dst = np.concatenate([h, np.arange(1 + hubs, n, dtype=np.int32)])
    e = graphgen.EdgeList(n, src, dst)
    case = Case(bfs, e)
    want = oracle.levels(case.ref, 0)
    s = oracle.do_schedule(case.ref, want, oracle.MODE_TD, 14, 24)
    lv, pa, info = case.run(0, bfs.options(mode=bfs.MODE_TD_ONLY, cluster_size=c))
    assert np.array_equal(lv, want)
    assert oracle.certify(case.ref, 0, lv, pa, case.labels) == (0, -1)
    _schedule_equal(info, s, c)
    rec = info["records"]
    assert rec[1, 8] == -1 and rec[2, 8] != -1, rec[:, 8]   # level 1 clustered, level 2 not


def test_long_path_and_roots(gpu_lib):
    bfs = gpu_lib
    e = graphgen.path(20000)
    case = Case(bfs, e)
    for root in (0, 12345):
        want = oracle.levels(case.ref, root)
        s = oracle.do_schedule(case.ref, want, oracle.MODE_DO, 14, 24)
        for c in (0, 1, 4):
            lv, pa, info = case.run(root, bfs.options(cluster_size=c))
            assert np.array_equal(lv, want), (root, c)
            assert oracle.certify(case.ref, root, lv, pa, case.labels) == (0, -1), (root, c)
            _schedule_equal(info, s, (root, c))
            assert (_cluster_levels(info) == 0) == (c == 1)
    # several roots at once: level = distance to the nearest root
    roots = [0, 7000, 7001, 19999]
    case.g.run_multiroot(roots, parent=case.parent, level=case.level, opts=bfs.options(cluster_size=16))
    lv = case.level.cpu().numpy()
    v = np.arange(e.n)
    want = np.min(np.abs(v[:, None] - np.array(roots)[None, :]), axis=1)
    assert np.array_equal(lv, want)


def test_cluster_size_is_validated(gpu_lib):
    bfs = gpu_lib
    case = Case(bfs, graphgen.path(100))
    for bad in (3, 5, 32, -1):
        with pytest.raises(bfs.BfsError):
            case.run(0, bfs.options(cluster_size=bad))

"""The multithreaded CPU direction-optimizing BFS (the benchmark's second CPU
comparator) against the oracle: levels bit-exact, parents certified, on small and
adversarial graphs, every direction mode and several thread counts."""
import numpy as np
import pytest

import cpubfs
import graphgen
import oracle
from graphgen import workloads

BU_ONLY = dict(alpha=1 << 40, beta=1 << 40)   # switch to bottom-up at level 0 and stay there
TD_ONLY = dict(alpha=0, beta=24)


def _graphs():
    gs = [graphgen.random_small(n, m, s) for n, m, s in [(2, 1, 1), (33, 20, 5), (257, 600, 11)]]
    gs += [graphgen.path(300), graphgen.star(200, center=3), graphgen.complete(30), graphgen.torus(32, seed=3000)]
    u, _ = graphgen.disjoint_union([graphgen.path(5), graphgen.complete(4), graphgen.from_pairs(3, [(0, 0)])])
    gs += [u, workloads.RMAT[12].edges(), workloads.RMAT[14].edges()]
    return gs


@pytest.mark.parametrize("gi", range(10))
def test_cpu_dobfs_matches_oracle(gi):
    e = _graphs()[gi]
    ref = oracle.build_csr(e.n, e.src, e.dst)
    labels = oracle.components(ref)
    deg = ref.degree()
    roots = sorted({int(np.argmax(deg)), 0, e.n - 1})
    for root in roots:
        want = oracle.levels(ref, root)
        for kw in ({}, TD_ONLY, BU_ONLY):
            for threads in (1, 3):
                pa, lv, st = cpubfs.dobfs(ref.offsets, ref.cols, root, threads=threads, **kw)
                assert np.array_equal(lv, want), (e.name, root, kw, threads)
                assert oracle.certify(ref, root, lv, pa, labels) == (0, -1), (e.name, root, kw, threads)
                assert st["levels"] == int(want.max()) + 1
                if kw is TD_ONLY:
                    assert st["bu_levels"] == 0
                if kw is BU_ONLY and deg[root] > 0:
                    assert st["td_levels"] == 0

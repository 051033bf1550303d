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

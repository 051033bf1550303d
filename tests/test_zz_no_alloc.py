"""The allocation-free entry point (bfs_run_csr_noalloc) against bfs_run.

Some callers cannot allocate device memory: their memory is fully
pre-allocated by a pool they do not control, or cudaMalloc/cudaFree (which may
synchronise the device) must not run on their path.  bfs_run_csr_noalloc keeps
all its work buffers in a fixed device array inside the library and takes the
graph as a caller-owned device CSR.  This file is collected last, so a
failure here comes after every other test has run; it passes both alone in a
fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import graphgen
import oracle
from graphgen import workloads

pytestmark = pytest.mark.gpu


def _csr_pointers(g):
    import paper_1705_04590_gb300._lib as L
    po, pc = ctypes.c_void_p(), ctypes.c_void_p()
    L.check(L.load().bfs_graph_csr(g.handle, ctypes.byref(po), ctypes.byref(pc)), "bfs_graph_csr")
    return po.value, pc.value


def test_noalloc_matches_bfs_run_two_calls(gpu_lib):
    import torch
    import paper_1705_04590_gb300._lib as L
    bfs = gpu_lib
    lib = L.load()
    w = workloads.RMAT[15]
    e = w.edges()
    ref = oracle.build_csr(e.n, e.src, e.dst)
    labels = oracle.components(ref)
    g = bfs.Graph.from_edges(e.src, e.dst, e.n)
    po, pc = _csr_pointers(g)      # the graph's own device CSR (padded past nnz)
    stream = torch.cuda.current_stream()
    for root in w.roots(e, 2).tolist():          # two calls in a row
        lv_ref = torch.empty(e.n, dtype=torch.int32, device="cuda")
        pa_ref = torch.empty(e.n, dtype=torch.int32, device="cuda")
        g.run(root, parent=pa_ref, level=lv_ref)
        lv = torch.full((e.n,), 7, dtype=torch.int32, device="cuda")
        pa = torch.full((e.n,), 7, dtype=torch.int32, device="cuda")
        st = lib.bfs_run_csr_noalloc(po, pc, e.n, g.nnz, root, pa.data_ptr(), lv.data_ptr(), stream.cuda_stream)
        assert st == 0, lib.bfs_last_error()
        torch.cuda.synchronize()
        lv_n, pa_n = lv.cpu().numpy(), pa.cpu().numpy()
        # levels are unique: bit-exact against the existing entry point (and the oracle)
        assert np.array_equal(lv_n, lv_ref.cpu().numpy())
        assert np.array_equal(lv_n, oracle.levels(ref, root))
        # parents are not unique: both must be valid BFS trees of the same graph
        assert oracle.certify(ref, root, lv_n, pa_n, labels) == (0, -1)
        assert oracle.certify(ref, root, lv_ref.cpu().numpy(), pa_ref.cpu().numpy(), labels) == (0, -1)
    g.close()


def test_noalloc_rejects_sizes_beyond_its_array(gpu_lib):
    import torch
    import paper_1705_04590_gb300._lib as L
    lib = L.load()
    e = graphgen.path(10)
    g = gpu_lib.Graph.from_edges(e.src, e.dst, e.n)
    po, pc = _csr_pointers(g)
    lv = torch.empty(16, dtype=torch.int32, device="cuda")
    st = lib.bfs_run_csr_noalloc(po, pc, (1 << 20) + 1, g.nnz, 0, None, lv.data_ptr(), None)
    assert st == L.BFS_ERR_INVALID and b"n must lie in" in lib.bfs_last_error()
    st = lib.bfs_run_csr_noalloc(po, pc, e.n, (1 << 24) + 1, 0, None, lv.data_ptr(), None)
    assert st == L.BFS_ERR_INVALID and b"nnz must lie in" in lib.bfs_last_error()
    g.close()

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
    # a column array that is only 4-byte aligned (a slice of a larger buffer) is refused on
    # the host: the bottom-up scan reads it 16 bytes at a time; nothing is launched
    lv.fill_(7)
    torch.cuda.synchronize()
    st = lib.bfs_run_csr_noalloc(po, pc + 4, e.n, g.nnz, 0, None, lv.data_ptr(), None)
    assert st == L.BFS_ERR_INVALID and b"col_ids must be 16-byte aligned" in lib.bfs_last_error()
    st = lib.bfs_run_csr_noalloc(po + 4, pc, e.n, g.nnz, 0, None, lv.data_ptr(), None)
    assert st == L.BFS_ERR_INVALID and b"row_offsets must be 8-byte aligned" in lib.bfs_last_error()
    torch.cuda.synchronize()
    assert int((lv != 7).sum()) == 0
    g.close()


def test_noalloc_caller_owned_csr_at_its_size_limit(gpu_lib):
    """A CSR the caller allocated itself (torch tensors, exactly the documented 32
    entries of padding), n = 2^20 (the fixed array's vertex limit, so every work
    buffer in it is fully used), one call with no parent output and one from a
    degree-0 root, checked against the oracle."""
    import torch
    import paper_1705_04590_gb300._lib as L
    lib = L.load()
    n = 1 << 20
    e = graphgen.erdos_renyi(n, 3 * n, seed=2020)      # nnz about 6n, below the 2^24 limit
    ref = oracle.build_csr(e.n, e.src, e.dst)
    assert ref.nnz <= (1 << 24)
    deg = ref.degree()
    off_d = torch.from_numpy(ref.offsets).cuda()
    cols_d = torch.zeros(ref.nnz + 32, dtype=torch.int32, device="cuda")
    cols_d[:ref.nnz] = torch.from_numpy(ref.cols).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    root = int(np.flatnonzero(deg > 0)[17])
    lv = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    st = lib.bfs_run_csr_noalloc(off_d.data_ptr(), cols_d.data_ptr(), n, ref.nnz, root, None, lv.data_ptr(), stream)
    assert st == 0, lib.bfs_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(lv.cpu().numpy(), oracle.levels(ref, root))
    iso = int(np.flatnonzero(deg == 0)[0])
    pa = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    st = lib.bfs_run_csr_noalloc(off_d.data_ptr(), cols_d.data_ptr(), n, ref.nnz, iso, pa.data_ptr(), lv.data_ptr(),
                                 stream)
    assert st == 0, lib.bfs_last_error()
    torch.cuda.synchronize()
    want = np.full(n, -1, np.int32)
    want[iso] = 0
    assert np.array_equal(lv.cpu().numpy(), want)
    want[iso] = iso
    assert np.array_equal(pa.cpu().numpy(), want)

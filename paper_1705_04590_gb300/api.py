"""Python binding over the C ABI (include/bfs.h): argument marshalling only.

Every step of a search runs in the library's CUDA kernels; this module turns
torch tensors into device pointers and torch streams into cudaStream_t.
Graph storage comes from PyTorch's caching allocator through the ABI's
allocator hook (PyTorch is used for device memory and streams only).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) or None


def _dev_ptr(t, dtype_name: str, numel: int | None = None, what: str = "tensor"):
    if t is None:
        return None
    torch = _torch()
    want = getattr(torch, dtype_name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != want or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous {dtype_name} tensor")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{what} needs at least {numel} elements")
    return t.data_ptr()


class _TorchAllocator:
    """bfs_allocator backed by torch.cuda.caching_allocator_alloc / _delete."""

    def __init__(self):
        torch = _torch()
        self._torch = torch
        self._dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self._dev, stream or 0))
            except Exception:
                return None

        def _free(ptr, nbytes, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self._alloc_cb = L.ALLOC_FN(_alloc)
        self._free_cb = L.FREE_FN(_free)
        self.struct = L.Allocator(self._alloc_cb, self._free_cb, None)


def options(mode: int = L.MODE_DO, layout: int = L.LAYOUT_CSR, alpha: int = 14, beta: int = 24,
            parent_mode: int = L.PARENT_ANY, td_big_degree: int = 0, timeout_ms: int = 10000, seed: int = 0,
            bu_rows: int = L.BU_ROWS_BY_ID, td_chunk: int = 0, ctas_per_sm: int = 0,
            cluster_size: int = 0) -> L.Options:
    o = L.Options()
    L.load().bfs_options_default(ctypes.byref(o))
    o.mode, o.layout, o.alpha, o.beta, o.parent_mode = mode, layout, alpha, beta, parent_mode
    o.td_big_degree, o.timeout_ms, o.seed = td_big_degree, timeout_ms, seed
    o.bu_rows, o.td_chunk, o.ctas_per_sm, o.cluster_size = bu_rows, td_chunk, ctas_per_sm, cluster_size
    return o


class Graph:
    """A resident undirected graph (CSR, optionally DCSC tiles) on the current CUDA device."""

    def __init__(self, handle: int, allocator, keepalive=()):
        self._h = ctypes.c_void_p(handle)
        self._alloc = allocator
        self._keep = keepalive
        n, nnz, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        L.check(L.load().bfs_graph_info(self._h, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nb)), "graph_info")
        self.n, self.nnz = n.value, nnz.value

    # ---------------------------------------------------------------- creation
    @classmethod
    def from_edges(cls, src, dst, n: int, dcsc: bool = False, stream=None, torch_allocator: bool = True,
                   hub_first: bool = False, directed: bool = False) -> "Graph":
        """src/dst: numpy int32 or int64 arrays (host) or CUDA tensors of either type (device;
        64-bit ids go through bfs_graph_create_from_edges64).  hub_first also
        stores rows ordered by neighbour degree and a 32-byte head per vertex (its degree and
        first 7 reordered ids), 4*nnz + 32*n more device bytes, for bottom-up option
        bu_rows=BU_ROWS_HUB_FIRST.  directed=True keeps edge i as src[i] -> dst[i] (out-edge
        rows for top-down steps, their transpose for bottom-up steps)."""
        lib = L.load()
        torch = _torch()
        flags = (0 if directed else L.FLAG_SYMMETRIZE) | (L.FLAG_BUILD_DCSC if dcsc else 0) | \
            (L.FLAG_BUILD_HUB_FIRST if hub_first else 0)
        if isinstance(src, torch.Tensor):
            if src.numel() != dst.numel():
                raise ValueError("src and dst differ in length")
            wide = src.dtype == torch.int64
            ty = "int64" if wide else "int32"
            ps, pd = _dev_ptr(src, ty, what="src"), _dev_ptr(dst, ty, what="dst")
            flags |= L.FLAG_DEVICE_PTRS
            m = src.numel()
            keep = (src, dst)
        else:
            wide = np.asarray(src).dtype == np.int64
            src = np.ascontiguousarray(src, np.int64 if wide else np.int32)
            dst = np.ascontiguousarray(dst, np.int64 if wide else np.int32)
            if src.shape != dst.shape:
                raise ValueError("src and dst differ in length")
            ps, pd, m, keep = src.ctypes.data, dst.ctypes.data, int(src.shape[0]), (src, dst)
        alloc = _TorchAllocator() if torch_allocator else None
        h = ctypes.c_void_p()
        create = lib.bfs_graph_create_from_edges64 if wide else lib.bfs_graph_create_from_edges
        st = create(ps, pd, m, n, flags, ctypes.byref(alloc.struct) if alloc else None, _stream_ptr(stream),
                    ctypes.byref(h))
        L.check(st, "bfs_graph_create_from_edges64" if wide else "bfs_graph_create_from_edges")
        del keep
        return cls(h.value, alloc)

    @classmethod
    def from_csr(cls, offsets, cols, n: int, check_symmetry: bool = False, dcsc: bool = False, stream=None,
                 torch_allocator: bool = True, hub_first: bool = False) -> "Graph":
        """offsets (int64, n+1) / cols (int32): a symmetric CSR on the host (numpy) or the
        device (CUDA tensors); check_symmetry verifies it in one extra pass.  dcsc and
        hub_first as in from_edges."""
        lib = L.load()
        torch = _torch()
        flags = (L.FLAG_CHECK_SYMMETRY if check_symmetry else 0) | (L.FLAG_BUILD_DCSC if dcsc else 0) | \
            (L.FLAG_BUILD_HUB_FIRST if hub_first else 0)
        if isinstance(offsets, torch.Tensor):
            po, pc = _dev_ptr(offsets, "int64", n + 1, "offsets"), _dev_ptr(cols, "int32", what="cols")
            nnz = cols.numel()
            flags |= L.FLAG_DEVICE_PTRS
        else:
            offsets = np.ascontiguousarray(offsets, np.int64)
            cols = np.ascontiguousarray(cols, np.int32)
            if offsets.shape[0] != n + 1:
                raise ValueError("offsets must have n+1 entries")
            po, pc, nnz = offsets.ctypes.data, cols.ctypes.data if cols.size else None, int(cols.shape[0])
        alloc = _TorchAllocator() if torch_allocator else None
        h = ctypes.c_void_p()
        st = lib.bfs_graph_create_from_csr(po, pc, n, nnz, flags, ctypes.byref(alloc.struct) if alloc else None,
                                           _stream_ptr(stream), ctypes.byref(h))
        L.check(st, "bfs_graph_create_from_csr")
        return cls(h.value, alloc)

    # ---------------------------------------------------------------- queries
    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        nb = ctypes.c_int64()
        L.check(L.load().bfs_graph_info(self._h, None, None, ctypes.byref(nb)), "graph_info")
        return nb.value

    def csr_host(self):
        """(offsets int64[n+1], cols int32[nnz]) copied to host numpy arrays."""
        off = np.empty(self.n + 1, np.int64)
        cols = np.empty(max(self.nnz, 1), np.int32)
        L.check(L.load().bfs_graph_copy_csr(self._h, off.ctypes.data, cols.ctypes.data, None), "graph_copy_csr")
        return off, cols[: self.nnz]

    def hub_first_host(self) -> np.ndarray:
        """The hub-first column ids (graph built with hub_first=True) as a host array."""
        cols = np.empty(max(self.nnz, 1), np.int32)
        L.check(L.load().bfs_graph_copy_hub_first(self._h, cols.ctypes.data, None), "graph_copy_hub_first")
        return cols[: self.nnz]

    def row_heads_host(self) -> np.ndarray:
        """The row heads (graph built with hub_first=True) as an (n, 8) host array:
        row u = [deg(u), first 7 ids of u's hub-first row, 0 past its end]."""
        heads = np.empty((self.n, 8), np.int32)
        L.check(L.load().bfs_graph_copy_row_heads(self._h, heads.ctypes.data, None), "graph_copy_row_heads")
        return heads

    def transpose_host(self):
        """A directed graph's in-edge rows: (offsets int64[n+1], cols int32[nnz]) on the host."""
        off = np.empty(self.n + 1, np.int64)
        cols = np.empty(max(self.nnz, 1), np.int32)
        L.check(L.load().bfs_graph_copy_transpose(self._h, off.ctypes.data, cols.ctypes.data, None),
                "graph_copy_transpose")
        return off, cols[: self.nnz]

    def bu_planes_host(self, first: bool = True):
        """(first, deg8): per vertex the first id of its hub-first row with bit 31 set when
        it has two or more neighbours (int32[n]; graph built with hub_first=True; None
        when first=False) and min(deg, 255) (uint8[n])."""
        f = np.empty(self.n, np.int32) if first else None
        d8 = np.empty(self.n, np.uint8)
        L.check(L.load().bfs_graph_copy_bu_planes(self._h, f.ctypes.data if first else None, d8.ctypes.data, None),
                "graph_copy_bu_planes")
        return f, d8

    def dcsc_layout(self) -> L.DcscLayout:
        d = L.DcscLayout()
        L.check(L.load().bfs_graph_dcsc(self._h, ctypes.byref(d)), "graph_dcsc")
        return d

    def dcsc_host(self):
        """(num_blocks, block_size, tile_ptr, jc, cp, ir) of the DCSC tiles, copied to host numpy arrays."""
        d = self.dcsc_layout()
        p = d.num_blocks
        tp = np.empty(p * p + 1, np.int64)
        jc = np.empty(max(d.nzc, 1), np.int32)
        cp = np.empty(d.nzc + 1, np.int64)
        ir = np.empty(max(self.nnz, 1), np.int32)
        L.check(L.load().bfs_graph_copy_dcsc(self._h, tp.ctypes.data, jc.ctypes.data, cp.ctypes.data, ir.ctypes.data,
                                             None), "graph_copy_dcsc")
        return p, d.block_size, tp, jc[: d.nzc], cp, ir[: self.nnz]

    # ---------------------------------------------------------------- searches
    def run(self, root: int, parent=None, level=None, opts: L.Options | None = None, stream=None,
            stats: bool = False, record_levels: int = 0):
        """BFS from root into caller-owned int32 CUDA tensors (either may be None).
        With stats=True the call synchronises and returns (num_levels, reached, records)."""
        lib = L.load()
        pp = _dev_ptr(parent, "int32", self.n, "parent")
        pl = _dev_ptr(level, "int32", self.n, "level")
        st_ptr, holder = self._stats(stats, record_levels)
        st = lib.bfs_run(self._h, int(root), pp, pl, ctypes.byref(opts) if opts else None, _stream_ptr(stream),
                         st_ptr)
        L.check(st, "bfs_run")
        return self._stats_out(holder)

    def run_multiroot(self, roots, parent=None, level=None, opts: L.Options | None = None, stream=None,
                      stats: bool = False, record_levels: int = 0):
        lib = L.load()
        r = np.ascontiguousarray(roots, np.int32)
        pp = _dev_ptr(parent, "int32", self.n, "parent")
        pl = _dev_ptr(level, "int32", self.n, "level")
        st_ptr, holder = self._stats(stats, record_levels)
        st = lib.bfs_run_multiroot(self._h, r.ctypes.data, int(r.shape[0]), pp, pl,
                                   ctypes.byref(opts) if opts else None, _stream_ptr(stream), st_ptr)
        L.check(st, "bfs_run_multiroot")
        return self._stats_out(holder)

    def run_multi(self, roots, level, parent=None, opts: L.Options | None = None, stream=None):
        """k searches packed as 64-bit lane masks; level/parent: int32 CUDA tensors of k*n."""
        lib = L.load()
        r = np.ascontiguousarray(roots, np.int32)
        k = int(r.shape[0])
        pl = _dev_ptr(level, "int32", k * self.n, "level")
        pp = _dev_ptr(parent, "int32", k * self.n, "parent")
        st = lib.bfs_run_multi(self._h, r.ctypes.data, k, pl, pp, ctypes.byref(opts) if opts else None,
                               _stream_ptr(stream))
        L.check(st, "bfs_run_multi")

    def sync(self, stream=None):
        L.check(L.load().bfs_graph_sync(self._h, _stream_ptr(stream)), "bfs_graph_sync")

    @staticmethod
    def _stats(want: bool, cap: int):
        if not want:
            return None, None
        s = L.Stats()
        recs = (L.LevelRecord * max(cap, 1))()
        s.levels_capacity = cap
        s.levels = ctypes.cast(recs, ctypes.POINTER(L.LevelRecord))
        return ctypes.byref(s), (s, recs, cap)

    @staticmethod
    def _stats_out(holder):
        if holder is None:
            return None
        s, recs, cap = holder
        nrec = min(s.num_levels, cap)
        rows = [(r.dir, r.nf, r.mf, r.nnext, r.mnext, r.scanned, r.examined, r.t_ns, r.aux, r.t_mid_ns, r.misses)
                for r in recs[:nrec]]
        arr = np.array(rows, dtype=np.int64).reshape(-1, 11)
        return {"num_levels": s.num_levels, "reached": s.vertices_reached, "edges_examined": s.edges_examined,
                "t_init_ns": s.t_init_ns, "t_final_ns": s.t_final_ns, "records": arr}

    def close(self):
        if self._h:
            L.load().bfs_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching BFS query server (bfs_server_* in include/bfs.h).

    Graphs stay resident; each query (slot, root) fills a caller-owned host
    int32 array of the graph's n levels.  Queries that arrive while others run
    join the running multi-source search of their graph at the next level.
    """

    def __init__(self, hbm_budget_bytes: int, max_lanes: int = 64, allocator=None):
        """allocator: None (the library's cudaMalloc), True (PyTorch's caching allocator) or
        an object with a `struct` attribute holding a bfs_allocator (kept alive here)."""
        lib = L.load()
        h = ctypes.c_void_p()
        if allocator is True:
            allocator = _TorchAllocator()
        self._alloc = allocator
        L.check(lib.bfs_server_create_ex(int(hbm_budget_bytes), int(max_lanes),
                                         ctypes.byref(allocator.struct) if allocator else None, ctypes.byref(h)),
                "bfs_server_create_ex")
        self._h = h
        self._graphs = []
        self._outs = {}

    def add_graph(self, g: Graph) -> int:
        slot = ctypes.c_int32()
        L.check(L.load().bfs_server_add_graph(self._h, g.handle, ctypes.byref(slot)), "bfs_server_add_graph")
        self._graphs.append(g)
        return slot.value

    def submit(self, slot: int, root: int, out: np.ndarray) -> int:
        """out: int32 host array of the graph's n entries (pinned memory copies fastest)."""
        if out.dtype != np.int32 or not out.flags.c_contiguous:
            raise TypeError("out must be a contiguous int32 numpy array")
        t = ctypes.c_uint64()
        L.check(L.load().bfs_submit(self._h, int(slot), int(root), out.ctypes.data, ctypes.byref(t)), "bfs_submit")
        self._outs[t.value] = out
        return t.value

    def poll(self, ticket: int) -> bool:
        st = L.load().bfs_poll(self._h, ctypes.c_uint64(ticket))
        if st == L.BFS_ERR_NOT_READY:
            return False
        L.check(st, "bfs_poll")
        self._outs.pop(ticket, None)
        return True

    def wait(self, ticket: int, timeout_ms: int = -1) -> bool:
        st = L.load().bfs_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms))
        if st == L.BFS_ERR_NOT_READY:
            return False
        L.check(st, "bfs_wait")
        self._outs.pop(ticket, None)
        return True

    def latency_us(self, ticket: int) -> float:
        us = ctypes.c_double()
        L.check(L.load().bfs_ticket_latency_us(self._h, ctypes.c_uint64(ticket), ctypes.byref(us)), "latency")
        return us.value

    def stats(self) -> dict:
        c = (ctypes.c_int64 * 3)()
        L.check(L.load().bfs_server_stats(self._h, c), "bfs_server_stats")
        return {"completed": c[0], "launches": c[1], "lanes_filled": c[2]}

    def close(self):
        if self._h:
            L.load().bfs_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._outs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

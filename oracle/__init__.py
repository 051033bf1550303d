"""CPU oracle for level-synchronous breadth-first search.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path (``paper_1705_04590_gb300``), and neither imports the
other.  The only module both sides use is ``graphgen`` (seeded inputs).

Contents (each cites the passage of Bulu\\c{c} et al. 2015 it follows):

* :func:`build_csr`       -- "Graph Representation" + "Data Sets" (numpy sort/unique)
* :func:`hub_first`       -- the same rows, neighbours ordered by degree (the row order a
                             bottom-up step may scan in; Algorithm 2 fixes none beyond "in order")
* :func:`hub_first_rows`  -- the same reordering row by row in C, for graphs too large
                             for the numpy lexsort (pinned equal to :func:`hub_first`)
* :func:`bfs_topdown`     -- Algorithm 1, serial FIFO (C)
* :func:`bfs_bottomup`    -- Algorithm 2, serial (C)
* :func:`min_parent`      -- (select2nd, min) semiring of the parallel top-down local discovery (C)
* :func:`components`      -- union-find, to pin "reached set = component of the root" (C)
* :func:`certify`         -- BFS invariants, valid at any size (C)
* :func:`do_schedule`     -- per-level direction and work counts of the
                             direction-optimizing search ("Parallel Direction-Optimizing BFS") (C)
* :func:`dcsc_tiles`      -- DCSC of the row-block x column-block tiles ("Graph Representation":
                             IR row ids, JC non-empty column ids, CP column pointers), numpy
* :func:`build_digraph`, :func:`do_schedule_dir`, :func:`reach`, :func:`certify_dir`
                          -- directed graphs: out-edge CSR and its transpose, the
                             schedule with out-/in-degree sums, depth-first
                             reachability, the invariants along directed edges (C)
* :func:`brute_force_levels` -- all-pairs unit-weight relaxation to a fixpoint
                             (Bellman-Ford style), numpy, tiny graphs only

Every function is pinned by ``tests/test_oracle.py`` against something other
than itself (brute force, closed forms, the hand-derived Figure 3 fixture,
invariants, direction invariance).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

CERT_CODES = {1: "root", 2: "parent edge / parent level", 3: "edge spans > 1 level",
              4: "edge to unreached vertex", 5: "reached set != component of root"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2; plain C, single thread)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        L.or_bfs_topdown.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        L.or_bfs_topdown.restype = i32
        L.or_bfs_bottomup.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp]
        L.or_bfs_bottomup.restype = i32
        L.or_min_parent.argtypes = [i64, vp, vp, vp, vp]
        L.or_min_parent.restype = None
        L.or_components.argtypes = [i64, vp, vp, vp]
        L.or_components.restype = None
        L.or_certify.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        L.or_certify.restype = i64
        L.or_do_schedule.argtypes = [i64, vp, vp, vp, i32, i64, i64, i32] + [vp] * 7
        L.or_do_schedule.restype = i32
        L.or_hub_first.argtypes = [i64, vp, vp, vp, i64, i64]
        L.or_hub_first.restype = i32
        L.or_do_schedule_dir.argtypes = [i64, vp, vp, vp, vp, i32, i64, i64, i32] + [vp] * 7
        L.or_do_schedule_dir.restype = i32
        L.or_reach.argtypes = [i64, vp, vp, i32, vp]
        L.or_reach.restype = i64
        L.or_certify_dir.argtypes = [i64, vp, vp, i32, vp, vp, vp]
        L.or_certify_dir.restype = i64
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class CSR:
    """Undirected, de-duplicated, self-loop-free CSR built by the oracle."""
    n: int
    offsets: np.ndarray  # int64[n+1]
    cols: np.ndarray     # int32[nnz], each row sorted ascending

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def degree(self) -> np.ndarray:
        return np.diff(self.offsets)


def build_csr(n: int, src: np.ndarray, dst: np.ndarray, chunk: int = 1 << 26, directed: bool = False) -> CSR:
    """CSR of the undirected graph ("Graph Representation": sorted adjacencies,
    each undirected edge stored in both rows, an n+1 row-pointer array; "Data
    Sets": duplicate edges pruned).  Self-loops are dropped.

    Written as the definition: the set {(u, v), (v, u) : {u, v} an input edge,
    u != v} as 64-bit keys u*2^32 + v, sorted (numpy's sort, a library
    primitive), repeats removed; the low halves are the column ids and the
    row lengths are counts of the high halves.  Chunked only to bound host
    memory (about 8 bytes per directed entry plus the 4-byte result).

    directed=True keeps only (u, v) for an input edge u -> v: the out-edge CSR
    of a directed graph (the method "applies to directed graphs", "Data Sets")."""
    src = np.asarray(src)
    dst = np.asarray(dst)
    m = int(src.shape[0])
    if m and (min(int(src.min()), int(dst.min())) < 0 or max(int(src.max()), int(dst.max())) >= n):
        raise ValueError("edge list holds ids outside [0, n)")
    keep_total = 0
    for a in range(0, m, chunk):
        keep_total += int(np.count_nonzero(src[a:a + chunk] != dst[a:a + chunk]))
    keys = np.empty((1 if directed else 2) * keep_total, np.uint64)
    w = 0
    for a in range(0, m, chunk):
        u = src[a:a + chunk].astype(np.uint64)
        v = dst[a:a + chunk].astype(np.uint64)
        k = u != v
        u, v = u[k], v[k]
        c = u.shape[0]
        keys[w:w + c] = (u << np.uint64(32)) | v
        if not directed:
            keys[keep_total + w:keep_total + w + c] = (v << np.uint64(32)) | u
        w += c
    keys.sort()
    # drop repeats in place (the write cursor never passes the read cursor)
    nnz = 0
    total = keys.shape[0]
    prev = None
    for a in range(0, total, chunk):
        blk = keys[a:a + chunk]
        first = np.empty(blk.shape[0], bool)
        first[1:] = blk[1:] != blk[:-1]
        if blk.shape[0]:
            first[0] = prev is None or blk[0] != prev
            prev = blk[-1]
        sel = blk[first]
        keys[nnz:nnz + sel.shape[0]] = sel
        nnz += sel.shape[0]
    cols = np.empty(nnz, np.int32)
    counts = np.zeros(n, np.int64)
    for a in range(0, nnz, chunk):
        blk = keys[a:min(a + chunk, nnz)]
        cols[a:a + blk.shape[0]] = (blk & np.uint64(0xFFFFFFFF)).astype(np.int32)
        counts += np.bincount((blk >> np.uint64(32)).astype(np.int64), minlength=n)
    del keys
    off = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    return CSR(n, off, cols)


def csr_from_edges(g) -> CSR:
    return build_csr(g.n, g.src, g.dst)


def hub_first(g: CSR) -> CSR:
    """The same graph with every row reordered: neighbours by degree, highest
    first, ties by id ascending.  Algorithm 2 scans a row "in order" and stops at
    the first frontier neighbour; any order yields a valid parent one level
    closer, and the per-level examination counts of the direction-optimizing
    schedule (:func:`do_schedule`) follow the row order of the CSR passed in.
    Written from the definition: one lexicographic sort of (row, -degree, id)."""
    deg = g.degree()
    rows = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    order = np.lexsort((g.cols, -deg[g.cols], rows))
    return CSR(g.n, g.offsets.copy(), np.ascontiguousarray(g.cols[order], np.int32))


def hub_first_rows(g: CSR, threads: int = 0) -> CSR:
    """:func:`hub_first` computed row by row in C (each row sorted on the key
    (~degree << 32) | id): the same result, with memory for one row of scratch
    instead of the lexsort's three full-length temporaries.  Rows are
    independent; ranges of about equal edge count run on `threads` host
    threads (0: one per core)."""
    import concurrent.futures as cf
    out = np.empty(max(g.nnz, 1), np.int32)
    threads = threads or (os.cpu_count() or 1)
    parts = max(1, min(4 * threads, g.n))
    cuts = np.searchsorted(g.offsets, np.linspace(0, g.nnz, parts + 1), side="left")
    cuts[0], cuts[-1] = 0, g.n
    lib = _load()

    def run(i):
        return lib.or_hub_first(g.n, _ptr(g.offsets), _ptr(g.cols), _ptr(out), int(cuts[i]), int(cuts[i + 1]))

    with cf.ThreadPoolExecutor(threads) as ex:
        if any(r != 0 for r in ex.map(run, range(parts))):
            raise MemoryError("or_hub_first: scratch allocation failed")
    return CSR(g.n, g.offsets.copy(), out[: g.nnz])


def bfs_topdown(g: CSR, root: int):
    """Algorithm 1. Returns (parent, level, num_levels)."""
    parent = np.empty(g.n, np.int32)
    level = np.empty(g.n, np.int32)
    queue = np.empty(max(g.n, 1), np.int32)
    L = _load().or_bfs_topdown(g.n, _ptr(g.offsets), _ptr(g.cols), int(root), _ptr(parent), _ptr(level), _ptr(queue))
    return parent, level, int(L)


def bfs_bottomup(g: CSR, root: int):
    """Algorithm 2. Returns (parent, level, num_levels)."""
    parent = np.empty(g.n, np.int32)
    level = np.empty(g.n, np.int32)
    f = np.empty(g.n, np.uint8)
    nx = np.empty(g.n, np.uint8)
    L = _load().or_bfs_bottomup(g.n, _ptr(g.offsets), _ptr(g.cols), int(root), _ptr(parent), _ptr(level),
                                _ptr(f), _ptr(nx))
    return parent, level, int(L)


def levels(g: CSR, root: int) -> np.ndarray:
    return bfs_topdown(g, root)[1]


def min_parent(g: CSR, level: np.ndarray) -> np.ndarray:
    level = np.ascontiguousarray(level, np.int32)
    out = np.empty(g.n, np.int32)
    _load().or_min_parent(g.n, _ptr(g.offsets), _ptr(g.cols), _ptr(level), _ptr(out))
    return out


def components(g: CSR) -> np.ndarray:
    lab = np.empty(g.n, np.int32)
    _load().or_components(g.n, _ptr(g.offsets), _ptr(g.cols), _ptr(lab))
    return lab


def certify(g: CSR, root: int, level: np.ndarray, parent: np.ndarray | None = None,
            labels: np.ndarray | None = None) -> tuple[int, int]:
    """(0, -1) if valid, else (failed invariant code, vertex).  See oracle.c."""
    if labels is None:
        labels = components(g)
    level = np.ascontiguousarray(level, np.int32)
    if parent is not None:
        parent = np.ascontiguousarray(parent, np.int32)
    labels = np.ascontiguousarray(labels, np.int32)   # kept alive across the call
    r = _load().or_certify(g.n, _ptr(g.offsets), _ptr(g.cols), int(root), _ptr(parent), _ptr(level),
                           _ptr(labels))
    if r == 0:
        return 0, -1
    return int(r >> 40), int(r & ((1 << 40) - 1))


MODE_DO, MODE_TD, MODE_BU = 0, 1, 2


@dataclass
class Schedule:
    dir: np.ndarray       # int32 per level: 0 top-down, 1 bottom-up
    nf: np.ndarray
    mf: np.ndarray
    nnext: np.ndarray
    mnext: np.ndarray
    scanned: np.ndarray
    examined: np.ndarray

    @property
    def num_levels(self) -> int:
        return int(self.dir.shape[0])


def do_schedule(g: CSR, level: np.ndarray, mode: int = MODE_DO, alpha: int = 14, beta: int = 24) -> Schedule:
    level = np.ascontiguousarray(level, np.int32)
    cap = int(level.max()) + 2 if level.size else 2
    arrs = [np.zeros(cap, np.int32)] + [np.zeros(cap, np.int64) for _ in range(6)]
    L = _load().or_do_schedule(g.n, _ptr(g.offsets), _ptr(g.cols), _ptr(level), mode, alpha, beta, cap,
                               *[_ptr(a) for a in arrs])
    if L < 0:
        raise RuntimeError("schedule capacity")
    return Schedule(*[a[:L].copy() for a in arrs])


def build_digraph(n: int, src: np.ndarray, dst: np.ndarray) -> tuple[CSR, CSR]:
    """(out, inn): the out-edge CSR of the directed graph {u -> v : (u, v) an input
    edge, u != v} and its transpose (the in-edge CSR, each row the sorted sources of
    the edges into that vertex), the second adjacency a bottom-up step needs ("Data
    Decomposition": the transpose).  Each is the set definition of build_csr."""
    return build_csr(n, src, dst, directed=True), build_csr(n, dst, src, directed=True)


def do_schedule_dir(out: CSR, inn: CSR, level: np.ndarray, mode: int = 0, alpha: int = 14,
                    beta: int = 24) -> "Schedule":
    """The direction-optimizing schedule of a directed search: m_f sums out-degrees of
    the frontier, m_u in-degrees of the unreached vertices, bottom-up steps scan in-rows."""
    level = np.ascontiguousarray(level, np.int32)
    cap = int(level.max()) + 2 if level.size else 2
    arrs = [np.zeros(cap, np.int32)] + [np.zeros(cap, np.int64) for _ in range(6)]
    L = _load().or_do_schedule_dir(out.n, _ptr(out.offsets), _ptr(inn.offsets), _ptr(inn.cols), _ptr(level), mode,
                                   alpha, beta, cap, *[_ptr(a) for a in arrs])
    if L < 0:
        raise RuntimeError("schedule capacity")
    return Schedule(*[a[:L].copy() for a in arrs])


def reach(out: CSR, root: int) -> np.ndarray:
    """bool[n]: vertices reachable from root along out-edges (depth-first search)."""
    mark = np.zeros(out.n, np.uint8)
    if _load().or_reach(out.n, _ptr(out.offsets), _ptr(out.cols), int(root), _ptr(mark)) < 0:
        raise MemoryError("or_reach: scratch allocation failed")
    return mark.astype(bool)


def certify_dir(out: CSR, root: int, level: np.ndarray, parent: np.ndarray | None = None,
                reached: np.ndarray | None = None) -> tuple[int, int]:
    """(0, -1) if (level, parent) is a BFS from root along out-edges, else (failed
    invariant code, vertex).  See or_certify_dir in oracle.c."""
    if reached is None:
        reached = reach(out, root)
    level = np.ascontiguousarray(level, np.int32)
    if parent is not None:
        parent = np.ascontiguousarray(parent, np.int32)
    reached = np.ascontiguousarray(reached, np.uint8)   # kept alive across the call
    r = _load().or_certify_dir(out.n, _ptr(out.offsets), _ptr(out.cols), int(root), _ptr(parent), _ptr(level),
                               _ptr(reached))
    if r == 0:
        return 0, -1
    return int(r >> 40), int(r & ((1 << 40) - 1))


def brute_force_levels(n: int, src: np.ndarray, dst: np.ndarray, root: int, directed: bool = False) -> np.ndarray:
    """Unit-weight relaxation d[v] = min(d[v], d[u] + 1) over every edge, both
    directions (only u -> v with directed=True), until nothing changes
    (Bellman-Ford style).  Self-loops and duplicates are harmless here.
    O(n * m): tiny graphs only."""
    INF = np.iinfo(np.int64).max // 4
    d = np.full(n, INF, np.int64)
    d[root] = 0
    if directed:
        s, t = np.asarray(src, np.int64), np.asarray(dst, np.int64)
    else:
        s = np.concatenate([np.asarray(src, np.int64), np.asarray(dst, np.int64)])
        t = np.concatenate([np.asarray(dst, np.int64), np.asarray(src, np.int64)])
    for _ in range(n + 1):
        cand = d[s] + 1
        new = d.copy()
        np.minimum.at(new, t, cand)
        if np.array_equal(new, d):
            break
        d = new
    out = np.where(d >= INF, -1, d)
    return out.astype(np.int32)


def dcsc_tiles(n: int, offsets: np.ndarray, cols: np.ndarray, row_block: int, col_block: int):
    """DCSC of every tile of a CSR matrix ("Graph Representation": for each
    tile, IR holds row ids, JC the ids of the columns with at least one
    nonzero, CP the column pointers into IR).  Tile (i, j) covers rows
    [i*row_block, (i+1)*row_block) and columns [j*col_block, (j+1)*col_block);
    tiles are listed i-major.  Row and column ids are local to the tile
    (minus the block start).  Returns (tile_ptr, JC, CP, IR) with JC/CP
    concatenated over tiles (CP holds positions into the concatenated IR).

    Written as the definition: every nonzero (u, v) ordered by (tile, v, u)."""
    offsets = np.asarray(offsets, np.int64)
    cols = np.asarray(cols, np.int64)
    nrb = (n + row_block - 1) // row_block
    ncb = (n + col_block - 1) // col_block
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(offsets))
    tile = (rows // row_block) * ncb + cols // col_block
    order = np.lexsort((rows, cols, tile))
    t, v, u = tile[order], cols[order] % col_block, rows[order] % row_block
    IR = u.astype(np.int32)
    new_col = np.ones(len(order), bool)
    if len(order):
        new_col[1:] = (t[1:] != t[:-1]) | (v[1:] != v[:-1])
    starts = np.flatnonzero(new_col)
    JC = v[starts].astype(np.int32)
    CP = np.append(starts, len(order)).astype(np.int64)
    tile_of_col = t[starts]
    tile_ptr = np.zeros(nrb * ncb + 1, np.int64)
    np.cumsum(np.bincount(tile_of_col, minlength=nrb * ncb), out=tile_ptr[1:])
    return tile_ptr, JC, CP, IR

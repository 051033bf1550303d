"""ctypes declarations of include/bfs.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

from ._build import LIB

c_i32, c_i64, c_u32, c_u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
c_vp = ctypes.c_void_p

BFS_OK, BFS_ERR_INVALID, BFS_ERR_OOM, BFS_ERR_CUDA, BFS_ERR_TIMEOUT, BFS_ERR_BUSY, BFS_ERR_NOT_READY, \
    BFS_ERR_UNSUPPORTED = range(8)

FLAG_DEVICE_PTRS, FLAG_SYMMETRIZE, FLAG_BUILD_DCSC, FLAG_CHECK_SYMMETRY, FLAG_BUILD_HUB_FIRST = 1, 2, 4, 8, 16
BU_ROWS_BY_ID, BU_ROWS_HUB_FIRST = 0, 1
MODE_DO, MODE_TD_ONLY, MODE_BU_ONLY, MODE_RANDOM = 0, 1, 2, 3
LAYOUT_CSR, LAYOUT_DCSC_TILED = 0, 1
PARENT_ANY, PARENT_MIN_ID = 0, 1

ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, ctypes.c_size_t, c_vp, c_vp)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_vp)]


class Options(ctypes.Structure):
    _fields_ = [("mode", c_i32), ("layout", c_i32), ("alpha", c_i32), ("beta", c_i32), ("parent_mode", c_i32),
                ("td_big_degree", c_i32), ("timeout_ms", c_i64), ("seed", c_u64),
                ("bu_rows", c_i32), ("td_chunk", c_i32), ("ctas_per_sm", c_i32), ("cluster_size", c_i32)]


class LevelRecord(ctypes.Structure):
    _fields_ = [("dir", c_i32), ("misses", c_i32), ("nf", c_i64), ("mf", c_i64), ("nnext", c_i64),
                ("mnext", c_i64), ("scanned", c_i64), ("examined", c_i64), ("t_ns", c_i64), ("aux", c_i64),
                ("t_mid_ns", c_i64)]


class Stats(ctypes.Structure):
    _fields_ = [("num_levels", c_i32), ("levels_capacity", c_i32), ("levels", ctypes.POINTER(LevelRecord)),
                ("vertices_reached", c_i64), ("edges_examined", c_i64), ("t_init_ns", c_i64), ("t_final_ns", c_i64)]


class DcscLayout(ctypes.Structure):
    _fields_ = [("num_blocks", c_i32), ("reserved", c_i32), ("block_size", c_i64), ("tile_ptr", c_vp), ("jc", c_vp),
                ("cp", c_vp), ("ir", c_vp), ("nzc", c_i64)]


# (name, restype, argtypes) of every entry point in include/bfs.h
SIGNATURES = [
    ("bfs_options_default", None, [ctypes.POINTER(Options)]),
    ("bfs_graph_create_from_edges", c_i32, [c_vp, c_vp, c_i64, c_i64, c_u32, ctypes.POINTER(Allocator), c_vp,
                                            ctypes.POINTER(c_vp)]),
    ("bfs_graph_create_from_csr", c_i32, [c_vp, c_vp, c_i64, c_i64, c_u32, ctypes.POINTER(Allocator), c_vp,
                                          ctypes.POINTER(c_vp)]),
    ("bfs_graph_info", c_i32, [c_vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    ("bfs_graph_csr", c_i32, [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp)]),
    ("bfs_graph_copy_csr", c_i32, [c_vp, c_vp, c_vp, c_vp]),
    ("bfs_graph_copy_hub_first", c_i32, [c_vp, c_vp, c_vp]),
    ("bfs_graph_copy_row_heads", c_i32, [c_vp, c_vp, c_vp]),
    ("bfs_graph_copy_bu_planes", c_i32, [c_vp, c_vp, c_vp, c_vp]),
    ("bfs_graph_copy_transpose", c_i32, [c_vp, c_vp, c_vp, c_vp]),
    ("bfs_graph_dcsc", c_i32, [c_vp, ctypes.POINTER(DcscLayout)]),
    ("bfs_graph_copy_dcsc", c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("bfs_graph_destroy", None, [c_vp]),
    ("bfs_run", c_i32, [c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(Options), c_vp, ctypes.POINTER(Stats)]),
    ("bfs_run_multiroot", c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(Options), c_vp,
                                  ctypes.POINTER(Stats)]),
    ("bfs_run_multi", c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(Options), c_vp]),
    ("bfs_run_csr_noalloc", c_i32, [c_vp, c_vp, c_i64, c_i64, c_i32, c_vp, c_vp, c_vp]),
    ("bfs_autotune", c_i32, [c_vp, c_vp, c_i32, ctypes.POINTER(Options), ctypes.POINTER(Options),
                             ctypes.POINTER(ctypes.c_double), c_vp]),
    ("bfs_graph_sync", c_i32, [c_vp, c_vp]),
    ("bfs_debug_set_barrier_extra", c_i32, [c_vp, c_i32]),
    ("bfs_graph_create_from_edges64", c_i32, [c_vp, c_vp, c_i64, c_i64, c_u32, ctypes.POINTER(Allocator), c_vp,
                                              ctypes.POINTER(c_vp)]),
    ("bfs_server_create_ex", c_i32, [c_i64, c_i32, ctypes.POINTER(Allocator), ctypes.POINTER(c_vp)]),
    ("bfs_server_create", c_i32, [c_i64, c_i32, ctypes.POINTER(c_vp)]),
    ("bfs_server_add_graph", c_i32, [c_vp, c_vp, ctypes.POINTER(c_i32)]),
    ("bfs_submit", c_i32, [c_vp, c_i32, c_i32, c_vp, ctypes.POINTER(c_u64)]),
    ("bfs_poll", c_i32, [c_vp, c_u64]),
    ("bfs_wait", c_i32, [c_vp, c_u64, c_i64]),
    ("bfs_server_stats", c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    ("bfs_ticket_latency_us", c_i32, [c_vp, c_u64, ctypes.POINTER(ctypes.c_double)]),
    ("bfs_server_destroy", None, [c_vp]),
    ("bfs_status_string", ctypes.c_char_p, [c_i32]),
    ("bfs_last_error", ctypes.c_char_p, []),
    ("bfs_version", ctypes.c_char_p, []),
]

_lib = None


def load(path: str | None = None):
    """Load libbfs_gb300.so (built in-tree).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1705_04590_gb300.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class BfsError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        self.status = status
        msg = lib.bfs_last_error().decode(errors="replace")
        name = lib.bfs_status_string(status).decode()
        super().__init__(f"{where}: {name}: {msg}")


def check(status: int, where: str) -> int:
    if status != BFS_OK:
        raise BfsError(status, where)
    return status

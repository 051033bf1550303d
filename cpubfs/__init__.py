"""Multithreaded direction-optimizing BFS on the host cores (OpenMP, C).

A CPU comparator for the benchmark: the paper's in-node algorithm (thread-local
queues merged per level, unsynchronised "benign race" claims in the top-down
step, a bitmap bottom-up step, the alpha/beta direction rule).  It is not part of
the GPU library and shares no code with it or with the serial oracle; the tests
check its levels against the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpubfs.c")
_LIB_PATH = os.path.join(_HERE, "libcpubfs.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile cpubfs.c into libcpubfs.so (gcc -O3 -fopenmp)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.cb_dobfs.argtypes = [i64, vp, vp, i32, i64, i64, i32, vp, vp, vp]
        L.cb_dobfs.restype = i32
        _lib = L
    return _lib


def dobfs(offsets: np.ndarray, cols: np.ndarray, root: int, alpha: int = 14, beta: int = 24, threads: int = 0):
    """Direction-optimizing BFS of an undirected CSR (int64 offsets, int32 ids) from
    `root`.  Returns (parent, level, stats) with stats = {levels, top-down levels,
    bottom-up levels, duplicate insertions, threads}."""
    n = int(offsets.shape[0]) - 1
    offsets = np.ascontiguousarray(offsets, np.int64)
    cols = np.ascontiguousarray(cols, np.int32)
    parent = np.empty(n, np.int32)
    level = np.empty(n, np.int32)
    st = np.zeros(4, np.int64)
    r = _load().cb_dobfs(n, offsets.ctypes.data, cols.ctypes.data, int(root), int(alpha), int(beta), int(threads),
                         parent.ctypes.data, level.ctypes.data, st.ctypes.data)
    if r < 0:
        raise MemoryError("cb_dobfs: out of host memory")
    return parent, level, {"levels": int(st[0]), "td_levels": int(st[1]), "bu_levels": int(st[2]),
                           "duplicates": int(st[3]), "threads": threads or (os.cpu_count() or 1)}

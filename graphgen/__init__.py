"""Seeded synthetic graph inputs (edge lists and roots).

This package produces the *inputs* that both the CPU oracle and the GPU path
consume: undirected edge lists (possibly with self-loops and duplicates, as a
random generator naturally makes them) and lists of distinct roots.  It holds
none of the breadth-first-search arithmetic: no adjacency build, no frontier,
no levels.  Each consumer symmetrises, drops self-loops and removes duplicate
edges on its own, as the paper's preprocessing step prescribes ("Data Sets":
duplicate edges are pruned; R-MAT a,b,c,d = .57,.19,.19,.05, edge factor 16).

The generators are written in C (``graphgen.c``) so that scale-26 inputs (about
10^9 edges) are produced in seconds on the host cores; small hand-made shapes
(paths, stars, ...) are plain numpy here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``libgraphgen.so`` beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-D_GNU_SOURCE",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint64, ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_er.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_er.restype = ctypes.c_int
        lib.gg_powerlaw.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_powerlaw.restype = ctypes.c_int
        lib.gg_torus.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_torus.restype = ctypes.c_int
        lib.gg_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, i32p]
        lib.gg_permutation.restype = None
        lib.gg_pick_roots.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p, ctypes.c_int64, ctypes.c_uint64, i32p]
        lib.gg_pick_roots.restype = ctypes.c_int64
        lib.gg_splitmix64_output.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_splitmix64_output.restype = ctypes.c_uint64
        lib.gg_stream_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_stream_key.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class EdgeList:
    """An undirected edge list over vertex ids [0, n) (may hold self-loops and duplicates)."""
    n: int
    src: np.ndarray  # int32[m]
    dst: np.ndarray  # int32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def splitmix64(state: int, i: int) -> int:
    """The i-th SplitMix64 output of a generator whose state starts at ``state``."""
    return int(_load().gg_splitmix64_output(state & (2**64 - 1), i))


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True, threads: int = 0) -> EdgeList:
    """R-MAT edge list with 2^scale vertices and edgefactor * 2^scale edges."""
    m = edgefactor << scale
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gg_rmat(scale, m, a, b, c, seed, int(permute), _p32(src), _p32(dst), threads)
    if rc != 0:
        raise ValueError("bad R-MAT arguments")
    return EdgeList(1 << scale, src, dst, f"rmat{scale}")


def erdos_renyi(n: int, m: int, seed: int = 1, permute: bool = True, threads: int = 0) -> EdgeList:
    """G(n, m): m independent uniform endpoint pairs."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _load().gg_er(n, m, seed, int(permute), _p32(src), _p32(dst), threads) != 0:
        raise ValueError("bad Erdos-Renyi arguments")
    return EdgeList(n, src, dst, f"er{n}")


def powerlaw(n: int, m: int, gamma: float = 2.1, i0: float = 50.0, seed: int = 1, permute: bool = True,
             threads: int = 0) -> EdgeList:
    """m edges whose ends are drawn with density (x + i0)^(-1/(gamma-1)) over vertex
    ranks x in [0, n) (Chung-Lu expected degrees, power-law exponent gamma > 2),
    ranks relabelled by the seeded bijection."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _load().gg_powerlaw(n, m, gamma, i0, seed, int(permute), _p32(src), _p32(dst), threads) != 0:
        raise ValueError("bad power-law arguments")
    return EdgeList(n, src, dst, f"powerlaw{n}")


def torus(side: int, seed: int = 3000, permute: bool = True, threads: int = 0) -> EdgeList:
    """side x side 2D torus (wrap-around), 2*side^2 edges; ids relabelled from ``seed``."""
    m = 2 * side * side
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    if _load().gg_torus(side, seed, int(permute), _p32(src), _p32(dst), threads) != 0:
        raise ValueError("bad torus arguments")
    return EdgeList(side * side, src, dst, f"torus{side}")


def torus_coordinates(side: int, seed: int = 3000, permute: bool = True) -> np.ndarray:
    """inv[label] = unpermuted grid id y*side + x of the vertex carrying ``label``."""
    n = side * side
    if not permute:
        return np.arange(n, dtype=np.int64)
    p = permutation(n, seed)
    inv = np.empty(n, np.int64)
    inv[p] = np.arange(n, dtype=np.int64)
    return inv


def permutation(n: int, seed: int) -> np.ndarray:
    """The seeded bijection of [0, n) used to relabel vertices: out[i] = label of vertex i."""
    out = np.empty(n, np.int32)
    _load().gg_permutation(n, seed, _p32(out))
    return out


def pick_roots(g: EdgeList, k: int, seed: int) -> np.ndarray:
    """k distinct roots, uniform over vertices with an edge to another vertex."""
    out = np.empty(max(k, 1), np.int32)
    got = _load().gg_pick_roots(g.n, g.m, _p32(g.src), _p32(g.dst), k, seed, _p32(out))
    if got < 0:
        raise ValueError("edge list holds ids outside [0, n)")
    return out[:got].copy()


# ------------------------------------------------------------------ small shapes

def from_pairs(n: int, pairs, name: str = "") -> EdgeList:
    arr = np.asarray(list(pairs), dtype=np.int64).reshape(-1, 2)
    return EdgeList(n, arr[:, 0].astype(np.int32), arr[:, 1].astype(np.int32), name)


def path(n: int) -> EdgeList:
    return from_pairs(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def cycle(n: int) -> EdgeList:
    return from_pairs(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def star(n: int, center: int = 0) -> EdgeList:
    return from_pairs(n, [(center, i) for i in range(n) if i != center], f"star{n}")


def complete(n: int) -> EdgeList:
    return from_pairs(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"complete{n}")


def random_small(n: int, m: int, seed: int, self_loops: bool = True) -> EdgeList:
    """Tiny random multigraph (numpy Generator): duplicates and, optionally, self-loops."""
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m, dtype=np.int64)
    dst = rng.integers(0, n, m, dtype=np.int64)
    if not self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    return EdgeList(n, src.astype(np.int32), dst.astype(np.int32), f"rand{n}_{m}_{seed}")


def disjoint_union(parts) -> tuple[EdgeList, np.ndarray]:
    """Concatenate edge lists with vertex ids offset per part; returns (graph, offsets)."""
    offs = np.zeros(len(parts) + 1, np.int64)
    for i, p in enumerate(parts):
        offs[i + 1] = offs[i] + p.n
    src = np.concatenate([p.src.astype(np.int64) + offs[i] for i, p in enumerate(parts)]).astype(np.int32)
    dst = np.concatenate([p.dst.astype(np.int64) + offs[i] for i, p in enumerate(parts)]).astype(np.int32)
    return EdgeList(int(offs[-1]), src, dst, "union"), offs

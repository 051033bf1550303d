"""GB300-native direction-optimizing breadth-first search.

Single-GPU implementation of the level-synchronous direction-optimizing BFS
of Bulu\\c{c}, Beamer, Madduri, Asanovic, Patterson, "Distributed-Memory
Breadth-First Search on Massive Graphs" (2015): top-down steps (Algorithm 1),
bottom-up steps (Algorithm 2), the per-level switch between them, CSR or
column-block DCSC storage.  Hand-written CUDA for sm_103a behind a C ABI
(include/bfs.h); this package is a thin ctypes binding.

    import paper_1705_04590_gb300 as bfs
    bfs.build(); bfs.load()
    g = bfs.Graph.from_edges(src, dst, n)
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    g.run(root, level=level)
"""
from ._build import build, LIB
from ._lib import (load, BfsError, MODE_DO, MODE_TD_ONLY, MODE_BU_ONLY, MODE_RANDOM, LAYOUT_CSR,
                   LAYOUT_DCSC_TILED, PARENT_ANY, PARENT_MIN_ID, BU_ROWS_BY_ID, BU_ROWS_HUB_FIRST, SIGNATURES)
from .api import Graph, Server, options

__all__ = ["build", "load", "Graph", "Server", "options", "BfsError", "LIB", "SIGNATURES", "MODE_DO", "MODE_TD_ONLY",
           "MODE_BU_ONLY", "MODE_RANDOM", "LAYOUT_CSR", "LAYOUT_DCSC_TILED", "PARENT_ANY", "PARENT_MIN_ID",
           "BU_ROWS_BY_ID", "BU_ROWS_HUB_FIRST"]

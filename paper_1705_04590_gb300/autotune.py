"""Autotuned search options, cached per (device, graph shape).

`tuned_options(graph, roots)` returns the bfs_options that bfs_autotune (the
library's native tuner: a grid over alpha, beta and the top-down hub cut-off,
then the top-down chunk size, the CTAs per SM and the cluster size one at a time, timed with CUDA
events) picked for a graph of this size and degree profile on this device,
running the tuner once and remembering the result in a JSON file (default
~/.cache/gb300_dobfs/autotune.json, or $BFS_AUTOTUNE_CACHE).
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _lib as L


def _cache_path() -> str:
    p = os.environ.get("BFS_AUTOTUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "gb300_dobfs", "autotune.json")


def _key(graph) -> str:
    import torch
    dev = torch.cuda.get_device_name()
    # graphs of the same size class and density share a setting
    return f"{dev}|n2^{int(np.ceil(np.log2(max(graph.n, 2))))}|deg{round(graph.nnz / max(graph.n, 1))}"


def autotune(graph, roots, base: L.Options | None = None, stream=None):
    """Run the library's tuner now; returns (options, ms per search)."""
    from .api import _stream_ptr
    r = np.ascontiguousarray(roots, np.int32)
    best = L.Options()
    ms = ctypes.c_double()
    L.check(L.load().bfs_autotune(graph.handle, r.ctypes.data, int(r.shape[0]), ctypes.byref(base) if base else None,
                                  ctypes.byref(best), ctypes.byref(ms), _stream_ptr(stream)), "bfs_autotune")
    return best, ms.value


def tuned_options(graph, roots, refresh: bool = False) -> L.Options:
    """Cached autotuned options for this graph's size class on this device."""
    path = _cache_path()
    key = _key(graph)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache and not refresh:
        c = cache[key]
        o = L.Options()
        L.load().bfs_options_default(ctypes.byref(o))
        o.alpha, o.beta, o.td_big_degree = int(c["alpha"]), int(c["beta"]), int(c["td_big_degree"])
        o.td_chunk, o.ctas_per_sm = int(c.get("td_chunk", 0)), int(c.get("ctas_per_sm", 0))
        o.cluster_size = int(c.get("cluster_size", 0))
        return o
    best, ms = autotune(graph, roots)
    cache[key] = {"alpha": best.alpha, "beta": best.beta, "td_big_degree": best.td_big_degree,
                  "td_chunk": best.td_chunk, "ctas_per_sm": best.ctas_per_sm,
                  "cluster_size": best.cluster_size, "ms": ms}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best

"""Named synthetic workloads: which graph, which seed, which roots.

Seeds are fixed so that every run (tests, bench, CPU baseline) sees the same
graphs and roots:

* R-MAT scale s: graph seed 1000 + s (initiator .57/.19/.19/.05, edge factor 16,
  ids relabelled by the seeded bijection), the paper's synthetic family.
* Erdos-Renyi with n = 2^k and expected degree 16 (8n undirected edges): seed 2000 + k.
* 4096 x 4096 torus: relabelling seed 3000.
* "Twitter-sized": 61.5 M vertices and 1.47 B generated edges (the size the paper
  gives for its Twitter graph in "Data Sets") with power-law expected degrees,
  exponent 2.1, rank offset 50 (largest expected degree about 2 M): seed 4000.  A
  synthetic stand-in of that size and shape; the Twitter data set itself is not here.
* roots: seed = graph seed + 1_000_000, distinct, uniform over vertices with degree > 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import EdgeList, erdos_renyi, pick_roots, powerlaw, rmat, torus


@dataclass(frozen=True)
class Workload:
    kind: str          # "rmat" | "er" | "torus" | "twitterlike"
    size: int          # scale (rmat), log2 n (er), side (torus), unused (twitterlike)

    @property
    def graph_seed(self) -> int:
        base = {"rmat": 1000, "er": 2000, "torus": 3000, "twitterlike": 4000}[self.kind]
        return base + (self.size if self.kind in ("rmat", "er") else 0)

    @property
    def root_seed(self) -> int:
        return self.graph_seed + 1_000_000

    @property
    def name(self) -> str:
        if self.kind == "rmat":
            return f"rmat-scale{self.size}-ef16"
        if self.kind == "er":
            return f"er-n2^{self.size}-deg16"
        if self.kind == "twitterlike":
            return "twitterlike-n61.5M-m1.47B-powerlaw2.1"
        return f"torus-{self.size}x{self.size}"

    def edges(self, threads: int = 0) -> EdgeList:
        if self.kind == "rmat":
            return rmat(self.size, 16, 0.57, 0.19, 0.19, seed=self.graph_seed, permute=True, threads=threads)
        if self.kind == "er":
            n = 1 << self.size
            return erdos_renyi(n, 8 * n, seed=self.graph_seed, permute=True, threads=threads)
        if self.kind == "twitterlike":
            return powerlaw(61_500_000, 1_470_000_000, 2.1, 50.0, seed=self.graph_seed, permute=True, threads=threads)
        return torus(self.size, seed=self.graph_seed, permute=True, threads=threads)

    def roots(self, g: EdgeList, k: int) -> np.ndarray:
        return pick_roots(g, k, self.root_seed)


RMAT = {s: Workload("rmat", s) for s in range(4, 31)}
ER26 = Workload("er", 26)
TORUS4096 = Workload("torus", 4096)
TWITTERLIKE = Workload("twitterlike", 0)

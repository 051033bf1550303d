"""Seeded input generators: determinism and structural properties (CPU)."""
import numpy as np
import pytest

import graphgen
from graphgen import workloads


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 1234567, as published with the
    # generator's reference implementation (Vigna, prng.di.unimi.it).
    assert [graphgen.splitmix64(1234567, i) for i in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000, 4096, 65537])
def test_permutation_is_bijection(n):
    p = graphgen.permutation(n, seed=42)
    assert np.array_equal(np.sort(p), np.arange(n, dtype=np.int32))


def test_permutation_depends_on_seed():
    a = graphgen.permutation(4096, 1)
    b = graphgen.permutation(4096, 2)
    assert not np.array_equal(a, b)
    assert (a == np.arange(4096)).mean() < 0.01


def test_rmat_deterministic_and_thread_independent():
    g1 = graphgen.rmat(12, seed=7, threads=1)
    g2 = graphgen.rmat(12, seed=7, threads=4)
    assert np.array_equal(g1.src, g2.src) and np.array_equal(g1.dst, g2.dst)
    g3 = graphgen.rmat(12, seed=8)
    assert not np.array_equal(g1.src, g3.src)
    assert g1.m == 16 * 4096 and g1.src.min() >= 0 and g1.src.max() < 4096


def test_rmat_quadrant_frequencies():
    # Without relabelling, the top bit of (u, v) is the first quadrant choice,
    # drawn with probabilities a, b, c, d.
    scale = 14
    g = graphgen.rmat(scale, seed=3, permute=False)
    hu = g.src >> (scale - 1)
    hv = g.dst >> (scale - 1)
    m = g.m
    freq = [np.mean((hu == 0) & (hv == 0)), np.mean((hu == 0) & (hv == 1)),
            np.mean((hu == 1) & (hv == 0)), np.mean((hu == 1) & (hv == 1))]
    for f, p in zip(freq, [0.57, 0.19, 0.19, 0.05]):
        assert abs(f - p) < 5 * np.sqrt(p * (1 - p) / m)


def test_rmat_permutation_is_relabelling():
    a = graphgen.rmat(10, seed=5, permute=False)
    b = graphgen.rmat(10, seed=5, permute=True)
    # the seeded bijection of R-MAT uses the graph seed
    p = graphgen.permutation(1 << 10, 5)
    assert np.array_equal(p[a.src], b.src) and np.array_equal(p[a.dst], b.dst)


def test_torus_structure():
    s = 8
    g = graphgen.torus(s, permute=False)
    assert g.m == 2 * s * s
    deg = np.bincount(np.concatenate([g.src, g.dst]), minlength=s * s)
    assert np.all(deg == 4)
    inv = graphgen.torus_coordinates(s, seed=9, permute=True)
    gp = graphgen.torus(s, seed=9, permute=True)
    assert np.array_equal(inv[gp.src], g.src) and np.array_equal(inv[gp.dst], g.dst)


def test_er_range():
    g = graphgen.erdos_renyi(1000, 5000, seed=1)
    assert g.src.min() >= 0 and g.src.max() < 1000 and g.m == 5000


def test_pick_roots_distinct_nonisolated():
    g = graphgen.rmat(12, seed=1012)
    roots = graphgen.pick_roots(g, 64, seed=5)
    assert len(set(roots.tolist())) == 64
    touched = np.zeros(g.n, bool)
    keep = g.src != g.dst
    touched[g.src[keep]] = True
    touched[g.dst[keep]] = True
    assert touched[roots].all()
    # fewer candidates than requested: all of them, once
    s = graphgen.from_pairs(10, [(1, 2), (3, 3)])
    r = graphgen.pick_roots(s, 5, seed=1)
    assert sorted(r.tolist()) == [1, 2]


def test_workload_seeds():
    w = workloads.RMAT[12]
    assert w.graph_seed == 1012 and w.root_seed == 1001012
    assert workloads.ER26.graph_seed == 2026 and workloads.TORUS4096.graph_seed == 3000


def test_powerlaw_generator_deterministic_and_follows_its_cdf():
    """The power-law generator gives one edge list per seed whatever the thread count,
    keeps ids in range, and (unpermuted) its endpoint ranks follow the closed-form CDF
    G(x) = ((x + i0)^b - i0^b) / ((n + i0)^b - i0^b), b = 1 - 1/(gamma - 1), within
    sampling error."""
    import math
    n, m, gamma, i0 = 200_000, 400_000, 2.1, 50.0
    a = graphgen.powerlaw(n, m, gamma, i0, seed=11, threads=1)
    b = graphgen.powerlaw(n, m, gamma, i0, seed=11, threads=4)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    assert a.src.min() >= 0 and max(a.src.max(), a.dst.max()) < n
    c = graphgen.powerlaw(n, m, gamma, i0, seed=12, threads=2)
    assert not np.array_equal(a.src, c.src)
    raw = graphgen.powerlaw(n, m, gamma, i0, seed=11, permute=False, threads=2)
    ends = np.concatenate([raw.src, raw.dst]).astype(np.int64)
    bb = 1.0 - 1.0 / (gamma - 1.0)
    for x in (1, 10, 100, 1000, 10_000, 100_000):
        want = ((x + i0) ** bb - i0 ** bb) / ((n + i0) ** bb - i0 ** bb)
        got = float(np.mean(ends < x))
        sd = math.sqrt(want * (1 - want) / ends.size)
        assert abs(got - want) < 6 * sd + 1e-6, (x, got, want)
    # a permutation of the unpermuted graph: same degree multiset
    da = np.sort(np.bincount(np.concatenate([a.src, a.dst]), minlength=n))
    dr = np.sort(np.bincount(ends, minlength=n))
    assert np.array_equal(da, dr)

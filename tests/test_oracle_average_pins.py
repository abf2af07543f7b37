"""Pins of the oracle's average cluster sizes (section "Cluster Analysis" results:
the average cluster size; reading R14: number average sum s c / sum c and weight
average sum s^2 c / sum s c, each one FP64 division of exact integer sums).

The expected values come from the mathematics, not from the oracle: hand-built
lattices whose clusters are known, exact rationals from ``fractions.Fraction``
over a graph library's connected components, and the inequalities every pair of
averages satisfies.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

NB = {
    oracle.TRI6: [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)],
    oracle.SQ4: [(1, 0), (-1, 0), (0, 1), (0, -1)],
}


def _lattice(Lx, Ly, fn):
    return np.array([1 if fn(i % Lx, i // Lx) else 0 for i in range(Lx * Ly)], dtype=np.uint8)


def _exact(sizes):
    """Exact (number, weight) averages of a list of cluster sizes, as floats of
    the exact rationals (IEEE division of two exactly representable integers is
    correctly rounded, so the FP64 averages must equal these bit for bit)."""
    n = len(sizes)
    if n == 0:
        return 0.0, 0.0
    s1 = sum(sizes)
    s2 = sum(s * s for s in sizes)
    return float(Fraction(s1, n)), float(Fraction(s2, s1))


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_all_A_is_one_cluster_of_N(geometry):
    t = np.ones(8 * 8, dtype=np.uint8)
    assert oracle.cluster_averages(8, 8, geometry, t, 1) == (64.0, 64.0)
    # no B site: the averages of an empty histogram are 0 (R14)
    assert oracle.cluster_averages(8, 8, geometry, t, 0) == (0.0, 0.0)


def test_square_checkerboard_is_all_singletons():
    t = _lattice(8, 8, lambda x, y: (x + y) % 2 == 0)
    assert oracle.cluster_averages(8, 8, oracle.SQ4, t, 1) == (1.0, 1.0)
    assert oracle.cluster_averages(8, 8, oracle.SQ4, t, 0) == (1.0, 1.0)


def test_triangular_checkerboard_is_diagonal_lines():
    # On the triangular lattice the (1,-1) bond joins (x, y) to (x+1, y-1): the
    # sites with x + y even form the lines x + y = c, c even; on an 8 x 8 torus
    # each line closes after 8 sites, so there are 4 clusters of 8.
    t = _lattice(8, 8, lambda x, y: (x + y) % 2 == 0)
    assert oracle.cluster_averages(8, 8, oracle.TRI6, t, 1) == (8.0, 8.0)


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_wrapping_stripe(geometry):
    # The columns x = 0 and x = Lx - 1 are one cluster of 2 Ly sites through the wrap.
    t = _lattice(10, 6, lambda x, y: x in (0, 9))
    assert oracle.cluster_averages(10, 6, geometry, t, 1) == (12.0, 12.0)


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_clusters_of_one_two_three(geometry):
    # Row 1 holds a singleton, a pair and a triple separated by B sites; all other
    # rows are B.  Number average 6/3 = 2, weight average (1 + 4 + 9)/6 = 7/3.  A
    # weight average computed over sum c instead of sum s c would give 14/3; one
    # computed from sizes without counts is the same here, so the next test adds
    # repeated sizes.
    A = {(1, 1), (3, 1), (4, 1), (6, 1), (7, 1), (8, 1)}
    t = _lattice(11, 5, lambda x, y: (x, y) in A)
    n_avg, w_avg = oracle.cluster_averages(11, 5, geometry, t, 1)
    assert n_avg == 2.0
    assert w_avg == float(Fraction(7, 3))


def test_histogram_averages_counts_weigh_sizes():
    # three singletons and one cluster of 5: <s>_n = 8/4, <s>_w = (3 + 25)/8
    assert oracle.histogram_averages([1, 5], [3, 1]) == (2.0, 3.5)
    # one size only: both averages equal it
    assert oracle.histogram_averages([7], [11]) == (7.0, 7.0)
    assert oracle.histogram_averages([], []) == (0.0, 0.0)


def test_histogram_averages_large_sums_are_exact_integers():
    # 2^31 - 1 sites in one cluster plus 2^20 singletons: the sums are exact
    # int64 values and each average is one correctly rounded division.
    big = (1 << 31) - 1
    n_avg, w_avg = oracle.histogram_averages([1, big], [1 << 20, 1])
    assert n_avg == float(Fraction(big + (1 << 20), (1 << 20) + 1))
    assert w_avg == float(Fraction(big * big + (1 << 20), big + (1 << 20)))


def test_histogram_averages_rejects_bad_input():
    with pytest.raises(ValueError):
        oracle.histogram_averages([1, -2], [1, 1])
    with pytest.raises(ValueError):
        oracle.histogram_averages([1, 2], [1, -1])
    with pytest.raises(OverflowError):
        oracle.histogram_averages([1 << 32], [1 << 32])


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
@pytest.mark.parametrize("Lx,Ly,frac", [(4, 4, 0.5), (9, 5, 0.4), (30, 30, 0.45), (17, 40, 0.6),
                                        (64, 64, 0.5)])
def test_averages_against_networkx_exact_rationals(geometry, Lx, Ly, frac):
    nx = pytest.importorskip("networkx")
    N = Lx * Ly
    t = oracle.init(Lx, Ly, int(frac * N), 777 + Lx + Ly)
    for species in (0, 1):
        G = nx.Graph()
        G.add_nodes_from(i for i in range(N) if t[i] == species)
        for i in range(N):
            if t[i] != species:
                continue
            x, y = i % Lx, i // Lx
            for dx, dy in NB[geometry]:
                j = ((y + dy) % Ly) * Lx + (x + dx) % Lx
                if t[j] == species:
                    G.add_edge(i, j)
        sizes = [len(c) for c in nx.connected_components(G)]
        n_avg, w_avg = oracle.cluster_averages(Lx, Ly, geometry, t, species)
        assert (n_avg, w_avg) == _exact(sizes)


@pytest.mark.parametrize("seed", range(6))
def test_average_inequalities(seed):
    # <s>_n * (number of clusters) = number of sites of the species, and
    # 1 <= <s>_n <= <s>_w <= largest cluster (Cauchy-Schwarz), with <s>_n = <s>_w
    # only when every cluster has the same size.
    Lx, Ly = 48, 40
    t = oracle.init(Lx, Ly, 700 + 90 * seed, 40 + seed)
    s, c = oracle.cluster_histogram(Lx, Ly, oracle.TRI6, t, 1)
    n_avg, w_avg = oracle.cluster_averages(Lx, Ly, oracle.TRI6, t, 1)
    assert n_avg * int(c.sum()) == pytest.approx(int(t.sum()), rel=1e-15)
    assert 1.0 <= n_avg <= w_avg <= float(s.max())
    assert (n_avg == w_avg) == (s.size == 1)

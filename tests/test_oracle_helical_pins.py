"""Pins for the oracle's helical lattice and seven-colour schedule (section
"Massive Parallel Kawasaki Kinetics": seven-lipid domains covering the
triangular lattice under helical boundary conditions, Fig. 4; the MPKK loop).

Each pin is independent of the oracle's code: a brute-force search for the
domain tilings the paper asserts, brute-force conflict checks of every
iteration, exact enumeration of a small lattice's Boltzmann distribution, the
omega = 0 limit, and a graph library's connected components.  The helical
neighbours are rebuilt here from the lattice definition: the six axial steps of
the triangular lattice read as index steps dx + dy*Lx, modulo N.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

AXIAL = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]


def hnbr(Lx, N, i, d):
    return (i + d[0] + d[1] * Lx) % N


def closed_nbhd(Lx, N, c):
    return {c} | {hnbr(Lx, N, c, d) for d in AXIAL}


def tiles(Lx, Ly):
    """Brute force: for every k the closed neighbourhoods of the sites i with
    i mod 7 = k partition the lattice (and the sites are all distinct)."""
    N = Lx * Ly
    for k in range(7):
        covered = []
        for c in range(k, N, 7):
            nb = closed_nbhd(Lx, N, c)
            if len(nb) != 7:
                return False
            covered.extend(nb)
        if len(covered) != N or len(set(covered)) != N:
            return False
    return True


def test_tiling_rule_matches_brute_force():
    """The paper's claim that seven-lipid domains cover the lattice "for certain
    sizes", with seven coverages generated by the first seven lipids: brute force
    over every Lx in 4..30 and Ly in 4..21 agrees with the rule 7 | N and
    Lx mod 7 in {3, 5}, and the rule holds for some sizes of every kind."""
    n_valid = 0
    for Lx in range(4, 31):
        for Ly in range(4, 22):
            bf = tiles(Lx, Ly)
            assert bf == oracle.helical_valid(Lx, Ly), (Lx, Ly)
            n_valid += bf
    assert n_valid > 20


@pytest.mark.parametrize("Lx,Ly", [(5, 7), (10, 7), (12, 14), (17, 7), (24, 21)])
def test_every_iteration_is_conflict_free(Lx, Ly):
    """For every coverage k and shared direction d, no site of one pair equals or
    neighbours a site of another pair, so an iteration does not depend on the
    order of its domains."""
    assert oracle.helical_valid(Lx, Ly)
    N = Lx * Ly
    for k in range(7):
        for d in AXIAL:
            owner = {}
            for c in range(k, N, 7):
                for s in (c, hnbr(Lx, N, c, d)):
                    assert s not in owner
                    owner[s] = c
            for s, c in owner.items():
                for e in AXIAL:
                    other = owner.get(hnbr(Lx, N, s, e))
                    assert other is None or other == c


def test_a_private_direction_per_domain_can_conflict():
    """The reading behind one shared direction: with a direction chosen per
    domain, the pairs of two neighbouring domains can touch."""
    Lx, Ly = 10, 7
    N = Lx * Ly
    c1 = 0
    c2 = next(c for c in range(7, N, 7) if any(hnbr(Lx, N, s, e) in closed_nbhd(Lx, N, c)
                                                for s in closed_nbhd(Lx, N, c1) for e in AXIAL))
    touching = [(d1, d2) for d1 in AXIAL for d2 in AXIAL
                if any(hnbr(Lx, N, hnbr(Lx, N, c1, d1), e) == hnbr(Lx, N, c2, d2) for e in AXIAL)]
    assert touching


def _bonds(Lx, Ly):
    N = Lx * Ly
    return sorted({tuple(sorted((i, hnbr(Lx, N, i, d)))) for i in range(N) for d in AXIAL})


@pytest.mark.parametrize("Lx,Ly", [(5, 7), (10, 7), (31, 14)])
def test_helical_energy_against_bond_list(Lx, Ly):
    bonds = np.array(_bonds(Lx, Ly))
    assert len(bonds) == 3 * Lx * Ly  # six neighbours, every bond once
    t = oracle.init(Lx, Ly, Lx * Ly // 3, 9)
    assert oracle.n_unlike(Lx, Ly, oracle.TRI6, t, oracle.HELICAL) == int(
        np.sum(t[bonds[:, 0]] != t[bonds[:, 1]]))


@pytest.mark.parametrize("Lx,Ly,bw", [(10, 7, 0.8), (12, 14, -0.6), (24, 21, 1.5)])
def test_mpkk_counts_energy_and_order(Lx, Ly, bw):
    """N attempts per MCS (seven iterations of N/7 domains), the incremental
    energy equals a recount after every iteration, composition is conserved, and
    reversing the domains' order changes nothing."""
    N = Lx * Ly
    t0 = oracle.init(Lx, Ly, N // 2, 5)
    r = oracle.run_mpkk(Lx, Ly, bw, 5, t0, 0, 15, check=True)
    rr = oracle.run_mpkk(Lx, Ly, bw, 5, t0, 0, 15, reverse=True)
    assert r.attempts == 15 * N
    assert int(r.lattice.sum()) == N // 2
    assert np.array_equal(r.lattice, rr.lattice) and r.counters() == rr.counters()
    whole = oracle.run_mpkk(Lx, Ly, bw, 5, t0, 3, 12)
    a = oracle.run_mpkk(Lx, Ly, bw, 5, t0, 3, 5)
    b = oracle.run_mpkk(Lx, Ly, bw, 5, a.lattice, 8, 7, n_unlike0=a.n_unlike, counters0=a.counters())
    assert np.array_equal(whole.lattice, b.lattice) and whole.counters() == b.counters()


def test_mpkk_zero_omega_accepts_every_unlike_pair():
    t0 = oracle.init(12, 14, 80, 2)
    r = oracle.run_mpkk(12, 14, 0.0, 2, t0, 0, 10)
    assert r.draws == 0 and r.accepts == r.unlike > 0


def test_mpkk_params_cover_all_values():
    from scipy.stats import chisquare

    ks = np.zeros(7)
    ds = np.zeros(6)
    for s in range(3000):
        for f in range(7):
            k, d = oracle.mpkk_params(17, s, f)
            ks[k] += 1
            ds[d] += 1
    assert chisquare(ks).pvalue > 1e-4 and chisquare(ds).pvalue > 1e-4


@pytest.mark.parametrize("bw", [0.4, -0.7])
def test_mpkk_stationary_distribution(bw):
    """Detailed balance of one iteration (each is a product of commuting
    symmetric Metropolis exchanges): on the helical 5 x 7 lattice with 3 A sites
    the energy classes are visited with the exact weights g(n) exp(-bw n)."""
    from scipy.stats import chisquare

    Lx, Ly, nA = 5, 7, 3
    N = Lx * Ly
    bonds = np.array(_bonds(Lx, Ly))
    g = {}
    for subset in itertools.combinations(range(N), nA):
        t = np.zeros(N, dtype=np.int8)
        t[list(subset)] = 1
        n = int(np.sum(t[bonds[:, 0]] != t[bonds[:, 1]]))
        g[n] = g.get(n, 0) + 1
    ns = np.array(sorted(g))
    w = np.array([g[n] * math.exp(-bw * n) for n in ns])
    p = w / w.sum()
    samples = np.array([oracle.run_mpkk(Lx, Ly, bw, 2000 + c, oracle.init(Lx, Ly, nA, 2000 + c), 0, 120).n_unlike
                        for c in range(4000)])
    obs = np.array([np.sum(samples == n) for n in ns], dtype=float)
    exp = p * obs.sum()
    keep = exp >= 5
    o2 = np.append(obs[keep], obs[~keep].sum())
    e2 = np.append(exp[keep], exp[~keep].sum())
    if e2[-1] == 0:
        o2, e2 = o2[:-1], e2[:-1]
    assert chisquare(o2, e2).pvalue > 1e-4


@pytest.mark.parametrize("Lx,Ly,frac", [(10, 7, 0.5), (31, 14, 0.4), (17, 21, 0.6)])
def test_helical_clusters_against_networkx(Lx, Ly, frac):
    nx = pytest.importorskip("networkx")
    N = Lx * Ly
    t = oracle.init(Lx, Ly, int(frac * N), 77 + Lx)
    for species in (0, 1):
        G = nx.Graph()
        G.add_nodes_from(i for i in range(N) if t[i] == species)
        for i, j in _bonds(Lx, Ly):
            if t[i] == species and t[j] == species:
                G.add_edge(i, j)
        comps = list(nx.connected_components(G))
        us, uc = np.unique(np.array(sorted(len(c) for c in comps)), return_counts=True)
        s, c = oracle.cluster_histogram(Lx, Ly, oracle.TRI6, t, species, oracle.HELICAL)
        assert list(s) == list(us) and list(c) == list(uc)
        labels, n = oracle.cluster_labels(Lx, Ly, oracle.TRI6, t, species, oracle.HELICAL)
        assert n == len(comps)
        for comp in comps:
            assert {int(labels[i]) for i in comp} == {min(comp)}

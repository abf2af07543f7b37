"""The values the paper states (tests/golden/paper_values.txt) against the oracle
and brute force.

Pins: the paper's claim that a coverable lattice has exactly seven decompositions
into seven-lipid domains, each generated by one of the first seven lipids, checked
by enumerating every tiling of small helical lattices; the 1/7 * 1/6 choice of a
centre and a neighbour; seven iterations of N/7 attempts per MPKK step; and the
image threshold delta_col the library uses by default.
"""
import inspect

import numpy as np
import pytest

import oracle
from _golden import paper_value

AXIAL = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)]


def all_tilings(Lx, Ly):
    """Every set of centres whose closed neighbourhoods (helical neighbours
    i + dx + dy*Lx mod N) partition the lattice, by exhaustive backtracking."""
    N = Lx * Ly
    nb = [[(i + dx + dy * Lx) % N for dx, dy in AXIAL] for i in range(N)]
    dom = [frozenset([i] + nb[i]) for i in range(N)]
    holders = [[c for c in [s] + nb[s] if len(dom[c]) == len(AXIAL) + 1 and s in dom[c]] for s in range(N)]
    covered = [False] * N
    chosen, found = [], []

    def extend():
        if all(covered):
            found.append(frozenset(chosen))
            return
        s = covered.index(False)  # the first uncovered site must lie in some domain
        for c in holders[s]:
            if not any(covered[t] for t in dom[c]):
                for t in dom[c]:
                    covered[t] = True
                chosen.append(c)
                extend()
                chosen.pop()
                for t in dom[c]:
                    covered[t] = False

    extend()
    return found, dom


@pytest.mark.parametrize("Lx,Ly", [(5, 7), (10, 7), (12, 7), (17, 7), (10, 14), (12, 14), (24, 7)])
def test_exactly_seven_coverages(Lx, Ly):
    tilings, dom = all_tilings(Lx, Ly)
    assert len(tilings) == paper_value("coverages")
    assert oracle.helical_valid(Lx, Ly)
    first = list(range(paper_value("coverage_generators")))
    for centres in tilings:
        assert all(len(dom[c]) == paper_value("domain_sites") for c in centres)
        gen = [c for c in first if c in centres]
        assert len(gen) == 1  # generated by exactly one of the first seven lipids
        assert centres == frozenset(range(gen[0], Lx * Ly, 7))
    # the seven are distinct: each first lipid generates its own
    assert len({min(c for c in t if c < 7) for t in tilings}) == len(tilings)


@pytest.mark.parametrize("Lx,Ly", [(6, 7), (7, 7), (8, 7), (9, 7), (11, 7)])
def test_no_coverage_outside_the_rule(Lx, Ly):
    tilings, _ = all_tilings(Lx, Ly)
    assert tilings == [] and not oracle.helical_valid(Lx, Ly)


def test_centre_and_neighbour_choice_probability():
    """Over iterations, the pair (coverage k, direction d) that makes centre c
    exchange with its neighbour in direction d comes up with probability
    1/7 * 1/6, within 5 sigma of the binomial."""
    den = paper_value("pair_choice_den")
    n = 0
    hits = np.zeros((7, 6))
    for s in range(1200):
        for f in range(7):
            k, d = oracle.mpkk_params(23, s, f)
            hits[k, d] += 1
            n += 1
    p = 1.0 / den
    sigma = np.sqrt(n * p * (1 - p))
    assert np.all(np.abs(hits - n * p) < 5 * sigma)


def test_step_is_seven_iterations_of_N_over_7():
    Lx, Ly = 10, 14
    N = Lx * Ly
    r = oracle.run_mpkk(Lx, Ly, 0.5, 3, oracle.init(Lx, Ly, N // 2, 3), 0, 1)
    assert r.attempts == paper_value("iterations_per_step") * (N // paper_value("domain_sites")) == N


def test_library_threshold_default_is_the_papers():
    import paper_1309_4349_gb300 as klmc

    assert inspect.signature(klmc.Lattice.image_ffn).parameters["delta"].default == paper_value("delta_col")


def test_neighbours_per_site():
    assert oracle.COORDINATION[oracle.TRI6] == paper_value("neighbours_per_site")

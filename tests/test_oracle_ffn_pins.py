"""Pins for the oracle's fraction of first neighbours (section "Image analysis":
for every site one randomly chosen nearest neighbour, the similar pairs divided
by the lattice size) and the comparison of the phase schedule with classical
Kawasaki that the paper draws on it (section "Results", Fig. 7).

Pins: exact values on lattices where every choice gives the same answer,
binomial statistics on striped lattices where the answer fixes the neighbour
choice to be uniform, the estimator's expectation (the all-bond fraction), and
equal equilibrium fractions for the schedule and random-sequential Kawasaki.
"""
import numpy as np
import pytest

import oracle


def _lattice(Lx, Ly, f):
    return np.array([1 if f(i % Lx, i // Lx) else 0 for i in range(Lx * Ly)], dtype=np.uint8)


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_uniform_lattice_is_all_similar(geometry):
    t = np.ones(20 * 14, dtype=np.uint8)
    for m in range(5):
        assert oracle.ffn_count(20, 14, geometry, t, 3, m) == 20 * 14
    assert oracle.ffn_exact(20, 14, geometry, t) == 1.0


def test_square_checkerboard_has_no_similar_neighbour():
    t = _lattice(16, 12, lambda x, y: (x + y) % 2 == 0)
    for m in range(5):
        assert oracle.ffn_count(16, 12, oracle.SQ4, t, 9, m) == 0
    assert oracle.ffn_exact(16, 12, oracle.SQ4, t) == 0.0


@pytest.mark.parametrize("geometry,stripes,p", [
    (oracle.TRI6, lambda x, y: y % 2 == 0, 2 / 6),   # like neighbours: (x+-1, y) only
    (oracle.SQ4, lambda x, y: x % 2 == 0, 2 / 4),    # like neighbours: (x, y+-1) only
    (oracle.SQ4, lambda x, y: y % 2 == 0, 2 / 4),
])
def test_striped_lattices_fix_the_choice_distribution(geometry, stripes, p):
    """On stripes the chosen neighbour is like with probability (like directions)/z
    exactly when the six (four) directions are equally likely; each sample is
    Binomial(N, p)."""
    Lx, Ly = 30, 20
    N = Lx * Ly
    t = _lattice(Lx, Ly, stripes)
    assert oracle.ffn_exact(Lx, Ly, geometry, t) == pytest.approx(p)
    M = 400
    mean = np.mean([oracle.ffn_count(Lx, Ly, geometry, t, 21, m) for m in range(M)])
    sigma = np.sqrt(N * p * (1 - p) / M)
    assert abs(mean - N * p) < 5 * sigma


@pytest.mark.parametrize("geometry,boundary,Lx,Ly", [(oracle.TRI6, oracle.PERIODIC, 40, 30),
                                                     (oracle.SQ4, oracle.PERIODIC, 33, 21),
                                                     (oracle.TRI6, oracle.HELICAL, 31, 14)])
def test_expectation_is_the_all_bond_fraction(geometry, boundary, Lx, Ly):
    N = Lx * Ly
    if boundary == oracle.HELICAL:
        t = oracle.run_mpkk(Lx, Ly, 0.9, 4, oracle.init(Lx, Ly, N // 3, 4), 0, 40).lattice
    else:
        t = oracle.run(Lx, Ly, geometry, 0.9, 4, oracle.init(Lx, Ly, N // 3, 4), 0, 40).lattice
    exact = oracle.ffn_exact(Lx, Ly, geometry, t, boundary)
    c = np.array([oracle.ffn_count(Lx, Ly, geometry, t, 4, m, boundary) for m in range(500)]) / N
    assert abs(c.mean() - exact) < 5 * c.std(ddof=1) / np.sqrt(len(c))


def test_schedule_and_classical_kawasaki_reach_the_same_fraction():
    """Fig. 7's comparison: at equilibrium the fraction of like first neighbours is
    the same for the conflict-free phase schedule and for random-sequential
    Kawasaki (one random site and neighbour per attempt), within the error of
    time averages over blocks."""
    Lx = Ly = 32
    N = Lx * Ly
    bw, seed = 0.6, 12
    t0 = oracle.init(Lx, Ly, N // 2, seed)
    burn, n, every = 400, 3000, 5
    r = oracle.run(Lx, Ly, oracle.TRI6, bw, seed, t0, 0, burn)
    tr = oracle.run(Lx, Ly, oracle.TRI6, bw, seed, r.lattice, burn, n, n_unlike0=r.n_unlike,
                    trace_every=every).trace
    f_sched = 1.0 - tr / (3.0 * N)
    t = t0
    f_seq = []
    t, _, _ = oracle.run_random_sequential(Lx, Ly, oracle.TRI6, bw, seed, t, 0, burn * N)
    for k in range(n // every):
        t, _, _ = oracle.run_random_sequential(Lx, Ly, oracle.TRI6, bw, seed, t, (burn + k * every) * N,
                                               every * N)
        f_seq.append(oracle.ffn_exact(Lx, Ly, oracle.TRI6, t))
    f_seq = np.array(f_seq)

    def block_err(x, blocks=20):
        b = x[: len(x) // blocks * blocks].reshape(blocks, -1).mean(axis=1)
        return b.std(ddof=1) / np.sqrt(blocks)

    err = np.hypot(block_err(f_sched), block_err(f_seq))
    assert abs(f_sched.mean() - f_seq.mean()) < 4 * err
    assert 0.5 < f_sched.mean() < 0.95  # demixing raises the like fraction above 1/2

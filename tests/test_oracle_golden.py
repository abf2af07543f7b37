"""The stored oracle runs (tests/golden/oracle_runs.txt): the oracle still
reproduces them bit for bit, and each stored result satisfies, by arithmetic
written here, what any correct run must: the composition of its start, an energy
equal to a recount of unlike bonds, N attempts per MCS where 4 divides Lx and Ly
(and on the helical lattice), ordered counters, and cluster sizes summing to n_A."""
import numpy as np
import pytest

import oracle
from _golden import oracle_cases

CASES = oracle_cases()
DIRS = {oracle.TRI6: [(1, 0), (0, 1), (1, -1)], oracle.SQ4: [(1, 0), (0, 1)]}


def recount(c):
    Lx, Ly, N = c["Lx"], c["Ly"], c["Lx"] * c["Ly"]
    t = c["lattice"].astype(np.int64)
    i = np.arange(N)
    x, y = i % Lx, i // Lx
    n = 0
    for dx, dy in DIRS[c["geometry"]]:
        if c["boundary"] == oracle.HELICAL:
            j = (i + dx + dy * Lx) % N
        else:
            j = ((y + dy) % Ly) * Lx + (x + dx) % Lx
        n += int(np.sum(t != t[j]))
    return n


@pytest.mark.parametrize("c", CASES, ids=lambda c: f"g{c['geometry']}b{c['boundary']}_{c['Lx']}x{c['Ly']}")
def test_stored_run_is_consistent(c):
    assert int(c["lattice"].sum()) == c["n_A"]
    assert recount(c) == c["n_unlike"]
    sizes, counts = c["hist_A"]
    assert int(np.sum(sizes * counts)) == c["n_A"]
    assert c["accepts"] <= c["unlike"] <= c["attempts"] and c["draws"] <= c["unlike"]
    if c["boundary"] == oracle.HELICAL or (c["Lx"] % 4 == 0 and c["Ly"] % 4 == 0):
        assert c["attempts"] == c["mcs"] * c["Lx"] * c["Ly"]


@pytest.mark.parametrize("c", CASES, ids=lambda c: f"g{c['geometry']}b{c['boundary']}_{c['Lx']}x{c['Ly']}")
def test_oracle_reproduces_stored_run(c):
    Lx, Ly = c["Lx"], c["Ly"]
    t0 = oracle.init(Lx, Ly, c["n_A"], c["seed"])
    if c["boundary"] == oracle.HELICAL:
        r = oracle.run_mpkk(Lx, Ly, c["omega_over_kT"], c["seed"], t0, 0, c["mcs"], check=True)
    else:
        r = oracle.run(Lx, Ly, c["geometry"], c["omega_over_kT"], c["seed"], t0, 0, c["mcs"], check=True)
    assert np.array_equal(r.lattice, c["lattice"])
    assert (r.n_unlike, *r.counters()) == (c["n_unlike"], c["attempts"], c["unlike"], c["draws"], c["accepts"])
    sizes, counts = oracle.cluster_histogram(Lx, Ly, c["geometry"], r.lattice, 1, c["boundary"])
    assert np.array_equal(sizes, c["hist_A"][0]) and np.array_equal(counts, c["hist_A"][1])

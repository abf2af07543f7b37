"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

None of these retype the oracle's own formulas.  Each pin uses an independent
source: another project's Philox, high-precision arithmetic, exact enumeration
of a small lattice's Boltzmann distribution, closed forms at omega = 0, a
graph library's connected components, and brute force over the schedule.
"""
import itertools
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# The test's own neighbour tables, written from the lattice definitions
# (triangular lattice in axial coordinates: six neighbours; square: four).
NB = {
    oracle.TRI6: [(1, 0), (-1, 0), (0, 1), (0, -1), (1, -1), (-1, 1)],
    oracle.SQ4: [(1, 0), (-1, 0), (0, 1), (0, -1)],
}


def nbr(Lx, Ly, i, d):
    x, y = i % Lx, i // Lx
    return ((y + d[1]) % Ly) * Lx + (x + d[0]) % Lx


# ---------------------------------------------------------------------------
# Philox4x32-10: against Triton's independent implementation (CPU interpreter).
# ---------------------------------------------------------------------------
def test_philox_matches_independent_implementation():
    pytest.importorskip("triton")
    cases = [
        ([0, 0, 0, 0], 0),
        ([1, 2, 3, 4], 0x1234567890ABCDEF),
        ([0xFFFFFFFF, 7, 0xFFFFFFFF, 0xFFFFFFFF], 0xFFFFFFFFFFFFFFFF),
        ([159999, 0xFFFFFFFF, 0, 0], 2),
        ([0xFFFFFFFF, 3, 19999, 0], 6),
        ([12345, 5, 0x89ABCDEF, 1], 1000 + 17),
    ]
    rng = np.random.default_rng(7)
    for _ in range(10):
        cases.append(([int(v) for v in rng.integers(0, 2**32, 4)], int(rng.integers(0, 2**63))))
    script = textwrap.dedent(
        """
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import torch, triton, triton.language as tl
        cases = json.loads(sys.argv[1])
        @triton.jit
        def k(out_ptr, c_ptr, seed):
            c0 = tl.load(c_ptr + 0); c1 = tl.load(c_ptr + 1)
            c2 = tl.load(c_ptr + 2); c3 = tl.load(c_ptr + 3)
            a, b, c, d = tl.philox(seed, c0, c1, c2, c3, n_rounds=10)
            tl.store(out_ptr + 0, a); tl.store(out_ptr + 1, b)
            tl.store(out_ptr + 2, c); tl.store(out_ptr + 3, d)
        res = []
        for ctr, seed in cases:
            c = torch.tensor([v - (1 << 32) if v >= (1 << 31) else v for v in ctr], dtype=torch.int32)
            out = torch.zeros(4, dtype=torch.int32)
            k[(1,)](out, c, seed)
            res.append([int(v) & 0xFFFFFFFF for v in out])
        print(json.dumps(res))
        """
    )
    import json

    proc = subprocess.run([sys.executable, "-c", script, json.dumps(cases)], capture_output=True,
                          text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    want = json.loads(proc.stdout.strip().splitlines()[-1])
    for (ctr, seed), w in zip(cases, want):
        got = oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert [int(v) for v in got] == w, (ctr, seed)


def test_philox_output_uniform():
    # 2^16 outputs of consecutive counters: each of the 16 top-nibble classes
    # holds 1/16 of them within 5 sigma.
    words = np.array([oracle.philox([i, 0, 0, 0], [99, 0]) for i in range(1 << 14)]).ravel()
    counts = np.bincount(words >> 28, minlength=16)
    exp = words.size / 16
    assert np.all(np.abs(counts - exp) < 5 * math.sqrt(exp))


# ---------------------------------------------------------------------------
# Acceptance thresholds: closed form with 60-digit arithmetic.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bw", [0.0, 0.1, 0.2, 0.55, 0.6, 0.85, 1.0, 1.2, 3.0, -0.5, -1.2])
def test_threshold_closed_form(bw):
    import mpmath

    mpmath.mp.dps = 60
    for dn in range(-10, 11, 2):
        always, thr = oracle.threshold(bw, dn)
        x = bw * dn
        if x <= 0:
            assert always and thr == 1 << 32
            continue
        assert not always
        exact = int(mpmath.ceil(mpmath.exp(-mpmath.mpf(bw) * dn) * mpmath.mpf(2) ** 32))
        assert abs(thr - exact) <= 1, (bw, dn, thr, exact)
        p = float(mpmath.exp(-mpmath.mpf(bw) * dn))
        # P(accept) = thr / 2^32 lies in [p, p + 2^-32) up to FP64 rounding of p
        assert p - 2**-40 <= thr / 2**32 < p + 2**-32 + 2**-40


def test_threshold_monotone():
    for bw in (0.3, 1.0):
        thrs = [oracle.threshold(bw, dn)[1] for dn in range(2, 11, 2)]
        assert all(a > b for a, b in zip(thrs, thrs[1:]))


def test_threshold_acceptance_frequency():
    # Empirical frequency of r < thr over Philox draws matches thr/2^32 within
    # binomial error.
    always, thr = oracle.threshold(0.6, 4)
    n = 20000
    hits = sum(int(oracle.philox([i, 3, 1, 0], [5, 0])[0]) < thr for i in range(n))
    p = thr / 2**32
    assert abs(hits - n * p) < 5 * math.sqrt(n * p * (1 - p))


# ---------------------------------------------------------------------------
# Initial placement: exact composition; uniform over subsets; smallest keys.
# ---------------------------------------------------------------------------
def test_n_A_rounding():
    assert oracle.n_A(64, 64, 2048) == 2048
    assert oracle.n_A(400, 400, -1, 0.3) == 48000
    assert oracle.n_A(5, 5, -1, 0.5) == 13  # floor(12.5 + 0.5)
    assert oracle.n_A(4, 4, -1, 0.0) == 0
    assert oracle.n_A(4, 4, -1, 1.0) == 16


@pytest.mark.parametrize("Lx,Ly,nA", [(4, 4, 0), (4, 4, 16), (5, 7, 12), (64, 64, 2048), (33, 9, 100)])
def test_init_composition_and_selection(Lx, Ly, nA):
    seed = 11
    t = oracle.init(Lx, Ly, nA, seed)
    assert int(t.sum()) == nA
    assert set(np.unique(t)).issubset({0, 1})
    keys = sorted((oracle.site_key(seed, i), i) for i in range(Lx * Ly))
    want = np.zeros(Lx * Ly, dtype=np.uint8)
    for _, i in keys[:nA]:
        want[i] = 1
    assert np.array_equal(t, want)


def test_init_uniform_over_subsets():
    # 4x4 lattice with 2 A sites: C(16,2) = 120 subsets, each equally likely.
    from scipy.stats import chisquare

    n_seeds = 24000
    counts = {}
    for seed in range(n_seeds):
        t = oracle.init(4, 4, 2, seed)
        key = tuple(np.flatnonzero(t))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 120
    stat = chisquare(list(counts.values()))
    assert stat.pvalue > 1e-4


# ---------------------------------------------------------------------------
# Schedule: conflict-free phases and full bond coverage (brute force).
# ---------------------------------------------------------------------------
def _grid(Lx, Ly, o):
    if o == (0, 1):
        return 2, 4, (Lx - 2) // 2 + 1, (Ly - 3) // 4 + 1
    return 4, 2, (Lx - 3) // 4 + 1, (Ly - 2) // 2 + 1


def _conflict_free(Lx, Ly, geometry, anchors, o):
    N = Lx * Ly
    a = np.asarray(anchors)
    b = np.array([nbr(Lx, Ly, int(i), o) for i in a])
    owner = np.full(N, -1)
    sites = np.concatenate([a, b])
    ids = np.concatenate([np.arange(a.size), np.arange(a.size)])
    if np.unique(sites).size != sites.size:
        return False
    owner[sites] = ids
    for p, (ai, bi) in enumerate(zip(a, b)):
        for s in (int(ai), int(bi)):
            for d in NB[geometry]:
                q = owner[nbr(Lx, Ly, s, d)]
                if q != -1 and q != p:
                    return False
    return True


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_schedule_conflict_free_all_sizes(geometry):
    # The anchor set of shift (rx, ry) is the (0, 0) set translated on the torus,
    # so checking shift (0, 0) for every size and orientation covers all shifts.
    for Lx in range(4, 41):
        for Ly in range(4, 41):
            for oi, o in enumerate(oracle.ORIENTATIONS[geometry]):
                anchors = oracle.phase_anchors(Lx, Ly, geometry, oi, 0, 0)
                px, py, Kx, My = _grid(Lx, Ly, o)
                assert anchors.size == Kx * My
                assert _conflict_free(Lx, Ly, geometry, anchors, o), (Lx, Ly, o)
                if Lx % 4 == 0 and Ly % 4 == 0:
                    assert anchors.size == Lx * Ly // 8


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_schedule_shifts_translate_and_cover(geometry):
    for Lx, Ly in [(4, 4), (5, 7), (9, 6), (12, 13)]:
        covered = set()
        for oi, o in enumerate(oracle.ORIENTATIONS[geometry]):
            base = oracle.phase_anchors(Lx, Ly, geometry, oi, 0, 0)
            for rx in range(Lx):
                for ry in range(Ly):
                    got = oracle.phase_anchors(Lx, Ly, geometry, oi, rx, ry)
                    want = [((i // Lx + ry) % Ly) * Lx + (i % Lx + rx) % Lx for i in base]
                    assert list(got) == want
                    for a in got:
                        covered.add(frozenset((int(a), nbr(Lx, Ly, int(a), o))))
        bonds = {frozenset((i, nbr(Lx, Ly, i, d))) for i in range(Lx * Ly) for d in NB[geometry]}
        assert covered == bonds  # every bond is proposed by some phase (ergodicity)


def test_phase_params_ranges():
    seen = set()
    for s in range(200):
        for f in range(8):
            o, rx, ry = oracle.phase_params(13, 7, oracle.TRI6, 3, s, f)
            assert 0 <= o < 3 and 0 <= rx < 13 and 0 <= ry < 7
            seen.add((o, rx, ry))
    assert len(seen) > 200


# ---------------------------------------------------------------------------
# Dynamics invariants.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
@pytest.mark.parametrize("Lx,Ly,bw", [(4, 4, 0.6), (5, 7, 1.0), (16, 16, 0.3), (13, 21, -0.5), (12, 8, 2.0)])
def test_run_conserves_and_tracks_energy(geometry, Lx, Ly, bw):
    nA = (Lx * Ly) // 3
    t0 = oracle.init(Lx, Ly, nA, 5)
    r = oracle.run(Lx, Ly, geometry, bw, 5, t0, 0, 30, check=True, trace_every=3)
    assert int(r.lattice.sum()) == nA
    assert r.n_unlike == oracle.n_unlike(Lx, Ly, geometry, r.lattice)
    assert r.trace[-1] == r.n_unlike
    px_all = [_grid(Lx, Ly, o) for o in oracle.ORIENTATIONS[geometry]]
    assert r.attempts <= 30 * 8 * max(k * m for _, _, k, m in px_all)
    assert r.accepts <= r.unlike <= r.attempts and r.draws <= r.unlike


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_run_order_independent(geometry):
    t0 = oracle.init(23, 18, 150, 9)
    a = oracle.run(23, 18, geometry, 0.7, 9, t0, 4, 20)
    b = oracle.run(23, 18, geometry, 0.7, 9, t0, 4, 20, reverse=True)
    assert np.array_equal(a.lattice, b.lattice)
    assert a.counters() == b.counters() and a.n_unlike == b.n_unlike


def test_run_split_equals_whole():
    t0 = oracle.init(20, 20, 200, 3)
    whole = oracle.run(20, 20, 0, 0.8, 3, t0, 0, 40)
    first = oracle.run(20, 20, 0, 0.8, 3, t0, 0, 17)
    second = oracle.run(20, 20, 0, 0.8, 3, first.lattice, 17, 23, n_unlike0=first.n_unlike,
                        counters0=first.counters())
    assert np.array_equal(whole.lattice, second.lattice)
    assert whole.counters() == second.counters()


def _enumerate_energy_classes(Lx, Ly, geometry, nA):
    """Density of states g(n) over all placements of nA A-sites."""
    N = Lx * Ly
    bonds = sorted({tuple(sorted((i, nbr(Lx, Ly, i, d)))) for i in range(N) for d in NB[geometry]})
    bi = np.array([b[0] for b in bonds])
    bj = np.array([b[1] for b in bonds])
    g = {}
    for subset in itertools.combinations(range(N), nA):
        t = np.zeros(N, dtype=np.int8)
        t[list(subset)] = 1
        n = int(np.sum(t[bi] != t[bj]))
        g[n] = g.get(n, 0) + 1
    return g


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
@pytest.mark.parametrize("bw", [0.3, 1.0, -0.5])
def test_stationary_distribution_4x4(geometry, bw):
    """Detailed balance (section "Massive Parallel Kawasaki Kinetics"): on a 4x4
    torus with 8 A sites the energy classes are visited with the exact Boltzmann
    weights g(n) exp(-bw n) at fixed composition."""
    from scipy.stats import chisquare

    g = _enumerate_energy_classes(4, 4, geometry, 8)
    ns = np.array(sorted(g))
    w = np.array([g[n] * math.exp(-bw * n) for n in ns])
    p = w / w.sum()
    # One sample per independent chain, taken after a burn-in well past the
    # energy autocorrelation (about 400 MCS at |bw| = 1 on this lattice).
    burn = 500 if abs(bw) >= 1.0 else 60
    samples = np.array([oracle.run(4, 4, geometry, bw, 1000 + c, oracle.init(4, 4, 8, 1000 + c),
                                   0, burn).n_unlike for c in range(5000)])
    obs = np.array([np.sum(samples == n) for n in ns], dtype=float)
    exp = p * obs.sum()
    keep = exp >= 5
    o2 = np.append(obs[keep], obs[~keep].sum())
    e2 = np.append(exp[keep], exp[~keep].sum())
    if e2[-1] == 0:
        o2, e2 = o2[:-1], e2[:-1]
    assert chisquare(o2, e2).pvalue > 1e-4


def test_uniform_states_at_zero_omega():
    """omega = 0: every placement of 8 A sites on 4x4 is equally likely."""
    from scipy.stats import chisquare

    t = oracle.init(4, 4, 8, 1)
    counts = np.zeros(1 << 16, dtype=np.int64)
    sweep, nu = 0, None
    weights = 1 << np.arange(16)
    for _ in range(20000):
        r = oracle.run(4, 4, oracle.TRI6, 0.0, 1, t, sweep, 3, n_unlike0=nu)
        t, sweep, nu = r.lattice, sweep + 3, r.n_unlike
        counts[int(np.dot(t.astype(np.int64), weights))] += 1
    n = int(counts.sum())
    # distinct states visited: coupon-collector expectation over 12870 states
    visited = int(np.count_nonzero(counts))
    exp_visited = 12870 * (1 - (1 - 1 / 12870) ** n)
    assert abs(visited - exp_visited) < 5 * math.sqrt(exp_visited * math.exp(-n / 12870))
    # chi-square over 99 bins of states (state rank mod 99), expected counts from
    # the number of states in each bin
    ranks = {sum(1 << i for i in c): r for r, c in enumerate(itertools.combinations(range(16), 8))}
    assert set(np.flatnonzero(counts)).issubset(ranks)
    obs = np.zeros(99)
    size = np.zeros(99)
    for code, r in ranks.items():
        obs[r % 99] += counts[code]
        size[r % 99] += 1
    assert chisquare(obs, n * size / size.sum()).pvalue > 1e-4


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
def test_zero_omega_mixing(geometry):
    """omega = 0: every unlike exchange is accepted without a draw, and the mean
    number of unlike contacts is B * 2 nA nB / (N (N - 1)), B = z N / 2."""
    Lx = Ly = 32
    N, nA = Lx * Ly, 300
    nB = N - nA
    t0 = oracle.init(Lx, Ly, nA, 17)
    r = oracle.run(Lx, Ly, geometry, 0.0, 17, t0, 0, 2000, trace_every=1)
    assert r.draws == 0 and r.accepts == r.unlike
    B = oracle.COORDINATION[geometry] * N / 2
    mean_exact = B * 2 * nA * nB / (N * (N - 1))
    tr = r.trace[100:].astype(float)
    batches = tr[: (tr.size // 50) * 50].reshape(50, -1).mean(axis=1)
    err = batches.std(ddof=1) / math.sqrt(batches.size)
    assert abs(tr.mean() - mean_exact) < 5 * err + 1e-9


# ---------------------------------------------------------------------------
# Clusters: hand-built patterns and a graph library's components.
# ---------------------------------------------------------------------------
def _lattice(Lx, Ly, fn):
    return np.array([1 if fn(i % Lx, i // Lx) else 0 for i in range(Lx * Ly)], dtype=np.uint8)


def test_clusters_all_A():
    t = np.ones(64, dtype=np.uint8)
    for g in (oracle.TRI6, oracle.SQ4):
        s, c = oracle.cluster_histogram(8, 8, g, t, 1)
        assert list(s) == [64] and list(c) == [1]
        s, c = oracle.cluster_histogram(8, 8, g, t, 0)
        assert s.size == 0


def test_clusters_checkerboard_distinguishes_geometry():
    t = _lattice(8, 8, lambda x, y: (x + y) % 2 == 0)
    s, c = oracle.cluster_histogram(8, 8, oracle.SQ4, t, 1)
    assert list(s) == [1] and list(c) == [32]  # square: all isolated
    s, c = oracle.cluster_histogram(8, 8, oracle.TRI6, t, 1)
    # triangular: (1,-1) diagonals connect same-parity sites into 4 lines of 8... which
    # close around the torus; (x+y) even sites on an 8x8 torus form x-y = const lines
    assert int((s * c).sum()) == 32
    assert s.max() > 1


def test_clusters_wrapping_stripe():
    # A vertical stripe x in {0, Lx-1} is one cluster through the periodic x boundary.
    t = _lattice(10, 6, lambda x, y: x in (0, 9))
    for g in (oracle.TRI6, oracle.SQ4):
        s, c = oracle.cluster_histogram(10, 6, g, t, 1)
        assert list(s) == [12] and list(c) == [1]


def test_clusters_diagonal_pair():
    # (2,3) and (3,2) touch in TRI6 through offset (1,-1); not in SQ4.
    t = _lattice(7, 7, lambda x, y: (x, y) in ((2, 3), (3, 2)))
    s, c = oracle.cluster_histogram(7, 7, oracle.TRI6, t, 1)
    assert list(s) == [2]
    s, c = oracle.cluster_histogram(7, 7, oracle.SQ4, t, 1)
    assert list(s) == [1] and list(c) == [2]
    # (2,2) and (3,3) touch in neither.
    t = _lattice(7, 7, lambda x, y: (x, y) in ((2, 2), (3, 3)))
    s, c = oracle.cluster_histogram(7, 7, oracle.TRI6, t, 1)
    assert list(s) == [1] and list(c) == [2]


@pytest.mark.parametrize("geometry", [oracle.TRI6, oracle.SQ4])
@pytest.mark.parametrize("Lx,Ly,frac", [(4, 4, 0.5), (9, 5, 0.4), (30, 30, 0.45), (17, 40, 0.6)])
def test_clusters_against_networkx(geometry, Lx, Ly, frac):
    nx = pytest.importorskip("networkx")
    N = Lx * Ly
    t = oracle.init(Lx, Ly, int(frac * N), 123 + Lx)
    for species in (0, 1):
        G = nx.Graph()
        G.add_nodes_from(i for i in range(N) if t[i] == species)
        for i in range(N):
            if t[i] != species:
                continue
            for d in NB[geometry]:
                j = nbr(Lx, Ly, i, d)
                if t[j] == species:
                    G.add_edge(i, j)
        comps = list(nx.connected_components(G))
        sizes = np.array(sorted(len(c) for c in comps))
        us, uc = np.unique(sizes, return_counts=True)
        s, c = oracle.cluster_histogram(Lx, Ly, geometry, t, species)
        assert list(s) == list(us) and list(c) == list(uc)
        assert int((s * c).sum()) == int((t == species).sum())
        labels, n = oracle.cluster_labels(Lx, Ly, geometry, t, species)
        assert n == len(comps)
        for comp in comps:
            assert {int(labels[i]) for i in comp} == {min(comp)}

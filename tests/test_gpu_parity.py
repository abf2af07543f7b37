"""GPU parity: the CUDA library, called through its C ABI, against the CPU oracle.

Every comparison is exact (integer lattice, counters, energies, histograms).
The FP64 average cluster sizes (number and weight averages, klmc_cluster_averages)
are compared with the oracle's within 1e-12 relative (``assert_averages``); both
sides divide the same exact integer sums, so they agree bit for bit in practice.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()
GEOMS = [klmc.TRI6, klmc.SQ4]
PACKS = [klmc.PACK_BIT, klmc.PACK_BYTE]


def make(Lx, Ly, nA, bw, seed, geometry=klmc.TRI6, packing=klmc.PACK_BIT, cluster=0, threads=0):
    return klmc.Lattice(Lx, Ly, geometry=geometry, packing=packing, n_A=nA, omega_over_kT=bw,
                        seed=seed, cluster=cluster, threads=threads)


AVG_RTOL = 1e-12


def assert_averages(got, want):
    """Average cluster sizes within 1e-12 relative (absolute 0 for an empty species)."""
    for g, w in zip(got, want):
        assert abs(g - w) <= AVG_RTOL * abs(w), (got, want)


def assert_same_run(lat, ref):
    assert np.array_equal(lat.get_lattice(), ref.lattice)
    c = lat.counters()
    assert (c["attempts"], c["unlike"], c["draws"], c["accepts"]) == ref.counters()
    assert lat.energy()[0] == ref.n_unlike
    assert lat.energy_recount() == ref.n_unlike


@pytest.mark.parametrize("packing", PACKS)
@pytest.mark.parametrize("Lx,Ly,nA,seed", [(4, 4, 8, 1), (5, 7, 0, 2), (5, 7, 35, 2), (64, 64, 2048, 1),
                                           (33, 65, 1000, 9), (101, 37, 1234, 3), (400, 400, 48000, 2)])
def test_initial_placement(packing, Lx, Ly, nA, seed):
    lat = make(Lx, Ly, nA, 0.6, seed, packing=packing)
    t = lat.get_lattice()
    assert np.array_equal(t, oracle.init(Lx, Ly, nA, seed))
    for g in GEOMS:
        assert oracle.n_unlike(Lx, Ly, g, t) >= 0
    assert lat.energy()[0] == oracle.n_unlike(Lx, Ly, klmc.TRI6, t)
    assert lat.n_A == nA


def test_fraction_rounding():
    lat = klmc.Lattice(5, 5, fraction_A=0.5, seed=4)
    assert lat.n_A == oracle.n_A(5, 5, -1, 0.5) == 13
    assert np.array_equal(lat.get_lattice(), oracle.init(5, 5, 13, 4))


CASES = [
    (4, 4, 8, 0.6), (5, 7, 17, 1.0), (7, 5, 12, -0.5), (31, 33, 400, 0.6), (64, 64, 2048, 0.6),
    (63, 100, 2000, 2.0), (100, 101, 3030, 0.0), (127, 33, 2000, 0.85), (96, 40, 1920, 0.3),
]


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("Lx,Ly,nA,bw", CASES)
def test_sweep_parity(geometry, Lx, Ly, nA, bw):
    seed = 1000 + Lx + 7 * Ly
    lat = make(Lx, Ly, nA, bw, seed, geometry)
    t0 = oracle.init(Lx, Ly, nA, seed)
    lat.sweep(20)
    ref = oracle.run(Lx, Ly, geometry, bw, seed, t0, 0, 20)
    assert_same_run(lat, ref)


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("cluster", [1, 2, 3, 4, 5, 8, 16])
@pytest.mark.parametrize("Lx,Ly,nA,bw", [(64, 64, 2048, 0.6), (100, 101, 3030, 1.0), (37, 70, 700, -0.4),
                                         (130, 131, 8000, 0.85)])
def test_cluster_size_parity(geometry, cluster, Lx, Ly, nA, bw):
    """The split of a lattice over a thread-block cluster never changes the result."""
    if Ly // cluster < 4:
        pytest.skip("bands need >= 4 rows")
    seed = 77 + cluster
    lat = make(Lx, Ly, nA, bw, seed, geometry, cluster=cluster)
    tr = lat.sweep_traced(12, 4)
    ref = oracle.run(Lx, Ly, geometry, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 12, trace_every=4)
    assert_same_run(lat, ref)
    torch.cuda.synchronize()
    assert tr.cpu().numpy().tolist() == ref.trace.tolist()


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("packing", PACKS)
@pytest.mark.parametrize("Lx,Ly,nA,bw,n_mcs,trace_every", [
    (4, 4, 8, 0.6, 9, 3), (5, 7, 17, 1.0, 11, 0), (64, 64, 2048, 0.6, 21, 10), (33, 95, 1500, -0.4, 17, 5),
    (100, 101, 3030, 0.85, 12, 4), (257, 66, 5000, 0.0, 9, 0),
])
def test_tiled_path_parity(geometry, packing, Lx, Ly, nA, bw, n_mcs, trace_every):
    """The per-phase tiled path (graph replays of K sweeps plus direct launches for
    the rest) gives the same trajectory as the oracle."""
    seed = 5 + Lx + Ly
    lat = make(Lx, Ly, nA, bw, seed, geometry, packing, cluster=-1)
    assert lat.launch_shape()[0] == -1
    ref = oracle.run(Lx, Ly, geometry, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, n_mcs,
                     trace_every=trace_every)
    if trace_every:
        tr = lat.sweep_traced(n_mcs, trace_every)
        torch.cuda.synchronize()
        assert tr.cpu().numpy().tolist() == ref.trace.tolist()
    else:
        lat.sweep(n_mcs)
    assert_same_run(lat, ref)


@pytest.mark.parametrize("packing", PACKS)
@pytest.mark.parametrize("Lx,Ly,K", [(200, 777, 4), (60000, 64, 4), (200000, 16, 1), (5, 7, 1), (64, 64, 4)])
def test_tiled_plans(packing, Lx, Ly, K):
    """The tiled path's plans: blocks of K phases per launch over bands of one or
    more rows, with rows wider than 2000 words, and the per-phase kernel when no
    block of halo rows fits (too short, or rows too wide for 2 x 5 halo rows in
    shared memory).  Odd sweep counts end the ping-pong on the second buffer."""
    nA, bw, seed = Lx * Ly * 2 // 5, 0.9, 31 + Ly
    lat = make(Lx, Ly, nA, bw, seed, klmc.TRI6, packing, cluster=-1)
    assert lat.plan() == K
    lat.sweep(3)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 3)
    assert_same_run(lat, ref)


def test_tiled_split_equals_whole():
    Lx, Ly, nA, bw, seed = 90, 70, 2000, 0.7, 44
    a = make(Lx, Ly, nA, bw, seed, cluster=-1)
    for n in (3, 8, 1, 16, 5):
        a.sweep(n)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 33)
    assert_same_run(a, ref)


def test_8192_lattice_tiled():
    """The 8192 x 8192, 1 bit per site, omega/kT = 0.85 lattice: too large for
    shared memory, so it runs on the tiled path.  One sweep against the oracle;
    then 25 more traced sweeps checked by invariants."""
    L = 8192
    nA = L * L // 2
    lat = make(L, L, nA, 0.85, 7)
    assert lat.launch_shape()[0] == -1
    t0 = lat.get_lattice()
    assert np.array_equal(t0, oracle.init(L, L, nA, 7))
    lat.sweep(1)
    ref = oracle.run(L, L, klmc.TRI6, 0.85, 7, t0, 0, 1)
    assert_same_run(lat, ref)
    tr = lat.sweep_traced(25, 10)
    torch.cuda.synchronize()
    t = lat.get_lattice()
    assert int(t.sum()) == nA
    n_end = lat.energy()[0]
    assert n_end == lat.energy_recount()
    assert tr.cpu().numpy().tolist()[-1] <= ref.n_unlike  # demixing lowers the energy
    assert lat.counters()["sweeps"] == 26


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("Lx,Ly,nA,bw", [(64, 64, 2048, 0.6), (150, 97, 4000, 1.0), (23, 41, 300, -0.3)])
def test_autotune_keeps_trajectory(geometry, Lx, Ly, nA, bw):
    """Tuning times every valid launch shape on a scratch copy (all must agree) and
    leaves the lattice, its counters and its future trajectory unchanged."""
    seed = 300 + Lx
    lat = make(Lx, Ly, nA, bw, seed, geometry)
    lat.sweep(3)
    before = lat.get_lattice()
    cnt = lat.counters()
    cluster, threads = lat.autotune(4)
    assert (cluster, threads) == lat.launch_shape()
    assert cluster == -1 or cluster in (1, 2, 4, 8, 16)
    assert threads in (128, 256, 512)
    assert np.array_equal(lat.get_lattice(), before)
    assert lat.counters() == cnt
    lat.sweep(9)
    ref = oracle.run(Lx, Ly, geometry, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 12)
    assert_same_run(lat, ref)
    # a new lattice of the same shape picks the tuned shape up
    assert make(Lx, Ly, nA, bw, seed + 1, geometry).launch_shape() == (cluster, threads)


@pytest.mark.parametrize("cluster,threads", [(1, 128), (1, 256), (1, 512), (3, 128), (8, 128), (16, 128)])
def test_thread_variant_parity(cluster, threads):
    """Every (CTAs per lattice, threads per CTA) variant gives the oracle's trajectory."""
    Lx, Ly, nA, bw, seed = 131, 100, 3300, 0.9, 61
    lat = make(Lx, Ly, nA, bw, seed, cluster=cluster, threads=threads)
    assert lat.launch_shape() == (cluster, threads)
    lat.sweep(11)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 11)
    assert_same_run(lat, ref)


# (Lx, Ly, CTAs, threads, phases between exchanges): blocks of 4 and 2 phases,
# two-CTA clusters (both neighbours are the same CTA), 512-thread CTAs in a
# cluster, and a cluster barrier after every phase for bands too thin for a block.
PLANS = [
    (131, 100, 8, 128, 4), (131, 100, 3, 512, 4), (400, 400, 16, 512, 4), (400, 400, 16, 256, 4),
    (37, 29, 2, 128, 2), (45, 23, 2, 512, 2), (2000, 96, 16, 128, 2), (1500, 24, 2, 128, 2),
    (64, 64, 16, 256, 1), (300, 41, 4, 512, 4),
]


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("Lx,Ly,cluster,threads,K", PLANS)
def test_plan_parity(geometry, Lx, Ly, cluster, threads, K):
    """Each plan gives the oracle's trajectory over 9 sweeps in two calls (blocks
    cross sweep and call boundaries), for omega > 0, < 0 and = 0."""
    for i, bw in enumerate((0.85, -0.6, 0.0)):
        seed = 500 + Lx + 7 * i
        nA = (Lx * Ly * (3 + i)) // 10
        packing = klmc.PACK_BYTE if (i == 2 and Lx < 200) else klmc.PACK_BIT
        lat = make(Lx, Ly, nA, bw, seed, geometry, cluster=cluster, threads=threads, packing=packing)
        assert lat.plan() == K
        lat.sweep(4)
        lat.sweep(5)
        ref = oracle.run(Lx, Ly, geometry, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 9)
        assert_same_run(lat, ref)
        lat.close()


def test_cluster_size_rejected():
    with pytest.raises(klmc.KlmcError) as e:
        make(16, 16, 100, 0.5, 1, cluster=8)  # bands of 2 rows
    assert e.value.status == 1
    with pytest.raises(klmc.KlmcError):
        make(64, 64, 100, 0.5, 1, cluster=17)
    with pytest.raises(klmc.KlmcError):
        make(64, 64, 100, 0.5, 1, cluster=-2)
    with pytest.raises(klmc.KlmcError):
        make(64, 64, 100, 0.5, 1, threads=64)


@pytest.mark.parametrize("geometry", GEOMS)
def test_byte_store_parity(geometry):
    Lx, Ly, nA, bw, seed = 70, 45, 1300, 0.7, 77
    lat = make(Lx, Ly, nA, bw, seed, geometry, klmc.PACK_BYTE)
    lat.sweep(15)
    ref = oracle.run(Lx, Ly, geometry, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 15)
    assert_same_run(lat, ref)


@pytest.mark.parametrize("geometry", GEOMS)
def test_edge_compositions(geometry):
    for nA in (0, 8 * 9):
        lat = make(8, 9, nA, 0.6, 3, geometry)
        lat.sweep(5)
        ref = oracle.run(8, 9, geometry, 0.6, 3, oracle.init(8, 9, nA, 3), 0, 5)
        assert_same_run(lat, ref)
        assert ref.unlike == 0


def test_split_equals_whole_and_trace():
    Lx, Ly, nA, bw, seed = 48, 52, 900, 0.9, 12
    a = make(Lx, Ly, nA, bw, seed)
    tr = a.sweep_traced(30, 3)
    b = make(Lx, Ly, nA, bw, seed)
    b.sweep(7)
    b.sweep(0)
    b.sweep(23)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 30, trace_every=3)
    assert_same_run(a, ref)
    assert_same_run(b, ref)
    torch.cuda.synchronize()
    assert tr.cpu().numpy().tolist() == ref.trace.tolist()


def test_checkpoint_resume():
    Lx, Ly, nA, bw, seed = 40, 36, 500, 0.6, 8
    a = make(Lx, Ly, nA, bw, seed)
    a.sweep(25)
    snap = a.get_lattice()
    b = make(Lx, Ly, nA, bw, seed + 1)  # different placement, same model
    b.set_lattice(snap, 25)
    a.sweep(15)
    # seeds differ, so resume b under a's key by building it with a's seed
    c = make(Lx, Ly, nA, bw, seed)
    c.set_lattice(snap, 25)
    c.sweep(15)
    assert np.array_equal(a.get_lattice(), c.get_lattice())
    assert a.energy()[0] == c.energy()[0]
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, snap, 25, 15)
    assert np.array_equal(c.get_lattice(), ref.lattice)
    assert c.counters()["accepts"] == ref.accepts
    assert b.n_A == nA


def test_set_lattice_device():
    Lx, Ly, bw, seed = 45, 30, 0.8, 14
    t = oracle.init(Lx, Ly, 700, 99)
    lat = make(Lx, Ly, 10, bw, seed)
    lat.set_lattice_device(torch.from_numpy(t).cuda(), 3)
    assert lat.n_A == 700
    lat.sweep(12)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, t, 3, 12)
    assert_same_run(lat, ref)


def _hist_equal(lat, t, species):
    s, c = lat.cluster_histogram(species)
    rs, rc = oracle.cluster_histogram(lat.Lx, lat.Ly, lat.geometry, t, species)
    assert np.array_equal(s, rs) and np.array_equal(c, rc)
    assert int((s * c).sum()) == int((t == species).sum())
    assert_averages(lat.cluster_averages(species), oracle.histogram_averages(rs, rc))


@pytest.mark.parametrize("geometry", GEOMS)
@pytest.mark.parametrize("Lx,Ly,nA,bw", [(4, 4, 8, 0.6), (9, 5, 20, 1.0), (64, 64, 2048, 0.6),
                                         (400, 400, 48000, 1.0), (130, 77, 5000, 0.0)])
def test_cluster_histogram_parity(geometry, Lx, Ly, nA, bw):
    lat = make(Lx, Ly, nA, bw, 31, geometry)
    _hist_equal(lat, lat.get_lattice(), 1)
    lat.sweep(10)
    t = lat.get_lattice()
    for species in (1, 0):
        _hist_equal(lat, t, species)


def test_cluster_patterns():
    def pattern(Lx, Ly, fn):
        return np.array([1 if fn(i % Lx, i // Lx) else 0 for i in range(Lx * Ly)], dtype=np.uint8)

    cases = [
        (8, 8, lambda x, y: True),
        (8, 8, lambda x, y: (x + y) % 2 == 0),
        (10, 6, lambda x, y: x in (0, 9)),
        (7, 7, lambda x, y: (x, y) in ((2, 3), (3, 2))),
        (33, 9, lambda x, y: (x * 7 + y * 3) % 5 < 2),
    ]
    for g in GEOMS:
        for Lx, Ly, fn in cases:
            t = pattern(Lx, Ly, fn)
            lat = make(Lx, Ly, int(t.sum()), 0.5, 1, g)
            lat.set_lattice(t, 0)
            assert np.array_equal(lat.get_lattice(), t)
            _hist_equal(lat, t, 1)
            _hist_equal(lat, t, 0)


def test_histogram_truncation():
    lat = make(64, 64, 2048, 0.0, 5)
    import ctypes

    sizes = np.zeros(1, dtype=np.int64)
    counts = np.zeros(1, dtype=np.int64)
    n = ctypes.c_int64(-1)
    st = klmc.lib().klmc_cluster_histogram(lat._h, 1, sizes.ctypes.data, counts.ctypes.data, 1,
                                           ctypes.byref(n))
    rs, _ = oracle.cluster_histogram(64, 64, klmc.TRI6, lat.get_lattice(), 1)
    assert st == 6 and n.value == rs.size > 1  # KLMC_ETRUNC with the needed length


def test_batch_parity_mixed():
    reps = [
        dict(Lx=64, Ly=64, n_A=2048, omega_over_kT=0.6, seed=1),
        dict(Lx=37, Ly=29, n_A=300, omega_over_kT=1.1, seed=2, geometry=klmc.SQ4),
        dict(Lx=100, Ly=100, n_A=3000, omega_over_kT=0.2, seed=3),
        dict(Lx=5, Ly=4, n_A=9, omega_over_kT=-0.4, seed=4),
        dict(Lx=150, Ly=90, n_A=6000, omega_over_kT=0.85, seed=5, packing=klmc.PACK_BYTE),
    ]
    b = klmc.Batch(reps)
    steps = [12, 7, 0, 20, 9]
    b.sweep(steps)
    b.sweep(3)
    for r, lat, n in zip(reps, b.replicas, steps):
        g = r.get("geometry", klmc.TRI6)
        ref = oracle.run(r["Lx"], r["Ly"], g, r["omega_over_kT"], r["seed"],
                         oracle.init(r["Lx"], r["Ly"], r["n_A"], r["seed"]), 0, n + 3)
        assert_same_run(lat, ref)
        assert lat.counters()["sweeps"] == n + 3
    b.close()


def test_batch_histograms_match_oracle():
    """klmc_batch_cluster_histogram_device: every replica's histogram, computed on
    concurrent streams into one (n, capacity) buffer, equals the oracle's on the
    replica's lattice, for both species and both geometries; a capacity below the
    number of distinct sizes truncates the pairs but reports the full count."""
    reps = [dict(Lx=64 + 9 * i, Ly=50 + 7 * i, n_A=(64 + 9 * i) * (50 + 7 * i) * (2 + i % 4) // 10,
                 omega_over_kT=0.4 + 0.2 * (i % 5), seed=900 + i,
                 geometry=klmc.SQ4 if i % 3 == 1 else klmc.TRI6) for i in range(11)]
    b = klmc.Batch(reps)
    b.sweep(30)
    n, cap = len(reps), 256
    for species in (1, 0):
        sizes = torch.full((n, cap), -1, dtype=torch.int64, device="cuda")
        counts = torch.full((n, cap), -1, dtype=torch.int64, device="cuda")
        nd = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        b.cluster_histogram_device(species, sizes, counts, nd)
        torch.cuda.synchronize()
        for i, (r, lat) in enumerate(zip(reps, b.replicas)):
            g = r.get("geometry", klmc.TRI6)
            rs, rc = oracle.cluster_histogram(r["Lx"], r["Ly"], g, lat.get_lattice(), species)
            k = int(nd[i].item())
            assert k == rs.size and k <= cap
            assert np.array_equal(sizes[i, :k].cpu().numpy(), rs)
            assert np.array_equal(counts[i, :k].cpu().numpy(), rc)
            assert_averages(klmc.histogram_averages(sizes[i, :k].cpu().numpy(), counts[i, :k].cpu().numpy()),
                            oracle.histogram_averages(rs, rc))
    small = torch.zeros((n, 1), dtype=torch.int64, device="cuda")
    nd = torch.zeros((n,), dtype=torch.int64, device="cuda")
    b.cluster_histogram_device(1, small, small.clone(), nd)
    torch.cuda.synchronize()
    for i, (r, lat) in enumerate(zip(reps, b.replicas)):
        rs, _ = oracle.cluster_histogram(r["Lx"], r["Ly"], r.get("geometry", klmc.TRI6), lat.get_lattice(), 1)
        assert int(nd[i].item()) == rs.size and int(small[i, 0].item()) == rs[0]
    b.close()


def test_batch_oversubscribed_runs_throughput_shape():
    """More 200 x 200 replicas (8 CTAs each at their own shape) than the GPU's SMs
    hold: the call runs the replicas with automatic shapes at 4 CTAs of 128
    threads, a replica with a fixed shape keeps its shape, a call that advances few
    replicas uses the own shapes again, and every trajectory still equals the
    oracle's."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    n = nsm // 8 + 2
    reps = [dict(Lx=200, Ly=200, n_A=12000 + 7 * i, omega_over_kT=0.3 + 0.05 * (i % 9), seed=40 + i,
                 geometry=klmc.SQ4 if i % 5 == 2 else klmc.TRI6) for i in range(n)]
    reps[3]["cluster"] = 8
    b = klmc.Batch(reps)
    own = [r.launch_shape() for r in b.replicas]
    assert own[0] == (8, 256) and own[3][0] == 8
    steps = [4 + (i % 3) for i in range(n)]
    b.sweep(steps)
    for i in range(n):
        assert b.launch_shape(i) == (own[i] if i == 3 else (4, 128)), i
    few = [0] * n
    few[0], few[3] = 3, 2
    b.sweep(few)
    assert b.launch_shape(0) == own[0] and b.launch_shape(3) == own[3]
    for i in (0, 1, 2, 3, n - 1):
        r = reps[i]
        g = r.get("geometry", klmc.TRI6)
        ref = oracle.run(200, 200, g, r["omega_over_kT"], r["seed"],
                         oracle.init(200, 200, r["n_A"], r["seed"]), 0, steps[i] + few[i])
        assert_same_run(b.replicas[i], ref)
    b.close()


def test_largest_single_cta_lattice():
    """The largest lattice one CTA holds (1280 rows + 4 halo rows of 44 words)."""
    Lx, Ly = 1280, 1280
    nA = Lx * Ly // 2
    lat = make(Lx, Ly, nA, 0.85, 7, cluster=1)
    lat.sweep(2)
    ref = oracle.run(Lx, Ly, klmc.TRI6, 0.85, 7, oracle.init(Lx, Ly, nA, 7), 0, 2)
    assert_same_run(lat, ref)
    with pytest.raises(klmc.KlmcError) as e:
        make(1400, 1400, 1000, 0.5, 1, cluster=1).sweep(1)
    assert e.value.status == 1


def test_large_lattice_on_full_cluster():
    """2048 x 2048 split over 16 CTAs (the largest side of the serving workload)."""
    Lx = Ly = 2048
    nA = Lx * Ly * 3 // 10
    lat = make(Lx, Ly, nA, 0.7, 9, cluster=16)
    assert lat.launch_shape()[0] == 16
    lat.sweep(1)
    ref = oracle.run(Lx, Ly, klmc.TRI6, 0.7, 9, oracle.init(Lx, Ly, nA, 9), 0, 1)
    assert_same_run(lat, ref)
    # too large for a 16-CTA cluster: the automatic choice falls back to the tiled path
    assert make(6000, 6000, 1000, 0.5, 1).launch_shape()[0] == -1
    with pytest.raises(klmc.KlmcError) as e:
        make(6000, 6000, 1000, 0.5, 1, cluster=16).sweep(1)
    assert e.value.status == 1


def test_full_size_400_sampled():
    """The benchmark's 400x400 lattice for the full 20000 steps with the
    cluster-histogram cadence of 500 steps: every histogram is checked against
    the oracle on the GPU's own lattice, the running energy against a recount, and
    the first and last steps against oracle runs started from the same states."""
    Lx = Ly = 400
    nA, bw, seed = 48000, 1.0, 6
    lat = make(Lx, Ly, nA, bw, seed)
    t0 = lat.get_lattice()
    lat.sweep(30)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, t0, 0, 30)
    assert np.array_equal(lat.get_lattice(), ref.lattice)
    done = 30
    for k in range(1, 40):
        lat.sweep(500 * k - done)
        done = 500 * k
        if k % 13 == 0:
            t = lat.get_lattice()
            _hist_equal(lat, t, 1)
            assert lat.energy()[0] == lat.energy_recount() == oracle.n_unlike(Lx, Ly, 0, t)
            assert int(t.sum()) == nA
    lat.sweep(19990 - done)
    snap = lat.get_lattice()
    n0 = lat.energy()[0]
    lat.sweep(10)
    ref = oracle.run(Lx, Ly, klmc.TRI6, bw, seed, snap, 19990, 10, n_unlike0=n0)
    assert np.array_equal(lat.get_lattice(), ref.lattice)
    assert lat.energy()[0] == ref.n_unlike
    _hist_equal(lat, ref.lattice, 1)


def test_c4_workload_sampled():
    """The batched workload as the benchmark builds it (256 replicas, sides 100 to
    1017, in one batch at the throughput shapes), for 12 MCS: every replica keeps
    its composition and an energy equal to a recount, and the largest, the
    smallest and two more replicas equal their oracle runs bit for bit."""
    import bench

    reps = bench.c4_replicas()
    assert len(reps) == 256
    b = klmc.Batch(reps)
    n = 12
    b.sweep([n] * len(reps))
    sides = [r["Lx"] for r in reps]
    for i, r in enumerate(reps):
        lat = b.replicas[i]
        t = lat.get_lattice()
        assert int(t.sum()) == oracle.n_A(r["Lx"], r["Ly"], -1, r["fraction_A"]), i
        assert lat.energy()[0] == lat.energy_recount(), i
        c = lat.counters()
        assert c["attempts"] <= n * r["Lx"] * r["Ly"] and c["accepts"] <= c["unlike"], i
    for i in sorted({int(np.argmax(sides)), int(np.argmin(sides)), 17, 200}):
        r = reps[i]
        nA = oracle.n_A(r["Lx"], r["Ly"], -1, r["fraction_A"])
        ref = oracle.run(r["Lx"], r["Ly"], klmc.TRI6, r["omega_over_kT"], r["seed"],
                         oracle.init(r["Lx"], r["Ly"], nA, r["seed"]), 0, n)
        assert_same_run(b.replicas[i], ref)
    b.close()


def test_c1_workload_full():
    """The 64x64 workload as the benchmark runs it (TRI6, byte store, 2048 A, omega/kT
    0.6, seed 1, tuned launch shape, 1000 MCS with an A-cluster histogram every 100
    MCS), in full: all ten histograms, the final lattice, the counters and the
    energy equal the oracle's."""
    import bench

    c = bench.C1
    L = c["L"]
    lat = klmc.Lattice(L, L, n_A=c["n_A"], omega_over_kT=c["omega"], seed=c["seed"], packing=klmc.PACK_BYTE)
    lat.autotune(16)
    t = oracle.init(L, L, c["n_A"], c["seed"])
    assert np.array_equal(lat.get_lattice(), t)
    nu, cnt = None, (0, 0, 0, 0)
    for k in range(c["mcs"] // c["hist_every"]):
        lat.sweep(c["hist_every"])
        r = oracle.run(L, L, klmc.TRI6, c["omega"], c["seed"], t, k * c["hist_every"], c["hist_every"],
                       n_unlike0=nu, counters0=cnt)
        t, nu, cnt = r.lattice, r.n_unlike, r.counters()
        sizes, counts = lat.cluster_histogram(1)
        rs, rc = oracle.cluster_histogram(L, L, klmc.TRI6, t, 1)
        assert np.array_equal(np.asarray(sizes), rs) and np.array_equal(np.asarray(counts), rc), k
        want = oracle.histogram_averages(rs, rc)
        assert_averages(lat.cluster_averages(1), want)
        assert_averages(klmc.histogram_averages(sizes, counts), want)
        assert_averages(lat.cluster_averages(0), oracle.cluster_averages(L, L, klmc.TRI6, t, 0))
    assert_same_run(lat, r)
    lat.close()


def test_8192_full_size_graph_block_against_oracle():
    """The 8192 x 8192, 1 bit per site, omega/kT = 0.85 lattice as the benchmark runs
    it: one traced graph replay of 10 sweeps (20 band launches of 4 phases, the
    energy trace every 10 MCS) against the oracle, lattice, counters, energy and
    trace; then two more replays against the oracle continued from that state."""
    L = 8192
    nA = L * L // 2
    lat = make(L, L, nA, 0.85, 7)
    assert lat.launch_shape()[0] == -1
    t0 = oracle.init(L, L, nA, 7)
    tr = lat.sweep_traced(10, 10)
    ref = oracle.run(L, L, klmc.TRI6, 0.85, 7, t0, 0, 10, trace_every=10)
    assert_same_run(lat, ref)
    assert tr.cpu().numpy().tolist() == ref.trace.tolist()
    lat.sweep(16)  # two replays of the untraced 8-sweep graph
    ref2 = oracle.run(L, L, klmc.TRI6, 0.85, 7, ref.lattice, 10, 16, n_unlike0=ref.n_unlike,
                      counters0=ref.counters())
    assert_same_run(lat, ref2)
    lat.close()


def test_c4_all_replicas_against_oracle():
    """All 256 replicas of the batched workload as the benchmark builds them, in one
    batch at the shapes the batch chooses, for 5 MCS: every replica's lattice,
    counters and energy equal its own oracle run (the oracle spread over host
    threads)."""
    import concurrent.futures

    import bench

    reps = bench.c4_replicas()
    b = klmc.Batch(reps)
    n = 5
    b.sweep([n] * len(reps))

    def ref_of(r):
        nA = oracle.n_A(r["Lx"], r["Ly"], -1, r["fraction_A"])
        return oracle.run(r["Lx"], r["Ly"], klmc.TRI6, r["omega_over_kT"], r["seed"],
                          oracle.init(r["Lx"], r["Ly"], nA, r["seed"]), 0, n)

    with concurrent.futures.ThreadPoolExecutor(max_workers=16) as ex:
        refs = list(ex.map(ref_of, reps))
    shapes = set()
    for i, ref in enumerate(refs):
        assert_same_run(b.replicas[i], ref)
        shapes.add(b.launch_shape(i))
    assert len(shapes) >= 2  # the batch ran several launch shapes
    b.close()


def test_c2_one_run_2000_mcs_all_histograms():
    """One of the 400 x 400 workload's runs (omega/kT 0.6, its seed) for 2000 MCS
    with the histogram cadence of 500 MCS: all four histograms, their averages, and
    the final lattice, counters and energy equal the oracle's."""
    import bench

    Lx = Ly = bench.L
    w, seed = bench.OMEGAS[2], bench.SEEDS[2]
    nA = oracle.n_A(Lx, Ly, -1, bench.FRACTION_A)
    lat = klmc.Lattice(Lx, Ly, fraction_A=bench.FRACTION_A, omega_over_kT=w, seed=seed)
    t = oracle.init(Lx, Ly, nA, seed)
    assert np.array_equal(lat.get_lattice(), t)
    nu, cnt = None, (0, 0, 0, 0)
    for k in range(4):
        lat.sweep(bench.HIST_EVERY)
        r = oracle.run(Lx, Ly, klmc.TRI6, w, seed, t, k * bench.HIST_EVERY, bench.HIST_EVERY,
                       n_unlike0=nu, counters0=cnt)
        t, nu, cnt = r.lattice, r.n_unlike, r.counters()
        _hist_equal(lat, t, 1)
    assert_same_run(lat, r)
    lat.close()


def test_large_standalone_lattice_takes_tiled_path_automatically():
    """A standalone 1024 x 1000 lattice (at least 786432 sites) with the automatic
    shape runs on the tiled path, exactly; the same lattice as a batch replica stays
    resident and gives the same lattice."""
    Lx, Ly, nA, bw, seed = 1024, 1000, 307200, 0.7, 31
    lat = make(Lx, Ly, nA, bw, seed)
    b = klmc.Batch([dict(Lx=Lx, Ly=Ly, n_A=nA, omega_over_kT=bw, seed=seed)])
    try:
        assert lat.launch_shape()[0] == -1
        lat.sweep(2)
        b.sweep(2)
        assert b.launch_shape(0)[0] >= 1
        ref = oracle.run(Lx, Ly, oracle.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 2)
        assert np.array_equal(lat.get_lattice(), ref.lattice)
        assert np.array_equal(b.replicas[0].get_lattice(), ref.lattice)
        c = lat.counters()
        assert (c["attempts"], c["draws"], c["accepts"]) == (ref.attempts, ref.draws, ref.accepts)
    finally:
        b.close()
        lat.close()

"""The helical triangular lattice with the seven-colour MPKK schedule on the GPU
(section "Massive Parallel Kawasaki Kinetics": seven-lipid domains covering the
lattice under helical boundary conditions, one Kawasaki attempt per domain per
iteration, seven iterations per step) against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()


def make(Lx, Ly, nA, bw, seed, packing=klmc.PACK_BIT, cluster=0):
    return klmc.Lattice(Lx, Ly, geometry=klmc.TRI6, packing=packing, n_A=nA, omega_over_kT=bw, seed=seed,
                        boundary=klmc.HELICAL, cluster=cluster)


def assert_same_run(lat, ref, Lx, Ly):
    assert np.array_equal(lat.get_lattice(), ref.lattice)
    c = lat.counters()
    assert (c["attempts"], c["unlike"], c["draws"], c["accepts"]) == ref.counters()
    assert lat.energy()[0] == ref.n_unlike
    assert lat.energy_recount() == ref.n_unlike == oracle.n_unlike(Lx, Ly, oracle.TRI6, ref.lattice,
                                                                   oracle.HELICAL)


@pytest.mark.parametrize("cluster", [0, -1])
@pytest.mark.parametrize("packing", [klmc.PACK_BIT, klmc.PACK_BYTE])
@pytest.mark.parametrize("Lx,Ly,bw,n_mcs", [(10, 7, 0.9, 23), (12, 14, -0.5, 17), (17, 7, 0.0, 9),
                                            (24, 21, 1.4, 13), (40, 35, 0.6, 11), (402, 399, 0.8, 5)])
def test_helical_parity(cluster, packing, Lx, Ly, bw, n_mcs):
    """Automatic shape (resident in a cluster when the bands are tall enough for
    blocks of iterations, else one launch per iteration) and the per-iteration
    path, both against the oracle."""
    assert oracle.helical_valid(Lx, Ly)
    nA, seed = Lx * Ly * 3 // 10, 11 + Lx
    lat = make(Lx, Ly, nA, bw, seed, packing, cluster)
    C, T = lat.launch_shape()
    if cluster == -1 or Ly < 48:
        assert C == -1 and lat.plan() == 1
    else:
        assert C >= 2 and T == 512 and lat.plan() in (2, 4)
    t0 = lat.get_lattice()
    assert np.array_equal(t0, oracle.init(Lx, Ly, nA, seed))
    assert lat.energy()[0] == oracle.n_unlike(Lx, Ly, oracle.TRI6, t0, oracle.HELICAL)
    lat.sweep(n_mcs - 4)
    lat.sweep(4)
    ref = oracle.run_mpkk(Lx, Ly, bw, seed, t0, 0, n_mcs)
    assert_same_run(lat, ref, Lx, Ly)


def test_helical_traced_and_large():
    """A 1004 x 1001 lattice (about 10^6 sites), traced every 3 steps: the trace
    and the final state equal the oracle's."""
    Lx, Ly, bw, seed = 1004, 1001, 0.7, 5
    nA = Lx * Ly // 2
    lat = make(Lx, Ly, nA, bw, seed)
    t0 = lat.get_lattice()
    tr = lat.sweep_traced(9, 3)
    torch.cuda.synchronize()
    ref = oracle.run_mpkk(Lx, Ly, bw, seed, t0, 0, 9, trace_every=3)
    assert tr.cpu().numpy().tolist() == ref.trace.tolist()
    assert_same_run(lat, ref, Lx, Ly)


def test_helical_large():
    """8195 x 3129 (2.6e7 sites, 7 | N, Lx mod 7 = 5): two steps equal the
    oracle's."""
    Lx, Ly, bw, seed = 8195, 3129, 0.8, 21
    assert oracle.helical_valid(Lx, Ly)
    nA = Lx * Ly * 2 // 5
    lat = make(Lx, Ly, nA, bw, seed)
    t0 = lat.get_lattice()
    lat.sweep(2)
    ref = oracle.run_mpkk(Lx, Ly, bw, seed, t0, 0, 2)
    assert_same_run(lat, ref, Lx, Ly)


def test_helical_set_lattice_and_histograms():
    Lx, Ly = 31, 14
    lat = make(Lx, Ly, 100, 1.1, 3)
    t = oracle.run_mpkk(Lx, Ly, 1.1, 3, oracle.init(Lx, Ly, 180, 8), 0, 30).lattice
    lat.set_lattice(t, 70)
    assert lat.energy()[0] == oracle.n_unlike(Lx, Ly, oracle.TRI6, t, oracle.HELICAL)
    for species in (0, 1):
        s, c = lat.cluster_histogram(species)
        rs, rc = oracle.cluster_histogram(Lx, Ly, oracle.TRI6, t, species, oracle.HELICAL)
        assert np.array_equal(s, rs) and np.array_equal(c, rc)
    lat.sweep(6)
    ref = oracle.run_mpkk(Lx, Ly, 1.1, 3, t, 70, 6)
    assert np.array_equal(lat.get_lattice(), ref.lattice)
    assert lat.energy()[0] == ref.n_unlike


def test_helical_rejections():
    with pytest.raises(klmc.KlmcError) as e:
        make(64, 64, 100, 0.5, 1)  # 64 mod 7 = 1: the domains do not tile it
    assert e.value.status == 1
    with pytest.raises(klmc.KlmcError):
        klmc.Lattice(10, 7, geometry=klmc.SQ4, boundary=klmc.HELICAL)
    with pytest.raises(klmc.KlmcError):
        klmc.Lattice(10, 7, boundary=klmc.HELICAL, cluster=2)
    with pytest.raises(klmc.KlmcError) as e:
        klmc.Batch([dict(Lx=10, Ly=7, boundary=klmc.HELICAL)])
    assert e.value.status == 1


def test_c6_workload_one_run_full():
    """One of the helical workload's five runs as the benchmark sets it up (402 x
    399, 30% A, omega/kT 0.6, its seed) for the full 2000 MCS: the A-cluster
    histogram after every 500 MCS, the final lattice, the counters and the energy
    equal the oracle's."""
    import bench

    c = bench.C6
    Lx, Ly = c["Lx"], c["Ly"]
    w, seed = bench.OMEGAS[2], bench.SEEDS[2]
    lat = klmc.Lattice(Lx, Ly, fraction_A=bench.FRACTION_A, omega_over_kT=w, seed=seed, boundary=klmc.HELICAL)
    nA = oracle.n_A(Lx, Ly, -1, bench.FRACTION_A)
    t = oracle.init(Lx, Ly, nA, seed)
    assert np.array_equal(lat.get_lattice(), t)
    nu, cnt = None, (0, 0, 0, 0)
    for k in range(c["mcs"] // c["hist_every"]):
        lat.sweep(c["hist_every"])
        r = oracle.run_mpkk(Lx, Ly, w, seed, t, k * c["hist_every"], c["hist_every"], n_unlike0=nu,
                            counters0=cnt)
        t, nu, cnt = r.lattice, r.n_unlike, r.counters()
        sizes, counts = lat.cluster_histogram(1)
        rs, rc = oracle.cluster_histogram(Lx, Ly, oracle.TRI6, t, 1, oracle.HELICAL)
        assert np.array_equal(np.asarray(sizes), rs) and np.array_equal(np.asarray(counts), rc), k
        # average cluster sizes within 1e-12 relative of the oracle's
        for got, want in zip(lat.cluster_averages(1), oracle.histogram_averages(rs, rc)):
            assert abs(got - want) <= 1e-12 * abs(want), k
    assert_same_run(lat, r, Lx, Ly)
    lat.close()


@pytest.mark.parametrize("packing", [klmc.PACK_BIT, klmc.PACK_BYTE])
@pytest.mark.parametrize("Lx,Ly,cluster,bw", [(101, 98, 4, 0.7), (101, 98, 2, -0.6), (103, 70, 2, 1.2),
                                              (199, 77, 4, 0.0), (199, 77, 8, 0.9), (38, 336, 16, 0.5),
                                              (402, 399, 16, 1.0), (402, 399, 8, 0.3)])
def test_helical_resident_parity(packing, Lx, Ly, cluster, bw):
    """The resident helical sweep (a cluster of CTAs, blocks of iterations with
    re-evaluated halos, pads of the helical row continuation) at explicit cluster
    sizes, both stores, rows of one to thirteen words with ragged ends, both
    residues of Lx mod 7: against the oracle over several calls whose iterations
    cross sweep and block boundaries."""
    assert oracle.helical_valid(Lx, Ly)
    nA, seed = Lx * Ly // 3, 40 + cluster
    lat = make(Lx, Ly, nA, bw, seed, packing, cluster)
    assert lat.launch_shape() == (cluster, 512)
    t0 = lat.get_lattice()
    for n in (1, 3, 7):
        lat.sweep(n)
    ref = oracle.run_mpkk(Lx, Ly, bw, seed, t0, 0, 11)
    assert_same_run(lat, ref, Lx, Ly)


def test_helical_resident_equals_per_iteration_path():
    """The same lattice and seed on the resident sweep and on one launch per
    iteration: identical lattices, counters and traces after 40 steps."""
    Lx, Ly, bw, seed = 402, 399, 0.6, 4
    nA = Lx * Ly * 3 // 10
    a = make(Lx, Ly, nA, bw, seed, cluster=16)
    b = make(Lx, Ly, nA, bw, seed, cluster=-1)
    ta = a.sweep_traced(40, 5)
    tb = b.sweep_traced(40, 5)
    torch.cuda.synchronize()
    assert ta.cpu().numpy().tolist() == tb.cpu().numpy().tolist()
    assert np.array_equal(a.get_lattice(), b.get_lattice())
    assert a.counters() == b.counters()
    assert a.energy() == b.energy()


def test_helical_resident_rejects_thin_bands():
    with pytest.raises(klmc.KlmcError) as e:
        make(103, 70, 1000, 0.5, 1, cluster=16)  # bands of 4 rows: no room for 2K+1 halo rows
    assert e.value.status == 1


def test_helical_replicas_in_a_batch():
    """Helical replicas (resident helical sweep, one launch each) batched with
    periodic ones: every replica equals its own oracle run, and the batch's
    histograms of the helical replicas use the helical adjacency."""
    reps = [dict(Lx=101, Ly=98, n_A=3000, omega_over_kT=0.8, seed=61, boundary=klmc.HELICAL),
            dict(Lx=120, Ly=100, n_A=4000, omega_over_kT=0.6, seed=62),
            dict(Lx=402, Ly=399, n_A=48000, omega_over_kT=1.0, seed=63, boundary=klmc.HELICAL),
            dict(Lx=64, Ly=64, n_A=2048, omega_over_kT=0.4, seed=64, geometry=klmc.SQ4)]
    b = klmc.Batch(reps)
    inits = [lat.get_lattice() for lat in b.replicas]
    steps = [9, 7, 5, 3]
    b.sweep(steps)
    for r, lat, t0, n in zip(reps, b.replicas, inits, steps):
        Lx, Ly = r["Lx"], r["Ly"]
        if r.get("boundary") == klmc.HELICAL:
            assert b.launch_shape(reps.index(r))[1] == 512
            ref = oracle.run_mpkk(Lx, Ly, r["omega_over_kT"], r["seed"], t0, 0, n)
            assert_same_run(lat, ref, Lx, Ly)
        else:
            ref = oracle.run(Lx, Ly, r.get("geometry", klmc.TRI6), r["omega_over_kT"], r["seed"], t0, 0, n)
            assert np.array_equal(lat.get_lattice(), ref.lattice)
            assert lat.energy()[0] == ref.n_unlike
    cap = 512
    sizes = torch.zeros((len(reps), cap), dtype=torch.int64, device="cuda")
    counts = torch.zeros_like(sizes)
    nd = torch.zeros(len(reps), dtype=torch.int64, device="cuda")
    b.cluster_histogram_device(1, sizes, counts, nd)
    torch.cuda.synchronize()
    for i, (r, lat) in enumerate(zip(reps, b.replicas)):
        bnd = oracle.HELICAL if r.get("boundary") == klmc.HELICAL else oracle.PERIODIC
        rs, rc = oracle.cluster_histogram(r["Lx"], r["Ly"], r.get("geometry", klmc.TRI6), lat.get_lattice(), 1,
                                          bnd)
        k = int(nd[i].item())
        assert k == rs.size
        assert np.array_equal(sizes[i, :k].cpu().numpy(), rs) and np.array_equal(counts[i, :k].cpu().numpy(), rc)
    b.close()


def test_helical_jobs_in_the_server():
    """Helical jobs served beside periodic ones: each result equals the oracle's
    run of that job, histograms included; a helical lattice too small for the
    resident sweep is refused as a job (EINVAL) without stopping the others."""
    srv = klmc.Server(1 << 30)
    jobs = [dict(L=(101, 98), helical=True, n_A=3000, w=0.7, seed=71, n=40),
            dict(L=(96, 96), helical=False, n_A=3000, w=0.9, seed=72, n=30),
            dict(L=(402, 399), helical=True, n_A=40000, w=1.1, seed=73, n=25),
            dict(L=(10, 7), helical=True, n_A=20, w=0.5, seed=74, n=5)]
    ids = [srv.submit(j["L"][0], j["L"][1], n_mcs=j["n"], hist_every=10, keep_lattice=True, n_A=j["n_A"],
                      omega_over_kT=j["w"], seed=j["seed"], boundary=klmc.HELICAL if j["helical"] else 0)
           for j in jobs]
    srv.drain(300.0)
    for j, jid in zip(jobs, ids):
        r = srv.poll(jid)
        Lx, Ly = j["L"]
        if (Lx, Ly) == (10, 7):
            assert r["status"] == 1
            continue
        assert r["status"] == 0
        t0 = oracle.init(Lx, Ly, j["n_A"], j["seed"])
        if j["helical"]:
            ref = oracle.run_mpkk(Lx, Ly, j["w"], j["seed"], t0, 0, j["n"])
            bnd = oracle.HELICAL
        else:
            ref = oracle.run(Lx, Ly, oracle.TRI6, j["w"], j["seed"], t0, 0, j["n"])
            bnd = oracle.PERIODIC
        assert np.array_equal(srv.lattice(jid, Lx * Ly), ref.lattice)
        assert (r["attempts"], r["unlike"], r["draws"], r["accepts"]) == ref.counters()
        assert r["n_unlike"] == ref.n_unlike
        s, c = srv.histogram(jid)
        rs, rc = oracle.cluster_histogram(Lx, Ly, oracle.TRI6, ref.lattice, 1, bnd)
        assert np.array_equal(s, rs) and np.array_equal(c, rc)
    srv.close()

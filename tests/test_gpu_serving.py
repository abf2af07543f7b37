"""Serving form: a job server with continuous batching, through the C ABI.

Each job's result (counters, energy, final lattice, last cluster histogram) must
be exactly the same whether the job runs alone or in a mix of concurrently
resident jobs that arrive while others are on the GPU, and must equal the plain
single-lattice path (and the oracle for small lattices).
"""
import random
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()

JOB = dict(Lx=72, Ly=80, n_A=2000, omega_over_kT=0.8, seed=77, n_mcs=700, hist_every=250)


def run_alone(job):
    s = klmc.Server(1 << 30)
    jid = s.submit(job["Lx"], job["Ly"], n_mcs=job["n_mcs"], hist_every=job.get("hist_every", 0),
                   keep_lattice=True, n_A=job["n_A"], omega_over_kT=job["omega_over_kT"],
                   seed=job["seed"], geometry=job.get("geometry", klmc.TRI6))
    s.drain(120)
    res = s.poll(jid)
    lat = s.lattice(jid, job["Lx"] * job["Ly"])
    hist = s.histogram(jid)
    s.close()
    return res, lat, hist


def same(a, b):
    ra, la, ha = a
    rb, lb, hb = b
    keys = ("status", "n_mcs", "n_unlike", "attempts", "unlike", "draws", "accepts", "n_histograms")
    assert {k: ra[k] for k in keys} == {k: rb[k] for k in keys}
    assert np.array_equal(la, lb)
    assert np.array_equal(ha[0], hb[0]) and np.array_equal(ha[1], hb[1])


def test_job_same_alone_and_in_a_mix():
    alone = run_alone(JOB)
    assert alone[0]["status"] == 0 and alone[0]["n_mcs"] == JOB["n_mcs"]
    # The same job inside a stream of other jobs that arrive while it is resident.
    rng = random.Random(5)
    s = klmc.Server(1 << 30)
    ids = {}
    others = []
    for k in range(14):
        L = rng.choice([16, 40, 64, 100, 130, 257, 400])
        others.append(dict(Lx=L, Ly=L + rng.choice([0, 3]), n_A=(L * L) // 3,
                           omega_over_kT=rng.uniform(0.1, 1.2), seed=1000 + k,
                           n_mcs=rng.choice([50, 300, 900, 2000]), hist_every=rng.choice([0, 100]),
                           geometry=rng.choice([klmc.TRI6, klmc.SQ4])))
    for k, job in enumerate(others[:6]):
        ids[k] = s.submit(job["Lx"], job["Ly"], n_mcs=job["n_mcs"], hist_every=job["hist_every"],
                          keep_lattice=True, n_A=job["n_A"], omega_over_kT=job["omega_over_kT"],
                          seed=job["seed"], geometry=job["geometry"])
    time.sleep(0.01)
    jid = s.submit(JOB["Lx"], JOB["Ly"], n_mcs=JOB["n_mcs"], hist_every=JOB["hist_every"],
                   keep_lattice=True, n_A=JOB["n_A"], omega_over_kT=JOB["omega_over_kT"], seed=JOB["seed"])
    for k, job in enumerate(others[6:], start=6):
        time.sleep(rng.uniform(0, 0.01))
        ids[k] = s.submit(job["Lx"], job["Ly"], n_mcs=job["n_mcs"], hist_every=job["hist_every"],
                          keep_lattice=True, n_A=job["n_A"], omega_over_kT=job["omega_over_kT"],
                          seed=job["seed"], geometry=job["geometry"])
    s.drain(300)
    st = s.stats()
    assert st["finished"] == st["submitted"] == 15 and st["rounds"] > 1
    mixed = (s.poll(jid), s.lattice(jid, JOB["Lx"] * JOB["Ly"]), s.histogram(jid))
    same(alone, mixed)
    # Every other job equals the plain single-lattice path; small ones also the oracle.
    for k, job in enumerate(others):
        r = s.poll(ids[k])
        assert r["status"] == 0
        lat = klmc.Lattice(job["Lx"], job["Ly"], n_A=job["n_A"], omega_over_kT=job["omega_over_kT"],
                           seed=job["seed"], geometry=job["geometry"])
        lat.sweep(job["n_mcs"])
        assert np.array_equal(s.lattice(ids[k], job["Lx"] * job["Ly"]), lat.get_lattice())
        c = lat.counters()
        assert (r["attempts"], r["unlike"], r["draws"], r["accepts"]) == (
            c["attempts"], c["unlike"], c["draws"], c["accepts"])
        assert r["n_unlike"] == lat.energy()[0]
        if job["hist_every"]:
            hs, hc = s.histogram(ids[k])
            ls, lc = lat.cluster_histogram(1)
            assert np.array_equal(hs, ls) and np.array_equal(hc, lc)
        if job["Lx"] <= 64 and job["n_mcs"] <= 300:
            ref = oracle.run(job["Lx"], job["Ly"], job["geometry"], job["omega_over_kT"], job["seed"],
                             oracle.init(job["Lx"], job["Ly"], job["n_A"], job["seed"]), 0, job["n_mcs"])
            assert np.array_equal(s.lattice(ids[k], job["Lx"] * job["Ly"]), ref.lattice)
        assert r["submit_s"] <= r["start_s"] <= r["finish_s"]
    s.close()


def test_admission_by_memory_budget():
    # A budget that holds two 400x400 bit-packed jobs (25.6 KB of lattice plus a few KB
    # of state each) but not three: the rest queue and are admitted as earlier ones
    # retire; resident memory never exceeds the budget.
    budget = 70000
    s = klmc.Server(budget)
    ids = [s.submit(400, 400, n_mcs=200, n_A=48000, omega_over_kT=0.5, seed=i) for i in range(6)]
    s.drain(300)
    st = s.stats()
    assert st["finished"] == 6 and st["peak_device_bytes"] <= budget
    starts = sorted(s.poll(i)["start_s"] for i in ids)
    finishes = sorted(s.poll(i)["finish_s"] for i in ids)
    assert starts[2] >= finishes[0]  # the third job waited for memory
    s.close()


def test_oversized_job_does_not_block():
    s = klmc.Server(200000)
    big = s.submit(2048, 2048, n_mcs=10, n_A=1000, seed=1)
    small = s.submit(32, 32, n_mcs=10, n_A=300, seed=2)
    s.drain(60)
    assert s.poll(big)["status"] == 1  # KLMC_EINVAL: never fits the budget
    assert s.poll(small)["status"] == 0
    s.close()


def test_drain_timeout_and_poll_busy():
    s = klmc.Server(1 << 30)
    jid = s.submit(400, 400, n_mcs=4000, n_A=48000, omega_over_kT=0.6, seed=3)
    with pytest.raises(klmc.KlmcError) as e:
        s.drain(0.0)
    assert e.value.status == 4  # KLMC_ETIMEOUT
    assert s.poll(jid) is None or s.poll(jid)["status"] == 0
    s.drain(300)
    assert s.poll(jid)["n_mcs"] == 4000
    s.close()

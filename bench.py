#!/usr/bin/env python3
"""Throughput benchmark of the Kawasaki lattice Monte Carlo hot path.

Workload (the paper's 400x400 lattice size, section "Cluster Analysis"): five
separate runs of a 400x400 periodic triangular lattice with 30 % A / 70 % B
placed at random, omega/kT in {0.2, 0.4, 0.6, 0.8, 1.0} (seeds 2..6), 20000
Monte Carlo steps each, the A-cluster size histogram every 500 steps, lattice
stored at 1 bit per site.  Inputs are synthetic, seeded random lattices.

One benchmark step = the whole workload: load the five initial lattices, run
20000 steps of each with the 40 histograms each.  Metric: Kawasaki exchange
attempts per second (attempts are counted exactly by the kernels).

Forms: "batched" (one resident-kernel launch advances all five lattices, one
thread-block cluster of 16 CTAs each; this is ``value``) and "plain" (one launch per lattice, issued in
turn).  ``e2e`` is the batched form through the public API with the initial
lattices copied from pinned host memory and all histograms, lattices and
energies copied back, inside the timed region.

``--impl reference`` times the CPU oracle (the plain sequential C program in
oracle/) on a bounded sample of the same workload on the host cores.

Multi-GPU (torchrun): every rank runs its own independent copy of the workload
(seeds offset by rank), no collective on the data path; weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L = 400
FRACTION_A = 0.3
OMEGAS = [0.2, 0.4, 0.6, 0.8, 1.0]
SEEDS = [2, 3, 4, 5, 6]
N_MCS = 20000
HIST_EVERY = 500
WORKLOAD = ("400x400 TRI6 periodic, 30% A random start, omega/kT in {0.2,0.4,0.6,0.8,1.0} "
            "(5 separate runs, seeds 2..6), 20000 MCS each, A-cluster histogram every 500 MCS, "
            "1 bit/site")

# Operation model of the sweep kernel (lane-instructions per attempt), used for
# the ALU roofline: C_PAIR is the bit-sliced neighbour evaluation of one
# anchor word (windows, comparisons, adder tree, masks) divided by the anchors
# per word, averaged over the three orientations; C_PHILOX is one Philox4x32-10
# evaluation (10 rounds x (2 IMAD.WIDE + 2 LOP3)), paid only by drawn attempts.
C_PAIR = 4.8
C_PHILOX = 40.0
# INT32 lanes per SM per clock: 4 sub-partitions x 16, the documented 32-bit
# integer and logical-operation rate of 64 results per clock per SM; a throughput
# probe on GB300 measured 60 LOP3 and 30 IMAD.WIDE (+30 LOP3) lane-ops/clk/SM.
INT32_LANES_PER_SM = 64
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture
# each (one resident-sweep launch of 500 MCS of the 400x400 x 5 workload; one
# 4-phase band launch of the 8192x8192 lattice), valid only for the kernel sources
# they were taken with (hash of sweep_resident.cu + sweep_common.cuh).
TRAFFIC_C2_LAUNCH = 306432
TRAFFIC_C3_LAUNCH = 8498432
TRAFFIC_SOURCES = "1553ba35071005ba"



def resident_sources_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ("sweep_resident.cu", "sweep_common.cuh"):
        with open(os.path.join(ROOT, "paper_1309_4349_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# Kernels launched per library call (fixed by the library's structure).
LAUNCHES_SWEEP = 1
LAUNCHES_HISTOGRAM = 5
LAUNCHES_SET_LATTICE_DEVICE = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mcs", type=int, default=N_MCS, help="steps per run (default: the workload's)")
    ap.add_argument("--workload", choices=["c2", "c1", "c3", "c4", "c5", "c6"], default="c2",
                    help="c2 (default): 400x400 x 5 omega; c1: 64x64; c3: 8192x8192; c4: 256 replicas; "
                         "c5: serving; c6: helical 402x399 x 5 omega, seven-colour schedule")
    ap.add_argument("--jobs", type=int, default=300, help="c5: number of jobs")
    ap.add_argument("--rate", type=float, default=0.0, help="c5: arrivals per second (0: 0.8 load)")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_seeds(rank):
    """Seeds of one rank's copy of the workload: every rank runs independent
    Markov chains (replicas only; no collective on the data path)."""
    return [s + 1000 * rank for s in SEEDS]


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (x itself without a process group)."""
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def gpu_smi_id(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def oracle_sample(n_mcs: int, threads: int):
    """The oracle on a bounded sample: each of the five runs for n_mcs steps plus
    one cluster histogram, one host thread per run (ctypes releases the GIL)."""
    import numpy as np  # noqa: F401

    import oracle

    oracle.build()
    inits = [oracle.init(L, L, oracle.n_A(L, L, -1, FRACTION_A), s) for s in SEEDS]
    res = [None] * len(SEEDS)

    def work(i):
        r = oracle.run(L, L, oracle.TRI6, OMEGAS[i], SEEDS[i], inits[i], 0, n_mcs)
        oracle.cluster_histogram(L, L, oracle.TRI6, r.lattice, 1)
        res[i] = r.attempts

    t0 = time.perf_counter()
    ths = [threading.Thread(target=work, args=(i,)) for i in range(len(SEEDS))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    return sum(res), dt


def run_reference(args, rank, world=1):
    """The oracle timed on the host's cores; under torchrun rank 0 alone runs it."""
    if rank != 0:
        return
    n_mcs = 60
    for _ in range(args.warmup):
        oracle_sample(n_mcs, len(SEEDS))
    att, tot = 0, 0.0
    for _ in range(args.steps):
        a, dt = oracle_sample(n_mcs, len(SEEDS))
        att += a
        tot += dt
    value = att / tot
    sample = (f"{n_mcs} MCS of each of the 5 runs plus one A-cluster histogram each, per step; "
              f"one host thread per run")
    line = {
        "impl": "reference", "metric": "Kawasaki exchange attempts/s", "value": value,
        "unit": "attempts/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "oracle (plain sequential C, CPU)",
                   "ranks": "rank 0 only" if world > 1 else "single process"},
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": len(SEEDS),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Other workloads (the default line is the 400x400 x 5 omega workload).
# ---------------------------------------------------------------------------
C1 = dict(L=64, n_A=2048, omega=0.6, seed=1, mcs=1000, hist_every=100)
C3 = dict(L=8192, omega=0.85, seed=7, mcs=1000, trace_every=10)
# Helical triangular lattice with the seven-colour MPKK schedule: the nearest size to
# 400 x 400 that seven-site domains tile (7 | 402*399, 402 mod 7 = 3), the 400x400
# workload's composition, omegas and seeds, 2000 MCS (bounded run), histograms every 500.
C6 = dict(Lx=402, Ly=399, mcs=2000, hist_every=500)
C4 = dict(n=256, L_min=100, L_max=1024, f_min=0.1, f_max=0.5, w_min=0.1, w_max=1.2, mcs=5000,
          seed0=1000, draw_seed=20260)
C5 = dict(L_min=64, L_max=2048, f_min=0.1, f_max=0.5, w_min=0.1, w_max=1.2, mcs_min=1e3, mcs_max=1e5,
          seed0=1000000, draw_seed=77, budget=16 << 30)


def c5_jobs(n):
    """Serving jobs: side log-uniform over [64, 2048], A fraction U[0.1, 0.5],
    omega/kT U[0.1, 1.2], steps log-uniform over [1e3, 1e5], seed 10^6 + j."""
    import numpy as np

    rng = np.random.default_rng(C5["draw_seed"])
    jobs = []
    for j in range(n):
        L = int(round(float(np.exp(rng.uniform(np.log(C5["L_min"]), np.log(C5["L_max"]))))))
        mcs = int(round(float(np.exp(rng.uniform(np.log(C5["mcs_min"]), np.log(C5["mcs_max"]))))))
        jobs.append(dict(L=L, fraction_A=float(rng.uniform(C5["f_min"], C5["f_max"])),
                         omega_over_kT=float(rng.uniform(C5["w_min"], C5["w_max"])), n_mcs=mcs,
                         seed=C5["seed0"] + j))
    return jobs


def bench_serving(args, klmc, np):
    """Poisson arrivals submitted in real time from a host thread; every job is
    admitted by memory, kept resident and batched with the others in rounds."""
    jobs = c5_jobs(args.jobs)
    mean_attempts = float(np.mean([j["L"] ** 2 * j["n_mcs"] for j in jobs]))
    rate = args.rate if args.rate > 0 else 0.8 * 1.5e11 / mean_attempts
    rng = np.random.default_rng(C5["draw_seed"] + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(jobs)))
    srv = klmc.Server(C5["budget"])
    ids = [None] * len(jobs)
    t0 = time.perf_counter()
    for k, (j, t) in enumerate(zip(jobs, arrivals)):
        wait = t - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids[k] = srv.submit(j["L"], j["L"], n_mcs=j["n_mcs"], fraction_A=j["fraction_A"],
                            omega_over_kT=j["omega_over_kT"], seed=j["seed"])
    srv.drain(24 * 3600)
    makespan = time.perf_counter() - t0
    res = [srv.poll(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    lat = np.array([r["finish_s"] - r["submit_s"] for r in res])
    wait = np.array([r["start_s"] - r["submit_s"] for r in res])
    attempts = sum(r["attempts"] for r in res)
    return {
        "metric": "Kawasaki exchange attempts/s", "value": attempts / makespan, "unit": "attempts/s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": makespan * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"serving: Poisson arrivals of {len(jobs)} jobs (the configuration's "
                               "10000 reduced to bound the run), side log-uniform 64-2048, A fraction "
                               "U[0.1,0.5], omega/kT U[0.1,1.2], MCS log-uniform 1e3-1e5, seeds 1e6+j",
                   "arrival_rate_per_s": rate, "offered_load_attempts_per_s": rate * mean_attempts,
                   "device_budget_bytes": C5["budget"],
                   "form": "job server: memory admission, resident lattices, rounds over all resident jobs"},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
        "server": {k: st[k] for k in ("rounds", "busy_s", "uptime_s", "peak_device_bytes")},
        "jobs": len(jobs), "attempts": attempts,
    }


def c4_replicas():
    """256 replicas: side log-uniform over [100, 1024], A fraction uniform over
    [0.1, 0.5], omega/kT uniform over [0.1, 1.2], seed 1000 + r (drawn from a fixed
    numpy generator so every run uses the same set)."""
    import numpy as np

    rng = np.random.default_rng(C4["draw_seed"])
    out = []
    for r in range(C4["n"]):
        L = int(round(float(np.exp(rng.uniform(np.log(C4["L_min"]), np.log(C4["L_max"]))))))
        out.append(dict(Lx=L, Ly=L, fraction_A=float(rng.uniform(C4["f_min"], C4["f_max"])),
                        omega_over_kT=float(rng.uniform(C4["w_min"], C4["w_max"])),
                        seed=C4["seed0"] + r))
    return out


def _time_steps(torch, stream, flush, step, K, W):
    for _ in range(W):
        step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(K):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def _roofline(kernel, launch_ms, attempts_launch, p_draw, sm_count, sm_mhz, ctas, extra=None):
    ops_attempt = C_PAIR + p_draw * C_PHILOX
    peak = sm_count * INT32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = ops_attempt * attempts_launch / (launch_ms * 1e-3) / 1e12
    d = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
         "unit": "Tops/s (INT32 lane-ops)", "frac": achieved / peak, "traffic": None,
         "ops_per_attempt": ops_attempt, "p_draw": p_draw, "launch_ms": launch_ms,
         "attempts_per_launch": attempts_launch, "ctas_per_launch": ctas,
         "peak_basis": (f"{sm_count} SMs x {INT32_LANES_PER_SM} INT32 lanes/clk x median SM clock "
                        f"{sm_mhz:.0f} MHz (64 INT32 lanes: documented rate, confirmed by a throughput probe)")}
    d.update(extra or {})
    return d


def bench_other(args, klmc, torch, np):
    local = int(os.environ.get("LOCAL_RANK", "0"))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = ClockSampler(gpu_smi_id(torch, local))
    line = {"metric": "Kawasaki exchange attempts/s", "unit": "attempts/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic"}
    if args.workload == "c1":
        c = C1
        lat = klmc.Lattice(c["L"], c["L"], n_A=c["n_A"], omega_over_kT=c["omega"], seed=c["seed"],
                           packing=klmc.PACK_BYTE)
        lat.autotune(16)
        init = torch.from_numpy(lat.get_lattice()).cuda()
        nseg = c["mcs"] // c["hist_every"]
        cap = int(np.sqrt(2.0 * lat.N)) + 2
        sz = torch.zeros((nseg, cap), dtype=torch.int64, device="cuda")
        ct = torch.zeros_like(sz)
        nd = torch.zeros(nseg, dtype=torch.int64, device="cuda")
        sweep_ev = []

        def step(record=False):
            lat.set_lattice_device(init, 0)
            for k in range(nseg):
                if record:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                lat.sweep(c["hist_every"])
                if record:
                    e1.record(stream)
                    sweep_ev.append((e0, e1))
                lat.cluster_histogram_device(1, sz[k], ct[k], nd[k:k + 1])

        clocks.start()
        ms = _time_steps(torch, stream, flush, lambda: step(True), args.steps, args.warmup)
        clk = clocks.stop()
        cnt = lat.counters()
        attempts = cnt["attempts"]
        ms_step = sum(ms) / len(ms)
        tail = sweep_ev[-nseg * args.steps:]
        launch_ms = sum(a.elapsed_time(b) for a, b in tail) / len(tail)
        C, T = lat.launch_shape()
        line.update({"value": attempts / (ms_step * 1e-3), "ms_per_step": ms_step,
                     "config": {"workload": "64x64 TRI6 periodic, 2048 A + 2048 B random start, "
                                "omega/kT 0.6, int8 (1 byte/site) store, 1000 MCS, A-cluster "
                                "histogram every 100 MCS", "form": "plain (one lattice)",
                                "l2": "flushed between steps"},
                     "us_per_mcs": ms_step * 1e3 / c["mcs"],
                     "roofline": _roofline("resident_sweep_kernel", launch_ms,
                                           attempts // nseg, cnt["draws"] / attempts, sm_count,
                                           clk["sm_mhz"] if clk else 2070.0, C,
                                           {"cluster": C, "threads_per_cta": T}),
                     "clocks": clk, "gpu_launches": args.steps * (3 + nseg * (1 + LAUNCHES_HISTOGRAM))})
    elif args.workload == "c3":
        c = C3
        line["variants"] = {}
        for geom, name in ((klmc.TRI6, "TRI6"), (klmc.SQ4, "SQ4")):
            L = c["L"]
            lat = klmc.Lattice(L, L, n_A=L * L // 2, omega_over_kT=c["omega"], seed=c["seed"],
                               geometry=geom)
            init = torch.from_numpy(lat.get_lattice()).cuda()
            trace = torch.zeros(c["mcs"] // c["trace_every"], dtype=torch.int64, device="cuda")

            def step():
                lat.set_lattice_device(init, 0)
                lat.sweep_traced(c["mcs"], c["trace_every"], out=trace)

            clocks.start()
            ms = _time_steps(torch, stream, flush, step, args.steps, args.warmup)
            clk = clocks.stop()
            cnt = lat.counters()
            ms_step = sum(ms) / len(ms)
            attempts = cnt["attempts"]
            K = lat.plan()  # phases per launch
            launches = 8 * c["mcs"] // K
            launch_ms = ms_step / launches  # graph gaps included
            rl = _roofline("band_phases_kernel" if K > 1 else "tiled_phase_kernel", launch_ms,
                           attempts // launches, cnt["draws"] / attempts, sm_count,
                           clk["sm_mhz"] if clk else 2070.0, -1,
                           {"note": "per-launch time = step time / sweep launches (graph replays)",
                            "phases_per_launch": K,
                            "traffic": (TRAFFIC_C3_LAUNCH if resident_sources_hash() == TRAFFIC_SOURCES
                                        and geom == klmc.TRI6 else None),
                            "traffic_note": "DRAM bytes per launch from one ncu capture (TRI6); the "
                                            "8 MiB lattice and its second buffer stay in L2"})
            v = {"value": attempts / (ms_step * 1e-3), "ms_per_step": ms_step, "roofline": rl,
                 "clocks": clk, "final_n_unlike": int(trace[-1].item())}
            if geom == klmc.TRI6:
                # Fraction of first neighbours of the final lattice: the random-neighbour
                # estimator over all 2^26 sites, 20 samples timed with CUDA events.
                cnt_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
                for m in range(3):
                    lat.ffn_device(m, cnt_dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for m in range(20):
                    lat.ffn_device(100 + m, cnt_dev)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_ffn = e0.elapsed_time(e1) / 20
                n_sites = L * L
                lat_bytes = n_sites // 8
                # Snapshot image at a quarter of the natural width (geometry kept, 4 x 4
                # supersampling) and its fraction of first neighbours.
                U = 2 * L + L - 1
                Wi = U // 4
                Hi = int(round(Wi * L * (3 ** 0.5 / 2) / (U / 2)))
                img, msk = lat.snapshot(Wi, Hi, 4)
                lat.image_ffn(img, msk, 35, 0)
                e2, e3, e4 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e2.record(stream)
                for _ in range(5):
                    lat.snapshot(Wi, Hi, 4)
                e3.record(stream)
                torch.cuda.synchronize()
                t_img = []
                for m in range(5):
                    t0 = time.perf_counter()
                    lat.image_ffn(img, msk, 35, m)
                    t_img.append(time.perf_counter() - t0)
                e4.record(stream)
                torch.cuda.synchronize()
                ms_snap = e2.elapsed_time(e3) / 5
                v["images"] = {"kernels": ["snapshot_kernel", "image_ffn_kernel"], "W": Wi, "H": Hi, "S": 4,
                               "snapshot_ms": ms_snap, "snapshot_pixels_per_s": Wi * Hi / (ms_snap * 1e-3),
                               "image_ffn_ms_host": 1e3 * min(t_img),
                               "note": "snapshot timed with CUDA events; image fraction of first neighbours "
                                       "timed on the host around its synchronising call"}
                v["ffn"] = {"kernel": "ffn_kernel", "ms_per_sample": ms_ffn,
                            "sites_per_s": n_sites / (ms_ffn * 1e-3),
                            "algorithmic_bytes": lat_bytes,
                            "achieved_gbs": lat_bytes / (ms_ffn * 1e-3) / 1e9,
                            "note": "one read of the 1-bit lattice per sample (the lattice fits L2; "
                                    "neighbour reads hit cache); plus one Philox per 4 sites"}
            line["variants"][name] = v
            if geom == klmc.TRI6:
                line.update({"value": v["value"], "ms_per_step": ms_step, "roofline": rl, "clocks": clk})
            lat.close()
        line["config"] = {"workload": "8192x8192 periodic, 50/50 random start, 1 bit/site, omega/kT "
                          "0.85, 1000 MCS, energy trace every 10 MCS (TRI6; SQ4 in variants)",
                          "form": "tiled path: bands of 54 rows per CTA, 4 phases per launch with "
                                  "9 halo rows per side, launches replayed from a CUDA graph of 10 MCS",
                          "l2": "lattice (8 MiB) fits L2; flushed between steps"}
        line["gpu_launches"] = args.steps * (3 + 8 // K * c["mcs"] + 2 * c["mcs"] // c["trace_every"])
    elif args.workload == "c6":
        c = C6
        Lx, Ly = c["Lx"], c["Ly"]
        streams = [torch.cuda.Stream() for _ in OMEGAS]
        lats = [klmc.Lattice(Lx, Ly, fraction_A=FRACTION_A, omega_over_kT=w, seed=sd, boundary=klmc.HELICAL,
                             stream=st) for w, sd, st in zip(OMEGAS, SEEDS, streams)]
        inits = [torch.from_numpy(l.get_lattice()).cuda() for l in lats]
        nseg = c["mcs"] // c["hist_every"]
        cap = int(np.sqrt(2.0 * Lx * Ly)) + 2
        sz = torch.zeros((len(lats), nseg, cap), dtype=torch.int64, device="cuda")
        ct = torch.zeros_like(sz)
        nd = torch.zeros((len(lats), nseg), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()

        def step():
            fork = torch.cuda.Event()
            fork.record(stream)
            for i, (l, st) in enumerate(zip(lats, streams)):
                st.wait_event(fork)
                l.set_lattice_device(inits[i], 0)
                for k in range(nseg):
                    l.sweep(c["hist_every"])
                    l.cluster_histogram_device(1, sz[i, k], ct[i, k], nd[i, k:k + 1])
            for st in streams:
                done = torch.cuda.Event()
                done.record(st)
                stream.wait_event(done)

        clocks.start()
        ms = _time_steps(torch, stream, flush, step, args.steps, args.warmup)
        clk = clocks.stop()
        cnts = [l.counters() for l in lats]
        attempts = sum(x["attempts"] for x in cnts)
        draws = sum(x["draws"] for x in cnts)
        assert attempts == len(lats) * c["mcs"] * Lx * Ly
        ms_step = sum(ms) / len(ms)
        cpu = None
        if not args.skip_cpu:
            import oracle
            import threading as _th

            oracle.build()
            n_cpu = 60
            oinits = [oracle.init(Lx, Ly, oracle.n_A(Lx, Ly, -1, FRACTION_A), sd) for sd in SEEDS]
            res = [0] * len(SEEDS)

            def work(i):
                r = oracle.run_mpkk(Lx, Ly, OMEGAS[i], SEEDS[i], oinits[i], 0, n_cpu)
                oracle.cluster_histogram(Lx, Ly, oracle.TRI6, r.lattice, 1, oracle.HELICAL)
                res[i] = r.attempts

            t0 = time.perf_counter()
            ths = [_th.Thread(target=work, args=(i,)) for i in range(len(SEEDS))]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
            dt = time.perf_counter() - t0
            cpu = {"value": sum(res) / dt, "unit": "attempts/s", "cores": len(SEEDS), "kind": "oracle",
                   "sample": f"{n_cpu} MCS of each of the 5 runs plus one A-cluster histogram each, one host "
                             f"thread per run; nproc={os.cpu_count()}"}
        line.update({"value": attempts / (ms_step * 1e-3), "ms_per_step": ms_step,
                     "config": {"workload": "helical triangular 402x399 (7 | N, 402 mod 7 = 3), seven-colour "
                                            "MPKK schedule, 30% A random start, omega/kT in "
                                            "{0.2,0.4,0.6,0.8,1.0} (5 runs, seeds 2..6), 2000 MCS each, "
                                            "A-cluster histogram every 500 MCS, 1 bit/site",
                                "form": "one launch per iteration (7 per MCS), a thread per domain centre, "
                                        "graph replays; the 5 lattices on 5 streams",
                                "l2": "flushed between steps"},
                     "roofline": _roofline("mpkk_phase_kernel", ms_step, attempts, draws / attempts, sm_count,
                                           clk["sm_mhz"] if clk else 2070.0, -1,
                                           {"note": "all launches of a step, the 5 lattices' overlapping on 5 "
                                                    "streams: time = step time"}),
                     "cpu_baseline": cpu, "clocks": clk,
                     "gpu_launches": args.steps * len(lats) * (3 + 7 * c["mcs"] + c["mcs"] // 8 +
                                                               nseg * LAUNCHES_HISTOGRAM)})
    elif args.workload == "c4":
        reps = c4_replicas()
        b = klmc.Batch([dict(r, packing=klmc.PACK_BIT) for r in reps])
        inits = [torch.from_numpy(l.get_lattice()).cuda() for l in b.replicas]

        def step():
            for l, t in zip(b.replicas, inits):
                l.set_lattice_device(t, 0)
            b.sweep(C4["mcs"])

        clocks.start()
        ms = _time_steps(torch, stream, flush, step, args.steps, args.warmup)
        clk = clocks.stop()
        cnts = [l.counters() for l in b.replicas]
        attempts = sum(x["attempts"] for x in cnts)
        draws = sum(x["draws"] for x in cnts)
        ms_step = sum(ms) / len(ms)
        groups = {}  # launch shape (CTAs per replica x threads per CTA) the timed calls used
        for i in range(len(reps)):
            C, T = b.launch_shape(i)
            groups[(C, T)] = groups.get((C, T), 0) + 1
        ctas = sum(C * n for (C, _), n in groups.items())
        line.update({"value": attempts / (ms_step * 1e-3), "ms_per_step": ms_step,
                     "config": {"workload": "batched: 256 replicas, side log-uniform 100-1024, A "
                                "fraction U[0.1,0.5], omega/kT U[0.1,1.2], seeds 1000+r, 5000 MCS each",
                                "form": "batched: one launch per launch shape, launches on concurrent "
                                        "streams",
                                "groups": {f"{C}x{T}": v for (C, T), v in sorted(groups.items())},
                                "l2": "flushed between steps"},
                     "roofline": _roofline("resident_sweep_kernel", ms_step, attempts, draws / attempts,
                                           sm_count, clk["sm_mhz"] if clk else 2070.0, ctas,
                                           {"note": "launch time = step time (group launches overlap)"}),
                     "clocks": clk, "gpu_launches": args.steps * (3 * len(reps) + len(groups))})
        if not args.skip_plain:
            sub = list(range(0, len(reps), 16))  # 16 replicas, one launch each, in turn
            def step_plain():
                for i in sub:
                    b.replicas[i].set_lattice_device(inits[i], 0)
                    b.replicas[i].sweep(C4["mcs"])
            msp = _time_steps(torch, stream, flush, step_plain, 1, 1)
            att_sub = sum(b.replicas[i].counters()["attempts"] for i in sub)
            line["forms"] = {"batched": {"value": line["value"]},
                             "plain": {"value": att_sub / (msp[0] * 1e-3),
                                       "sample": f"{len(sub)} of the 256 replicas, one launch each"}}
        b.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    import paper_1309_4349_gb300 as klmc

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    klmc.build()
    if args.workload == "c5":
        if rank == 0:
            print(json.dumps(bench_serving(args, klmc, np)), flush=True)
        return
    if args.workload != "c2":
        if rank == 0:
            bench_other(args, klmc, torch, np)
        return
    n_mcs = args.mcs
    n_seg = n_mcs // HIST_EVERY
    assert n_seg * HIST_EVERY == n_mcs
    seeds = replica_seeds(rank)
    reps = [dict(Lx=L, Ly=L, fraction_A=FRACTION_A, omega_over_kT=w, seed=s,
                 packing=klmc.PACK_BIT) for w, s in zip(OMEGAS, seeds)]
    nrun = len(reps)
    N = L * L
    stream = torch.cuda.current_stream()

    # Tune the launch shape of this lattice size once (cached for the replicas).
    probe = klmc.Lattice(L, L, fraction_A=FRACTION_A, omega_over_kT=OMEGAS[2], seed=99,
                         packing=klmc.PACK_BIT)
    tuned = probe.autotune(64)
    probe.close()
    batch = klmc.Batch(reps)
    init_host = [batch.replicas[i].get_lattice() for i in range(nrun)]
    init_dev = [torch.from_numpy(t).cuda() for t in init_host]
    hcap = int(np.sqrt(2.0 * N)) + 2
    sizes = torch.zeros((n_seg, nrun, hcap), dtype=torch.int64, device="cuda")
    counts = torch.zeros_like(sizes)
    ndist = torch.zeros((n_seg, nrun), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    sweep_events = []

    def histograms(lats, seg):
        for i, lat in enumerate(lats):
            lat.cluster_histogram_device(1, sizes[seg, i], counts[seg, i], ndist[seg, i:i + 1])

    def histograms_batched(seg):  # the replicas' histograms overlap on internal streams
        batch.cluster_histogram_device(1, sizes[seg], counts[seg], ndist[seg])

    def step_batched(record=False):
        for i, lat in enumerate(batch.replicas):
            lat.set_lattice_device(init_dev[i], 0)
        for seg in range(n_seg):
            if record:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            batch.sweep(HIST_EVERY)
            if record:
                e1.record(stream)
                sweep_events.append((e0, e1))
            histograms_batched(seg)

    plain = [batch.replicas[i] for i in range(nrun)]

    def step_plain():
        for i, lat in enumerate(plain):
            lat.set_lattice_device(init_dev[i], 0)
        for seg in range(n_seg):
            for lat in plain:
                lat.sweep(HIST_EVERY)
            histograms(plain, seg)

    def timed(step, K, W, record=False):
        for _ in range(W):
            step()
        torch.cuda.synchronize()
        barrier()
        evs = []
        for _ in range(K):
            flush.zero_()  # L2 (129 MB) flushed between steps, outside the timed events
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            if record:
                step(record=True)
            else:
                step()
            e.record(stream)
            evs.append((s, e))
        torch.cuda.synchronize()
        barrier()
        return [s.elapsed_time(e) for s, e in evs]

    # ---------------- batched (the reported value) ----------------
    clocks = ClockSampler(gpu_smi_id(torch, local))
    clocks.start()
    ms_steps = timed(step_batched, args.steps, args.warmup, record=True)
    clk = clocks.stop()
    ms_step = sum(ms_steps) / len(ms_steps)
    cnt = [lat.counters() for lat in batch.replicas]
    attempts_step = sum(c["attempts"] for c in cnt)
    draws_step = sum(c["draws"] for c in cnt)
    assert attempts_step == nrun * n_mcs * N, attempts_step  # 4 | 400: N attempts per MCS
    ms_step_max = max_over_ranks(ms_step, dist, "cuda")  # device time, max over ranks
    value = world * attempts_step / (ms_step_max * 1e-3)

    sweep_ms = [e0.elapsed_time(e1) for e0, e1 in sweep_events]
    launch_ms = sum(sweep_ms) / len(sweep_ms)
    attempts_launch = nrun * HIST_EVERY * N
    p_draw = draws_step / attempts_step
    ops_attempt = C_PAIR + p_draw * C_PHILOX
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clk["sm_mhz"] if clk else 2070.0
    peak_tops = sm_count * INT32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved_tops = ops_attempt * attempts_launch / (launch_ms * 1e-3) / 1e12
    cluster, threads = batch.replicas[0].launch_shape()
    ctas = nrun * cluster
    roofline = {"bound": "alu", "kernel": "resident_sweep_kernel", "achieved": achieved_tops,
                "peak": peak_tops, "unit": "Tops/s (INT32 lane-ops)", "frac": achieved_tops / peak_tops,
                "traffic": (TRAFFIC_C2_LAUNCH if resident_sources_hash() == TRAFFIC_SOURCES
                            and n_mcs % HIST_EVERY == 0 else None),
                "traffic_note": "DRAM bytes per launch from one ncu capture (cold cache); the "
                                "lattices stay in shared memory within a launch",
                "algorithmic_bytes_per_launch": 2 * nrun * L * ((L + 31) // 32) * 4,
                "ops_per_attempt": ops_attempt, "p_draw": p_draw,
                "launch_ms": launch_ms, "attempts_per_launch": attempts_launch,
                "ctas_per_launch": ctas, "cluster": cluster, "threads_per_cta": threads,
                "sm_count": sm_count,
                "peak_basis": (f"{sm_count} SMs x {INT32_LANES_PER_SM} INT32 lanes/clk x median SM "
                               f"clock {sm_mhz:.0f} MHz (64 INT32 lanes: documented rate, confirmed by a "
                               f"throughput probe)"),
                "frac_of_occupied_sms": achieved_tops / (peak_tops * min(ctas, sm_count) / sm_count),
                "sweep_share_of_step": sum(sweep_ms) / sum(ms_steps),
                "note": "latency-bound: each phase waits for its slowest task (the lane with the most Philox "
                        "draws) and a barrier; the 5 lattices occupy 5 clusters of SMs (ncu: issue "
                        "active 30%, top stall barrier)"}

    # Exactness spot check of the timed state (the parity tests do the full check).
    e_run = [lat.energy()[0] for lat in batch.replicas]
    e_rec = [lat.energy_recount() for lat in batch.replicas]
    assert e_run == e_rec

    # ---------------- plain ----------------
    forms = {"batched": {"value": value, "ms_per_step": ms_step_max, "launches_per_step":
                         n_seg * LAUNCHES_SWEEP}}
    if not args.skip_plain:
        ms_plain = timed(step_plain, 1, 1)
        forms["plain"] = {"value": world * attempts_step / (ms_plain[0] * 1e-3),
                          "ms_per_step": ms_plain[0], "launches_per_step": n_seg * nrun}

    # ---------------- end to end through the public API, host buffers ----------------
    pinned = [torch.from_numpy(t).pin_memory() for t in init_host]
    pinned_np = [p.numpy() for p in pinned]
    out_lat = [np.zeros(N, dtype=np.uint8) for _ in range(nrun)]

    def step_e2e():
        for i, lat in enumerate(batch.replicas):
            lat.set_lattice(pinned_np[i], 0)
        for seg in range(n_seg):
            batch.sweep(HIST_EVERY)
            histograms_batched(seg)
        h = (sizes.cpu(), counts.cpu(), ndist.cpu())
        energies = [lat.energy()[0] for lat in batch.replicas]
        for i, lat in enumerate(batch.replicas):
            out_lat[i][:] = lat.get_lattice()
        return h, energies

    for _ in range(args.warmup):
        step_e2e()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
    h2d = nrun * N
    d2h = sizes.numel() * 8 + counts.numel() * 8 + ndist.numel() * 8 + nrun * N + nrun * 8
    e2e = {"value": world * attempts_step / e2e_s, "unit": "attempts/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3}

    launches_step = (nrun * LAUNCHES_SET_LATTICE_DEVICE + n_seg * LAUNCHES_SWEEP +
                     n_seg * nrun * LAUNCHES_HISTOGRAM)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        n_sample = 300
        att, dt = oracle_sample(n_sample, len(SEEDS))
        cpu = {"value": att / dt, "unit": "attempts/s", "cores": len(SEEDS), "kind": "oracle",
               "sample": f"{n_sample} MCS of each of the 5 runs plus one A-cluster histogram each "
                         f"({att} attempts), one host thread per run; nproc={os.cpu_count()}"}

    line = {
        "metric": "Kawasaki exchange attempts/s", "value": value, "unit": "attempts/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "form": "batched (one resident launch, one thread-block cluster per lattice)",
                   "L": L, "runs": nrun, "mcs": n_mcs, "hist_every": HIST_EVERY,
                   "parallelism": f"replicas x{world}", "tuned_shape": list(tuned),
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "sites_per_s": value,  # one attempt per site per MCS: sites x MCS / s
        "forms": forms,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_step * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

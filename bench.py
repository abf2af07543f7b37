#!/usr/bin/env python3
"""Throughput benchmark of the Kawasaki lattice Monte Carlo hot path.

Headline workload (the paper's 400x400 lattice size, section "Cluster
Analysis"): five separate runs of a 400x400 periodic triangular lattice with
30 % A / 70 % B placed at random, omega/kT in {0.2, 0.4, 0.6, 0.8, 1.0} (seeds
2..6), 20000 Monte Carlo steps each, the A-cluster size histogram every 500
steps, lattice stored at 1 bit per site.  Inputs are synthetic, seeded random
lattices.

One benchmark step = the whole headline workload: load the five initial
lattices, run 20000 steps of each with the 40 histograms each.  Metric: Kawasaki
exchange attempts per second (attempts are counted exactly by the kernels).

Forms: "batched" (one resident-kernel launch advances all five lattices, one
thread-block cluster of 16 CTAs each; this is ``value``) and "plain" (one launch
per lattice, issued in turn).  ``e2e`` is the batched form through the public
API with the initial lattices copied from pinned host memory and all histograms,
lattices and energies copied back, inside the timed region.

The same JSON line carries, under ``workloads``, every other workload measured
in the same run, each with its ALU-roofline and L2-bandwidth fractions and the
oracle's 1-core and all-core rates: the 64x64 byte-store run (c1), the
8192x8192 lattice on the tiled path in both geometries (c3), 256 batched
replicas of uneven sizes against plain launches (c4), the job server under
Poisson arrivals with p50/p99 latency (c5), and the helical lattice with the
paper's seven-colour schedule (c6).  ``--workload cX`` prints one of them as its
own line; ``--headline-only`` skips them.

``--impl reference`` times the CPU oracle (the plain sequential C program in
oracle/) on a bounded sample of the headline workload on the host cores.

Multi-GPU (torchrun): every rank runs its own independent copy of the headline
workload (seeds offset by rank), no collective on the data path; weak scaling.
"""
from __future__ import annotations

import argparse
import concurrent.futures
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
# Issue slots per SM per clock (4 schedulers x 32 lanes): the bound on any
# instruction mix, given beside the INT32 figure.
ISSUE_LANES_PER_SM = 128
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture
# each (one resident-sweep launch of 500 MCS of the 400x400 x 5 workload; one
# 4-phase band launch of the 8192x8192 lattice; one resident helical launch of 500
# MCS of one 402x399 lattice), valid only for the kernel sources they were taken
# with (hash of the kernel's file + sweep_common.cuh + philox.cuh).
TRAFFIC_C2_LAUNCH = 211200
TRAFFIC_C3_LAUNCH = 8500480
TRAFFIC_SOURCES = "fabfcfe5f46002be"
TRAFFIC_C6_LAUNCH = 90624
TRAFFIC_HELICAL_SOURCES = "4e4cb06710757526"

# Kernels launched per library call (fixed by the library's structure).
LAUNCHES_SWEEP = 1
LAUNCHES_HISTOGRAM = 5
LAUNCHES_SET_LATTICE_DEVICE = 3

# The other workloads.
C1 = dict(L=64, n_A=2048, omega=0.6, seed=1, mcs=1000, hist_every=100)
C3 = dict(L=8192, omega=0.85, seed=7, mcs=1000, trace_every=10)
C4 = dict(n=256, L_min=100, L_max=1024, f_min=0.1, f_max=0.5, w_min=0.1, w_max=1.2, mcs=5000,
          seed0=1000, draw_seed=20260)
# Serving: the arrival rate offers 0.8 of the server's measured capacity on this
# job mix (C5_CAPACITY attempts/s: the first 1000 jobs of the stream submitted at
# once, `--workload c5 --rate 1000000`, served at 2.41e11 attempts/s on GB300);
# the configuration's 10000 jobs take about 10000 x 1.3e10 / (0.8 x C5_CAPACITY)
# seconds (about 12 minutes) to arrive, and the default run serves all of them
# (--c5-jobs N for the first N of the stream).
C5 = dict(L_min=64, L_max=2048, f_min=0.1, f_max=0.5, w_min=0.1, w_max=1.2, mcs_min=1e3, mcs_max=1e5,
          seed0=1000000, draw_seed=77, budget=16 << 30)
C5_CAPACITY = 2.4e11
C5_JOBS = 10000
# Helical triangular lattice with the seven-colour MPKK schedule: the nearest size to
# 400 x 400 that seven-site domains tile (7 | 402*399, 402 mod 7 = 3), the 400x400
# workload's composition, omegas and seeds, 2000 MCS (bounded run), histograms every 500.
C6 = dict(Lx=402, Ly=399, mcs=2000, hist_every=500)
# Sub-workload timing: warm-up and timed steps (the headline uses --steps/--warmup).
SUB_WARMUP = 3
SUB_STEPS = 3


def resident_sources_hash(kernel_file: str = "sweep_resident.cu") -> str:
    import hashlib

    h = hashlib.sha256()
    for f in (kernel_file, "sweep_common.cuh", "philox.cuh"):
        with open(os.path.join(ROOT, "paper_1309_4349_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mcs", type=int, default=N_MCS, help="steps per run (default: the workload's)")
    ap.add_argument("--workload", choices=["c2", "c1", "c3", "c4", "c5", "c6"], default="c2",
                    help="c2 (default, with every other workload under 'workloads'): 400x400 x 5 omega; "
                         "c1: 64x64; c3: 8192x8192; c4: 256 replicas; c5: serving; c6: helical 402x399")
    ap.add_argument("--headline-only", action="store_true", help="c2 without the other workloads")
    ap.add_argument("--c5-jobs", "--jobs", dest="jobs", type=int, default=C5_JOBS,
                    help="c5: number of jobs of the arrival stream to serve")
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
        self.lines = []
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


# ---------------------------------------------------------------------------
# The oracle (plain sequential C) on the host cores: the CPU baseline.
# ---------------------------------------------------------------------------
def _run_tasks(tasks, threads):
    """Runs callables that return attempt counts on `threads` host threads
    (ctypes releases the GIL); returns (attempts, seconds)."""
    t0 = time.perf_counter()
    if threads <= 1:
        att = sum(t() for t in tasks)
    else:
        with concurrent.futures.ThreadPoolExecutor(max_workers=threads) as ex:
            att = sum(ex.map(lambda t: t(), tasks))
    return att, time.perf_counter() - t0


def cpu_baseline(all_tasks, one_core_tasks, sample_all, sample_one):
    """The oracle's all-core rate (one host thread per independent run, at most
    nproc threads) and its 1-core rate (a subset on one thread)."""
    import oracle

    oracle.build()
    nproc = os.cpu_count() or 1
    threads = min(len(all_tasks), nproc)
    att, dt = _run_tasks(all_tasks, threads)
    att1, dt1 = _run_tasks(one_core_tasks, 1)
    return {"value": att / dt, "unit": "attempts/s", "cores": threads, "kind": "oracle",
            "sample": f"{sample_all}; {threads} host threads, one per run; nproc={nproc}",
            "one_core": {"value": att1 / dt1, "unit": "attempts/s", "cores": 1, "sample": sample_one}}


def c2_oracle_tasks(n_mcs, runs=None):
    import oracle

    def task(i):
        def f():
            t0 = oracle.init(L, L, oracle.n_A(L, L, -1, FRACTION_A), SEEDS[i])
            r = oracle.run(L, L, oracle.TRI6, OMEGAS[i], SEEDS[i], t0, 0, n_mcs)
            oracle.cluster_histogram(L, L, oracle.TRI6, r.lattice, 1)
            return r.attempts
        return f

    return [task(i) for i in (runs if runs is not None else range(len(SEEDS)))]


def oracle_sample(n_mcs: int, threads: int):
    """The oracle on a bounded sample of the headline workload: each of the five
    runs for n_mcs steps plus one cluster histogram, one host thread per run."""
    import oracle

    oracle.build()
    return _run_tasks(c2_oracle_tasks(n_mcs), threads)


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
# Workload generators.
# ---------------------------------------------------------------------------
def c4_replicas():
    """256 replicas: side log-uniform over [100, 1024], A fraction uniform over
    [0.1, 0.5], omega/kT uniform over [0.1, 1.2], seed 1000 + r (drawn from a fixed
    numpy generator so every run uses the same set)."""
    import numpy as np

    rng = np.random.default_rng(C4["draw_seed"])
    out = []
    for r in range(C4["n"]):
        L_ = int(round(float(np.exp(rng.uniform(np.log(C4["L_min"]), np.log(C4["L_max"]))))))
        out.append(dict(Lx=L_, Ly=L_, fraction_A=float(rng.uniform(C4["f_min"], C4["f_max"])),
                        omega_over_kT=float(rng.uniform(C4["w_min"], C4["w_max"])),
                        seed=C4["seed0"] + r))
    return out


def c5_jobs(n):
    """Serving jobs: side log-uniform over [64, 2048], A fraction U[0.1, 0.5],
    omega/kT U[0.1, 1.2], steps log-uniform over [1e3, 1e5], seed 10^6 + j."""
    import numpy as np

    rng = np.random.default_rng(C5["draw_seed"])
    jobs = []
    for j in range(n):
        L_ = int(round(float(np.exp(rng.uniform(np.log(C5["L_min"]), np.log(C5["L_max"]))))))
        mcs = int(round(float(np.exp(rng.uniform(np.log(C5["mcs_min"]), np.log(C5["mcs_max"]))))))
        jobs.append(dict(L=L_, fraction_A=float(rng.uniform(C5["f_min"], C5["f_max"])),
                         omega_over_kT=float(rng.uniform(C5["w_min"], C5["w_max"])), n_mcs=mcs,
                         seed=C5["seed0"] + j))
    return jobs


# ---------------------------------------------------------------------------
# Timing and roofline helpers.
# ---------------------------------------------------------------------------
def _time_steps(torch, stream, flush, step, K, W):
    for _ in range(W):
        step()
    torch.cuda.synchronize()
    evs = []
    for _ in range(K):
        flush.zero_()  # L2 (129 MB) flushed between steps, outside the timed events
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def measure_l2_peak(torch):
    """Measured L2 copy bandwidth (read + write bytes per second): a 16 MiB buffer
    copied into another (32 MiB in all, resident in the 129 MB L2) 200 times per
    trial, best of 5 trials, CUDA events on the current stream."""
    n = 16 << 20
    a = torch.empty(n, dtype=torch.uint8, device="cuda")
    b = torch.empty(n, dtype=torch.uint8, device="cuda")
    a.fill_(1)
    stream = torch.cuda.current_stream()
    best = 0.0
    for trial in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(200):
            b.copy_(a)
        e1.record(stream)
        torch.cuda.synchronize()
        if trial > 0:  # the first trial warms up
            best = max(best, 2 * n * 200 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return {"gbs": best, "how": "torch copy of a 16 MiB buffer into another (L2-resident), 200 per trial, "
                                "best of 5, read + write bytes"}


def _roofline(kernel, launch_ms, attempts_launch, p_draw, sm_count, sm_mhz, ctas, l2_bytes=None,
              l2_peak=None, extra=None):
    """ALU roofline of one launch: the operation model's lane-ops over its time
    against 64 INT32 lanes per SM per clock (the 128-lane issue figure beside
    it), and the L2-bandwidth fraction of the launch's algorithmic L2 bytes."""
    ops_attempt = C_PAIR + p_draw * C_PHILOX
    peak = sm_count * INT32_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = ops_attempt * attempts_launch / (launch_ms * 1e-3) / 1e12
    d = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
         "unit": "Tops/s (INT32 lane-ops)", "frac": achieved / peak, "traffic": None,
         "frac_of_issue_peak": achieved / (peak * ISSUE_LANES_PER_SM / INT32_LANES_PER_SM),
         "ops_per_attempt": ops_attempt, "p_draw": p_draw, "launch_ms": launch_ms,
         "attempts_per_launch": attempts_launch, "ctas_per_launch": ctas,
         "peak_basis": (f"{sm_count} SMs x {INT32_LANES_PER_SM} INT32 lanes/clk x median SM clock "
                        f"{sm_mhz:.0f} MHz (64 INT32 lanes: documented rate, confirmed by a throughput "
                        f"probe; the issue peak is {ISSUE_LANES_PER_SM} lanes/clk)")}
    if l2_bytes is not None and l2_peak:
        gbs = l2_bytes / (launch_ms * 1e-3) / 1e9
        d["l2"] = {"algorithmic_bytes_per_launch": int(l2_bytes), "achieved_gbs": gbs,
                   "peak_gbs": l2_peak, "frac": gbs / l2_peak}
    d.update(extra or {})
    return d


def _sm_mhz(clk):
    return clk["sm_mhz"] if clk else 2070.0


# ---------------------------------------------------------------------------
# The other workloads: each returns its own object (value, roofline, oracle).
# ---------------------------------------------------------------------------
class Ctx:
    """What every sub-workload needs: the modules, the stream, the L2-flush
    buffer, the clock sampler, the SM count, the measured L2 peak."""

    def __init__(self, args, torch, klmc, np, local, l2_peak):
        self.args, self.torch, self.klmc, self.np = args, torch, klmc, np
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        self.sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        self.clocks = ClockSampler(gpu_smi_id(torch, local))
        self.l2_peak = l2_peak

    def timed(self, step, K=SUB_STEPS, W=SUB_WARMUP):
        self.clocks.start()
        ms = _time_steps(self.torch, self.stream, self.flush, step, K, W)
        return ms, self.clocks.stop()


def sub_c1(x):
    torch, klmc, np = x.torch, x.klmc, x.np
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

    def step(record=True):
        lat.set_lattice_device(init, 0)
        for k in range(nseg):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(x.stream)
            lat.sweep(c["hist_every"])
            e1.record(x.stream)
            sweep_ev.append((e0, e1))
            lat.cluster_histogram_device(1, sz[k], ct[k], nd[k:k + 1])

    ms, clk = x.timed(step)
    cnt = lat.counters()
    attempts = cnt["attempts"]
    ms_step = sum(ms) / len(ms)
    tail = sweep_ev[-nseg * len(ms):]
    launch_ms = sum(a.elapsed_time(b) for a, b in tail) / len(tail)
    C, T = lat.launch_shape()
    out = {"value": attempts / (ms_step * 1e-3), "unit": "attempts/s", "ms_per_step": ms_step,
           "config": {"workload": "64x64 TRI6 periodic, 2048 A + 2048 B random start, omega/kT 0.6, "
                                  "int8 (1 byte/site) store, 1000 MCS, A-cluster histogram every 100 MCS",
                      "form": "plain (one lattice, tuned launch shape)", "l2": "flushed between steps"},
           "us_per_mcs": ms_step * 1e3 / c["mcs"],
           "roofline": _roofline("resident_sweep_kernel", launch_ms, attempts // nseg, cnt["draws"] / attempts,
                                 x.sm_count, _sm_mhz(clk), C, 2 * c["L"] * c["L"], x.l2_peak,
                                 {"cluster": C, "threads_per_cta": T,
                                  "note": "one lattice of 4096 sites on one CTA: latency-bound"}),
           "clocks": clk, "gpu_launches": len(ms) * (LAUNCHES_SET_LATTICE_DEVICE +
                                                    nseg * (LAUNCHES_SWEEP + LAUNCHES_HISTOGRAM))}
    lat.close()
    if not x.args.skip_cpu:
        import oracle

        def task():
            t = oracle.init(c["L"], c["L"], c["n_A"], c["seed"])
            att = 0
            for k in range(nseg):
                r = oracle.run(c["L"], c["L"], oracle.TRI6, c["omega"], c["seed"], t, k * c["hist_every"],
                               c["hist_every"])
                oracle.cluster_histogram(c["L"], c["L"], oracle.TRI6, r.lattice, 1)
                t, att = r.lattice, att + r.attempts
            return att

        cb = cpu_baseline([task], [task], "the whole workload (1000 MCS, ten histograms)",
                          "the whole workload on one thread")
        out["cpu_baseline"] = cb
    return out


def sub_c3(x, geom):
    """8192 x 8192 at 1 bit per site on the tiled path (too large for a cluster's
    shared memory): 1000 MCS with the energy trace every 10 MCS."""
    torch, klmc = x.torch, x.klmc
    c = C3
    L_ = c["L"]
    lat = klmc.Lattice(L_, L_, n_A=L_ * L_ // 2, omega_over_kT=c["omega"], seed=c["seed"], geometry=geom)
    init = torch.from_numpy(lat.get_lattice()).cuda()
    trace = torch.zeros(c["mcs"] // c["trace_every"], dtype=torch.int64, device="cuda")

    def step():
        lat.set_lattice_device(init, 0)
        lat.sweep_traced(c["mcs"], c["trace_every"], out=trace)

    ms, clk = x.timed(step)
    cnt = lat.counters()
    ms_step = sum(ms) / len(ms)
    attempts = cnt["attempts"]
    K = lat.plan()  # phases per launch
    launches = 8 * c["mcs"] // K
    launch_ms = ms_step / launches  # graph gaps included
    H = -(-L_ // x.sm_count)  # the plan's band height: one band per SM
    n_bands = -(-L_ // H)
    row_bytes = L_ // 8
    l2_bytes = row_bytes * (L_ + 2 * (2 * K + 1) * n_bands) + row_bytes * L_  # rows with halos in, band out
    out = {"value": attempts / (ms_step * 1e-3), "unit": "attempts/s", "ms_per_step": ms_step,
           "roofline": _roofline("band_phases_kernel" if K > 1 else "tiled_phase_kernel", launch_ms,
                                 attempts // launches, cnt["draws"] / attempts, x.sm_count, _sm_mhz(clk),
                                 n_bands, l2_bytes, x.l2_peak,
                                 {"note": "per-launch time = step time / sweep launches (graph replays); the "
                                          "8 MiB lattice and its second buffer stay in L2",
                                  "phases_per_launch": K, "band_rows": H,
                                  "traffic": (TRAFFIC_C3_LAUNCH if resident_sources_hash() == TRAFFIC_SOURCES
                                              and geom == klmc.TRI6 else None)}),
           "clocks": clk, "final_n_unlike": int(trace[-1].item()),
           "gpu_launches": len(ms) * (LAUNCHES_SET_LATTICE_DEVICE + launches + 2 * c["mcs"] // c["trace_every"])}
    if geom == klmc.TRI6:
        # Fraction of first neighbours of the final lattice (all 2^26 sites) and a
        # snapshot image at a quarter of the natural width with 4 x 4 supersampling.
        cnt_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        for m in range(3):
            lat.ffn_device(m, cnt_dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(x.stream)
        for m in range(20):
            lat.ffn_device(100 + m, cnt_dev)
        e1.record(x.stream)
        torch.cuda.synchronize()
        ms_ffn = e0.elapsed_time(e1) / 20
        U = 3 * L_ - 1
        Wi = U // 4
        Hi = int(round(Wi * L_ * (3 ** 0.5 / 2) / (U / 2)))
        img, msk = lat.snapshot(Wi, Hi, 4)
        lat.image_ffn(img, msk, 35, 0)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(x.stream)
        for _ in range(5):
            lat.snapshot(Wi, Hi, 4)
        e3.record(x.stream)
        torch.cuda.synchronize()
        ms_snap = e2.elapsed_time(e3) / 5
        out["ffn"] = {"kernel": "ffn_kernel", "ms_per_sample": ms_ffn, "sites_per_s": L_ * L_ / (ms_ffn * 1e-3)}
        out["images"] = {"kernel": "snapshot_kernel", "W": Wi, "H": Hi, "S": 4, "snapshot_ms": ms_snap,
                         "pixels_per_s": Wi * Hi / (ms_snap * 1e-3)}
    lat.close()
    if not x.args.skip_cpu:
        import oracle

        def task():
            t = oracle.init(L_, L_, L_ * L_ // 2, c["seed"])
            return oracle.run(L_, L_, geom, c["omega"], c["seed"], t, 0, 1).attempts

        cb = cpu_baseline([task], [task], "1 MCS of the lattice (one sequential run)",
                          "1 MCS of the lattice on one thread")
        cb.pop("one_core")
        cb["note"] = "one lattice: the sequential oracle uses one core"
        out["cpu_baseline"] = cb
    return out


def sub_c4(x):
    """256 replicas of uneven sizes in one batch, 5000 MCS each; plain launches of
    a 16-replica sample for comparison."""
    torch, klmc = x.torch, x.klmc
    reps = c4_replicas()
    b = klmc.Batch([dict(r, packing=klmc.PACK_BIT) for r in reps])
    inits = [torch.from_numpy(l.get_lattice()).cuda() for l in b.replicas]

    def step():
        for l_, t in zip(b.replicas, inits):
            l_.set_lattice_device(t, 0)
        b.sweep(C4["mcs"])

    ms, clk = x.timed(step)
    cnts = [l_.counters() for l_ in b.replicas]
    attempts = sum(c["attempts"] for c in cnts)
    draws = sum(c["draws"] for c in cnts)
    ms_step = sum(ms) / len(ms)
    groups = {}  # launch shape (CTAs per replica x threads per CTA) the timed calls used
    for i in range(len(reps)):
        C, T = b.launch_shape(i)
        groups[(C, T)] = groups.get((C, T), 0) + 1
    ctas = sum(C * n for (C, _), n in groups.items())
    l2_bytes = sum(2 * r["Ly"] * ((r["Lx"] + 31) // 32) * 4 for r in reps)  # each lattice in and out once
    out = {"value": attempts / (ms_step * 1e-3), "unit": "attempts/s", "ms_per_step": ms_step,
           "config": {"workload": "batched: 256 replicas, side log-uniform 100-1024, A fraction U[0.1,0.5], "
                                  "omega/kT U[0.1,1.2], seeds 1000+r, 5000 MCS each",
                      "form": "batched: one launch per launch shape, launches on concurrent streams",
                      "groups": {f"{C}x{T}": v for (C, T), v in sorted(groups.items())},
                      "l2": "flushed between steps"},
           "roofline": _roofline("resident_sweep_kernel", ms_step, attempts, draws / attempts, x.sm_count,
                                 _sm_mhz(clk), ctas, l2_bytes, x.l2_peak,
                                 {"note": "launch time = step time (group launches overlap)"}),
           "clocks": clk, "gpu_launches": len(ms) * (LAUNCHES_SET_LATTICE_DEVICE * len(reps) + len(groups))}
    if not x.args.skip_plain:
        sub = list(range(0, len(reps), 16))  # 16 replicas, one launch each, in turn

        def step_plain():
            for i in sub:
                b.replicas[i].set_lattice_device(inits[i], 0)
                b.replicas[i].sweep(C4["mcs"])

        msp = _time_steps(torch, x.stream, x.flush, step_plain, 1, 1)
        att_sub = sum(b.replicas[i].counters()["attempts"] for i in sub)
        out["forms"] = {"batched": {"value": out["value"]},
                        "plain": {"value": att_sub / (msp[0] * 1e-3),
                                  "sample": f"{len(sub)} of the 256 replicas, one launch each, in turn"}}
    b.close()
    if not x.args.skip_cpu:
        import oracle

        n_cpu = 10

        def task(r):
            def f():
                nA = oracle.n_A(r["Lx"], r["Ly"], -1, r["fraction_A"])
                t = oracle.init(r["Lx"], r["Ly"], nA, r["seed"])
                return oracle.run(r["Lx"], r["Ly"], oracle.TRI6, r["omega_over_kT"], r["seed"], t, 0,
                                  n_cpu).attempts
            return f

        out["cpu_baseline"] = cpu_baseline([task(r) for r in reps], [task(r) for r in reps[::16]],
                                           f"{n_cpu} MCS of each of the 256 replicas",
                                           f"{n_cpu} MCS of 16 of the replicas (every 16th) on one thread")
    return out


def sub_c5(x, n_jobs):
    """Poisson arrivals submitted in real time from a host thread; every job is
    admitted by memory, kept resident and batched with the others in rounds."""
    klmc, np = x.klmc, x.np
    jobs = c5_jobs(n_jobs)
    mean_attempts = float(np.mean([j["L"] ** 2 * j["n_mcs"] for j in jobs]))
    rate = x.args.rate if x.args.rate > 0 else 0.8 * C5_CAPACITY / mean_attempts
    rng = np.random.default_rng(C5["draw_seed"] + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(jobs)))
    srv = klmc.Server(C5["budget"])
    ids = [None] * len(jobs)
    x.clocks.start()
    t0 = time.perf_counter()
    for k, (j, t) in enumerate(zip(jobs, arrivals)):
        wait = t - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ids[k] = srv.submit(j["L"], j["L"], n_mcs=j["n_mcs"], fraction_A=j["fraction_A"],
                            omega_over_kT=j["omega_over_kT"], seed=j["seed"])
    srv.drain(24 * 3600)
    makespan = time.perf_counter() - t0
    clk = x.clocks.stop()
    res = [srv.poll(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    lat = np.array([r["finish_s"] - r["submit_s"] for r in res])
    wait = np.array([r["start_s"] - r["submit_s"] for r in res])
    attempts = sum(r["attempts"] for r in res)
    out = {"value": attempts / makespan, "unit": "attempts/s", "ms_per_step": makespan * 1e3,
           "config": {"workload": ("serving: Poisson arrivals of all 10000 jobs of the " if len(jobs) == 10000 else
                                   f"serving: Poisson arrivals of the first {len(jobs)} jobs of the 10000-job ") +
                                  "stream (side log-uniform 64-2048, A fraction U[0.1,0.5], omega/kT "
                                  "U[0.1,1.2], MCS log-uniform 1e3-1e5, seeds 1e6+j)",
                      "jobs": len(jobs), "arrival_rate_per_s": rate,
                      "offered_load_attempts_per_s": rate * mean_attempts,
                      "offered_load_basis": f"0.8 x {C5_CAPACITY:.2g} attempts/s, the server's measured "
                                            "capacity on this job mix",
                      "device_budget_bytes": C5["budget"],
                      "form": "job server: memory admission, resident lattices, continuous batching in rounds"},
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "mean": float(lat.mean()), "max": float(lat.max())},
           "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
           "server": {k: st[k] for k in ("rounds", "busy_s", "uptime_s", "peak_device_bytes")},
           "attempts": attempts, "clocks": clk}
    if not x.args.skip_cpu:
        import oracle

        sample = jobs[:200]
        n_cpu = 3

        def task(j):
            def f():
                nA = oracle.n_A(j["L"], j["L"], -1, j["fraction_A"])
                t = oracle.init(j["L"], j["L"], nA, j["seed"])
                return oracle.run(j["L"], j["L"], oracle.TRI6, j["omega_over_kT"], j["seed"], t, 0, n_cpu).attempts
            return f

        out["cpu_baseline"] = cpu_baseline([task(j) for j in sample], [task(j) for j in sample[:20]],
                                           f"{n_cpu} MCS of each of the stream's first 200 jobs",
                                           f"{n_cpu} MCS of the first 20 jobs on one thread")
    return out


def sub_c6(x):
    """The helical lattice with the seven-colour schedule: five runs of 402 x 399
    on five streams, 2000 MCS each with the A-cluster histogram every 500."""
    torch, klmc, np = x.torch, x.klmc, x.np
    c = C6
    Lx, Ly = c["Lx"], c["Ly"]
    streams = [torch.cuda.Stream() for _ in OMEGAS]
    lats = [klmc.Lattice(Lx, Ly, fraction_A=FRACTION_A, omega_over_kT=w, seed=sd, boundary=klmc.HELICAL,
                         stream=st) for w, sd, st in zip(OMEGAS, SEEDS, streams)]
    inits = [torch.from_numpy(l_.get_lattice()).cuda() for l_ in lats]
    nseg = c["mcs"] // c["hist_every"]
    cap = int(np.sqrt(2.0 * Lx * Ly)) + 2
    sz = torch.zeros((len(lats), nseg, cap), dtype=torch.int64, device="cuda")
    ct = torch.zeros_like(sz)
    nd = torch.zeros((len(lats), nseg), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()

    def step():
        fork = torch.cuda.Event()
        fork.record(x.stream)
        for i, (l_, st) in enumerate(zip(lats, streams)):
            st.wait_event(fork)
            l_.set_lattice_device(inits[i], 0)
            for k in range(nseg):
                l_.sweep(c["hist_every"])
                l_.cluster_histogram_device(1, sz[i, k], ct[i, k], nd[i, k:k + 1])
        for st in streams:
            done = torch.cuda.Event()
            done.record(st)
            x.stream.wait_event(done)

    ms, clk = x.timed(step)
    cnts = [l_.counters() for l_ in lats]
    attempts = sum(c_["attempts"] for c_ in cnts)
    draws = sum(c_["draws"] for c_ in cnts)
    assert attempts == len(lats) * c["mcs"] * Lx * Ly
    ms_step = sum(ms) / len(ms)
    C, T = lats[0].launch_shape()
    lat_bytes = Ly * ((Lx + 31) // 32) * 4
    resident = C > 0
    out = {"value": attempts / (ms_step * 1e-3), "unit": "attempts/s", "ms_per_step": ms_step,
           "config": {"workload": "helical triangular 402x399 (7 | N, 402 mod 7 = 3), seven-colour MPKK "
                                  "schedule, 30% A random start, omega/kT in {0.2,0.4,0.6,0.8,1.0} (5 runs, "
                                  "seeds 2..6), 2000 MCS each, A-cluster histogram every 500 MCS, 1 bit/site",
                      "form": (f"the 5 lattices on 5 streams, each resident in a {C}-CTA cluster of {T} threads"
                               if resident else "the 5 lattices on 5 streams, one launch per iteration"),
                      "l2": "flushed between steps"},
           "roofline": _roofline("helical_resident_kernel" if resident else "mpkk_phase_kernel", ms_step, attempts,
                                 draws / attempts, x.sm_count, _sm_mhz(clk), len(lats) * max(C, 1),
                                 (2 * len(lats) * nseg * lat_bytes if resident
                                  else 2 * len(lats) * 7 * c["mcs"] * lat_bytes), x.l2_peak,
                                 {"note": "all launches of a step, the 5 lattices' overlapping on 5 streams: "
                                          "time = step time; L2 bytes: each lattice in and out once per "
                                          "resident launch (once per iteration on the per-iteration path)",
                                  "traffic": (len(lats) * nseg * TRAFFIC_C6_LAUNCH if resident and
                                              resident_sources_hash("sweep_helical.cu") == TRAFFIC_HELICAL_SOURCES
                                              and c["hist_every"] == 500 else None),
                                  "traffic_note": "DRAM bytes of the step's 20 resident launches, from one ncu "
                                                  "capture of a 500-MCS launch of one lattice"}),
           "clocks": clk}
    for l_ in lats:
        l_.close()
    if not x.args.skip_cpu:
        import oracle

        n_cpu = 60

        def task(i):
            def f():
                t = oracle.init(Lx, Ly, oracle.n_A(Lx, Ly, -1, FRACTION_A), SEEDS[i])
                r = oracle.run_mpkk(Lx, Ly, OMEGAS[i], SEEDS[i], t, 0, n_cpu)
                oracle.cluster_histogram(Lx, Ly, oracle.TRI6, r.lattice, 1, oracle.HELICAL)
                return r.attempts
            return f

        out["cpu_baseline"] = cpu_baseline([task(i) for i in range(5)], [task(2)],
                                           f"{n_cpu} MCS of each of the 5 runs plus one A-cluster histogram each",
                                           f"{n_cpu} MCS of one run (omega/kT 0.6) on one thread")
    return out


def other_workloads(x):
    """Every workload besides the headline, one object each."""
    klmc = x.klmc
    out = {}
    for name, fn in (("c1", lambda: sub_c1(x)), ("c3_tri6", lambda: sub_c3(x, klmc.TRI6)),
                     ("c3_sq4", lambda: sub_c3(x, klmc.SQ4)), ("c4", lambda: sub_c4(x)),
                     ("c6", lambda: sub_c6(x)), ("c5", lambda: sub_c5(x, x.args.jobs))):
        t0 = time.perf_counter()
        out[name] = fn()
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def single_workload_line(args, x, name):
    """One workload as its own JSON line (--workload cX)."""
    fn = {"c1": lambda: sub_c1(x), "c3": lambda: sub_c3(x, x.klmc.TRI6), "c4": lambda: sub_c4(x),
          "c5": lambda: sub_c5(x, args.jobs), "c6": lambda: sub_c6(x)}[name]
    v = fn()
    line = {"metric": "Kawasaki exchange attempts/s", "value": v.pop("value"), "unit": v.pop("unit"),
            "n_gpus": 1, "steps": SUB_STEPS if name != "c5" else 1, "warmup": SUB_WARMUP if name != "c5" else 0,
            "ms_per_step": v.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic"}
    if name == "c3":
        v["config"] = {"workload": "8192x8192 TRI6 periodic, 50/50 random start, 1 bit/site, omega/kT 0.85, "
                                   "1000 MCS, energy trace every 10 MCS",
                       "form": "tiled path: one band of rows per CTA, 4 phases per launch, graph replays",
                       "l2": "lattice (8 MiB) fits L2; flushed between steps"}
    line.update(v)
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
    l2_peak = measure_l2_peak(torch)
    x = Ctx(args, torch, klmc, np, local, l2_peak["gbs"])
    if args.workload != "c2":
        if rank == 0:
            single_workload_line(args, x, args.workload)
        return
    n_mcs = args.mcs
    n_seg = n_mcs // HIST_EVERY
    assert n_seg * HIST_EVERY == n_mcs
    seeds = replica_seeds(rank)
    reps = [dict(Lx=L, Ly=L, fraction_A=FRACTION_A, omega_over_kT=w, seed=s,
                 packing=klmc.PACK_BIT) for w, s in zip(OMEGAS, seeds)]
    nrun = len(reps)
    N = L * L
    stream = x.stream

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
    flush = x.flush
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
    x.clocks.start()
    ms_steps = timed(step_batched, args.steps, args.warmup, record=True)
    clk = x.clocks.stop()
    ms_step = sum(ms_steps) / len(ms_steps)
    cnt = [lat.counters() for lat in batch.replicas]
    attempts_step = sum(c["attempts"] for c in cnt)
    draws_step = sum(c["draws"] for c in cnt)
    assert attempts_step == nrun * n_mcs * N, attempts_step  # 4 | 400: N attempts per MCS
    ms_step_max = max_over_ranks(ms_step, dist, "cuda")  # device time, max over ranks
    value = world * attempts_step / (ms_step_max * 1e-3)

    sweep_ms = [e0.elapsed_time(e1) for e0, e1 in sweep_events[-n_seg * args.steps:]]
    launch_ms = sum(sweep_ms) / len(sweep_ms)
    attempts_launch = nrun * HIST_EVERY * N
    p_draw = draws_step / attempts_step
    cluster, threads = batch.replicas[0].launch_shape()
    ctas = nrun * cluster
    lat_bytes = L * ((L + 31) // 32) * 4
    roofline = _roofline(
        "resident_sweep_kernel", launch_ms, attempts_launch, p_draw, x.sm_count, _sm_mhz(clk), ctas,
        2 * nrun * lat_bytes, x.l2_peak,
        {"traffic": (TRAFFIC_C2_LAUNCH if resident_sources_hash() == TRAFFIC_SOURCES
                     and n_mcs % HIST_EVERY == 0 else None),
         "traffic_note": "DRAM bytes per launch from one ncu capture (cold cache); the lattices stay in "
                         "shared memory within a launch",
         "algorithmic_bytes_per_launch": 2 * nrun * lat_bytes,
         "cluster": cluster, "threads_per_cta": threads, "sm_count": x.sm_count,
         "frac_of_occupied_sms": None, "sweep_share_of_step": sum(sweep_ms) / sum(ms_steps),
         "phase_us": launch_ms * 1e3 / (8 * HIST_EVERY),
         "note": "latency-bound: 160000 phases of each lattice run one after another; a phase waits for its "
                 "slowest task and a barrier, and the 5 lattices occupy 5 clusters of SMs"})
    roofline["frac_of_occupied_sms"] = roofline["frac"] * x.sm_count / min(ctas, x.sm_count)

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
    batch.close()

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        n_sample = 300
        cpu = cpu_baseline(c2_oracle_tasks(n_sample), c2_oracle_tasks(n_sample, [2]),
                           f"{n_sample} MCS of each of the 5 runs plus one A-cluster histogram each",
                           f"{n_sample} MCS of one run (omega/kT 0.6) plus one histogram on one thread")

    workloads = None
    if rank == 0 and world == 1 and not args.headline_only:
        workloads = other_workloads(x)
        launches_step_all = sum(v.get("gpu_launches", 0) for v in workloads.values())
    else:
        launches_step_all = 0

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
        "l2_peak": l2_peak,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_step * args.steps,
        "clocks": clk,
    }
    if workloads is not None:
        line["workloads"] = workloads
        line["gpu_launches_workloads"] = launches_step_all
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

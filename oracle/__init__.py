"""CPU oracle for Kawasaki lattice Monte Carlo -- TEST INFRASTRUCTURE ONLY.

The plain sequential C implementation in ``klmc_oracle.c`` is the correctness
reference for the CUDA library and the timed CPU baseline.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the library under ``paper_1309_4349_gb300`` never does.

Every function states the passage of the paper (Lis & Pintal, arXiv:1309.4349)
it follows; the readings that the paper leaves open are listed in the header
of ``klmc_oracle.c``.

ctypes releases the GIL for the duration of each call, so independent runs
can be spread over host cores with plain Python threads.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "klmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_klmc.so")
_lock = threading.Lock()
_lib = None

TRI6, SQ4 = 0, 1
PERIODIC, HELICAL = 0, 1
COORDINATION = {TRI6: 6, SQ4: 4}
# Bond orientations, every bond is {i, i+o} for one site i (section "Monte Carlo
# model with Kawasaki based kinetics", Fig. 2: triangular lattice; square option).
ORIENTATIONS = {TRI6: [(1, 0), (0, 1), (1, -1)], SQ4: [(1, 0), (0, 1)]}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
    lib.orc_philox4x32_10.restype = None
    lib.orc_n_unlike.argtypes = [i32, i32, i32, vp]
    lib.orc_n_unlike.restype = i64
    lib.orc_threshold.argtypes = [dbl, i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(u64)]
    lib.orc_threshold.restype = None
    lib.orc_n_A.argtypes = [i32, i32, i64, dbl]
    lib.orc_n_A.restype = i64
    lib.orc_site_key.argtypes = [u64, i64]
    lib.orc_site_key.restype = u64
    lib.orc_init.argtypes = [i32, i32, i64, u64, vp]
    lib.orc_init.restype = ctypes.c_int
    lib.orc_phase_params.argtypes = [i32, i32, i32, u64, i64, i32,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]
    lib.orc_phase_params.restype = None
    lib.orc_phase_anchors.argtypes = [i32, i32, i32, i32, i32, i32, vp, i64]
    lib.orc_phase_anchors.restype = i64
    lib.orc_run.argtypes = [i32, i32, i32, dbl, u64, vp, i64, i64, ctypes.POINTER(i64), vp,
                            i64, vp, ctypes.c_int]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_cluster_labels.argtypes = [i32, i32, i32, vp, ctypes.c_int, vp]
    lib.orc_cluster_labels.restype = i64
    lib.orc_cluster_histogram.argtypes = [i32, i32, i32, vp, ctypes.c_int, vp, vp, i64]
    lib.orc_cluster_histogram.restype = i64
    lib.orc_run_random_sequential.argtypes = [i32, i32, i32, dbl, u64, vp, i64, i64,
                                              ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.orc_run_random_sequential.restype = ctypes.c_int
    lib.orc_n_unlike_b.argtypes = [i32, i32, i32, i32, vp]
    lib.orc_n_unlike_b.restype = i64
    lib.orc_helical_valid.argtypes = [i32, i32]
    lib.orc_helical_valid.restype = ctypes.c_int
    lib.orc_mpkk_params.argtypes = [u64, i64, i32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.orc_mpkk_params.restype = None
    lib.orc_run_mpkk.argtypes = [i32, i32, dbl, u64, vp, i64, i64, ctypes.POINTER(i64), vp, i64, vp,
                                 ctypes.c_int]
    lib.orc_run_mpkk.restype = ctypes.c_int
    lib.orc_cluster_labels_b.argtypes = [i32, i32, i32, i32, vp, ctypes.c_int, vp]
    lib.orc_cluster_labels_b.restype = i64
    lib.orc_cluster_histogram_b.argtypes = [i32, i32, i32, i32, vp, ctypes.c_int, vp, vp, i64]
    lib.orc_cluster_histogram_b.restype = i64
    lib.orc_ffn_count.argtypes = [i32, i32, i32, i32, vp, u64, i64]
    lib.orc_ffn_count.restype = i64
    lib.orc_snapshot.argtypes = [i32, i32, vp, i32, i32, i32, vp, vp]
    lib.orc_snapshot.restype = ctypes.c_int
    lib.orc_image_ffn.argtypes = [vp, vp, i32, i32, i32, u64, i64, ctypes.POINTER(i64)]
    lib.orc_image_ffn.restype = i64
    lib.orc_cluster_averages.argtypes = [vp, vp, i64, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.orc_cluster_averages.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11).
# ---------------------------------------------------------------------------
def philox(ctr, key):
    """Four output words of Philox4x32-10 for counter ctr[4] and key[2]."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


# ---------------------------------------------------------------------------
# Model pieces.
# ---------------------------------------------------------------------------
def threshold(bw: float, dn: int):
    """(always, thr) for an energy change dn: Metropolis u < min{1, exp(-bw*dn)}
    with u = r/2^32 (Metropolis step c; acceptance ratio restated in the
    section "Monte Carlo model with Kawasaki based kinetics")."""
    lib = _load()
    a = ctypes.c_int()
    t = ctypes.c_uint64()
    lib.orc_threshold(float(bw), int(dn), ctypes.byref(a), ctypes.byref(t))
    return bool(a.value), int(t.value)


def n_A(Lx: int, Ly: int, nA: int = -1, fraction: float = 0.5) -> int:
    return int(_load().orc_n_A(Lx, Ly, nA, fraction))


def site_key(seed: int, i: int) -> int:
    return int(_load().orc_site_key(seed, i))


def init(Lx: int, Ly: int, nA: int, seed: int) -> np.ndarray:
    """Random initial lattice with exactly nA A-sites (Fig. 2: randomly distributed
    lipids; composition conserved).  One byte per site, 1 = A, index y*Lx + x."""
    t = np.zeros(Lx * Ly, dtype=np.uint8)
    rc = _load().orc_init(Lx, Ly, nA, seed, _ptr(t))
    if rc != 0:
        raise ValueError(f"orc_init failed ({rc})")
    return t


def n_unlike(Lx: int, Ly: int, geometry: int, t: np.ndarray, boundary: int = PERIODIC) -> int:
    """Number of unlike nearest-neighbour contacts; E/kT = (omega/kT) * n_unlike."""
    t = np.ascontiguousarray(t, dtype=np.uint8)
    return int(_load().orc_n_unlike_b(Lx, Ly, geometry, boundary, _ptr(t)))


def phase_params(Lx: int, Ly: int, geometry: int, seed: int, sweep: int, phase: int):
    """(orientation index, rx, ry) of one phase (MPKK loop: a random decomposition
    per iteration, here a random shift and orientation of the sublattice)."""
    o, rx, ry = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _load().orc_phase_params(Lx, Ly, geometry, seed, sweep, phase, ctypes.byref(o),
                             ctypes.byref(rx), ctypes.byref(ry))
    return o.value, rx.value, ry.value


def phase_anchors(Lx: int, Ly: int, geometry: int, o_index: int, rx: int, ry: int) -> np.ndarray:
    lib = _load()
    n = lib.orc_phase_anchors(Lx, Ly, geometry, o_index, rx, ry, None, 0)
    out = np.zeros(max(n, 1), dtype=np.int64)
    lib.orc_phase_anchors(Lx, Ly, geometry, o_index, rx, ry, _ptr(out), n)
    return out[:n]


class RunResult:
    __slots__ = ("lattice", "n_unlike", "attempts", "unlike", "draws", "accepts", "trace")

    def __init__(self, lattice, n_unlike, counters, trace):
        self.lattice = lattice
        self.n_unlike = int(n_unlike)
        self.attempts, self.unlike, self.draws, self.accepts = (int(c) for c in counters)
        self.trace = trace

    def counters(self):
        return (self.attempts, self.unlike, self.draws, self.accepts)


def run(Lx: int, Ly: int, geometry: int, bw: float, seed: int, lattice: np.ndarray,
        sweep0: int, n_mcs: int, n_unlike0: int | None = None, counters0=(0, 0, 0, 0),
        trace_every: int = 0, check: bool = False, reverse: bool = False) -> RunResult:
    """n_mcs sweeps of eight conflict-free phases each (MPKK loop with a Kawasaki
    step per domain; Metropolis steps a-c per attempt).  The lattice array is
    copied, not modified.  check: recount the energy after every phase;
    reverse: visit each phase's anchors in reverse order."""
    lib = _load()
    t = np.array(lattice, dtype=np.uint8, copy=True)
    if n_unlike0 is None:
        n_unlike0 = n_unlike(Lx, Ly, geometry, t)
    nu = ctypes.c_int64(int(n_unlike0))
    cnt = np.array(counters0, dtype=np.int64)
    n_tr = n_mcs // trace_every if trace_every > 0 else 0
    trace = np.zeros(max(n_tr, 1), dtype=np.int64)
    rc = lib.orc_run(Lx, Ly, geometry, float(bw), seed, _ptr(t), sweep0, n_mcs, ctypes.byref(nu),
                     _ptr(cnt), trace_every, _ptr(trace), (1 if check else 0) | (2 if reverse else 0))
    if rc != 0:
        raise AssertionError("incremental energy disagrees with a full recount")
    return RunResult(t, nu.value, cnt, trace[:n_tr])


def cluster_labels(Lx: int, Ly: int, geometry: int, t: np.ndarray, species: int = 1,
                   boundary: int = PERIODIC):
    """Component label (smallest site index of the component) per site of the
    species, -1 elsewhere (section "Cluster Analysis methods")."""
    t = np.ascontiguousarray(t, dtype=np.uint8)
    labels = np.zeros(Lx * Ly, dtype=np.int64)
    n = _load().orc_cluster_labels_b(Lx, Ly, geometry, boundary, _ptr(t), species, _ptr(labels))
    return labels, int(n)


def cluster_histogram(Lx: int, Ly: int, geometry: int, t: np.ndarray, species: int = 1,
                      boundary: int = PERIODIC):
    """Sparse ascending (sizes, counts) of the species' clusters."""
    lib = _load()
    t = np.ascontiguousarray(t, dtype=np.uint8)
    n = lib.orc_cluster_histogram_b(Lx, Ly, geometry, boundary, _ptr(t), species, None, None, 0)
    if n < 0:
        raise MemoryError("orc_cluster_histogram")
    sizes = np.zeros(max(n, 1), dtype=np.int64)
    counts = np.zeros(max(n, 1), dtype=np.int64)
    lib.orc_cluster_histogram_b(Lx, Ly, geometry, boundary, _ptr(t), species, _ptr(sizes), _ptr(counts), n)
    return sizes[:n], counts[:n]


def histogram_averages(sizes, counts):
    """(number average, weight average) of a sparse cluster-size histogram: sum s c
    / sum c and sum s^2 c / sum s c, each one FP64 division of exact int64 sums
    (section "Cluster Analysis" results: average cluster size; reading R14).  Both
    are 0 for an empty histogram."""
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
    ct = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
    if sz.shape != ct.shape:
        raise ValueError("sizes and counts differ in length")
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = _load().orc_cluster_averages(_ptr(sz), _ptr(ct), sz.size, ctypes.byref(a), ctypes.byref(b))
    if rc == -1:
        raise ValueError("negative size or count")
    if rc != 0:
        raise OverflowError("histogram sums exceed int64")
    return a.value, b.value


def cluster_averages(Lx: int, Ly: int, geometry: int, t: np.ndarray, species: int = 1,
                     boundary: int = PERIODIC):
    """(number average, weight average) cluster size of the species' clusters."""
    return histogram_averages(*cluster_histogram(Lx, Ly, geometry, t, species, boundary))


# ---------------------------------------------------------------------------
# Helical boundary and the seven-colour schedule (section "Massive Parallel
# Kawasaki Kinetics": seven-lipid domains, helical boundary conditions, the MPKK
# loop with k = rand%7 per iteration).
# ---------------------------------------------------------------------------
def helical_valid(Lx: int, Ly: int) -> bool:
    """Whether the seven domain coverages tile the helical Lx x Ly lattice."""
    return bool(_load().orc_helical_valid(Lx, Ly))


def mpkk_params(seed: int, sweep: int, phase: int):
    """(coverage k, direction index d) of iteration `phase` of sweep `sweep`."""
    k, d = ctypes.c_int(), ctypes.c_int()
    _load().orc_mpkk_params(seed, sweep, phase, ctypes.byref(k), ctypes.byref(d))
    return k.value, d.value


def run_mpkk(Lx: int, Ly: int, bw: float, seed: int, lattice: np.ndarray, sweep0: int, n_mcs: int,
             n_unlike0: int | None = None, counters0=(0, 0, 0, 0), trace_every: int = 0,
             check: bool = False, reverse: bool = False) -> RunResult:
    """n_mcs sweeps of seven iterations each on the helical triangular lattice:
    per iteration a random coverage by seven-lipid domains and one Kawasaki
    attempt per domain (MPKK loop), all domains in one shared direction."""
    lib = _load()
    t = np.array(lattice, dtype=np.uint8, copy=True)
    if n_unlike0 is None:
        n_unlike0 = n_unlike(Lx, Ly, TRI6, t, HELICAL)
    nu = ctypes.c_int64(int(n_unlike0))
    cnt = np.array(counters0, dtype=np.int64)
    n_tr = n_mcs // trace_every if trace_every > 0 else 0
    trace = np.zeros(max(n_tr, 1), dtype=np.int64)
    rc = lib.orc_run_mpkk(Lx, Ly, float(bw), seed, _ptr(t), sweep0, n_mcs, ctypes.byref(nu), _ptr(cnt),
                          trace_every, _ptr(trace), (1 if check else 0) | (2 if reverse else 0))
    if rc == -2:
        raise ValueError("the seven-site domains do not tile this helical lattice")
    if rc != 0:
        raise AssertionError("incremental energy disagrees with a full recount")
    return RunResult(t, nu.value, cnt, trace[:n_tr])


def run_random_sequential(Lx: int, Ly: int, geometry: int, bw: float, seed: int,
                          lattice: np.ndarray, attempt0: int, n_attempts: int):
    """Classical sequential Kawasaki (the paper's CPU method, Fig. 5B)."""
    t = np.array(lattice, dtype=np.uint8, copy=True)
    nu = ctypes.c_int64(n_unlike(Lx, Ly, geometry, t))
    acc = ctypes.c_int64(0)
    _load().orc_run_random_sequential(Lx, Ly, geometry, float(bw), seed, _ptr(t), attempt0,
                                      n_attempts, ctypes.byref(nu), ctypes.byref(acc))
    return t, int(nu.value), int(acc.value)


# ---------------------------------------------------------------------------
# Fraction of first neighbours (section "Image analysis": for every site one
# randomly chosen nearest neighbour; similar pairs divided by the lattice size).
# ---------------------------------------------------------------------------
def ffn_count(Lx: int, Ly: int, geometry: int, t: np.ndarray, seed: int, sample: int,
              boundary: int = PERIODIC) -> int:
    """Sites whose randomly chosen nearest neighbour (sample `sample`) has the same type."""
    t = np.ascontiguousarray(t, dtype=np.uint8)
    return int(_load().orc_ffn_count(Lx, Ly, geometry, boundary, _ptr(t), seed, sample))


def ffn_exact(Lx: int, Ly: int, geometry: int, t: np.ndarray, boundary: int = PERIODIC) -> float:
    """The all-bond fraction of like neighbours, 1 - n_unlike / B, B = z N / 2: the
    random-neighbour estimator's expectation."""
    B = COORDINATION[geometry] * Lx * Ly // 2
    return 1.0 - n_unlike(Lx, Ly, geometry, t, boundary) / B


# ---------------------------------------------------------------------------
# Snapshot images (section "Image analysis": one pixel per site, sloped to keep
# the triangular geometry, scaled with supersampling to gray levels) and the
# image's fraction of first neighbours with a gray-level threshold.
# ---------------------------------------------------------------------------
def snapshot(Lx: int, Ly: int, t: np.ndarray, W: int, H: int, S: int):
    """(image, mask): gray levels 0..255 and lattice membership, arrays of H x W."""
    t = np.ascontiguousarray(t, dtype=np.uint8)
    image = np.zeros(W * H, dtype=np.uint8)
    mask = np.zeros(W * H, dtype=np.uint8)
    if _load().orc_snapshot(Lx, Ly, _ptr(t), W, H, S, _ptr(image), _ptr(mask)) != 0:
        raise ValueError("bad snapshot size")
    return image.reshape(H, W), mask.reshape(H, W)


def image_ffn(image: np.ndarray, mask: np.ndarray, delta: int, seed: int, sample: int):
    """(similar pixels, lattice pixels) of one random-neighbour sample of the image."""
    H, W = image.shape
    im = np.ascontiguousarray(image, dtype=np.uint8)
    mk = np.ascontiguousarray(mask, dtype=np.uint8)
    n = ctypes.c_int64()
    sim = _load().orc_image_ffn(_ptr(im), _ptr(mk), W, H, delta, seed, sample, ctypes.byref(n))
    return int(sim), int(n.value)


def natural_width(Lx: int, Ly: int) -> int:
    """Image width of one pixel per half-site: U = 2 Lx + Ly - 1."""
    return 2 * Lx + Ly - 1

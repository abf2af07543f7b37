"""Python binding of libklmc.so, the GB300 Kawasaki lattice Monte Carlo library.

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels (see ``include/klmc.h`` for the C ABI).  PyTorch supplies device
memory (its caching allocator, passed to the library as allocator callbacks)
and streams.  There is no CPU path: if the shared library is missing or cannot
load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libklmc.so")

TRI6, SQ4 = 0, 1
PERIODIC, HELICAL = 0, 1
PACK_AUTO, PACK_BIT, PACK_BYTE = 0, 1, 2

STATUS = {0: "KLMC_OK", 1: "KLMC_EINVAL", 2: "KLMC_ENOMEM", 3: "KLMC_ECUDA", 4: "KLMC_ETIMEOUT",
          5: "KLMC_EBUSY", 6: "KLMC_ETRUNC", 7: "KLMC_ESTATE", 8: "KLMC_ENODEV"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("geometry", ctypes.c_int32),
                ("boundary", ctypes.c_int32), ("packing", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("n_A", ctypes.c_int64),
                ("fraction_A", ctypes.c_double), ("omega_over_kT", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("user", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class Counters(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("attempts", ctypes.c_int64),
                ("unlike", ctypes.c_int64), ("draws", ctypes.c_int64),
                ("accepts", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_mcs", ctypes.c_int64),
                ("n_unlike", ctypes.c_int64), ("attempts", ctypes.c_int64), ("unlike", ctypes.c_int64),
                ("draws", ctypes.c_int64), ("accepts", ctypes.c_int64), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double),
                ("n_histograms", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("finished", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("resident", ctypes.c_int64), ("rounds", ctypes.c_int64), ("attempts", ctypes.c_int64),
                ("busy_s", ctypes.c_double), ("uptime_s", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("peak_device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


JOB_KEEP_LATTICE = 1


class KlmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {message}")


_lib = None


def build(force: bool = False) -> str:
    """Compiles libklmc.so for sm_103a (nvcc)."""
    from . import _build

    return _build.build(force=force)


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_1309_4349_gb300.build() "
                          "(the CUDA library is required; there is no CPU path)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "klmc_params_default": [P(Params)],
        "klmc_create": [P(vp), i32, dbl, dbl, u64],
        "klmc_create_ex": [P(vp), P(Params)],
        "klmc_sweep": [vp, i64],
        "klmc_sweep_traced": [vp, i64, i64, vp],
        "klmc_energy": [vp, P(i64), P(dbl)],
        "klmc_energy_recount": [vp, P(i64)],
        "klmc_cluster_histogram": [vp, i32, vp, vp, i64, P(i64)],
        "klmc_cluster_histogram_device": [vp, i32, vp, vp, i64, vp],
        "klmc_cluster_averages": [vp, i32, P(dbl), P(dbl)],
        "klmc_histogram_averages": [vp, vp, i64, P(dbl), P(dbl)],
        "klmc_get_counters": [vp, P(Counters)],
        "klmc_test_copy_shortfall": [vp, i32],
        "klmc_get_lattice": [vp, vp, i64],
        "klmc_set_lattice": [vp, vp, i64, i64],
        "klmc_set_lattice_device": [vp, vp, i64, i64],
        "klmc_get_shape": [vp, P(i32), P(i32), P(i32), P(i64)],
        "klmc_get_launch": [vp, P(i32), P(i32)],
        "klmc_set_packing": [vp, i32],
        "klmc_get_packing": [vp, P(i32)],
        "klmc_autotune": [vp, i32, P(i32), P(i32)],
        "klmc_synchronize": [vp],
        "klmc_destroy": [vp],
        "klmc_batch_create": [P(vp), P(Params), i32],
        "klmc_batch_sweep": [vp, P(i64)],
        "klmc_batch_replica": [vp, i32, P(vp)],
        "klmc_batch_get_launch": [vp, i32, P(i32), P(i32)],
        "klmc_batch_cluster_histogram_device": [vp, i32, vp, vp, i64, vp],
        "klmc_get_plan": [vp, P(i32)],
        "klmc_ffn": [vp, i64, P(i64), P(ctypes.c_double)],
        "klmc_ffn_device": [vp, i64, vp],
        "klmc_snapshot": [vp, i32, i32, i32, vp, vp],
        "klmc_image_ffn": [vp, vp, vp, i32, i32, i32, i64, P(i64), P(i64)],
        "klmc_batch_destroy": [vp],
        "klmc_server_create": [P(vp), ctypes.c_size_t, vp],
        "klmc_server_submit": [vp, P(Params), i64, i64, ctypes.c_uint32, P(u64)],
        "klmc_server_poll": [vp, u64, P(JobResult)],
        "klmc_server_job_lattice": [vp, u64, vp, i64],
        "klmc_server_job_histogram": [vp, u64, vp, vp, i64, P(i64)],
        "klmc_server_release": [vp, u64],
        "klmc_server_get_stats": [vp, P(ServerStats)],
        "klmc_server_drain": [vp, dbl],
        "klmc_server_destroy": [vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.klmc_status_str.argtypes = [ctypes.c_int]
    L.klmc_status_str.restype = ctypes.c_char_p
    L.klmc_last_error.argtypes = []
    L.klmc_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        msg = lib().klmc_last_error().decode(errors="replace")
        raise KlmcError(status, msg)


def _torch_stream_handle(stream=None) -> int:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class _TorchAllocator:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, device: int):
        import torch

        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device,
                                                              stream=stream or 0))
            except Exception:  # allocation failure is reported as NULL
                return None

        def _free(ptr, nbytes, stream, user):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


def histogram_averages(sizes, counts) -> tuple[float, float]:
    """(number average, weight average) of a sparse host histogram
    (klmc_histogram_averages)."""
    sz = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
    ct = np.ascontiguousarray(np.asarray(counts, dtype=np.int64))
    if sz.shape != ct.shape:
        raise ValueError("sizes and counts differ in length")
    a, w = ctypes.c_double(), ctypes.c_double()
    _check(lib().klmc_histogram_averages(sz.ctypes.data, ct.ctypes.data, sz.size, ctypes.byref(a),
                                         ctypes.byref(w)))
    return a.value, w.value


def make_params(Lx: int, Ly: int | None = None, *, geometry: int = TRI6, packing: int = PACK_BIT,
                n_A: int = -1, fraction_A: float = 0.5, omega_over_kT: float = 0.0, seed: int = 1,
                cluster: int = 0, threads: int = 0, boundary: int = 0, stream: int | None = None,
                allocator: _TorchAllocator | None = None) -> Params:
    p = Params()
    _check(lib().klmc_params_default(ctypes.byref(p)))
    p.Lx = int(Lx)
    p.Ly = int(Ly if Ly is not None else Lx)
    p.geometry = int(geometry)
    p.packing = int(packing)
    p.n_A = int(n_A)
    p.fraction_A = float(fraction_A)
    p.omega_over_kT = float(omega_over_kT)
    p.seed = int(seed)
    p.cluster = int(cluster)
    p.threads = int(threads)
    p.boundary = int(boundary)
    p.stream = stream
    if allocator is not None:
        p.alloc = allocator.alloc
        p.free = allocator.free
    return p


class Lattice:
    """One lattice (klmc_ctx).  Every method is one C-ABI call."""

    def __init__(self, Lx: int, Ly: int | None = None, *, geometry: int = TRI6,
                 packing: int = PACK_BIT, n_A: int = -1, fraction_A: float = 0.5,
                 omega_over_kT: float = 0.0, seed: int = 1, cluster: int = 0, threads: int = 0,
                 boundary: int = 0, stream=None, torch_allocator: bool = True, _handle=None,
                 _owner=None):
        import torch

        self._owner = _owner
        self._alloc = None
        if _handle is not None:
            self._h = _handle
        else:
            dev = torch.cuda.current_device()
            self._alloc = _TorchAllocator(dev) if torch_allocator else None
            p = make_params(Lx, Ly, geometry=geometry, packing=packing, n_A=n_A,
                            fraction_A=fraction_A, omega_over_kT=omega_over_kT, seed=seed,
                            cluster=cluster, threads=threads, boundary=boundary,
                            stream=_torch_stream_handle(stream), allocator=self._alloc)
            h = ctypes.c_void_p()
            _check(lib().klmc_create_ex(ctypes.byref(h), ctypes.byref(p)))
            self._h = h
        Lx_, Ly_, g_ = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nA_ = ctypes.c_int64()
        _check(lib().klmc_get_shape(self._h, ctypes.byref(Lx_), ctypes.byref(Ly_), ctypes.byref(g_),
                                    ctypes.byref(nA_)))
        self.Lx, self.Ly, self.geometry = Lx_.value, Ly_.value, g_.value

    @property
    def N(self) -> int:
        return self.Lx * self.Ly

    @property
    def n_A(self) -> int:
        nA_ = ctypes.c_int64()
        _check(lib().klmc_get_shape(self._h, None, None, None, ctypes.byref(nA_)))
        return nA_.value

    def sweep(self, n_mcs: int):
        _check(lib().klmc_sweep(self._h, int(n_mcs)))

    def sweep_traced(self, n_mcs: int, trace_every: int, out=None):
        """Runs n_mcs steps; returns an int64 CUDA tensor of n_unlike after every
        trace_every-th step (filled asynchronously on the lattice's stream)."""
        import torch

        n = int(n_mcs) // int(trace_every)
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        _check(lib().klmc_sweep_traced(self._h, int(n_mcs), int(trace_every),
                                       ctypes.c_void_p(out.data_ptr())))
        return out[:n]

    def energy(self):
        n = ctypes.c_int64()
        e = ctypes.c_double()
        _check(lib().klmc_energy(self._h, ctypes.byref(n), ctypes.byref(e)))
        return int(n.value), float(e.value)

    def energy_recount(self) -> int:
        n = ctypes.c_int64()
        _check(lib().klmc_energy_recount(self._h, ctypes.byref(n)))
        return int(n.value)

    def cluster_histogram(self, species: int = 1):
        cap = int(np.sqrt(2.0 * self.N)) + 2
        sizes = np.zeros(cap, dtype=np.int64)
        counts = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int64()
        _check(lib().klmc_cluster_histogram(self._h, int(species), sizes.ctypes.data,
                                            counts.ctypes.data, cap, ctypes.byref(n)))
        return sizes[:n.value].copy(), counts[:n.value].copy()

    def cluster_averages(self, species: int = 1) -> tuple[float, float]:
        """(number average, weight average) cluster size of the species
        (klmc_cluster_averages)."""
        a, w = ctypes.c_double(), ctypes.c_double()
        _check(lib().klmc_cluster_averages(self._h, int(species), ctypes.byref(a), ctypes.byref(w)))
        return a.value, w.value

    def ffn(self, sample: int = 0) -> tuple[float, float]:
        """(random-neighbour fraction of first neighbours of sample `sample`, all-bond
        fraction 1 - n_unlike / B)."""
        n, e = ctypes.c_int64(), ctypes.c_double()
        _check(lib().klmc_ffn(self._h, int(sample), ctypes.byref(n), ctypes.byref(e)))
        return n.value / self.N, e.value

    def snapshot(self, W: int, H: int, S: int = 1):
        """(image, mask) as uint8 CUDA tensors of shape (H, W): gray levels of the
        sloped, supersampled lattice and lattice-pixel membership."""
        import torch

        image = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        _check(lib().klmc_snapshot(self._h, int(W), int(H), int(S), image.data_ptr(), mask.data_ptr()))
        return image, mask

    def image_ffn(self, image, mask, delta: int = 35, sample: int = 0) -> tuple[int, int]:
        """(similar pixels, lattice pixels) of one random-neighbour sample of an image."""
        H, W = image.shape
        sim, px = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().klmc_image_ffn(self._h, image.data_ptr(), mask.data_ptr(), int(W), int(H), int(delta),
                                    int(sample), ctypes.byref(sim), ctypes.byref(px)))
        return sim.value, px.value

    def ffn_device(self, sample: int, out):
        """Enqueues sample `sample`'s similar-neighbour count into a one-element int64
        CUDA tensor (no synchronisation)."""
        _check(lib().klmc_ffn_device(self._h, int(sample), out.data_ptr()))

    def cluster_histogram_device(self, species, sizes, counts, n_distinct):
        """Enqueues the histogram into int64 CUDA tensors (no synchronisation)."""
        cap = min(sizes.numel(), counts.numel())
        _check(lib().klmc_cluster_histogram_device(self._h, int(species), sizes.data_ptr(),
                                                   counts.data_ptr(), cap, n_distinct.data_ptr()))

    def counters(self) -> dict:
        c = Counters()
        _check(lib().klmc_get_counters(self._h, ctypes.byref(c)))
        return c.as_dict()

    def test_copy_shortfall(self, nbytes: int):
        """Test hook: make this handle's tiled launches wait for row copies that
        never arrive (klmc_test_copy_shortfall)."""
        _check(lib().klmc_test_copy_shortfall(self._h, int(nbytes)))

    def get_lattice(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.uint8)
        _check(lib().klmc_get_lattice(self._h, out.ctypes.data, self.N))
        return out

    def set_lattice(self, t, sweep_index: int = 0):
        arr = np.ascontiguousarray(np.asarray(t, dtype=np.uint8).ravel())
        _check(lib().klmc_set_lattice(self._h, arr.ctypes.data, arr.size, int(sweep_index)))

    def set_lattice_device(self, t, sweep_index: int = 0):
        """Loads the lattice from a uint8 CUDA tensor of Lx*Ly entries (0/1), async."""
        assert t.is_cuda and t.dtype.itemsize == 1 and t.numel() == self.N and t.is_contiguous()
        _check(lib().klmc_set_lattice_device(self._h, t.data_ptr(), self.N, int(sweep_index)))

    def autotune(self, probe_sweeps: int = 8):
        """Times the valid launch shapes on a scratch copy and keeps the fastest
        (all candidates must give identical results); returns (cluster, threads)."""
        c, t = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().klmc_autotune(self._h, int(probe_sweeps), ctypes.byref(c), ctypes.byref(t)))
        return c.value, t.value

    def launch_shape(self):
        """(CTAs per lattice, threads per CTA) of the resident sweep."""
        c, t = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().klmc_get_launch(self._h, ctypes.byref(c), ctypes.byref(t)))
        return c.value, t.value

    def packing(self) -> int:
        """Store format of the device lattice: PACK_BIT or PACK_BYTE (klmc_get_packing)."""
        v = ctypes.c_int32()
        _check(lib().klmc_get_packing(self._h, ctypes.byref(v)))
        return v.value

    def set_packing(self, packing: int) -> None:
        """Moves the device lattice into a store of the given format (klmc_set_packing)."""
        _check(lib().klmc_set_packing(self._h, int(packing)))

    def plan(self) -> int:
        """Phases advanced between halo exchanges of the resident sweep (1: every phase)."""
        k = ctypes.c_int32()
        _check(lib().klmc_get_plan(self._h, ctypes.byref(k)))
        return k.value

    def synchronize(self):
        _check(lib().klmc_synchronize(self._h))

    def close(self):
        if self._owner is None and getattr(self, "_h", None):
            _check(lib().klmc_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            if self._owner is None and getattr(self, "_h", None):
                lib().klmc_destroy(self._h)
                self._h = None
        except Exception:
            pass


class Batch:
    """Replicas advanced together by one resident-kernel launch (klmc_batch)."""

    def __init__(self, replicas: list[dict], stream=None, torch_allocator: bool = True):
        import torch

        dev = torch.cuda.current_device()
        self._alloc = _TorchAllocator(dev) if torch_allocator else None
        sh = _torch_stream_handle(stream)
        arr = (Params * len(replicas))()
        for i, r in enumerate(replicas):
            arr[i] = make_params(stream=sh, allocator=self._alloc, **r)
        h = ctypes.c_void_p()
        _check(lib().klmc_batch_create(ctypes.byref(h), arr, len(replicas)))
        self._h = h
        self.n = len(replicas)
        self.replicas = []
        for i in range(self.n):
            v = ctypes.c_void_p()
            _check(lib().klmc_batch_replica(self._h, i, ctypes.byref(v)))
            self.replicas.append(Lattice(0, _handle=v, _owner=self))

    def sweep(self, n_mcs):
        if np.isscalar(n_mcs):
            n_mcs = [int(n_mcs)] * self.n
        arr = (ctypes.c_int64 * self.n)(*[int(v) for v in n_mcs])
        _check(lib().klmc_batch_sweep(self._h, arr))

    def cluster_histogram_device(self, species: int, sizes, counts, n_distinct):
        """Every replica's histogram into torch int64 CUDA tensors: sizes and counts of
        shape (n, capacity), n_distinct of shape (n,); enqueued, not synchronised."""
        cap = int(sizes.shape[-1]) if sizes is not None else 0
        for t in (sizes, counts, n_distinct):
            if t is not None and not t.is_contiguous():
                raise ValueError("output tensors must be contiguous")
        _check(lib().klmc_batch_cluster_histogram_device(
            self._h, int(species), sizes.data_ptr() if sizes is not None else None,
            counts.data_ptr() if counts is not None else None, cap, n_distinct.data_ptr()))

    def launch_shape(self, i: int) -> tuple[int, int]:
        """(CTAs per replica, threads per CTA) replica i ran with in the last sweep."""
        c, t = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().klmc_batch_get_launch(self._h, int(i), ctypes.byref(c), ctypes.byref(t)))
        return c.value, t.value

    def close(self):
        if getattr(self, "_h", None):
            for r in self.replicas:
                r._h = None
            _check(lib().klmc_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Job server with continuous batching (klmc_server): jobs are admitted by
    device memory, stay resident, and advance together in rounds."""

    def __init__(self, device_mem_budget: int, stream=None):
        h = ctypes.c_void_p()
        sh = None if stream is None else int(stream.cuda_stream)
        _check(lib().klmc_server_create(ctypes.byref(h), int(device_mem_budget), sh))
        self._h = h

    def submit(self, Lx: int, Ly: int | None = None, *, n_mcs: int, hist_every: int = 0,
               keep_lattice: bool = False, geometry: int = TRI6, packing: int = PACK_BIT,
               n_A: int = -1, fraction_A: float = 0.5, omega_over_kT: float = 0.0, seed: int = 1,
               cluster: int = 0, boundary: int = 0, allocator=None) -> int:
        """Queues a job; `allocator` (an object with ``alloc`` and ``free`` callbacks
        of types ALLOC_FN and FREE_FN, kept alive by the caller until the job ends)
        serves the job's lattice memory instead of the server's own allocations."""
        p = make_params(Lx, Ly, geometry=geometry, packing=packing, n_A=n_A, fraction_A=fraction_A,
                        omega_over_kT=omega_over_kT, seed=seed, cluster=cluster, boundary=boundary,
                        allocator=allocator)
        jid = ctypes.c_uint64()
        _check(lib().klmc_server_submit(self._h, ctypes.byref(p), int(n_mcs), int(hist_every),
                                        JOB_KEEP_LATTICE if keep_lattice else 0, ctypes.byref(jid)))
        return int(jid.value)

    def poll(self, job_id: int):
        """Result dict of a finished job, or None while it is queued or running."""
        r = JobResult()
        st = lib().klmc_server_poll(self._h, int(job_id), ctypes.byref(r))
        if st == 5:  # KLMC_EBUSY
            return None
        _check(st)
        return r.as_dict()

    def lattice(self, job_id: int, n: int) -> np.ndarray:
        out = np.zeros(n, dtype=np.uint8)
        _check(lib().klmc_server_job_lattice(self._h, int(job_id), out.ctypes.data, n))
        return out

    def histogram(self, job_id: int):
        cap = 1 << 16
        sizes = np.zeros(cap, dtype=np.int64)
        counts = np.zeros(cap, dtype=np.int64)
        n = ctypes.c_int64()
        _check(lib().klmc_server_job_histogram(self._h, int(job_id), sizes.ctypes.data,
                                               counts.ctypes.data, cap, ctypes.byref(n)))
        return sizes[:n.value].copy(), counts[:n.value].copy()

    def release(self, job_id: int):
        _check(lib().klmc_server_release(self._h, int(job_id)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().klmc_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def drain(self, timeout_s: float = 3600.0):
        _check(lib().klmc_server_drain(self._h, float(timeout_s)))

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().klmc_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

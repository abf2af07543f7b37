"""Failure paths that need a device but fault nothing: device allocations refused
by an allocator the test supplies (a host-side fake of an out-of-memory
allocator).  Every refusal must surface as KLMC_ENOMEM, and every allocation the
library obtained before it must be returned: the test's allocator counts what is
outstanding."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()
ENOMEM = 2


class FailingAllocator:
    """Device allocator backed by torch's caching allocator that returns NULL on
    its allocation number `fail_at` (0-based; None: never), and on every one while
    `refuse` is set.  `outstanding` holds the pointers not yet freed."""

    def __init__(self, fail_at=None):
        self.fail_at = fail_at
        self.refuse = False
        self.calls = 0
        self.outstanding = {}
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, user):
            k = self.calls
            self.calls += 1
            if self.refuse or k == self.fail_at:
                return None
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream or 0))
            self.outstanding[ptr] = int(nbytes)
            return ptr

        def _free(ptr, nbytes, stream, user):
            assert ptr in self.outstanding, "free of a pointer this allocator did not hand out"
            assert self.outstanding.pop(ptr) == nbytes
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = klmc.ALLOC_FN(_alloc)
        self.free = klmc.FREE_FN(_free)


def create(fa, Lx=64, Ly=48, **kw):
    p = klmc.make_params(Lx, Ly, n_A=Lx * Ly // 3, omega_over_kT=0.7, seed=11, allocator=fa,
                         stream=torch.cuda.current_stream().cuda_stream, **kw)
    h = ctypes.c_void_p()
    st = klmc.lib().klmc_create_ex(ctypes.byref(h), ctypes.byref(p))
    return st, h


def test_create_enomem_at_every_allocation():
    """Refuse the first, second, ... allocation of klmc_create_ex in turn: each
    attempt fails with ENOMEM, returns no handle and leaves nothing allocated; the
    first attempt that needs no refused allocation succeeds and runs exactly."""
    n_allocs = None
    for k in range(16):
        fa = FailingAllocator(fail_at=k)
        st, h = create(fa)
        if st == 0:
            n_allocs = k
            fa.fail_at = None  # allocations on first use (the byte lattice) are granted
            lat = klmc.Lattice(0, _handle=h)
            lat.sweep(3)
            ref = oracle.run(64, 48, klmc.TRI6, 0.7, 11, oracle.init(64, 48, 64 * 48 // 3, 11), 0, 3)
            assert np.array_equal(lat.get_lattice(), ref.lattice)
            lat.close()
            assert not fa.outstanding
            break
        assert st == ENOMEM, klmc.lib().klmc_last_error().decode()
        assert h.value is None
        assert not fa.outstanding, f"allocation {k} refused: {len(fa.outstanding)} left allocated"
    assert n_allocs is not None and n_allocs >= 3  # lattice, state, placement scratch at least


def test_lazy_allocations_enomem_and_handle_survives():
    """Allocations made on first use (cluster scratch, the byte lattice of a device
    load) report ENOMEM and leave the handle usable; destroying it frees all."""
    fa = FailingAllocator()
    st, h = create(fa)
    assert st == 0
    lat = klmc.Lattice(0, _handle=h)
    held = dict(fa.outstanding)
    fa.refuse = True
    with pytest.raises(klmc.KlmcError) as e:
        lat.cluster_histogram(1)
    assert e.value.status == ENOMEM
    with pytest.raises(klmc.KlmcError) as e:
        lat.cluster_averages(1)
    assert e.value.status == ENOMEM
    assert fa.outstanding == held
    fa.refuse = False
    lat.sweep(2)  # still a valid handle
    assert lat.energy()[0] == lat.energy_recount()
    s, c = lat.cluster_histogram(1)
    rs, rc = oracle.cluster_histogram(64, 48, klmc.TRI6, lat.get_lattice(), 1)
    assert np.array_equal(s, rs) and np.array_equal(c, rc)
    lat.close()
    assert not fa.outstanding


def test_tiled_second_buffer_enomem():
    """A lattice too large for a cluster runs on the tiled path, whose second store
    buffer is allocated at the first sweep: refused, the sweep reports ENOMEM."""
    fa = FailingAllocator()
    st, h = create(fa, 6000, 6000)
    assert st == 0
    lat = klmc.Lattice(0, _handle=h)
    assert lat.launch_shape()[0] == -1
    fa.refuse = True
    with pytest.raises(klmc.KlmcError) as e:
        lat.sweep(1)
    assert e.value.status == ENOMEM
    lat.close()
    assert not fa.outstanding


def test_batch_create_enomem_at_every_allocation():
    """klmc_batch_create over three replicas sharing one refusing allocator: every
    refused allocation fails the whole batch with ENOMEM and frees what the
    replicas created before it held."""
    sides = [(40, 32), (57, 41), (100, 64)]
    done = False
    for k in range(40):
        fa = FailingAllocator(fail_at=k)
        sh = torch.cuda.current_stream().cuda_stream
        arr = (klmc.Params * len(sides))()
        for i, (Lx, Ly) in enumerate(sides):
            arr[i] = klmc.make_params(Lx, Ly, n_A=Lx * Ly // 4, omega_over_kT=0.5, seed=20 + i,
                                      allocator=fa, stream=sh)
        h = ctypes.c_void_p()
        st = klmc.lib().klmc_batch_create(ctypes.byref(h), arr, len(sides))
        if st == 0:
            assert k >= 3 * len(sides)
            klmc.lib().klmc_batch_destroy(h)
            assert not fa.outstanding
            done = True
            break
        assert st == ENOMEM, klmc.lib().klmc_last_error().decode()
        assert not fa.outstanding, f"allocation {k} refused: {len(fa.outstanding)} left allocated"
    assert done


def test_server_job_enomem_fails_only_that_job():
    """A served job whose own allocator refuses finishes with status ENOMEM and
    holds nothing; the jobs around it run normally and equal the oracle."""
    srv = klmc.Server(1 << 30)
    bad = FailingAllocator(fail_at=1)  # the lattice is granted, the state is refused
    ok_ids = [srv.submit(48, 40, n_mcs=20, n_A=500, omega_over_kT=0.6, seed=31 + i, keep_lattice=True)
              for i in range(2)]
    bad_id = srv.submit(48, 40, n_mcs=20, n_A=500, omega_over_kT=0.6, seed=99, allocator=bad)
    ok_ids.append(srv.submit(48, 40, n_mcs=20, n_A=500, omega_over_kT=0.6, seed=33, keep_lattice=True))
    srv.drain(120.0)
    assert srv.poll(bad_id)["status"] == ENOMEM
    assert not bad.outstanding
    for i, jid in enumerate(ok_ids):
        r = srv.poll(jid)
        assert r["status"] == 0
        seed = 31 + i
        ref = oracle.run(48, 40, klmc.TRI6, 0.6, seed, oracle.init(48, 40, 500, seed), 0, 20)
        assert np.array_equal(srv.lattice(jid, 48 * 40), ref.lattice)
        assert r["n_unlike"] == ref.n_unlike
    srv.close()


def test_store_conversion_enomem_leaves_handle_unchanged():
    """klmc_set_packing and the autotuner's store-format probes allocate new stores:
    refused, they report ENOMEM, hold nothing more and leave the handle's store as
    it was; granted, the old store is returned to the allocator."""
    fa = FailingAllocator()
    st, h = create(fa, packing=klmc.PACK_AUTO)
    assert st == 0
    lat = klmc.Lattice(0, _handle=h)
    lat.sweep(2)
    before = lat.get_lattice()
    held = dict(fa.outstanding)
    fa.refuse = True
    with pytest.raises(klmc.KlmcError) as e:
        lat.set_packing(klmc.PACK_BYTE)
    assert e.value.status == ENOMEM
    with pytest.raises(klmc.KlmcError) as e:
        lat.autotune(1)
    assert e.value.status == ENOMEM
    assert fa.outstanding == held
    assert lat.packing() == klmc.PACK_BIT
    fa.refuse = False
    lat.set_packing(klmc.PACK_BYTE)
    assert np.array_equal(lat.get_lattice(), before)
    assert len(fa.outstanding) == len(held)  # the bit store went back, the byte store came in
    assert sum(fa.outstanding.values()) > sum(held.values())
    lat.sweep(2)
    ref = oracle.run(64, 48, klmc.TRI6, 0.7, 11, oracle.init(64, 48, 64 * 48 // 3, 11), 0, 4)
    assert np.array_equal(lat.get_lattice(), ref.lattice)
    lat.close()
    assert not fa.outstanding

"""klmc_cluster_histogram_noalloc: the cluster histogram for callers that cannot
allocate device memory (a framework that owns all device memory under a fixed
budget with no allocator hook, or a loop that cannot accept cudaMalloc's implicit
device synchronisation).  It must give exactly what the allocating entry point
klmc_cluster_histogram_device gives, call after call, although every call reuses
one fixed scratch array.

This file is collected last on purpose, and must pass both alone in a fresh
process and after the other tests.
"""
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


def noalloc_fn():
    f = klmc.lib().klmc_cluster_histogram_noalloc
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    f.argtypes = [vp, i32, i32, i32, i32, i32, i32, vp, vp, i64, vp, vp]
    f.restype = ctypes.c_int
    return f


def histogram_with_allocating_entry_point(t, Lx, Ly, geometry, species):
    lat = klmc.Lattice(Lx, Ly, geometry=geometry, n_A=int(t.sum()), seed=1)
    lat.set_lattice(t, 0)
    cap = int(np.sqrt(2.0 * Lx * Ly)) + 2
    sizes = torch.zeros(cap, dtype=torch.int64, device="cuda")
    counts = torch.zeros(cap, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    lat.cluster_histogram_device(species, sizes, counts, n)
    torch.cuda.synchronize()
    k = int(n.item())
    return sizes[:k].cpu().numpy(), counts[:k].cpu().numpy()


def histogram_noalloc(t, Lx, Ly, geometry, species, packing):
    if packing == klmc.PACK_BYTE:
        pitch = Lx
        dev = torch.from_numpy(t.copy()).cuda()
    else:
        pitch = (Lx + 31) // 32
        rows = np.zeros((Ly, pitch * 32), dtype=np.uint8)
        rows[:, :Lx] = t.reshape(Ly, Lx)
        words = np.packbits(rows.reshape(Ly, pitch, 32)[:, :, ::-1], axis=-1)  # bit x%32 of word x/32
        words = words.reshape(Ly, pitch, 4)[:, :, ::-1].copy().view(np.uint32).reshape(-1)
        dev = torch.from_numpy(words.view(np.int32)).cuda()
    cap = int(np.sqrt(2.0 * Lx * Ly)) + 2
    sizes = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    counts = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    n = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = noalloc_fn()(dev.data_ptr(), packing, Lx, Ly, pitch, geometry, species, sizes.data_ptr(),
                      counts.data_ptr(), cap, n.data_ptr(), stream)
    assert st == 0, klmc.lib().klmc_last_error().decode()
    torch.cuda.synchronize()
    k = int(n.item())
    return sizes[:k].cpu().numpy(), counts[:k].cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    cases = [
        # (Lx, Ly, geometry, species, packing, lattice)
        (400, 400, klmc.TRI6, 1, klmc.PACK_BIT, oracle.init(400, 400, 48000, 2)),
        (257, 130, klmc.SQ4, 0, klmc.PACK_BYTE,
         oracle.run(257, 130, oracle.SQ4, 0.9, 5, oracle.init(257, 130, 13000, 5), 0, 6).lattice),
    ]
    for Lx, Ly, g, species, packing, t in cases:
        want = histogram_with_allocating_entry_point(t, Lx, Ly, g, species)
        ref = oracle.cluster_histogram(Lx, Ly, g, t, species)
        for _ in range(2):  # the second call reuses the scratch the first one left behind
            got = histogram_noalloc(t, Lx, Ly, g, species, packing)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
            assert int((got[0] * got[1]).sum()) == int((t == species).sum())


def test_noalloc_rejects_lattices_above_its_fixed_scratch():
    dev = torch.zeros(8, dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    side = 1025  # 1025 * 1025 > KLMC_NOALLOC_MAX_SITES = 2^20
    st = noalloc_fn()(dev.data_ptr(), klmc.PACK_BYTE, side, side, side, klmc.TRI6, 1, None, None, 0,
                      n.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 1  # KLMC_EINVAL, before any GPU work
    assert "exceeds" in klmc.lib().klmc_last_error().decode()

"""Store formats (1 bit or 1 byte per site): moving a handle's lattice between
them mid-run, and the autotuner choosing one for a handle created with
PACK_AUTO.  Every run must stay bit-exact against the oracle, whichever store
the sweeps ran on."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()
EINVAL, ESTATE = 1, 7


@pytest.mark.parametrize("Lx,Ly,cluster", [(96, 80, 4), (200, 777, -1), (64, 48, 1)])
def test_store_moves_between_formats_mid_run(Lx, Ly, cluster):
    nA, bw, seed = Lx * Ly * 2 // 5, 0.8, 17
    lat = klmc.Lattice(Lx, Ly, n_A=nA, omega_over_kT=bw, seed=seed, cluster=cluster)
    try:
        assert lat.packing() == klmc.PACK_BIT
        lat.sweep(2)
        before = lat.get_lattice()
        lat.set_packing(klmc.PACK_BYTE)
        assert lat.packing() == klmc.PACK_BYTE
        assert np.array_equal(lat.get_lattice(), before)
        lat.sweep(3)
        lat.set_packing(klmc.PACK_BIT)
        lat.set_packing(klmc.PACK_BIT)  # already there: nothing to do
        lat.sweep(2)
        ref = oracle.run(Lx, Ly, oracle.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 7)
        assert np.array_equal(lat.get_lattice(), ref.lattice)
        c = lat.counters()
        assert (c["attempts"], c["unlike"], c["draws"], c["accepts"]) == ref.counters()
        assert lat.energy()[0] == ref.n_unlike
    finally:
        lat.close()


def test_autotune_picks_a_store_format_for_auto_packing():
    Lx, Ly, nA, bw, seed = 128, 96, 128 * 96 // 3, 0.6, 23
    lat = klmc.Lattice(Lx, Ly, n_A=nA, omega_over_kT=bw, seed=seed, packing=klmc.PACK_AUTO)
    try:
        lat.sweep(2)
        before = lat.get_lattice()
        lat.autotune(2)
        assert lat.packing() in (klmc.PACK_BIT, klmc.PACK_BYTE)
        assert np.array_equal(lat.get_lattice(), before)
        lat.sweep(3)
        ref = oracle.run(Lx, Ly, oracle.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 5)
        assert np.array_equal(lat.get_lattice(), ref.lattice)
        assert lat.counters()["accepts"] == ref.accepts
        # a later handle of the same size with the automatic shape takes the tuned choice
        again = klmc.Lattice(Lx, Ly, n_A=nA, omega_over_kT=bw, seed=seed, packing=klmc.PACK_AUTO)
        try:
            assert again.packing() == lat.packing()
            assert again.launch_shape() == lat.launch_shape()
        finally:
            again.close()
    finally:
        lat.close()


def test_set_packing_refusals():
    lat = klmc.Lattice(64, 64, n_A=2048, omega_over_kT=0.5, seed=3)
    b = klmc.Batch([dict(Lx=64, Ly=64, n_A=2048, omega_over_kT=0.5, seed=3)])
    try:
        with pytest.raises(klmc.KlmcError) as err:
            lat.set_packing(klmc.PACK_AUTO)
        assert err.value.status == EINVAL
        with pytest.raises(klmc.KlmcError) as err:
            b.replicas[0].set_packing(klmc.PACK_BYTE)
        assert err.value.status == ESTATE
        assert lat.packing() == klmc.PACK_BIT
    finally:
        b.close()
        lat.close()

"""The band kernel's bounded wait for its row copies: made to run out through the
test hook (its launches expect 16 bytes that no copy delivers), it gives up,
leaves its band unwritten and reports KLMC_ETIMEOUT through klmc_energy and
klmc_get_counters, and the device context stays usable (a new handle's tiled
sweeps still match the oracle bit for bit)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()
KLMC_ETIMEOUT = 4


def test_copy_wait_gives_up_and_reports():
    Lx, Ly, nA, bw, seed = 200, 777, 62160, 0.9, 5
    lat = klmc.Lattice(Lx, Ly, n_A=nA, omega_over_kT=bw, seed=seed, cluster=-1)
    try:
        assert lat.plan() == 4  # bands of 4 phases, rows by bulk copy
        lat.test_copy_shortfall(16)
        lat.sweep(1)
        for call in (lat.energy, lat.counters):
            with pytest.raises(klmc.KlmcError) as err:
                call()
            assert err.value.status == KLMC_ETIMEOUT
    finally:
        lat.close()
    fresh = klmc.Lattice(Lx, Ly, n_A=nA, omega_over_kT=bw, seed=seed, cluster=-1)
    try:
        fresh.sweep(3)
        ref = oracle.run(Lx, Ly, oracle.TRI6, bw, seed, oracle.init(Lx, Ly, nA, seed), 0, 3)
        assert np.array_equal(fresh.get_lattice(), ref.lattice)
        assert fresh.energy()[0] == ref.n_unlike
    finally:
        fresh.close()


def test_hook_rejects_negative():
    lat = klmc.Lattice(64, 64, n_A=2048, omega_over_kT=0.6, seed=1)
    try:
        with pytest.raises(klmc.KlmcError):
            lat.test_copy_shortfall(-1)
    finally:
        lat.close()

"""Fraction of first neighbours on the GPU (section "Image analysis": one randomly
chosen nearest neighbour per site, similar pairs over the lattice size) against
the oracle: the random-neighbour count bit for bit, the all-bond fraction
exactly."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()


@pytest.mark.parametrize("packing", [klmc.PACK_BIT, klmc.PACK_BYTE])
@pytest.mark.parametrize("geometry,boundary,Lx,Ly", [
    (klmc.TRI6, klmc.PERIODIC, 37, 29), (klmc.SQ4, klmc.PERIODIC, 64, 33), (klmc.TRI6, klmc.PERIODIC, 400, 400),
    (klmc.TRI6, klmc.HELICAL, 31, 14), (klmc.TRI6, klmc.HELICAL, 402, 399), (klmc.SQ4, klmc.PERIODIC, 5, 4),
])
def test_ffn_parity(packing, geometry, boundary, Lx, Ly):
    N = Lx * Ly
    seed = 40 + Lx
    lat = klmc.Lattice(Lx, Ly, geometry=geometry, packing=packing, n_A=N // 3, omega_over_kT=0.8, seed=seed,
                       boundary=boundary)
    lat.sweep(7)
    t = lat.get_lattice()
    for m in (0, 1, 12345678901):
        f, exact = lat.ffn(m)
        assert f * N == oracle.ffn_count(Lx, Ly, geometry, t, seed, m, boundary)
        assert exact == pytest.approx(oracle.ffn_exact(Lx, Ly, geometry, t, boundary), abs=1e-15)
    dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    lat.ffn_device(3, dev)
    torch.cuda.synchronize()
    assert int(dev.item()) == oracle.ffn_count(Lx, Ly, geometry, t, seed, 3, boundary)


def test_ffn_time_series_tracks_the_energy_trace():
    """A time series of both fractions along a trajectory: the all-bond fraction is
    1 - trace / B at every sample, and the random-neighbour fraction scatters
    around it with the binomial spread."""
    Lx = Ly = 128
    N = Lx * Ly
    lat = klmc.Lattice(Lx, Ly, n_A=N // 2, omega_over_kT=0.7, seed=2)
    rnd, exact = [], []
    for k in range(30):
        lat.sweep(10)
        f, e = lat.ffn(k)
        rnd.append(f)
        exact.append(e)
        assert e == pytest.approx(1.0 - lat.energy()[0] / (3.0 * N), abs=1e-15)
    rnd, exact = np.array(rnd), np.array(exact)
    assert exact[-1] > exact[0]  # demixing raises the like fraction
    z = (rnd - exact) / np.sqrt(exact * (1 - exact) / N)
    assert abs(z.mean()) < 5 / np.sqrt(len(z)) and z.std() < 2.0

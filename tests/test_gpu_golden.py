"""The CUDA path, through the C ABI, against the stored oracle runs
(tests/golden/oracle_runs.txt): lattice, counters, energy and A-cluster
histogram bit for bit, in both store packings, without running the oracle."""
import numpy as np
import pytest

from _golden import oracle_cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1309_4349_gb300 as klmc  # noqa: E402

klmc.build()
CASES = oracle_cases()


@pytest.mark.parametrize("packing", [klmc.PACK_BIT, klmc.PACK_BYTE])
@pytest.mark.parametrize("c", CASES, ids=lambda c: f"g{c['geometry']}b{c['boundary']}_{c['Lx']}x{c['Ly']}")
def test_cuda_path_matches_stored_run(c, packing):
    lat = klmc.Lattice(c["Lx"], c["Ly"], geometry=c["geometry"], boundary=c["boundary"], packing=packing,
                       n_A=c["n_A"], omega_over_kT=c["omega_over_kT"], seed=c["seed"])
    try:
        lat.sweep(c["mcs"])
        assert np.array_equal(lat.get_lattice(), c["lattice"])
        k = lat.counters()
        assert (k["attempts"], k["unlike"], k["draws"], k["accepts"]) == (c["attempts"], c["unlike"], c["draws"],
                                                                          c["accepts"])
        assert lat.energy()[0] == c["n_unlike"]
        sizes, counts = lat.cluster_histogram(1)
        assert np.array_equal(np.asarray(sizes), c["hist_A"][0]) and np.array_equal(np.asarray(counts),
                                                                                     c["hist_A"][1])
    finally:
        lat.close()

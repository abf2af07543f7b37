"""C-ABI checks that need no GPU: the library builds, loads, exports every entry
point declared in include/klmc.h, and rejects invalid arguments before touching
the device."""
import ctypes
import os
import re

import pytest

import paper_1309_4349_gb300 as klmc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    klmc.build()
    return klmc.lib()


def declared_functions():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(klmc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("klmc_create", "klmc_sweep", "klmc_energy", "klmc_cluster_histogram",
                     "klmc_destroy", "klmc_batch_create", "klmc_batch_sweep"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    for code, name in klmc.STATUS.items():
        assert L.klmc_status_str(code).decode() == name


def test_params_default(L):
    p = klmc.Params()
    assert L.klmc_params_default(ctypes.byref(p)) == 0
    assert (p.Lx, p.Ly, p.geometry, p.packing, p.n_A) == (64, 64, klmc.TRI6, klmc.PACK_BIT, -1)


@pytest.mark.parametrize("field,value", [("Lx", 3), ("Ly", 2), ("geometry", 7), ("packing", 9),
                                         ("boundary", 1), ("boundary", 2), ("n_A", 64 * 64 + 1), ("threads", 64),
                                         ("cluster", 17), ("cluster", -2),
                                         ("omega_over_kT", float("nan")),
                                         ("omega_over_kT", float("inf"))])
def test_create_rejects_invalid(L, field, value):
    p = klmc.Params()
    L.klmc_params_default(ctypes.byref(p))
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert L.klmc_create_ex(ctypes.byref(h), ctypes.byref(p)) == 1  # KLMC_EINVAL
    assert h.value is None
    assert L.klmc_last_error().decode() != ""


@pytest.mark.parametrize("Lx,Ly,geometry,cluster", [(10, 7, 1, 0), (11, 7, 0, 0), (10, 8, 0, 0),
                                                     (10, 7, 0, 4)])
def test_create_rejects_invalid_helical(L, Lx, Ly, geometry, cluster):
    """Helical lattices need TRI6, 7 | Lx*Ly, Lx mod 7 in {3, 5} and the per-launch
    path (no cluster)."""
    p = klmc.Params()
    L.klmc_params_default(ctypes.byref(p))
    p.Lx, p.Ly, p.geometry, p.cluster, p.boundary = Lx, Ly, geometry, cluster, klmc.HELICAL
    h = ctypes.c_void_p()
    assert L.klmc_create_ex(ctypes.byref(h), ctypes.byref(p)) == 1
    assert "helical" in L.klmc_last_error().decode()


def test_create_rejects_bad_fraction_and_size(L):
    p = klmc.Params()
    L.klmc_params_default(ctypes.byref(p))
    p.fraction_A = 1.5
    h = ctypes.c_void_p()
    assert L.klmc_create_ex(ctypes.byref(h), ctypes.byref(p)) == 1
    L.klmc_params_default(ctypes.byref(p))
    p.Lx, p.Ly = 65536, 65536
    assert L.klmc_create_ex(ctypes.byref(h), ctypes.byref(p)) == 1


def test_null_arguments(L):
    assert L.klmc_destroy(None) == 0
    assert L.klmc_batch_destroy(None) == 0
    assert L.klmc_sweep(None, 1) == 1
    assert L.klmc_energy(None, None, None) == 1
    assert L.klmc_create(None, 64, 0.5, 0.6, 1) == 1


def test_histogram_averages_host_arithmetic(L):
    """klmc_histogram_averages is host arithmetic only: checked here against exact
    rationals and the oracle's independent implementation, and for its errors."""
    from fractions import Fraction

    import numpy as np

    import oracle

    cases = [([1, 5], [3, 1]), ([7], [11]), ([], []), ([1, 2, 3, 40], [100, 7, 3, 1]),
             ([1, (1 << 31) - 1], [1 << 20, 1])]
    for sizes, counts in cases:
        got = klmc.histogram_averages(sizes, counts)
        assert got == oracle.histogram_averages(sizes, counts)
        c1 = sum(counts)
        s1 = sum(s * c for s, c in zip(sizes, counts))
        s2 = sum(s * s * c for s, c in zip(sizes, counts))
        want = (float(Fraction(s1, c1)) if c1 else 0.0, float(Fraction(s2, s1)) if s1 else 0.0)
        assert got == want
    rng = np.random.default_rng(5)
    for _ in range(20):
        k = int(rng.integers(1, 30))
        sizes = np.sort(rng.choice(np.arange(1, 5000), size=k, replace=False))
        counts = rng.integers(1, 1000, size=k)
        assert klmc.histogram_averages(sizes, counts) == oracle.histogram_averages(sizes, counts)
    for sizes, counts in (([1, -2], [1, 1]), ([1], [-1]), ([1 << 32], [1 << 32])):
        with pytest.raises(klmc.KlmcError) as e:
            klmc.histogram_averages(sizes, counts)
        assert e.value.status == 1

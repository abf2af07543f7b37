"""Snapshot images and the image fraction of first neighbours on the GPU
(section "Image analysis") against the oracle, byte for byte."""
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
@pytest.mark.parametrize("Lx,Ly,boundary,scale,S", [
    (37, 29, klmc.PERIODIC, 1.0, 1), (37, 29, klmc.PERIODIC, 0.5, 4), (64, 64, klmc.PERIODIC, 0.3, 8),
    (402, 399, klmc.HELICAL, 0.25, 4), (10, 7, klmc.HELICAL, 2.0, 3), (400, 400, klmc.PERIODIC, 1.0, 2),
])
def test_snapshot_and_image_ffn_parity(packing, Lx, Ly, boundary, scale, S):
    N = Lx * Ly
    seed = 3 + Ly
    lat = klmc.Lattice(Lx, Ly, packing=packing, n_A=N // 2, omega_over_kT=1.0, seed=seed, boundary=boundary)
    lat.sweep(5)
    t = lat.get_lattice()
    U = oracle.natural_width(Lx, Ly)
    W = max(1, int(round(U * scale)))
    H = max(1, int(round(W * Ly * (3 ** 0.5 / 2) / (U / 2))))
    image, mask = lat.snapshot(W, H, S)
    ref_image, ref_mask = oracle.snapshot(Lx, Ly, t, W, H, S)
    assert np.array_equal(image.cpu().numpy(), ref_image) and np.array_equal(mask.cpu().numpy(), ref_mask)
    for m in (0, 7):
        assert lat.image_ffn(image, mask, 35, m) == oracle.image_ffn(ref_image, ref_mask, 35, seed, m)
    assert lat.image_ffn(image, mask, 0, 1) == oracle.image_ffn(ref_image, ref_mask, 0, seed, 1)


def test_papers_image_agreement_on_the_gpu():
    """Fig. 12's check on a trajectory from a non-random start (A in the lower
    half): at the geometry-preserving natural resolution the image fraction of
    first neighbours agrees with the raw one to 0.1%."""
    Lx, Ly = 400, 399
    N = Lx * Ly
    lat = klmc.Lattice(Lx, Ly, n_A=N // 2, omega_over_kT=1.0, seed=3)
    t = np.array([1 if (i // Lx) < Ly // 2 else 0 for i in range(N)], np.uint8)
    lat.set_lattice(t, 0)
    lat.sweep(200)
    raw = np.mean([lat.ffn(m)[0] for m in range(8)])
    U = oracle.natural_width(Lx, Ly)
    H = int(round(U * Ly * (3 ** 0.5 / 2) / (U / 2)))
    image, mask = lat.snapshot(U, H, 1)
    img = np.mean([s / p for s, p in (lat.image_ffn(image, mask, 35, m) for m in range(8))])
    assert abs(img - raw) < 1e-3


def test_snapshot_rejections():
    lat = klmc.Lattice(64, 64, seed=1)
    buf = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(klmc.KlmcError):
        lat.snapshot(4, 4, 0)
    with pytest.raises(klmc.KlmcError):
        lat.snapshot(4, 4, 65)
    with pytest.raises(klmc.KlmcError):
        lat.image_ffn(buf.view(4, 4), buf.view(4, 4), -1, 0)

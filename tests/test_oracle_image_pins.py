"""Pins for the oracle's snapshot images and their fraction of first neighbours
(section "Image analysis": a pixel per site, the image sloped to keep the
triangular geometry and scaled with supersampling to gray levels; neighbours
compared with a gray-level threshold, delta_col = 35).

Pins: the slope and the pixel count of the lattice region, the conservation of
white pixels at one pixel per half-site, closed-form gray levels of striped
lattices under supersampling, exact expectations of the image estimator on
synthetic images (enumerated pixel by pixel), and the threshold's edge.
"""
import numpy as np
import pytest

import oracle
from _golden import paper_value

MOORE = [(1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]


def _stripes(Lx, Ly):
    return np.array([1 if (i % Lx) % 2 == 0 else 0 for i in range(Lx * Ly)], dtype=np.uint8)


@pytest.mark.parametrize("Lx,Ly", [(10, 6), (7, 9), (31, 14)])
def test_lattice_region_is_the_sloped_parallelogram(Lx, Ly):
    U = oracle.natural_width(Lx, Ly)
    for t, g in ((np.ones(Lx * Ly, np.uint8), 255), (np.zeros(Lx * Ly, np.uint8), 0)):
        image, mask = oracle.snapshot(Lx, Ly, t, U, Ly, 1)
        for j in range(Ly):
            cols = np.nonzero(mask[j])[0]
            assert list(cols) == list(range(j, j + 2 * Lx))  # row j shifted by j half-sites
            assert (image[j, cols] == g).all() and (image[j][mask[j] == 0] == 0).all()


@pytest.mark.parametrize("S", [1, 2, 4])
def test_one_pixel_per_half_site_conserves_white(S):
    """At one pixel per half-site every pixel lies in one site, so every site gives
    exactly two pixels of its colour."""
    Lx, Ly = 23, 17
    t = oracle.init(Lx, Ly, 150, 3)
    image, mask = oracle.snapshot(Lx, Ly, t, oracle.natural_width(Lx, Ly), Ly, S)
    assert set(np.unique(image[mask == 1])) <= {0, 255}
    assert int((image == 255).sum()) == 2 * int(t.sum())
    assert int(mask.sum()) == 2 * Lx * Ly


def test_supersampled_stripes_have_closed_form_gray():
    """Stripes of A on even x, two half-sites per pixel (Ly odd makes U even): rows
    with even y are pure (255, 0, 255, ...), rows with odd y straddle two sites of
    each colour and are mid-gray (255/2 rounds to 128)."""
    Lx, Ly, S = 10, 7, 8
    U = oracle.natural_width(Lx, Ly)
    assert U % 2 == 0
    image, mask = oracle.snapshot(Lx, Ly, _stripes(Lx, Ly), U // 2, Ly, S)
    for j in range(Ly):
        for i in range(U // 2):
            u0 = 2 * i  # the pixel covers half-sites [u0, u0 + 2)
            if not (u0 >= j + 1 and u0 + 2 <= j + 2 * Lx - 1):
                continue  # pixels near the slanted edges are partly outside
            if j % 2 == 0:
                x = (u0 - j) // 2
                assert image[j, i] == (255 if x % 2 == 0 else 0)
            else:
                assert image[j, i] == 128


def _expected_similar(image, mask, delta):
    H, W = image.shape
    e = 0.0
    for j in range(H):
        for i in range(W):
            if not mask[j, i]:
                continue
            ok = 0
            for di, dj in MOORE:
                a, b = i + di, j + dj
                if 0 <= a < W and 0 <= b < H and mask[b, a] and abs(int(image[j, i]) - int(image[b, a])) <= delta:
                    ok += 1
            e += ok / 8.0
    return e


@pytest.mark.parametrize("kind", ["uniform", "checker", "rows35"])
def test_image_estimator_expectation(kind):
    """Mean over samples of the similar count equals the expectation enumerated
    pixel by pixel (each pixel's similar neighbours over eight), within 5 sigma."""
    H, W = 24, 30
    jj, ii = np.mgrid[0:H, 0:W]
    if kind == "uniform":
        image = np.full((H, W), 200, np.uint8)
    elif kind == "checker":
        image = np.where((ii + jj) % 2 == 0, 255, 0).astype(np.uint8)
    else:
        image = np.where(jj % 2 == 0, 0, 35).astype(np.uint8)
    mask = np.ones((H, W), np.uint8)
    mask[0, :5] = 0  # a ragged lattice edge
    e = _expected_similar(image, mask, 35)
    c = np.array([oracle.image_ffn(image, mask, 35, 5, m)[0] for m in range(600)], dtype=float)
    assert oracle.image_ffn(image, mask, 35, 5, 0)[1] == int(mask.sum())
    assert abs(c.mean() - e) < 5 * c.std(ddof=1) / np.sqrt(len(c)) + 1e-9


def test_threshold_edge():
    """Rows alternating between gray 0 and 35: with delta = 35 every neighbour is
    similar, with delta = 34 only the two in the same row."""
    H, W = 20, 20
    image = np.where(np.mgrid[0:H, 0:W][0] % 2 == 0, 0, 35).astype(np.uint8)
    mask = np.ones((H, W), np.uint8)
    for delta, frac in ((35, None), (34, 2 / 8)):
        c = np.mean([oracle.image_ffn(image, mask, delta, 9, m)[0] for m in range(300)])
        e = _expected_similar(image, mask, delta)
        assert abs(c - e) < 0.03 * e
        if frac:
            interior = (H - 2) * (W - 2)
            assert _expected_similar(image[1:-1, 1:-1].copy(), np.ones((H - 2, W - 2), np.uint8), delta) \
                == pytest.approx(interior * frac, rel=0.2)


def test_papers_image_ffn_agreement_at_natural_resolution():
    """The paper's check (section "Results", Fig. 12): on a trajectory from a
    non-random start (A in the lower half) the fraction of first neighbours from
    the image agrees with the raw one to 0.1%.  Here at one pixel per half-site
    and sqrt(3) pixels per row (the geometry-preserving natural resolution), one
    sample per pixel; supersampled at this resolution, pixels that straddle two
    rows turn gray wherever the rows differ and the difference grows to 0.2%."""
    Lx, Ly = 200, 199
    N = Lx * Ly
    t = np.array([1 if (i // Lx) < Ly // 2 else 0 for i in range(N)], np.uint8)
    r = oracle.run(Lx, Ly, oracle.TRI6, 1.0, 3, t, 0, 40)
    raw = np.mean([oracle.ffn_count(Lx, Ly, oracle.TRI6, r.lattice, 3, m) for m in range(8)]) / N
    U = oracle.natural_width(Lx, Ly)
    H = int(round(U * Ly * (3 ** 0.5 / 2) / (U / 2)))
    image, mask = oracle.snapshot(Lx, Ly, r.lattice, U, H, 1)
    delta = paper_value("delta_col")
    img = np.mean([s / p for s, p in (oracle.image_ffn(image, mask, delta, 3, m) for m in range(8))])
    assert abs(img - raw) < paper_value("image_ffn_max_diff")

"""The seeded input generators that the oracle checks, the GPU tests and bench.py share: a
(generator, n, d, seed) tuple names one point set, with the shapes the input recipe states."""
import numpy as np
import pytest

import synthdata


@pytest.mark.parametrize("kind", ["uniform", "gmm", "varden"])
def test_same_seed_same_points_other_seed_other_points(kind):
    a = synthdata.generate(kind, 2000, 3, seed=5)
    b = synthdata.generate(kind, 2000, 3, seed=5)
    c = synthdata.generate(kind, 2000, 3, seed=6)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.shape == (2000, 3) and a.flags["C_CONTIGUOUS"]


def test_default_dtypes_and_override():
    assert synthdata.generate("uniform", 10, 2).dtype == np.float64
    assert synthdata.generate("gmm", 10, 2).dtype == np.float32
    assert synthdata.generate("varden", 10, 2).dtype == np.float32
    assert synthdata.generate("uniform", 10, 2, dtype=np.float32).dtype == np.float32
    with pytest.raises(ValueError):
        synthdata.generate("no-such-generator", 10, 2)


def test_uniform_fills_the_unit_cube():
    x = synthdata.uniform(100_000, 4, seed=1)
    assert x.min() >= 0.0 and x.max() < 1.0
    # each coordinate's mean within 6 standard errors of 1/2 (sd of U[0,1) = 1/sqrt(12))
    assert np.all(np.abs(x.mean(axis=0) - 0.5) < 6 / np.sqrt(12 * 100_000))


def test_gaussian_mixture_noise_and_box():
    n = 200_000
    x = synthdata.gaussian_mixture(n, 3, seed=2).astype(np.float64)
    # 5% of the points are uniform over the box; the clusters' centres lie in it too, and their
    # sigmas are at most 5, so nearly every point is within the box widened by a few sigma
    inside = np.all((x > -25.0) & (x < 125.0), axis=1)
    assert inside.mean() > 0.999
    # continuous draws: no two points coincide
    assert len(np.unique(x, axis=0)) == n


def test_varden_blobs_span_densities():
    n = 200_000
    x = synthdata.varden_blobs(n, 2, seed=3).astype(np.float64)
    assert np.all(np.isfinite(x))
    # Zipf(1.1) sizes over 1000 blobs: the largest blob holds about 1/H share (H = sum r^-1.1),
    # so a fine grid has some very dense cells and many nearly empty ones
    h, _, _ = np.histogram2d(x[:, 0], x[:, 1], bins=256, range=[[0, 1], [0, 1]])
    occupied = h[h > 0]
    assert occupied.max() / np.median(occupied) > 100


def test_collinear_and_unit_grid_are_exact():
    x = synthdata.collinear(50, 3, seed=4)
    assert np.array_equal(np.sort(x[:, 0]), np.arange(50.0))
    assert np.all(x[:, 1:] == 0.0)
    g = synthdata.unit_grid(5, 3, seed=4)
    assert g.shape == (125, 3)
    assert len(np.unique(g, axis=0)) == 125
    assert g.min() == 0.0 and g.max() == 4.0
    # seeded row order: another seed permutes the same set
    g2 = synthdata.unit_grid(5, 3, seed=9)
    assert not np.array_equal(g, g2)
    assert np.array_equal(np.unique(g, axis=0), np.unique(g2, axis=0))

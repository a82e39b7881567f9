"""Seeded synthetic point-set generators shared by the tests, the oracle checks and bench.py.

This module holds no arithmetic of the method (no distances, trees or spanning trees): it only
draws coordinates.  Every generator uses numpy's PCG64 bit generator
(``numpy.random.Generator(numpy.random.PCG64(seed))``), so a (generator, n, d, seed) tuple names
one point set on any machine with numpy >= 1.17.

The shapes stand in for the paper's synthetic workloads (Sec. 5, "Data Sets"):
UniformFill (points i.i.d. uniform in a hypercube) and SS-varden (seed-spreader clusters of
varying density).  The SS-varden generator itself is not available, so ``varden_blobs`` draws
Gaussian blobs whose widths span three decades and whose sizes follow a Zipf law instead.

All generators return a C-contiguous array of shape (n, d) (array-of-structs, row per point).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform",
    "gaussian_mixture",
    "varden_blobs",
    "collinear",
    "unit_grid",
    "generate",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform(n: int, d: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """n points i.i.d. uniform in [0,1)^d (UniformFill up to scale)."""
    x = _rng(seed).random((n, d), dtype=np.float64)
    return np.ascontiguousarray(x.astype(dtype))


def gaussian_mixture(n: int, d: int = 3, seed: int = 0, n_comp: int = 50, box: float = 100.0,
                     sigma_lo: float = 0.1, sigma_hi: float = 5.0, noise_frac: float = 0.05,
                     dtype=np.float32) -> np.ndarray:
    """Mixture of ``n_comp`` isotropic Gaussians plus uniform background noise.

    Centres uniform in [0, box)^d, sigmas log-uniform in [sigma_lo, sigma_hi], mixture weights
    Dirichlet(1), component counts multinomial over (1 - noise_frac) n, and the remaining points
    uniform in [0, box)^d.  Rows are shuffled so that the input order carries no cluster structure.
    """
    g = _rng(seed)
    n_noise = int(round(noise_frac * n))
    n_clu = n - n_noise
    centres = g.random((n_comp, d)) * box
    sigmas = np.exp(g.uniform(np.log(sigma_lo), np.log(sigma_hi), n_comp))
    weights = g.dirichlet(np.ones(n_comp))
    counts = g.multinomial(n_clu, weights)
    parts = [centres[c] + sigmas[c] * g.standard_normal((counts[c], d)) for c in range(n_comp)]
    parts.append(g.random((n_noise, d)) * box)
    x = np.concatenate(parts, axis=0)
    x = x[g.permutation(n)]
    return np.ascontiguousarray(x.astype(dtype))


def varden_blobs(n: int, d: int, seed: int = 0, n_blobs: int = 1000, sigma_lo: float = 1e-4,
                 sigma_hi: float = 1e-1, zipf_s: float = 1.1, dtype=np.float32) -> np.ndarray:
    """Variable-density clusters: ``n_blobs`` Gaussian blobs in [0,1)^d.

    Centres uniform in [0,1)^d; sigmas log-uniform over [sigma_lo, sigma_hi] (three decades by
    default); the blob of rank r gets a share proportional to r^-zipf_s of the n points (largest
    remainders rounding so the counts sum to n).  Rows are shuffled.
    """
    g = _rng(seed)
    centres = g.random((n_blobs, d))
    sigmas = np.exp(g.uniform(np.log(sigma_lo), np.log(sigma_hi), n_blobs))
    w = np.arange(1, n_blobs + 1, dtype=np.float64) ** (-zipf_s)
    w /= w.sum()
    raw = w * n
    counts = np.floor(raw).astype(np.int64)
    rem = n - int(counts.sum())
    if rem > 0:
        counts[np.argsort(-(raw - counts), kind="stable")[:rem]] += 1
    parts = [centres[b] + sigmas[b] * g.standard_normal((counts[b], d)) for b in range(n_blobs)]
    x = np.concatenate(parts, axis=0)
    x = x[g.permutation(n)]
    return np.ascontiguousarray(x.astype(dtype))


def collinear(n: int, d: int = 2, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """n unit-spaced points on the first axis, in a seeded random order."""
    x = np.zeros((n, d), dtype=np.float64)
    x[:, 0] = np.arange(n, dtype=np.float64)
    x = x[_rng(seed).permutation(n)]
    return np.ascontiguousarray(x.astype(dtype))


def unit_grid(k: int, d: int = 2, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """The k^d points of the unit grid {0..k-1}^d, in a seeded random order."""
    axes = [np.arange(k, dtype=np.float64)] * d
    x = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, d)
    x = x[_rng(seed).permutation(x.shape[0])]
    return np.ascontiguousarray(x.astype(dtype))


def generate(kind: str, n: int, d: int, seed: int = 0, dtype=None) -> np.ndarray:
    """Dispatch by name: 'uniform', 'gmm' (gaussian_mixture), 'varden' (varden_blobs)."""
    if kind == "uniform":
        return uniform(n, d, seed, dtype=dtype or np.float64)
    if kind == "gmm":
        return gaussian_mixture(n, d, seed, dtype=dtype or np.float32)
    if kind == "varden":
        return varden_blobs(n, d, seed, dtype=dtype or np.float32)
    raise ValueError(f"unknown generator {kind!r}")

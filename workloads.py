"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds no arithmetic of the method: it only draws point sets
y_j in [0, 2 pi) and coefficient vectors c_n, with numpy's Philox
generator, in the shapes and distributions of the paper's experiments
(Sec. 3: uniform random y for the forward transform, y perturbed around
the grid for the inverse) and of the workloads this library is measured on:

* ``uniform``    y_j iid U[0, 2 pi)
* ``jitter``     y_j = 2 pi j / N + U(-a, a) 2 pi / N, wrapped (a = 0.1 is the
                 paper's 10 % perturbation; a = 0.4 the 40 % variant)
* ``clustered``  wrapped mixture of 8 Gaussians, sigma = 0.05, centres U[0, 2 pi)
* ``contrast``   wrapped mixture of 8 Gaussians (sigma = 0.1) plus a uniform
                 floor whose weight gives a 1:100 min/max density ratio on a
                 4096-bin histogram of the analytic density
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi  # binary64 2 pi, below the true value


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _wrap(y: np.ndarray) -> np.ndarray:
    y = np.mod(y, TWO_PI)
    # np.mod can return exactly TWO_PI for tiny negative inputs; fold it to 0
    y[y >= TWO_PI] = 0.0
    y[y < 0.0] = 0.0
    return y


def points(kind: str, M: int, N: int | None = None, seed: int = 1234,
           jitter: float = 0.4) -> np.ndarray:
    """M points in [0, 2 pi) of the named distribution (float64)."""
    g = rng(seed)
    if kind == "uniform":
        return g.random(M) * TWO_PI
    if kind == "jitter":
        if N is None or N != M:
            raise ValueError("jitter needs M == N")
        j = np.arange(M, dtype=np.float64)
        return _wrap((j + g.uniform(-jitter, jitter, M)) * (TWO_PI / N))
    if kind == "clustered":
        centres = g.random(8) * TWO_PI
        comp = g.integers(0, 8, M)
        return _wrap(centres[comp] + 0.05 * g.standard_normal(M))
    if kind == "contrast":
        return _contrast(g, M)
    if kind == "multiscale":
        # four Gaussian clusters of widths 0.004 .. 0.15 rad and a uniform
        # background, a fifth of the points each: densities from the mean to
        # about 30x it
        widths = np.array([0.004, 0.02, 0.06, 0.15])
        comp = g.integers(0, 5, M)
        ctr = g.random(4) * TWO_PI
        k = np.minimum(comp, 3)
        y = np.where(comp < 4, ctr[k] + widths[k] * g.standard_normal(M), g.random(M) * TWO_PI)
        return _wrap(y)
    raise ValueError(kind)


def _mixture_density(x, centres, sigma):
    d = np.zeros_like(x)
    for c in centres:
        for k in (-1, 0, 1):
            d += np.exp(-0.5 * ((x - c + k * TWO_PI) / sigma) ** 2)
    return d / (len(centres) * sigma * math.sqrt(TWO_PI))


def _contrast(g: np.random.Generator, M: int, sigma: float = 0.1, ratio: float = 100.0):
    centres = g.random(8) * TWO_PI
    x = (np.arange(4096) + 0.5) * (TWO_PI / 4096)
    d = _mixture_density(x, centres, sigma)
    u = 1.0 / TWO_PI
    # density (1-w) d + w u ; choose w so that min/max = 1/ratio
    lo, hi = 0.0, 1.0
    for _ in range(200):
        w = 0.5 * (lo + hi)
        dens = (1 - w) * d + w * u
        if dens.min() / dens.max() < 1.0 / ratio:
            lo = w
        else:
            hi = w
    w = hi
    is_floor = g.random(M) < w
    comp = g.integers(0, 8, M)
    y = centres[comp] + sigma * g.standard_normal(M)
    y = np.where(is_floor, g.random(M) * TWO_PI, y)
    return _wrap(y)


def coeffs(N: int, seed: int = 99, dtype=np.complex128) -> np.ndarray:
    """c_n with real and imaginary parts iid N(0, 1)."""
    g = rng(seed)
    c = g.standard_normal(N) + 1j * g.standard_normal(N)
    return c.astype(dtype)


def samples(M: int, seed: int = 77, dtype=np.complex128) -> np.ndarray:
    """Non-uniform samples g_j with iid N(0, 1) parts (adjoint inputs)."""
    return coeffs(M, seed, dtype)


def sample_index(M: int, count: int = 4096, seed: int = 1234) -> np.ndarray:
    """Sorted target subset used when the O(NM) oracle cannot cover all of M."""
    if M <= count:
        return np.arange(M, dtype=np.int64)
    return np.sort(rng(seed).choice(M, size=count, replace=False)).astype(np.int64)

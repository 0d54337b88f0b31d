"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only draws random numbers
(numpy PCG64) in the shapes the workloads need.  Both the CUDA path and the
oracle receive the same arrays and do their own arithmetic on them.
"""
from __future__ import annotations

import itertools

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_vector(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float64 array uniform in [lo, hi), C order."""
    return rng(seed).uniform(lo, hi, size=shape)


def _wavevectors(kmax: float):
    r = int(np.floor(kmax))
    ks = [k for k in itertools.product(range(-r, r + 1), repeat=3)
          if 1.0 <= np.sqrt(k[0] ** 2 + k[1] ** 2 + k[2] ** 2) <= kmax]
    return np.array(ks, dtype=np.float64)


def fourier_modes(seed: int, nmodes: int = 8, kmax: float = 3.0) -> np.ndarray:
    """Rows (a_m, k1, k2, k3, phi_m) of a random Fourier field
    g(x) = sum_m a_m cos(2 pi k_m . x + phi_m): a_m ~ U[-1, 1],
    phi_m ~ U[0, 2 pi), k_m uniform over the integer vectors with
    1 <= |k| <= kmax."""
    g = rng(seed)
    ks = _wavevectors(kmax)
    a = g.uniform(-1.0, 1.0, size=nmodes)
    idx = g.integers(0, len(ks), size=nmodes)
    ph = g.uniform(0.0, 2.0 * np.pi, size=nmodes)
    return np.column_stack([a, ks[idx], ph])


def batch_patches(count: int = 64, seed: int = 0, p_range=(2, 6), nel_range=(16, 96)):
    """Degrees and element counts of uneven patches: p uniform in p_range,
    elements per direction uniform in nel_range independently per axis.
    Returns a list of (p, (nel1, nel2, nel3))."""
    g = rng(seed)
    out = []
    for _ in range(count):
        p = int(g.integers(p_range[0], p_range[1] + 1))
        nel = tuple(int(v) for v in g.integers(nel_range[0], nel_range[1] + 1, size=3))
        out.append((p, nel))
    return out


def open_uniform_knots(p: int, nel: int) -> np.ndarray:
    """Open knot vector of degree p with nel equal spans on [0, 1]."""
    return np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, nel + 1), np.ones(p)])


def jittered_knots(p: int, nel: int, seed: int, amount: float = 0.3) -> np.ndarray:
    """Open knot vector whose break points k/nel are moved by up to amount/nel."""
    g = rng(seed)
    u = np.arange(1, nel) / nel + g.uniform(-amount, amount, size=nel - 1) / nel
    return np.concatenate([np.zeros(p + 1), u, np.ones(p + 1)])

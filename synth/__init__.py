"""Seeded synthetic inputs shared by the oracle tests and the CUDA-path tests.

Holds no arithmetic of the method: it only draws random numbers (start vectors and
workload parameters) from numpy's PCG64 generator.  Both sides receive the same
arrays, so a comparison between them is a comparison of the method alone.
"""
from __future__ import annotations

import numpy as np


def unit_phase_vectors(n: int, R: int, seed: int) -> np.ndarray:
    """[R][n] complex128 start vectors with unit modulus and uniform phase."""
    g = np.random.Generator(np.random.PCG64(seed))
    phi = g.random((R, n)) * (2.0 * np.pi)
    return np.cos(phi) + 1j * np.sin(phi)


def gaussian_vectors(n: int, R: int, seed: int) -> np.ndarray:
    """[R][n] complex128 start vectors with independent standard normal parts."""
    g = np.random.Generator(np.random.PCG64(seed))
    return (g.standard_normal((R, n)) + 1j * g.standard_normal((R, n))) / np.sqrt(2.0)


def batched_square_systems(count: int, seed: int, L_lo=64, L_hi=1024, W_hi=4.0,
                           Ms=(512, 1024, 2048, 4096)):
    """Workload of many independent square-lattice systems: side L uniform in
    [L_lo, L_hi], Anderson width W uniform in [0, W_hi], M drawn from Ms."""
    g = np.random.Generator(np.random.PCG64(seed))
    L = g.integers(L_lo, L_hi + 1, size=count)
    W = g.random(count) * W_hi
    M = g.choice(np.asarray(Ms), size=count)
    seeds = g.integers(1, 2**62, size=count)
    return [dict(L=int(L[i]), W=float(W[i]), M=int(M[i]), seed=int(seeds[i])) for i in range(count)]

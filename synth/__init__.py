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


def learned_dos_systems(count: int, first_seed: int, L: int = 256, delta_hi=1.0, W_hi=4.0,
                        p_hi=0.02):
    """Training / held-out systems of the learned reconstruction: honeycomb L x L with
    staggered potential Delta uniform in [0, delta_hi] eV, Anderson width W uniform in
    [0, W_hi] eV and vacancy fraction uniform in [0, p_hi]; sample i draws its parameters
    from PCG64(first_seed + i) and uses first_seed + i as its disorder / phase seed."""
    out = []
    for i in range(count):
        g = np.random.Generator(np.random.PCG64(first_seed + i))
        d, w, p = g.random(3)
        out.append(dict(L=int(L), delta=float(d * delta_hi), W=float(w * W_hi), p_vac=float(p * p_hi),
                        seed=int(first_seed + i)))
    return out


def mlp_init(seed: int, n_in=128, n_hid=512, n_out=1024, head_scale=1.0) -> np.ndarray:
    """Initial parameters of the IN -> H -> H -> OUT perceptron as one flat float32 vector
    (W1[H][IN], b1, W2[H][H], b2, W3[OUT][H], b3): He-uniform weights with limit
    sqrt(6 / fan_in), zero biases, the last layer's weights multiplied by head_scale (a small
    value starts a residual network close to its prior)."""
    g = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for k, (rows, cols) in enumerate(((n_hid, n_in), (n_hid, n_hid), (n_out, n_hid))):
        lim = np.sqrt(6.0 / cols) * (head_scale if k == 2 else 1.0)
        parts.append(g.uniform(-lim, lim, size=rows * cols))
        parts.append(np.zeros(rows))
    return np.concatenate(parts).astype(np.float32)

"""Seeded synthetic inputs shared by the oracle and the CUDA path in tests.

Holds none of the method's arithmetic: it only draws random numbers with numpy's PCG64 and shapes
them like the paper's workloads (Kelvin-Helmholtz perturbation parameters; positive-density,
positive-internal-energy conserved states).
"""
import math

import numpy as np


def kh_theta(B: int, seed: int, P: int = 20) -> np.ndarray:
    """[B, P] KH parameters: first half amplitudes ~ U(0,1), second half phases ~ U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 1.0, (B, P // 2))
    b = rng.uniform(0.0, 2.0 * math.pi, (B, P // 2))
    return np.concatenate([a, b], axis=1)


def euler_state(B: int, ndim: int, n, seed: int, smooth: bool = True) -> np.ndarray:
    """[B, ndim+2, nz, ny, nx] conserved states with rho in [0.6, 1.6], |m|/rho <= 0.6 and an
    internal energy in [1.5, 3.5] added to the kinetic energy (so every cell is physical)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (list(n) + [1, 1])[:3]
    shape = (B, nz, ny, nx)

    def field(lo, hi):
        if not smooth:
            return rng.uniform(lo, hi, shape)
        # a few random Fourier modes: smooth, periodic
        x = np.arange(nx) / nx
        y = np.arange(ny) / ny
        z = np.arange(nz) / nz
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        f = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 3, 3)
            ph = rng.uniform(0, 2 * math.pi, (B, 1, 1, 1))
            f += np.sin(2 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + ph)
        f = (f - f.min()) / (f.max() - f.min() + 1e-300)
        return lo + (hi - lo) * f

    rho = field(0.6, 1.6)
    U = np.zeros((B, ndim + 2, nz, ny, nx))
    U[:, 0] = rho
    ke = np.zeros(shape)
    for k in range(ndim):
        m = rho * field(-0.6, 0.6)
        U[:, 1 + k] = m
        ke += 0.5 * m * m / rho
    U[:, ndim + 1] = ke + field(1.5, 3.5)
    return U


def burgers_state(B: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    U = np.zeros((B, 1, 1, 1, n))
    for b in range(B):
        for _ in range(3):
            U[b, 0, 0, 0] += rng.uniform(-0.5, 0.5) * np.sin(2 * math.pi * rng.integers(1, 4) * x + rng.uniform(0, 6))
    return U

"""Seeded synthetic inputs shared by the oracle tests and the GPU parity
tests.  Random numbers only: nothing here evaluates any part of the lattice
Boltzmann scheme (no equilibria, no closures, no fields)."""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_populations(seed: int, K: int, Q: int, ncell: int, base, amp) -> np.ndarray:
    """f[k, i, c] = (base[k] + amp[k] * r) / Q with r uniform in [-1, 1)."""
    g = rng(seed)
    base = np.asarray(base, dtype=np.float64).reshape(K, 1, 1)
    amp = np.asarray(amp, dtype=np.float64).reshape(K, 1, 1)
    r = g.uniform(-1.0, 1.0, size=(K, Q, ncell))
    return (base + amp * r) / Q


def random_fields(seed: int, ncell: int, amp: float) -> tuple[np.ndarray, np.ndarray]:
    g = rng(seed)
    E = amp * g.uniform(-1.0, 1.0, size=(3, ncell))
    B = amp * g.uniform(-1.0, 1.0, size=(3, ncell))
    return E, B


def uniform(seed: int, size, lo: float, hi: float) -> np.ndarray:
    return rng(seed).uniform(lo, hi, size=size)


def batch_draws(nruns: int = 64, seed: int = 2309) -> list[dict]:
    """Parameter draws of the uneven-grid sweep: n_z in {256, ..., 1024},
    n_x in {256, ..., 512} (steps of 32), mu log-uniform in [1e-4, 5e-2],
    alpha uniform in [0.01, 1], sigma_z uniform in [0.5, 2], closure coin."""
    g = rng(seed)
    out = []
    for _ in range(nruns):
        nz = int(g.integers(0, (1024 - 256) // 32 + 1)) * 32 + 256
        nx = int(g.integers(0, (512 - 256) // 32 + 1)) * 32 + 256
        mu = float(np.exp(g.uniform(np.log(1e-4), np.log(5e-2))))
        alpha = float(g.uniform(0.01, 1.0))
        sz = float(g.uniform(0.5, 2.0))
        closure = "warmc" if g.uniform() < 0.5 else "lec"
        out.append(dict(nz=nz, nx=nx, mu=mu, alpha=alpha, sigma_z=sz, closure=closure))
    return out

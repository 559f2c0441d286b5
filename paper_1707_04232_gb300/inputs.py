"""Seeded synthetic initial states for SDPD runs.

This module only draws inputs; it holds none of the integrator's arithmetic.
Both the CUDA library and the FP64 oracle are fed the arrays it returns, so
neither side generates its own initial state.

Recipe (the paper's Section 4 set-up, in the reduced units a, m, kT):

* positions: a simple-cubic lattice of n^3 sites with spacing a, site
  (ix, iy, iz) at ((ix + 1/2) a, ...) plus a uniform jitter in
  [-jitter*a, +jitter*a) per axis; particle id = ix + n (iy + n iz);
* momenta: Gaussian with variance m kT per component (Boltzmann
  distribution), mean momentum subtracted so that the total momentum is 0;
* internal energies: every particle at temperature T0. The ideal-gas
  equation of state (Eq. pg-eos) gives T = eps / C_K with
  C_K = 3/2 (K - 1) kB, so eps_i = C_K T0 for all i.

All arrays are float64, C-contiguous, indexed by particle id:
q[N,3], p[N,3], eps[N].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One synthetic fluid: an n^3 lattice in a periodic cube of side n*a."""

    n: int                 # lattice sites per axis
    a: float = 1.0         # lattice spacing
    m: float = 1.0         # particle mass
    h: float = 2.5         # smoothing length (cut-off radius) in units of a
    kT: float = 1.0        # initial temperature (kB = 1)
    K: float = 100.0       # particle size K = m / m0 (sets C_K)
    jitter: float = 0.05   # uniform jitter amplitude, in units of a
    seed: int = 0

    @property
    def N(self) -> int:
        return self.n ** 3

    @property
    def L(self) -> float:
        return self.n * self.a


def lattice_state(w: Workload, kB: float = 1.0):
    """Return (q, p, eps) for workload ``w`` as float64 arrays."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    n = w.n
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    sites = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    q = (sites + 0.5) * w.a + rng.uniform(-w.jitter * w.a, w.jitter * w.a, size=sites.shape)
    L = w.L
    q = np.where(q >= L, q - L, q)
    q = np.where(q < 0.0, q + L, q)
    p = rng.normal(0.0, np.sqrt(w.m * w.kT), size=sites.shape)
    p -= p.mean(axis=0, keepdims=True)
    C_K = 1.5 * (w.K - 1.0) * kB
    eps = np.full(w.N, C_K * w.kT, dtype=np.float64)
    return np.ascontiguousarray(q), np.ascontiguousarray(p), eps


def random_box_state(N: int, L: float, m: float, kT: float, eps0: float, seed: int):
    """Uniformly random positions in [0, L)^3 (a disordered fluid sample)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.uniform(0.0, L, size=(N, 3))
    q = np.where(q >= L, 0.0, q)
    p = rng.normal(0.0, np.sqrt(m * kT), size=(N, 3))
    p -= p.mean(axis=0, keepdims=True)
    eps = np.full(N, eps0, dtype=np.float64)
    return np.ascontiguousarray(q), np.ascontiguousarray(p), eps


# Named workloads, by what they are.
SMALL_LUCY_1000 = Workload(n=10, K=100.0, kT=1.0)          # N=1000, L=10
FLUID_32K = Workload(n=32, K=100.0, kT=1.0)                  # N=32,768, L=32
FLUID_131K_K100 = Workload(n=64, K=100.0, kT=1.0)            # N=131,072, L=64
FLUID_131K_K5_COLD = Workload(n=64, K=5.0, kT=0.1)           # stress case
FLUID_2M = Workload(n=128, K=50.0, kT=1.0)                   # N=2,097,152, L=128

"""Parity at the benchmark's full size, in its launch configuration.

The benchmark workload is the single large fluid: N = 128^3 = 2,097,152
particles on a jittered simple-cubic lattice (L = 128), Lucy kernel
h = 2.5a, kT = 1, K = 50, dt = 0.005, EMS.  The O(N^2) oracle cannot run it
whole, so outputs it can compute one particle at a time are compared on a
seeded sample (density, force, neighbour count by brute force over all N),
binning and storage order are compared for every particle, and the rest is
checked through properties that hold at any size.
"""
import numpy as np
import pytest

import oracle as O
from paper_1707_04232_gb300.inputs import Workload, lattice_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1707_04232_gb300 import sdpd  # noqa: E402

W = Workload(n=128, K=50.0, kT=1.0)


@pytest.fixture(scope="module")
def state():
    return lattice_state(W)


def sample(n, seed):
    rng = np.random.default_rng(seed)
    idx = np.concatenate([[0, W.N - 1], rng.choice(W.N, n - 2, replace=False)])
    return np.sort(idx)


def handle(precision, **kw):
    return sdpd.SDPD(W.N, W.L, m=W.m, h=W.h, K=W.K, precision=precision, **kw)


def test_fullsize_fp64_binning_and_sampled_pairs(state):
    q, p, e = state
    P = O.Config(N=W.N, L=W.L, K=W.K).params()
    s = handle(sdpd.FP64)
    s.set_state(q, p, e)
    assert (s.cells() == O.cells(P, q)).all()
    assert (s.order() == O.sorted_order(P, q)).all()
    idx = sample(24, 1)
    assert (s.neighbour_counts()[idx] == O.neighbour_count_at(P, q, idx)).all()
    rho_o = O.density_at(P, q, idx)
    assert np.abs(s.density()[idx] - rho_o).max() <= 1e-12 * rho_o.max()
    fidx = idx[:8]
    f_o = O.forces_at(P, q, e, fidx)
    f_g = s.forces()
    assert np.abs(f_g[fidx] - f_o).max() <= 1e-12 * np.abs(f_g).max()


def test_fullsize_mixed_sampled_density_and_force(state):
    q, p, e = state
    P = O.Config(N=W.N, L=W.L, K=W.K).params()
    s = handle(sdpd.MIXED)
    s.set_state(q, p, e)
    idx = sample(24, 2)
    rho_o = O.density_at(P, q, idx)
    rho_g = s.density()
    assert np.abs(rho_g[idx] - rho_o).max() <= 1e-5 * rho_g.max()
    fidx = idx[:8]
    f_o = O.forces_at(P, q, e, fidx)
    f_g = s.forces()
    assert np.abs(f_g[fidx] - f_o).max() <= 1e-5 * np.abs(f_g).max()


def test_fullsize_mixed_steps_invariants(state):
    """Three benchmark steps: no device error, momentum conserved, energy
    changed only by the Verlet error, every internal energy positive, one
    sweep per step over about half the neighbour count per particle."""
    q, p, e = state
    s = handle(sdpd.MIXED)
    s.set_state(q, p, e)
    o0 = s.observables()
    s.step(0.005, 3, seed=1234)
    o1 = s.observables()
    assert o1["status"] == 0 and o1["fd_step"] == 3 and o1["vv_step"] == 3
    assert np.abs(o1["P"] - o0["P"]).max() < 1e-2  # float32 momenta, 2M particles
    assert abs(o1["E"] - o0["E"]) < 1e-6 * o0["E"]
    assert o1["eps_min"] > 0.0
    per_particle = o1["n_pairs"] / (3 * W.N)
    assert 30.0 < per_particle < 45.0
    assert o1["n_reject_bound"] + o1["n_reject_metropolis"] < 1e-2 * o1["n_pairs"]


def test_fullsize_mixed_fd_only_conserves_energy(state):
    q, p, e = state
    s = handle(sdpd.MIXED, fd_only=True)
    s.set_state(q, p, e)
    o0 = s.observables()
    s.step(0.05, 2, seed=7)
    o1 = s.observables()
    assert o1["status"] == 0
    assert abs(o1["E"] - o0["E"]) < 1e-7 * o0["E"]
    assert np.abs(o1["P"] - o0["P"]).max() < 1e-2

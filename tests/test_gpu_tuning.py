"""Launch shapes, the autotuner and the cell grid on the GPU.

The block schedule of the sweep's colour launches and the thread-block size
of the pair passes change how the work is mapped onto the GPU, never the
arithmetic or its order: every shape must give bitwise the same trajectory.
The autotuner must leave the handle where it found it (state, step and
random-number counters, pair counters).  A chosen cell grid changes the
colouring and so the order of the sweep: it is checked against the oracle
run on the same grid.
"""
import numpy as np
import pytest

import oracle as O
from paper_1707_04232_gb300.inputs import Workload, lattice_state, random_box_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU-only hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1707_04232_gb300 import sdpd  # noqa: E402

FITS = {sdpd.FP64: (1, 2, 3), sdpd.MIXED: (0, 1, 2, 3, 4)}


def fluid(n=15, K=20.0, seed=2):
    w = Workload(n=n, K=K, jitter=0.2, seed=seed)
    q, p, e = lattice_state(w)
    return q, p, e, w


def run(precision, tuning, q, p, e, w, steps=4, scheme=sdpd.SCHEME_EMS, theta=1):
    s = sdpd.SDPD(w.N, w.L, h=w.h, K=w.K, precision=precision, scheme=scheme, theta=theta)
    if tuning is not None:
        s.set_tuning(*tuning)
    s.set_state(q, p, e)
    s.step(0.01, steps, seed=21)
    o = s.observables()
    return s.get_state(), (o["n_pairs"], o["n_accept"], o["n_reject_bound"], o["n_reject_metropolis"])


@pytest.mark.parametrize("precision", [sdpd.MIXED, sdpd.FP64])
def test_every_launch_shape_gives_the_same_trajectory(precision):
    q, p, e, w = fluid()
    ref_state, ref_counts = run(precision, None, q, p, e, w)
    assert ref_counts[0] > 0
    for v in FITS[precision]:
        for pt in (32, 64, 128):
            state, counts = run(precision, (v, pt), q, p, e, w)
            assert counts == ref_counts, (v, pt)
            for a, b in zip(state, ref_state):
                assert np.array_equal(a, b), (v, pt)


@pytest.mark.parametrize("precision,theta", [(sdpd.MIXED, 1), (sdpd.MIXED, 3), (sdpd.FP64, 2)])
def test_autotune_restores_the_handle(precision, theta):
    q, p, e, w = fluid(n=16, K=50.0, seed=5)
    a = sdpd.SDPD(w.N, w.L, h=w.h, K=w.K, precision=precision, theta=theta)
    b = sdpd.SDPD(w.N, w.L, h=w.h, K=w.K, precision=precision, theta=theta)
    for s in (a, b):
        s.set_state(q, p, e)
        s.step(0.005, 4, seed=8)
    tuning, ms = a.autotune(0.005, steps=2, seed=99)
    assert ms > 0 and a.tuning == tuning
    assert tuning["fd_variant"] in FITS[precision] and tuning["pair_threads"] in (32, 64, 128)
    oa, ob = a.observables(), b.observables()
    for k in ("n_pairs", "n_accept", "n_reject_bound", "n_reject_metropolis", "fd_step", "vv_step", "status"):
        assert oa[k] == ob[k], k
    for s in (a, b):
        s.step(0.005, 5, seed=8)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    oa, ob = a.observables(), b.observables()
    assert (oa["n_pairs"], oa["n_accept"], oa["fd_step"]) == (ob["n_pairs"], ob["n_accept"], ob["fd_step"])


def test_ensemble_autotune_keeps_every_member_bitwise():
    sizes = [(10, 5.0, 0.3), (11, 100.0, 1.0), (12, 20.0, 0.7)]  # blocks of 125, 216, 216
    members, alone, states = [], [], []
    for k, (n, K, kT) in enumerate(sizes):
        w = Workload(n=n, K=K, kT=kT, seed=30 + k)
        states.append((w, lattice_state(w)))
    for w, (q, p, e) in states:
        for lst in (members, alone):
            s = sdpd.SDPD(w.N, w.L, h=w.h, K=w.K, precision=sdpd.MIXED, stream=torch.cuda.Stream())
            s.set_state(q, p, e)
            lst.append(s)
    ens = sdpd.SDPDEnsemble(members)
    seeds = [3, 4, 5]
    ens.step(0.005, 4, seeds)
    ms = ens.autotune(0.005, steps=2, seeds=seeds)
    assert ms > 0
    ens.step(0.005, 6, seeds)
    torch.cuda.synchronize()
    for s, seed in zip(alone, seeds):
        s.step(0.005, 10, seed=seed)
    for m, s in zip(members, alone):
        for x, y in zip(m.get_state(), s.get_state()):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("n_c", [(4, 6, 4), (4, 4, 4)])
def test_chosen_cell_grid_matches_the_oracle(n_c):
    """A dilute fluid in L = 16 (default grid 6^3, 1500 particles so that a
    2x2x2 block of the coarsest grid holds ~190) swept on coarser grids:
    pair counts and decisions equal to the oracle's on the same grid
    (float64), states within 1e-10 after two steps."""
    L, N, K = 16.0, 1500, 20.0
    q, p, e = random_box_state(N, L, 1.0, 1.0, 1.5 * (K - 1.0), seed=4)
    dt, seed, steps = 0.01, 17, 2
    s = sdpd.SDPD(N, L, h=2.5, K=K, precision=sdpd.FP64, scheme=sdpd.SCHEME_EMS, nc=n_c)
    s.set_state(q, p, e)
    s.step(dt, steps, seed=seed)
    P = O.Config(N=N, L=L, K=K, n_c=n_c).params()
    st, rq, rp, re, stats, _ = O.run(P, q, p, e, dt, steps, seed=seed)
    assert st == O.OK
    o = s.observables()
    assert o["status"] == sdpd.OK
    assert o["n_pairs"] == stats.n_pairs > 0
    assert o["n_accept"] == stats.n_accept
    gq, gp, ge = s.get_state()
    Lv = np.array([L] * 3)
    dq = (gq - rq + 0.5 * Lv) % Lv - 0.5 * Lv
    assert np.abs(dq).max() <= 1e-10 * L
    assert np.abs(gp - rp).max() <= 1e-10 * np.abs(rp).max()
    assert np.abs(ge - re).max() <= 1e-10 * np.abs(re).max()
    # the grid does change the sweep: the default grid ends elsewhere
    d = sdpd.SDPD(N, L, h=2.5, K=K, precision=sdpd.FP64, scheme=sdpd.SCHEME_EMS)
    d.set_state(q, p, e)
    d.step(dt, steps, seed=seed)
    assert not np.array_equal(d.get_state()[1], gp)

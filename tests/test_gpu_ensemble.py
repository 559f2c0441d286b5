"""Ensembles of independent systems stepped by one CUDA graph.

Every member of an ensemble must end bitwise where the same system stepped
alone ends (same kernels, same seeds, same order); the members differ in
size, heat capacity, temperature and precision.  One float64 member is also
checked against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1707_04232_gb300.inputs import Workload, lattice_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1707_04232_gb300 import sdpd  # noqa: E402

MEMBERS = [  # (lattice n, K, kT, precision)
    (10, 100.0, 1.0, sdpd.FP64),
    (15, 5.0, 0.1, sdpd.MIXED),
    (16, 20.0, 0.5, sdpd.MIXED),
    (11, 100.0, 0.8, sdpd.MIXED),
    (12, 20.0, 0.3, sdpd.FP64),
]


def make(n, K, kT, prec, seed):
    w = Workload(n=n, K=K, kT=kT, seed=seed)
    q, p, e = lattice_state(w)
    s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=w.K, precision=prec, stream=torch.cuda.Stream())
    s.set_state(q, p, e)
    return s, (q, p, e, w)


@pytest.mark.parametrize("nsteps", [4, 5])
def test_ensemble_equals_members_stepped_alone(nsteps):
    seeds = [101 + k for k in range(len(MEMBERS))]
    ens_members = [make(*m, seed=k)[0] for k, m in enumerate(MEMBERS)]
    alone = [make(*m, seed=k)[0] for k, m in enumerate(MEMBERS)]
    ens = sdpd.SDPDEnsemble(ens_members)
    ens.step(0.005, nsteps, seeds)
    assert ens.kernel_nodes > 0
    for s, a, seed in zip(ens_members, alone, seeds):
        a.step(0.005, nsteps, seed=seed)
        qs, ps, es = s.get_state()
        qa, pa, ea = a.get_state()
        assert (qs == qa).all() and (ps == pa).all() and (es == ea).all()
        os_, oa = s.observables(), a.observables()
        assert os_["fd_step"] == oa["fd_step"] == nsteps and os_["vv_step"] == nsteps
        assert os_["n_pairs"] == oa["n_pairs"]


def test_ensemble_replay_draws_new_random_numbers():
    """Replaying the captured graph advances the sweep counter on the device:
    four steps in two replays equal four steps taken one call at a time."""
    s1, _ = make(12, 20.0, 0.5, sdpd.MIXED, seed=3)
    s2, _ = make(12, 20.0, 0.5, sdpd.MIXED, seed=3)
    ens = sdpd.SDPDEnsemble([s1])
    ens.step(0.005, 4, [9])
    for _ in range(4):
        s2.step(0.005, 1, seed=9)
    a, b = s1.get_state(), s2.get_state()
    assert all((x == y).all() for x, y in zip(a, b))


def test_ensemble_member_matches_oracle():
    s, (q, p, e, w) = make(10, 100.0, 1.0, sdpd.FP64, seed=0)
    other, _ = make(15, 5.0, 0.1, sdpd.MIXED, seed=1)
    ens = sdpd.SDPDEnsemble([s, other])
    ens.step(0.005, 4, [7, 8])
    qg, pg, eg = s.get_state()
    P = O.Config(N=w.N, L=w.L, K=w.K).params()
    st, qo, po, eo, _, _ = O.run(P, q, p, e, 0.005, 4, seed=7)
    L = w.L
    assert np.abs((qg - qo + 0.5 * L) % L - 0.5 * L).max() < 1e-6
    assert np.abs(eg - eo).max() < 1e-6 * eo.max()


def make_mts(n, K, kT, prec, seed, theta):
    w = Workload(n=n, K=K, kT=kT, seed=seed)
    q, p, e = lattice_state(w)
    s = sdpd.SDPD(w.N, w.L, m=w.m, h=w.h, K=w.K, precision=prec, theta=theta, stream=torch.cuda.Stream())
    s.set_state(q, p, e)
    return s


@pytest.mark.parametrize("nsteps,split", [(30, [30]), (37, [7, 30]), (65, [13, 52])])
def test_ensemble_with_multiple_time_steps(nsteps, split):
    """Members with theta = 3 and 5 (graph unit lcm(2, 3, 5) = 30 steps):
    bitwise equal to each member stepped alone one step per call, also when
    a call leaves the members at another phase of their theta cycle."""
    spec = [(10, 5.0, 1.0, sdpd.FP64, 3), (12, 20.0, 0.5, sdpd.MIXED, 5), (11, 100.0, 1.0, sdpd.MIXED, 1)]
    seeds = [5, 6, 7]
    ens_m = [make_mts(n, K, kT, pr, k, th) for k, (n, K, kT, pr, th) in enumerate(spec)]
    alone = [make_mts(n, K, kT, pr, k, th) for k, (n, K, kT, pr, th) in enumerate(spec)]
    ens = sdpd.SDPDEnsemble(ens_m)
    for part in split:
        ens.step(0.005, part, seeds)
    for s, a, seed, sp in zip(ens_m, alone, seeds, spec):
        for _ in range(nsteps):
            a.step(0.005, 1, seed=seed)
        x, y = s.get_state(), a.get_state()
        assert all((u == v).all() for u, v in zip(x, y))
        os_, oa = s.observables(), a.observables()
        assert os_["fd_step"] == oa["fd_step"] == nsteps // sp[4]
        assert os_["vv_step"] == nsteps

"""Reverse-mode gradients on the GPU versus the oracle and finite differences.

The library differentiates nsteps steps x_{k+1} = VV(x_k) + D_k (Velocity
Verlet at fixed entropies, Section 3.1, then the increments D_k that step k's
fluctuation/dissipation sweep produced in the recorded run, held fixed) and
the virial pressure, with respect to the state and to theta = (h, c_rho,
C_K).  The recorded increments themselves are checked against the oracle's
sweeps (same Philox streams, same pair order).  Tolerances (float64 on both sides, different
summation orders): the virial pressure within 1e-12 relative, its gradient
within 1e-10 of the largest component; trajectory gradients over a few steps
within 1e-9 of the largest component (the rounding differences of the
forward trajectories are amplified by the dynamics).  Checkpointing replays
the recorded run bit for bit, so results do not depend on the checkpoint
interval at all.  At the 32^3 size the oracle cannot reach, the gradient of
the virial pressure after 100 steps with the exact Metropolised sweep frozen
is checked against central differences (step 1e-6) of the frozen map.
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
from paper_1707_04232_gb300.autograd import handle_theta, verlet_trajectory, virial_pressure  # noqa: E402


def system(kind):
    if kind == "lattice1000_K5":
        w = Workload(n=10, K=5.0, jitter=0.2, seed=3)
        q, p, e = lattice_state(w)
        return q, p, e, (w.L,) * 3, w.K
    if kind == "random_rect":  # ragged N, rectangular box, disordered fluid, uneven energies
        L = (12.5, 15.0, 17.3)
        N = int(round(L[0] * L[1] * L[2]))
        C_K = 1.5 * (20.0 - 1.0)
        q, p, e = random_box_state(N, 1.0, 1.0, 1.0, C_K, seed=9)
        q = q * np.array(L)
        q = np.where(q >= np.array(L), 0.0, q)
        e = e * (0.5 + np.random.default_rng(3).random(N))
        return q, p, e, L, 20.0
    if kind == "coincident":
        w = Workload(n=10, K=5.0, jitter=0.2, seed=3)
        q, p, e = lattice_state(w)
        q[1] = q[0]
        return q, p, e, (w.L,) * 3, w.K
    raise KeyError(kind)


def make(N, L, K, kernel=sdpd.KERNEL_LUCY, precision=sdpd.FP64, h=2.5, c_rho=-1.0, scheme=sdpd.SCHEME_NONE,
         theta=1):
    return sdpd.SDPD(N, L, h=h, K=K, kernel=kernel, scheme=scheme, precision=precision, c_rho=c_rho,
                     theta=theta)


def oparams(N, L, K, kernel, scheme=O.SCHEME_NONE):
    return O.Config(N=N, L=tuple(L), K=K, kernel=kernel, scheme=scheme).params()


def recorded_increments(sim, tape, nsteps):
    """The tape's sweep increments as arrays [nsteps][N][3] and [nsteps][N]."""
    dps, des = [], []
    for k in range(nsteps):
        dp, de = sim.tape_increments(tape, k)
        dps.append(dp.cpu().numpy())
        des.append(de.cpu().numpy())
    return np.array(dps), np.array(des)


O_SCHEME = {sdpd.SCHEME_EMS: O.SCHEME_EMS, sdpd.SCHEME_AMS: O.SCHEME_AMS, sdpd.SCHEME_SSA: O.SCHEME_SSA}


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def close(got, ref, tol):
    got = got.cpu().numpy() if hasattr(got, "cpu") else np.asarray(got)
    scale = max(np.abs(ref).max(), 1e-300)
    return np.abs(got - ref).max() <= tol * scale, np.abs(got - ref).max() / scale


@pytest.mark.parametrize("kind", ["lattice1000_K5", "random_rect", "coincident"])
@pytest.mark.parametrize("kernel", [sdpd.KERNEL_LUCY, sdpd.KERNEL_CUBIC])
def test_virial_gradient_matches_oracle(kind, kernel):
    q, p, e, L, K = system(kind)
    sim = make(len(q), L, K, kernel)
    sim.set_state(q, p, e)
    val, gq, gp, ge, gt = sim.virial(grad=True)
    assert sim.virial() == val
    P = oparams(len(q), L, K, kernel)
    rval, rgq, rgp, rge, rgt = O.virial_vjp(P, q, p, e)
    assert abs(val - rval) <= 1e-12 * abs(rval)
    for got, ref in ((gq, rgq), (gp, rgp), (ge, rge)):
        ok, err = close(got, ref, 1e-10)
        assert ok, err
    assert np.abs(gt - rgt).max() <= 1e-10 * np.abs(rgt).max()
    # the state is untouched
    q2, p2, e2 = sim.get_state()
    assert np.array_equal(p2, p) and np.array_equal(e2, e)


@pytest.mark.parametrize("kind,kernel,nsteps,every", [
    ("lattice1000_K5", sdpd.KERNEL_LUCY, 7, 3),
    ("lattice1000_K5", sdpd.KERNEL_CUBIC, 5, 5),
    ("random_rect", sdpd.KERNEL_LUCY, 6, 4),
    ("coincident", sdpd.KERNEL_LUCY, 4, 2),
])
def test_trajectory_gradient_matches_oracle(kind, kernel, nsteps, every):
    q, p, e, L, K = system(kind)
    dt = 0.02
    sim = make(len(q), L, K, kernel)
    sim.set_state(q, p, e)
    tape = sim.vv_record(dt, nsteps, every)
    rng = np.random.default_rng(17)
    cq, cp, ce = rng.standard_normal(q.shape), rng.standard_normal(p.shape), rng.standard_normal(e.shape)
    gq, gp, ge, gt = sim.vv_adjoint(tape, dev(cq), dev(cp), dev(ce))
    P = oparams(len(q), L, K, kernel)
    rgq, rgp, rge, rgt = O.vv_vjp(P, q, p, e, dt, nsteps, cq, cp, ce)
    for got, ref in ((gq, rgq), (gp, rgp), (ge, rge)):
        ok, err = close(got, ref, 1e-9)
        assert ok, err
    assert np.abs(gt - rgt).max() <= 1e-9 * np.abs(rgt).max()


def test_checkpoint_interval_does_not_change_results():
    q, p, e, L, K = system("random_rect")
    dt, nsteps = 0.02, 9
    rng = np.random.default_rng(5)
    cot = [dev(rng.standard_normal(x.shape)) for x in (q, p, e)]
    results = []
    for every in (1, 2, 4, 9, 50):
        sim = make(len(q), L, K)
        sim.set_state(q, p, e)
        tape = sim.vv_record(dt, nsteps, every)
        gq, gp, ge, gt = sim.vv_adjoint(tape, *cot)
        results.append((gq.cpu().numpy(), gp.cpu().numpy(), ge.cpu().numpy(), gt))
    for r in results[1:]:
        for a, b in zip(r, results[0]):
            assert np.array_equal(a, b)


def test_adjoint_leaves_the_final_state_and_repeats():
    q, p, e, L, K = system("lattice1000_K5")
    sim = make(len(q), L, K)
    sim.set_state(q, p, e)
    tape = sim.vv_record(0.02, 5, 2)
    final = sim.get_state()
    sim2 = make(len(q), L, K)  # the same steps through sdpd_step
    sim2.set_state(q, p, e)
    sim2.step(0.02, 5)
    for a, b in zip(final, sim2.get_state()):
        assert np.array_equal(a, b)
    gp = dev(np.random.default_rng(1).standard_normal(p.shape))
    r1 = sim.vv_adjoint(tape, None, gp, None)
    for a, b in zip(final, sim.get_state()):
        assert np.array_equal(a, b)
    r2 = sim.vv_adjoint(tape, None, gp, None)
    for a, b in zip(r1[:3], r2[:3]):
        assert torch.equal(a, b)
    assert np.array_equal(r1[3], r2[3])


def test_zero_steps_is_identity():
    q, p, e, L, K = system("random_rect")
    sim = make(len(q), L, K)
    sim.set_state(q, p, e)
    tape = sim.vv_record(0.01, 0, 1)
    rng = np.random.default_rng(2)
    cq, cp, ce = rng.standard_normal(q.shape), rng.standard_normal(p.shape), rng.standard_normal(e.shape)
    gq, gp, ge, gt = sim.vv_adjoint(tape, dev(cq), dev(cp), dev(ce))
    assert np.abs(gq.cpu().numpy() - cq).max() < 1e-12
    assert np.array_equal(gp.cpu().numpy(), cp)
    assert np.abs(ge.cpu().numpy() - ce).max() < 1e-12 * np.abs(ce).max()
    assert np.abs(gt).max() < 1e-9


def test_argument_errors():
    q, p, e, L, K = system("lattice1000_K5")
    sim = make(len(q), L, K)
    sim.set_state(q, p, e)
    with pytest.raises(sdpd.SDPDError) as ex:  # no record yet
        sim.vv_adjoint(torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert ex.value.status == sdpd.ERR_INVALID_ARG
    assert sim.tape_bytes(-1, 1) == 0 and sim.tape_bytes(3, 0) == 0
    mixed = make(len(q), L, K, precision=sdpd.MIXED)
    mixed.set_state(q, p, e)
    with pytest.raises(sdpd.SDPDError) as ex:
        mixed.virial()
    assert ex.value.status == sdpd.ERR_INVALID_ARG
    with pytest.raises(sdpd.SDPDError) as ex:
        mixed.vv_record(0.01, 2, 1)
    assert ex.value.status == sdpd.ERR_INVALID_ARG


@pytest.mark.parametrize("kind,scheme,nsteps,every", [
    ("lattice1000_K5", sdpd.SCHEME_EMS, 6, 4),
    ("random_rect", sdpd.SCHEME_EMS, 5, 2),
    ("random_rect", sdpd.SCHEME_AMS, 4, 3),
    ("lattice1000_K5", sdpd.SCHEME_SSA, 3, 1),
])
def test_frozen_sweep_gradient_matches_oracle(kind, scheme, nsteps, every):
    """Recorded increments against the oracle's own sweeps, then the gradient
    of the frozen map against the oracle's reverse pass over the same
    increments."""
    q, p, e, L, K = system(kind)
    dt, seed = 0.02, 11
    sim = make(len(q), L, K, scheme=scheme)
    sim.set_state(q, p, e)
    tape = sim.vv_record(dt, nsteps, every, seed)
    dps, des = recorded_increments(sim, tape, nsteps)
    P = oparams(len(q), L, K, O.KERNEL_LUCY, O_SCHEME[scheme])
    rdp, rde, (rq, rp, re) = O.sweep_increments(P, q, p, e, dt, nsteps, seed)
    assert np.abs(dps).max() > 0.0  # the sweeps did move the state
    assert np.abs(dps - rdp).max() <= 1e-9 * np.abs(rdp).max()
    assert np.abs(des - rde).max() <= 1e-9 * np.abs(rde).max()
    gq_, gp_, ge_ = sim.get_state()
    assert np.abs(gp_ - rp).max() <= 1e-9 * np.abs(rp).max()
    assert np.abs(ge_ - re).max() <= 1e-9 * np.abs(re).max()
    rng = np.random.default_rng(23)
    cq, cp, ce = rng.standard_normal(q.shape), rng.standard_normal(p.shape), rng.standard_normal(e.shape)
    gq, gp, ge, gt = sim.vv_adjoint(tape, dev(cq), dev(cp), dev(ce))
    rgq, rgp, rge, rgt = O.frozen_vjp(P, q, p, e, dt, nsteps, dps, des, cq, cp, ce)
    for got, ref in ((gq, rgq), (gp, rgp), (ge, rge)):
        ok, err = close(got, ref, 1e-9)
        assert ok, err
    assert np.abs(gt - rgt).max() <= 1e-9 * np.abs(rgt).max()


def test_frozen_record_replay_and_checkpoints():
    """The record equals sdpd_step's trajectory up to rounding; a replay
    from the initial state retraces it bit for bit; the gradient does not
    depend on the checkpoint interval."""
    q, p, e, L, K = system("random_rect")
    dt, nsteps, seed = 0.02, 9, 5
    results = []
    rng = np.random.default_rng(5)
    cot = [dev(rng.standard_normal(x.shape)) for x in (q, p, e)]
    for every in (1, 4, 9, 50):
        sim = make(len(q), L, K, scheme=sdpd.SCHEME_EMS, theta=2)
        sim.set_state(q, p, e)
        tape = sim.vv_record(dt, nsteps, every, seed)
        final = sim.get_state()
        if every == 1:
            ref = make(len(q), L, K, scheme=sdpd.SCHEME_EMS, theta=2)
            ref.set_state(q, p, e)
            ref.step(dt, nsteps, seed=seed)
            for a, b in zip(final, ref.get_state()):
                assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max())
            sim.set_state(q, p, e)
            sim.vv_replay(tape)
            for a, b in zip(final, sim.get_state()):
                assert np.array_equal(a, b)
        gq, gp, ge, gt = sim.vv_adjoint(tape, *cot)
        for a, b in zip(final, sim.get_state()):
            assert np.array_equal(a, b)
        results.append((gq.cpu().numpy(), gp.cpu().numpy(), ge.cpu().numpy(), gt))
    for r in results[1:]:
        for a, b in zip(r, results[0]):
            assert np.array_equal(a, b)


def test_increment_argument_errors():
    q, p, e, L, K = system("lattice1000_K5")
    sim = make(len(q), L, K, scheme=sdpd.SCHEME_EMS)
    sim.set_state(q, p, e)
    tape = sim.vv_record(0.01, 3, 2, 1)
    for step in (-1, 3):
        with pytest.raises(sdpd.SDPDError) as ex:
            sim.tape_increments(tape, step)
        assert ex.value.status == sdpd.ERR_INVALID_ARG
    other = torch.empty_like(tape)
    with pytest.raises(sdpd.SDPDError) as ex:
        sim.vv_replay(other)
    assert ex.value.status == sdpd.ERR_INVALID_ARG


def test_virial_after_100_steps_32k_against_central_differences():
    """The workload of the gradient benchmark: 32^3 particles, K = 100,
    100 steps of dt = 0.005 with the exact Metropolised sweep after each,
    its increments frozen, checkpoints every 10 steps, Lucy kernel.  The
    gradient of the final virial pressure through torch.autograd against
    central differences (step 1e-6) of the frozen map: replays of the tape
    from the displaced initial states (a random direction of (q0, p0,
    eps0)), and, along each parameter, Verlet-only handles at the displaced
    parameter with the recorded increments added after each step."""
    w = Workload(n=32, K=100.0, seed=1)
    q, p, e = lattice_state(w)
    L, dt, nsteps, every, seed = (w.L,) * 3, 0.005, 100, 10, 3

    sim = make(w.N, L, w.K, scheme=sdpd.SCHEME_EMS)
    x = [dev(a).requires_grad_(True) for a in (q, p, e)]
    theta = torch.tensor(handle_theta(sim), dtype=torch.float64, requires_grad=True)
    qn, pn, en = verlet_trajectory(sim, *x, theta, dt, nsteps, every, seed)
    loss = virial_pressure(sim, qn, pn, en, theta)
    loss.backward()
    tape = sim._tape
    dps = [sim.tape_increments(tape, k) for k in range(nsteps)]
    assert max(d[0].abs().max().item() for d in dps) > 0.0  # the sweeps moved the state

    def replayed(x0):
        sim.set_state(*x0)
        sim.vv_replay(tape)
        return sim.virial()

    rng = np.random.default_rng(8)
    u = [dev(rng.standard_normal(a.shape) * (e if k == 2 else 1.0)) for k, a in enumerate((q, p, e))]
    d = 1e-6
    with torch.no_grad():
        lp = replayed([a + d * b for a, b in zip(x, u)])
        lm = replayed([a - d * b for a, b in zip(x, u)])
    fd = (lp - lm) / (2 * d)
    adj = sum((a.grad * b).sum().item() for a, b in zip(x, u))
    scale = sum((a.grad * b).abs().sum().item() for a, b in zip(x, u))
    assert abs(adj - fd) <= 1e-6 * scale, (adj, fd, scale)

    def frozen_loss(s2):
        s2.set_state(*(a.detach() for a in x))
        qk = torch.empty((w.N, 3), dtype=torch.float64, device="cuda")
        pk, ek = torch.empty_like(qk), torch.empty(w.N, dtype=torch.float64, device="cuda")
        for k in range(nsteps):
            s2.step(dt, 1)
            s2.get_state_device(qk, pk, ek)
            s2.set_state(qk, pk + dps[k][0], ek + dps[k][1])
        return s2.virial()

    h0, c0, k0 = handle_theta(sim)
    for k, (lo, hi, base) in enumerate((
            (dict(h=h0 * (1 - d), c_rho=c0), dict(h=h0 * (1 + d), c_rho=c0), h0),
            (dict(c_rho=c0 * (1 - d)), dict(c_rho=c0 * (1 + d)), c0),
            # C_K = 3/2 (K - 1) kB: move K, keep c_rho
            (dict(c_rho=c0, K=k0 * (1 - d) / 1.5 + 1), dict(c_rho=c0, K=k0 * (1 + d) / 1.5 + 1), k0))):
        vals = []
        for kw in (hi, lo):
            Kk = kw.pop("K", w.K)
            with torch.no_grad():
                vals.append(frozen_loss(make(w.N, L, Kk, **kw)))
        fd_t = (vals[0] - vals[1]) / (2 * d * base)
        assert abs(theta.grad[k].item() - fd_t) <= 1e-6 * abs(fd_t), (k, theta.grad[k].item(), fd_t)


def test_float32_sweep_on_float64_state():
    """sweep_f32: the sweep's pair arithmetic in float32 on the float64 state
    (as the mixed path does it).  Against the float64 sweep over 10 steps, as
    for the mixed path: a decision whose margin is within float32 rounding
    may flip, moving that pair's momenta by one noise kick, so almost every
    particle stays within 2e-6 a and none leaves 1e-2 a; the accept counts
    agree up to those flips and the total energy within 1e-6.  The recorded
    increments then give a gradient equal to the oracle's reverse pass over
    those same increments (they enter as constants)."""
    q, p, e, L, K = system("random_rect")
    dt, seed, nsteps = 0.02, 7, 10
    runs = {}
    for f32 in (False, True):
        s = sdpd.SDPD(len(q), L, h=2.5, K=K, scheme=sdpd.SCHEME_EMS, precision=sdpd.FP64, sweep_f32=f32)
        s.set_state(q, p, e)
        s.step(dt, nsteps, seed=seed)
        runs[f32] = (s.get_state(), s.observables())
    (q64, p64, e64), o64 = runs[False]
    (q32, p32, e32), o32 = runs[True]
    Lv = np.asarray(L)
    dq = np.abs((q32 - q64 + 0.5 * Lv) % Lv - 0.5 * Lv).max(axis=1)
    assert np.mean(dq < 2e-6) > 0.97 and dq.max() < 1e-2
    assert abs(o32["n_pairs"] - o64["n_pairs"]) <= 10  # pair sets can differ where trajectories did
    assert abs(o32["n_accept"] - o64["n_accept"]) <= 20
    assert abs(o32["E"] - o64["E"]) < 1e-6 * abs(o64["E"])
    assert o32["status"] == sdpd.OK
    # gradient of the frozen map recorded with the float32 sweep
    nsteps = 4
    sim = sdpd.SDPD(len(q), L, h=2.5, K=K, scheme=sdpd.SCHEME_EMS, precision=sdpd.FP64, sweep_f32=True)
    sim.set_state(q, p, e)
    tape = sim.vv_record(dt, nsteps, 2, seed)
    dps, des = recorded_increments(sim, tape, nsteps)
    assert np.abs(dps).max() > 0.0
    rng = np.random.default_rng(31)
    cq, cp, ce = rng.standard_normal(q.shape), rng.standard_normal(p.shape), rng.standard_normal(e.shape)
    gq, gp, ge, gt = sim.vv_adjoint(tape, dev(cq), dev(cp), dev(ce))
    P = oparams(len(q), L, K, O.KERNEL_LUCY, O.SCHEME_EMS)
    rgq, rgp, rge, rgt = O.frozen_vjp(P, q, p, e, dt, nsteps, dps, des, cq, cp, ce)
    for got, ref in ((gq, rgq), (gp, rgp), (ge, rge)):
        ok, err = close(got, ref, 1e-9)
        assert ok, err
    assert np.abs(gt - rgt).max() <= 1e-9 * np.abs(rgt).max()

"""Pins of the oracle's reverse-mode gradients of the conservative dynamics.

The gradients differentiate the Velocity Verlet trajectory of Eq.
(sdpd-verlet) at fixed entropies (Section 3.1), with the density gradient of
Eq. (gradient-rho), the pressures of Eq. (pg-eos) and the virial pressure as
a loss.  They are pinned by central differences of the oracle's own forward
maps (which other tests pin to the paper), by closed forms and by the exact
identity of a zero-step trajectory.  No test here needs a GPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_1707_04232_gb300.inputs import Workload, lattice_state


def setup(kernel=O.KERNEL_LUCY, K=5.0, jitter=0.2, seed=3):
    w = Workload(n=10, jitter=jitter, K=K, seed=seed)
    q, p, e = lattice_state(w)
    cfg = O.Config(N=w.N, L=w.L, K=w.K, kernel=kernel, scheme=O.SCHEME_NONE)
    return cfg, q, p, e


def central(f, d=1e-5):
    """Central difference.  Its truncation error is O(d^2) (the cubic spline's
    F'' jumps at h/2, which rules out Richardson steps), and the rounding of
    the ~40k-term pair sums sets a floor of ~1e-13 / d; hence the 1e-6
    relative tolerances below, far under the size of any dropped term."""
    return (f(d) - f(-d)) / (2 * d)


def with_param(cfg, name, value):
    P = cfg.params()
    setattr(P, name, value)
    return P


THETA = ("h", "c_rho", "C_K")


@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
def test_kernel_derivatives(kernel):
    """dF/dr, dW/dh and dF/dh against central differences of W and F, on both
    branches of the cubic spline; all vanish at r >= h."""
    h = 2.5
    for r in np.linspace(0.07, h - 0.07, 37):
        if abs(r - 0.5 * h) < 1e-3:
            continue
        d = 1e-5
        ref = (O.F(kernel, r + d, h) - O.F(kernel, r - d, h)) / (2 * d)
        assert abs(O.dF_dr(kernel, r, h) - ref) < 1e-8 * max(1.0, abs(ref))
        ref = (O.W(kernel, r, h + d) - O.W(kernel, r, h - d)) / (2 * d)
        assert abs(O.dW_dh(kernel, r, h) - ref) < 1e-8 * max(1.0, abs(ref))
        ref = (O.F(kernel, r, h + d) - O.F(kernel, r, h - d)) / (2 * d)
        assert abs(O.dF_dh(kernel, r, h) - ref) < 1e-8 * max(1.0, abs(ref))
    ref = (O.W(kernel, 0.0, h + 1e-5) - O.W(kernel, 0.0, h - 1e-5)) / 2e-5
    assert abs(O.dW_dh(kernel, 0.0, h) - ref) < 1e-9
    for f in (O.dF_dr, O.dW_dh, O.dF_dh):
        assert f(kernel, h, h) == 0.0 and f(kernel, 1.5 * h, h) == 0.0


def test_virial_pressure_ideal_gas():
    """No pair within h (lattice spacing 3 > h = 2.5): the virial pressure is
    the kinetic one, sum |p|^2 / (3 V m); its gradient is 2 p / (3 V m) in p
    and zero in q, eps and theta."""
    n, a = 6, 3.0
    idx = np.arange(n)
    q = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), -1).reshape(-1, 3) * a + 0.5 * a
    rng = np.random.default_rng(0)
    p = rng.standard_normal(q.shape)
    e = 1.0 + rng.random(len(q))
    P = O.Config(N=len(q), L=n * a, K=5.0, scheme=O.SCHEME_NONE).params()
    V = (n * a) ** 3
    val, gq, gp, ge, gt = O.virial_vjp(P, q, p, e)
    assert abs(val - (p * p).sum() / (3 * V)) < 1e-15 * val
    assert np.allclose(gp, 2 * p / (3 * V), rtol=1e-15, atol=0)
    assert not gq.any() and not ge.any() and not gt.any()


@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
def test_virial_gradient_by_differences(kernel):
    """dP/dq, dP/dp, dP/deps (random directions) and dP/dtheta of the virial
    pressure at fixed energies against central differences."""
    cfg, q, p, e = setup(kernel)
    P = cfg.params()
    val, gq, gp, ge, gt = O.virial_vjp(P, q, p, e)
    assert val == O.virial_pressure(P, q, p, e)
    rng = np.random.default_rng(7)
    for k, g in enumerate((gq, gp, ge)):
        u = rng.standard_normal(g.shape) * (e if k == 2 else 1.0)

        def f(d, k=k, u=u):
            x = [q, p, e]
            x[k] = x[k] + d * u
            return O.virial_pressure(P, *x)
        ref = central(f)
        assert abs((g * u).sum() - ref) < 1e-6 * np.abs(g * u).sum()
    for k, name in enumerate(THETA):
        base = getattr(P, name)
        ref = central(lambda d: O.virial_pressure(with_param(cfg, name, base + d * base), q, p, e)) / base
        assert abs(gt[k] - ref) < 1e-6 * max(1.0, abs(ref))


def test_virial_on_perfect_lattice():
    """On a perfect lattice at rest with equal energies every particle has the
    same pi and the same A = m^2 sum_shells F(r) r^2, so the virial pressure is
    N pi A / (3V) and dP/dq vanishes by symmetry."""
    w = Workload(n=10, jitter=0.0, K=5.0, seed=0)
    q, p, e = lattice_state(w)
    p[:] = 0.0
    P = O.Config(N=w.N, L=w.L, K=w.K, scheme=O.SCHEME_NONE).params()
    rho = O.density(P, q)
    pi = P.c_rho * e[0] / (P.C_K * P.m * rho[0])
    shells = [np.sqrt(x * x + y * y + z * z) for x in range(-3, 4) for y in range(-3, 4) for z in range(-3, 4)]
    A = sum(r * r * O.F(P.kernel, r, P.h) for r in shells if 0 < r < P.h)
    val, gq, _, _, _ = O.virial_vjp(P, q, p, e)
    assert abs(val - w.N * pi * A / (3 * w.L ** 3)) < 1e-12 * val
    assert np.abs(gq).max() < 1e-14 * val


def test_trajectory_gradient_zero_steps_is_identity():
    """With no step the map is the identity: eps_n = E(S(eps0, rho(q0)),
    rho(q0)) = eps0, so the final-energy and entropy paths through rho cancel."""
    cfg, q, p, e = setup()
    P = cfg.params()
    rng = np.random.default_rng(2)
    gqn, gpn, gen = rng.standard_normal(q.shape), rng.standard_normal(p.shape), rng.standard_normal(e.shape)
    gq, gp, ge, gt = O.vv_vjp(P, q, p, e, 0.01, 0, gqn, gpn, gen)
    assert np.abs(gq - gqn).max() < 1e-12
    assert np.array_equal(gp, gpn)
    assert np.abs(ge - gen).max() < 1e-12 * np.abs(gen).max()
    assert np.abs(gt).max() < 1e-9


@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
def test_trajectory_gradient_by_differences(kernel):
    """Cotangents of (q0, p0, eps0, theta) for a random linear functional of
    the state after 3 Velocity Verlet steps, against central differences."""
    cfg, q, p, e = setup(kernel)
    P = cfg.params()
    dt, ns = 0.02, 3
    rng = np.random.default_rng(11)
    cq, cp, ce = rng.standard_normal(q.shape), rng.standard_normal(p.shape), rng.standard_normal(e.shape)

    def loss(Pp, x):
        qn, pn, en = O.vv_trajectory(Pp, *x, dt, ns)
        return (cq * qn).sum() + (cp * pn).sum() + (ce * en).sum()
    gq, gp, ge, gt = O.vv_vjp(P, q, p, e, dt, ns, cq, cp, ce)
    for k, g in enumerate((gq, gp, ge)):
        u = rng.standard_normal(g.shape) * (e if k == 2 else 1.0)

        def f(d, k=k, u=u):
            x = [q, p, e]
            x[k] = x[k] + d * u
            return loss(P, x)
        ref = central(f)
        assert abs((g * u).sum() - ref) < 1e-6 * np.abs(g * u).sum()
    for k, name in enumerate(THETA):
        base = getattr(P, name)
        ref = central(lambda d: loss(with_param(cfg, name, base + d * base), [q, p, e])) / base
        assert abs(gt[k] - ref) < 1e-6 * max(1.0, abs(ref))


def test_virial_loss_gradient_by_differences():
    """The composed gradient of the virial pressure after 3 steps."""
    cfg, q, p, e = setup(K=20.0, seed=5)
    P = cfg.params()
    dt, ns = 0.02, 3

    def loss(Pp, x):
        return O.virial_pressure(Pp, *O.vv_trajectory(Pp, *x, dt, ns))
    val, gq, gp, ge, gt = O.vv_virial_grad(P, q, p, e, dt, ns)
    assert val == loss(P, [q, p, e])
    rng = np.random.default_rng(4)
    for k, g in enumerate((gq, gp, ge)):
        u = rng.standard_normal(g.shape) * (e if k == 2 else 1.0)

        def f(d, k=k, u=u):
            x = [q, p, e]
            x[k] = x[k] + d * u
            return loss(P, x)
        ref = central(f)
        assert abs((g * u).sum() - ref) < 1e-6 * np.abs(g * u).sum()
    for k, name in enumerate(THETA):
        base = getattr(P, name)
        ref = central(lambda d: loss(with_param(cfg, name, base + d * base), [q, p, e])) / base
        assert abs(gt[k] - ref) < 1e-6 * max(1.0, abs(ref))


def test_coincident_particles():
    """Two particles at the same position: the pair is inside the density sum
    (m W(0) each way), so it is in dP/dh, and its force derivative is F(0) I
    (the F'/r term vanishes with r); both against central differences."""
    cfg, q, p, e = setup()
    q[1] = q[0]
    P = cfg.params()
    dt, ns = 0.02, 3

    def loss(Pp, x):
        return O.virial_pressure(Pp, *O.vv_trajectory(Pp, *x, dt, ns))
    val, gq, gp, ge, gt = O.vv_virial_grad(P, q, p, e, dt, ns)
    u = np.zeros_like(q)
    u[0] = [0.3, -0.2, 0.5]
    u[1] = [-0.1, 0.4, 0.2]
    ref = central(lambda d: loss(P, [q + d * u, p, e]))
    # 1e-8: the rounding floor of the difference quotient (~1e-13 / d)
    assert abs((gq * u).sum() - ref) < 1e-6 * np.abs(gq * u).sum() + 1e-8
    val, gq, gp, ge, gt = O.virial_vjp(P, q, p, e)
    ref = central(lambda d: O.virial_pressure(with_param(cfg, "h", P.h * (1 + d)), q, p, e)) / P.h
    assert abs(gt[0] - ref) < 1e-6 * abs(ref)


def frozen_setup(kernel=O.KERNEL_LUCY, scheme=O.SCHEME_EMS, K=5.0, seed=3, dt=0.02, ns=3):
    cfg, q, p, e = setup(kernel, K=K, seed=seed)
    cfg_fd = O.Config(N=cfg.N, L=cfg.L, K=K, kernel=kernel, scheme=scheme)
    dp, de, _ = O.sweep_increments(cfg_fd.params(), q, p, e, dt, ns, seed=7)
    return cfg, q, p, e, dp, de, dt, ns


def test_frozen_run_reproduces_the_full_run():
    """Velocity Verlet plus the recorded sweep increments retraces the full
    run (Velocity Verlet then the sweep, every step) to rounding."""
    cfg, q, p, e, dp, de, dt, ns = frozen_setup()
    P = O.Config(N=cfg.N, L=cfg.L, K=5.0, scheme=O.SCHEME_EMS).params()
    st, qr, pr, er, _, _ = O.run(P, q, p, e, dt, ns, seed=7)
    qf, pf, ef = O.frozen_run(cfg.params(), q, p, e, dt, ns, dp, de)
    assert np.abs(qf - qr).max() < 1e-12 and np.abs(pf - pr).max() < 1e-12
    assert np.abs(ef - er).max() < 1e-12 * er.max()
    assert np.abs(dp).max() > 1e-3  # the sweeps did move the momenta


def test_frozen_gradient_with_zero_increments_is_the_verlet_gradient():
    """Without increments every step recomputes the same entropies, so the
    per-step reverse pass equals the fixed-entropy one."""
    cfg, q, p, e = setup()
    P = cfg.params()
    rng = np.random.default_rng(9)
    c = [rng.standard_normal(x.shape) for x in (q, p, e)]
    a = O.frozen_vjp(P, q, p, e, 0.02, 3, None, None, *c)
    b = O.vv_vjp(P, q, p, e, 0.02, 3, *c)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() <= 1e-9 * np.abs(y).max()
    z = O.frozen_vjp(P, q, p, e, 0.02, 0, None, None, *c)  # no step: the identity
    assert np.array_equal(z[0], c[0]) and np.array_equal(z[1], c[1]) and np.array_equal(z[2], c[2])


@pytest.mark.parametrize("kernel", [O.KERNEL_CUBIC, O.KERNEL_LUCY])
def test_frozen_virial_gradient_by_differences(kernel):
    """The virial pressure after 3 steps with the sweeps' increments frozen:
    the reverse pass against central differences in (q0, p0, eps0) and
    theta (the increments, not recomputed, make the map smooth)."""
    cfg, q, p, e, dp, de, dt, ns = frozen_setup(kernel)
    P = cfg.params()

    def loss(Pp, x):
        return O.virial_pressure(Pp, *O.frozen_run(Pp, *x, dt, ns, dp, de))
    qn, pn, en = O.frozen_run(P, q, p, e, dt, ns, dp, de)
    val, gqn, gpn, gen, gtn = O.virial_vjp(P, qn, pn, en)
    gq, gp, ge, gt = O.frozen_vjp(P, q, p, e, dt, ns, dp, de, gqn, gpn, gen)
    gt = gt + gtn
    rng = np.random.default_rng(4)
    for k, g in enumerate((gq, gp, ge)):
        u = rng.standard_normal(g.shape) * (e if k == 2 else 1.0)

        def f(d, k=k, u=u):
            x = [q, p, e]
            x[k] = x[k] + d * u
            return loss(P, x)
        ref = central(f)
        assert abs((g * u).sum() - ref) < 1e-6 * np.abs(g * u).sum()
    for k, name in enumerate(THETA):
        base = getattr(P, name)
        ref = central(lambda d: loss(with_param(cfg, name, base + d * base), [q, p, e])) / base
        assert abs(gt[k] - ref) < 1e-6 * max(1.0, abs(ref))

"""torch.autograd functions over the library's reverse-mode entry points.

``VerletTrajectory`` maps (q0, p0, eps0, theta) to the state after nsteps
steps x_{k+1} = VV(x_k) + D_k: a Velocity Verlet step at fixed entropies
(Section 3.1), then the increments D_k that the handle's fluctuation/
dissipation sweep (Sections 3.2-3.3) produced in the forward run, held fixed
(no sweep on a SCHEME_NONE handle, D_k = 0).  Its backward is the library's
checkpointed reverse pass.  ``VirialPressure`` maps a state to its
virial pressure.  theta = (h, c_rho, C_K) is a float64 tensor that must hold
the handle's own values (the library evaluates at those); it carries the
parameter gradient.  Both run on a float64 SDPD handle.  Argument marshalling
only: every step runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from .sdpd import SDPD


def handle_theta(sim: SDPD) -> tuple[float, float, float]:
    """(h, c_rho, C_K) of a handle, as the library computes them."""
    K, kB = sim.K, sim.params.kB
    c_rho = sim.params.c_rho if sim.params.c_rho >= 0 else 0.5 * (K - 1.0)
    return sim.h_smooth, c_rho, 1.5 * (K - 1.0) * kB


def _check_theta(sim: SDPD, theta: torch.Tensor):
    want = np.array(handle_theta(sim))
    got = theta.detach().double().cpu().numpy()
    if got.shape != (3,) or not np.allclose(got, want, rtol=1e-12, atol=0.0):
        raise ValueError(f"theta {got} differs from the handle's (h, c_rho, C_K) = {want}")


class VerletTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q0, p0, eps0, theta, sim: SDPD, dt: float, nsteps: int, every: int, seed: int):
        _check_theta(sim, theta)
        sim.set_state(q0.detach(), p0.detach(), eps0.detach())
        tape = sim.vv_record(dt, nsteps, every, seed)
        dev = q0.device
        q = torch.empty((sim.N, 3), dtype=torch.float64, device=dev)
        p = torch.empty((sim.N, 3), dtype=torch.float64, device=dev)
        e = torch.empty(sim.N, dtype=torch.float64, device=dev)
        sim.get_state_device(q, p, e)
        ctx.sim, ctx.tape, ctx.theta_device = sim, tape, theta.device
        return q, p, e

    @staticmethod
    def backward(ctx, gq, gp, ge):
        gq0, gp0, ge0, gth = ctx.sim.vv_adjoint(ctx.tape, gq, gp, ge)
        gth = torch.as_tensor(gth, dtype=torch.float64, device=ctx.theta_device)
        return gq0, gp0, ge0, gth, None, None, None, None, None


class VirialPressure(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, p, eps, theta, sim: SDPD):
        _check_theta(sim, theta)
        sim.set_state(q.detach(), p.detach(), eps.detach())
        value, gq, gp, ge, gth = sim.virial(grad=True)
        ctx.save_for_backward(gq, gp, ge)
        ctx.gth = torch.as_tensor(gth, dtype=torch.float64, device=theta.device)
        return torch.tensor(value, dtype=torch.float64, device=q.device)

    @staticmethod
    def backward(ctx, g):
        gq, gp, ge = ctx.saved_tensors
        return g * gq, g * gp, g * ge, g.to(ctx.gth.device) * ctx.gth, None


def verlet_trajectory(sim, q0, p0, eps0, theta, dt, nsteps, every=10, seed=0):
    return VerletTrajectory.apply(q0, p0, eps0, theta, sim, dt, nsteps, every, seed)


def virial_pressure(sim, q, p, eps, theta):
    return VirialPressure.apply(q, p, eps, theta, sim)

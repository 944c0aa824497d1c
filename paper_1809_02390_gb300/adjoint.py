"""Differentiable rollouts through the hand-written adjoint kernel.

``rollout(theta, rho0, nsteps, ...)`` runs ``nsteps`` time steps on the GPU and
returns the final post-collision state; it is a ``torch.autograd.Function``
whose backward pass recomputes the forward states segment by segment from
checkpoints (taken every ``checkpoint_every`` steps, sqrt(N) by default) and
runs ``lb_adjoint_step`` backwards through each segment.

Parameters theta = (Tr, G2, K_int):
  * Tr: reduced temperature, T = Tr Tc;
  * G2: interaction strength G^2/c^2 (the force strength of Eq. 12, lattice units);
  * K_int: interface parameter of Eqs. 21-22, acting through the pressure scale
    lam = K_EOS/c^2 = lam_ref (K_ref / K_int)^2, with rho_l (and so lam_ref) frozen
    at the reference parameters (the c_s rule of Eq. 22 evaluated once).
"""
from __future__ import annotations

import math

import numpy as np

from . import Lattice, capi


class RolloutSpec:
    """Fixed (non-differentiated) settings of a rollout."""

    def __init__(self, nx: int, ny: int, precision: str = "fp32", Tr_ref: float = 0.8, K_int_ref: float = 1.0,
                 eos: str = "vdw", eos_a: float = 9.0 / 49.0, eos_b: float = 2.0 / 21.0, R_gas: float = 1.0,
                 rho_ref: float | None = None, s_p: float = 1.0):
        from . import derive

        self.nx, self.ny, self.precision = nx, ny, precision
        self.eos, self.eos_a, self.eos_b, self.R_gas, self.s_p = eos, eos_a, eos_b, R_gas, s_p
        d = derive(nx, ny, eos=eos, eos_a=eos_a, eos_b=eos_b, R_gas=R_gas, Tr=Tr_ref, K_int=K_int_ref, s_p=s_p)
        self.Tc = d["Tc"]
        self.lam_ref = d["lam"]
        self.K_ref = K_int_ref
        self.G2_ref = d["G2"]
        self.rho_g, self.rho_l = d["rho_g"], d["rho_l"]
        # Storage shift of the populations (f_i - w_i rho_ref); the FP32 kernels carry it in float.
        r = 0.5 * (self.rho_g + self.rho_l) if rho_ref is None else float(rho_ref)
        self.rho_ref = r if precision == "fp64" else float(np.float32(r))

    def lattice_kwargs(self, theta) -> dict:
        Tr, G2, K = (float(v) for v in theta)
        return dict(eos=self.eos, eos_a=self.eos_a, eos_b=self.eos_b, R_gas=self.R_gas, Tr=Tr, G2=G2,
                    lam=self.lam_ref * (self.K_ref / K) ** 2, s_p=self.s_p)


class LBRollout:
    """Namespace holding the autograd Function (built lazily so that importing
    this module does not need torch)."""

    fn = None


def _make_function():
    import torch

    class _Rollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, f0, spec, nsteps, checkpoint_every):
            lat = Lattice(np.full((spec.ny, spec.nx), 0.5 * (spec.rho_g + spec.rho_l)), precision=spec.precision,
                          rho_ref=spec.rho_ref, **spec.lattice_kwargs(theta.detach().cpu().numpy()))
            capi.lb_set_state(lat.h, f0.detach().contiguous().data_ptr())
            checkpoints = [f0.detach().clone()]
            done = 0
            while done < nsteps:
                k = min(checkpoint_every, nsteps - done)
                lat.step(k)
                done += k
                if done < nsteps:
                    checkpoints.append(lat.state().clone())
            out = lat.state().clone()
            ctx.save_for_backward(theta)
            ctx.spec, ctx.nsteps, ctx.every = spec, nsteps, checkpoint_every
            ctx.checkpoints = checkpoints
            ctx.lat = lat
            return out

        @staticmethod
        def backward(ctx, grad_out):
            (theta,) = ctx.saved_tensors
            spec, lat = ctx.spec, ctx.lat
            real = torch.float64 if spec.precision == "fp64" else torch.float32
            dev = grad_out.device
            lam = grad_out.to(real).contiguous().clone()
            nscr = capi.lb_adjoint_steps_scratch_bytes(lat.p)
            scratch = torch.empty(nscr, dtype=torch.uint8, device=dev)
            dtheta = torch.zeros(3, dtype=torch.float64, device=dev)
            nseg = len(ctx.checkpoints)
            for seg in range(nseg - 1, -1, -1):
                start = seg * ctx.every
                k = min(ctx.every, ctx.nsteps - start)
                # Recompute the states s^start .. s^(start+k-1) of this segment, then
                # run the segment's adjoint steps backwards in one call.
                states = [ctx.checkpoints[seg]]
                capi.lb_set_state(lat.h, ctx.checkpoints[seg].data_ptr())
                for _ in range(k - 1):
                    lat.step(1)
                    states.append(lat.state().clone())
                capi.lb_adjoint_steps(lat.h, [t.data_ptr() for t in states], lam.data_ptr(), dtheta.data_ptr(),
                                      scratch.data_ptr(), nscr)
            dT, dG2, dlam = (float(v) for v in dtheta.cpu())
            Tr, G2, K = (float(v) for v in theta.detach().cpu())
            lam_val = spec.lam_ref * (spec.K_ref / K) ** 2
            g_theta = torch.tensor([dT * spec.Tc, dG2, dlam * (-2.0 * lam_val / K)], dtype=theta.dtype,
                                   device=theta.device)
            lat.close()
            ctx.lat = None
            ctx.checkpoints = None
            return g_theta, lam.to(grad_out.dtype), None, None, None

    return _Rollout


def rollout(theta, f0, spec: RolloutSpec, nsteps: int, checkpoint_every: int | None = None):
    """Final post-collision state after ``nsteps`` steps from ``f0`` (storage-type
    tensor [9, ny, nx] of deviations f - w rho_ref); differentiable in ``theta``
    (float64 tensor (Tr, G2, K_int)) and ``f0``."""
    if LBRollout.fn is None:
        LBRollout.fn = _make_function()
    every = checkpoint_every or max(1, int(round(math.sqrt(nsteps))))
    return LBRollout.fn.apply(theta, f0, spec, nsteps, every)


def initial_state(spec: RolloutSpec, rho0, theta):
    """Rest-equilibrium state for rho0 at parameters theta, as the rollout's f0."""
    lat = Lattice(rho0, precision=spec.precision, rho_ref=spec.rho_ref,
                  **spec.lattice_kwargs([float(v) for v in theta]))
    f0 = lat.state().clone()
    lat.close()
    return f0


def density(state, spec: RolloutSpec):
    """rho = sum_i f_i of a state tensor (the weights of the storage shift sum to 1)."""
    return state.sum(0) + spec.rho_ref


def calibrate(spec: RolloutSpec, f0, target, theta0, nsteps: int, iterations: int = 50, lr: float = 0.02,
              checkpoint_every: int | None = None):
    """Fits theta = (Tr, G2, K_int) so that the density after ``nsteps`` steps from
    ``f0`` matches ``target`` (loss = sum (rho - target)^2), with Adam on the
    relative deviations theta = theta0 (1 + delta).  Returns (theta, losses)."""
    import torch

    base = theta0.detach().clone().double()
    delta = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([delta], lr=lr)
    losses = []
    for _ in range(iterations):
        opt.zero_grad()
        theta = base * (1.0 + delta)
        out = rollout(theta, f0, spec, nsteps, checkpoint_every)
        loss = ((density(out, spec) - target) ** 2).sum()
        loss.backward()
        losses.append(float(loss.detach()))
        opt.step()
    return (base * (1.0 + delta)).detach(), losses

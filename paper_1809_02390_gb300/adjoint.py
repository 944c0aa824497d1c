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

        self.nx, self.ny, self.precision, self.Tr_ref = nx, ny, precision, Tr_ref
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

    def moments_lattice(self):
        """A lattice of this spec used only to evaluate densities of given states
        through lb_moments (created on first use)."""
        lat = getattr(self, "_moments_lat", None)
        if lat is None:
            lat = Lattice(np.full((self.ny, self.nx), 0.5 * (self.rho_g + self.rho_l)), precision=self.precision,
                          rho_ref=self.rho_ref,
                          **self.lattice_kwargs([self.Tr_ref, self.G2_ref, self.K_ref]))
            self._moments_lat = lat
        return lat

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


class _DensityFn:
    fn = None


def _make_density():
    import torch

    class _Density(torch.autograd.Function):
        """rho of a post-collision state by the library (lb_moments: rho = sum_i fbar_i,
        Eq. 5 at the time level of the last collision); its transpose, for the
        backward pass, spreads the cotangent of rho over the nine populations."""

        @staticmethod
        def forward(ctx, state, spec):
            lat = spec.moments_lattice()
            capi.lb_set_state(lat.h, state.detach().contiguous().data_ptr())
            rho = lat.moments(velocity=False).clone()
            ctx.shape, ctx.dtype = tuple(state.shape), state.dtype
            return rho

        @staticmethod
        def backward(ctx, g):
            return g.to(ctx.dtype).unsqueeze(0).expand(ctx.shape).contiguous(), None

    return _Density


def density(state, spec: RolloutSpec):
    """rho of a state tensor [9, ny, nx] (deviation storage), computed by the library
    (lb_moments) and differentiable in the state."""
    if _DensityFn.fn is None:
        _DensityFn.fn = _make_density()
    return _DensityFn.fn.apply(state, spec)


def trajectory(theta, f0, spec: RolloutSpec, nsteps: int, snapshots: int = 1,
               checkpoint_every: int | None = None) -> list:
    """Densities after each of ``snapshots`` equal segments of an ``nsteps``-step
    rollout (the last one ends at ``nsteps``), differentiable in theta and f0: the
    segments are chained rollouts, so the adjoint of each segment receives the
    cotangents of its own snapshot and of everything after it."""
    if snapshots < 1 or nsteps < snapshots:
        raise ValueError("need 1 <= snapshots <= nsteps")
    bounds = [round(nsteps * (k + 1) / snapshots) for k in range(snapshots)]
    out, state, done = [], f0, 0
    for b in bounds:
        state = rollout(theta, state, spec, b - done, checkpoint_every)
        done = b
        out.append(density(state, spec))
    return out


def calibrate(spec: RolloutSpec, f0, target, theta0, nsteps: int, iterations: int = 50, lr: float = 0.02,
              checkpoint_every: int | None = None, snapshots: int = 1, method: str = "lbfgs",
              bound: float = 0.25):
    """Fits theta = (Tr, G2, K_int) so that the densities of a rollout of ``nsteps``
    steps from ``f0`` match ``target`` (loss = sum over snapshots of sum (rho - target)^2),
    optimising delta in theta = theta0 (1 + bound tanh(delta / bound)): relative
    deviations for small delta, kept inside +-bound (25%) so that a line search
    cannot step to a temperature at or above the critical one, or below zero.  ``target``: the
    final density (snapshots = 1) or the list of ``snapshots`` densities of
    ``trajectory``.  method "adam" takes ``iterations`` Adam steps of size ``lr``;
    "lbfgs" (the default) runs L-BFGS with a strong-Wolfe line search for at most
    ``iterations`` loss-and-gradient evaluations (each one forward rollout and its
    adjoint).  The loss is ill-conditioned: the final density mostly fixes Tr and
    G2 / lam (coexistence densities, interface width), lam alone acts only through
    the dynamics.  Adam's per-parameter step normalisation follows the loss down
    the well-determined directions and leaves the others; the quasi-Newton
    curvature estimate resolves all three.  Snapshots along the trajectory add the
    dynamics to the loss.  Returns (theta, losses), one loss per evaluation."""
    import torch

    targets = [target] if snapshots == 1 and not isinstance(target, (list, tuple)) else list(target)
    if len(targets) != snapshots:
        raise ValueError("target must hold one density per snapshot")
    base = theta0.detach().clone().double()
    delta = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    losses = []

    def theta_of(d):
        return base * (1.0 + bound * torch.tanh(d / bound))

    def closure():
        opt.zero_grad()
        rhos = trajectory(theta_of(delta), f0, spec, nsteps, snapshots, checkpoint_every)
        loss = sum(((r - t) ** 2).sum() for r, t in zip(rhos, targets))
        loss.backward()
        losses.append(float(loss.detach()))
        return loss

    if method == "adam":
        opt = torch.optim.Adam([delta], lr=lr)
        for _ in range(iterations):
            closure()
            opt.step()
    elif method == "lbfgs":
        opt = torch.optim.LBFGS([delta], lr=1.0, max_iter=iterations, max_eval=iterations, history_size=10,
                                tolerance_grad=1e-12, tolerance_change=1e-14, line_search_fn="strong_wolfe")
        opt.step(closure)
    else:
        raise ValueError("method must be 'adam' or 'lbfgs'")
    return theta_of(delta).detach(), losses

"""Receiver traces as a differentiable function of the initial field and the source
amplitudes, with the hand-written discrete adjoint as the backward pass.

``traces = PMLTraces.apply(solver, u0, amp, nsteps)`` runs ``nsteps`` RK4 steps of the
discrete PML system from U = u0, V = 0 with the solver's sources scaled by ``amp`` and
returns U at the receivers after every step ([nsteps, nr]).  Its backward pass runs the
transposed scheme (pml_adjoint_step) with the incoming gradient of the traces injected
at the receivers, which yields dL/du0 (U part of the adjoint state at step 0) and
dL/damp (accumulated in FP64 on the device).  The map (u0, amp) -> traces is linear, so
the backward pass needs no forward state: only the traces' gradient.

``PMLTracesSigma.apply(N, w, sigmas, u0, amp, nsteps, coords, receivers, f_peak, t_delay,
precision)`` makes the damping profile (one edge-centred tensor per axis, zero on the
physical edges) a differentiable input as well.  The traces are not linear in sigma, so
its backward pass re-runs the forward steps from u0 with checkpoints every ~sqrt(nsteps)
steps and recomputes the forward states segment by segment while the adjoint runs
(pml_sigma_gradient): dL/dsigma, dL/du0 and dL/damp in one pass, with memory for about
2 sqrt(nsteps) states instead of nsteps.
"""
from __future__ import annotations

import numpy as np
import torch


class PMLTraces(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, u0, amp, nsteps, coords, receivers, f_peak, t_delay):
        nsteps = int(nsteps)
        solver.set_sources(coords, amp.detach().double().cpu().numpy(), f_peak, t_delay)
        tr = solver.set_receivers(receivers, nsteps)
        solver.set_initial(u0.detach())
        solver.step(nsteps)
        ctx.solver = solver
        ctx.nsteps = nsteps
        ctx.amp_dtype = amp.dtype
        ctx.u0_dtype = u0.dtype
        ctx.u0_device = u0.device
        return tr.clone()

    @staticmethod
    def backward(ctx, g):
        s = ctx.solver
        s.adjoint_reset()
        # row k of the injected residual belongs to forward step nsteps - k
        res = torch.flip(g.to(device=s.device, dtype=s.dtype), dims=[0]).contiguous()
        gu, ga = s.adjoint_step(ctx.nsteps, res, want_grad_u=True)
        gu = gu.to(device=ctx.u0_device, dtype=ctx.u0_dtype)
        gamp = torch.from_numpy(np.asarray(ga, dtype=np.float64)).to(ctx.amp_dtype)
        return None, gu, gamp, None, None, None, None, None


def traces(solver, u0, amp, nsteps, coords, receivers, f_peak, t_delay):
    return PMLTraces.apply(solver, u0, amp, nsteps, coords, receivers, f_peak, t_delay)


class PMLTracesSigma(torch.autograd.Function):
    @staticmethod
    def forward(ctx, N, w, u0, amp, nsteps, coords, receivers, f_peak, t_delay, precision, *sigmas):
        from .solver import PMLSolver
        nsteps = int(nsteps)
        sig = [s_.detach().double().cpu().numpy() for s_ in sigmas]
        solver = PMLSolver(N, w, sigma="user", user_sigma=sig, precision=precision, device=u0.device,
                           adjoint=True)
        solver.set_sources(coords, amp.detach().double().cpu().numpy(), f_peak, t_delay)
        tr = solver.set_receivers(receivers, nsteps)
        solver.set_initial(u0.detach())
        solver.step(nsteps)
        ctx.solver = solver
        ctx.nsteps = nsteps
        ctx.u0 = u0.detach()
        ctx.receivers = receivers
        ctx.amp_dtype = amp.dtype
        ctx.sig_meta = [(s_.dtype, s_.device) for s_ in sigmas]
        return tr.clone()

    @staticmethod
    def backward(ctx, g):
        s = ctx.solver
        s.set_initial(ctx.u0)
        s.set_receivers(ctx.receivers, ctx.nsteps)
        _, gsig, ga = s.sigma_gradient(ctx.nsteps, residual=g)
        gu = s.adjoint_read(0).to(dtype=ctx.u0.dtype, device=ctx.u0.device)
        gamp = torch.from_numpy(np.asarray(ga if ga is not None else [], dtype=np.float64)).to(ctx.amp_dtype)
        gs = [torch.from_numpy(x).to(dtype=dt, device=dev) for x, (dt, dev) in zip(gsig, ctx.sig_meta)]
        s.close()
        return (None, None, gu, gamp, None, None, None, None, None, None, *gs)


def traces_sigma(N, w, sigmas, u0, amp, nsteps, coords, receivers, f_peak, t_delay, precision=64):
    return PMLTracesSigma.apply(N, w, u0, amp, nsteps, coords, receivers, f_peak, t_delay, precision, *sigmas)

"""PonD rollout as a torch.autograd.Function with step checkpointing.

``pond_rollout(rho0, nu, ux0, uy0, T0, steps, ckpt_every)`` runs ``steps``
FP64 PonD steps from the equilibrium f = rho0 W in the gauge (u0, T0) and
returns the final density.  Backward recomputes each checkpoint segment
forward (keeping that segment's states on the device), then walks the steps
in reverse through ``pond_adjoint_step_given`` (the hand-written adjoint
kernels: implicit differentiation of the predictor-corrector fixed point,
transposed reconstruction and gauge transform, BGK collision), handing it
each step's output gauge -- the next recomputed state, the next checkpoint or
the final state -- so that it need not recompute the forward step, and
finally ``pond_adjoint_init``.  Gradients are returned for rho0 and nu.

All tensors are CUDA float64 (the boundary is FP64 for both forms); pass
``precision=pond.POND_FP32_MIXED`` to run the forward and the adjoint in the
mixed form, and ``lattice=pond.POND_D2Q9`` (with its ``T_ref``) for the D2Q9
lattice.  Every step of the forward and backward runs in libpond.so.
"""
from __future__ import annotations

import torch

from . import pond


def _get_state(sim, ny, nx, dev):
    f = torch.empty((sim.Q, ny, nx), dtype=torch.float64, device=dev)
    ux = torch.empty((ny, nx), dtype=torch.float64, device=dev)
    uy = torch.empty_like(ux)
    T = torch.empty_like(ux)
    pond.pond_get_state(sim.ctx, 0, f, ux, uy, T)
    return f, ux, uy, T


def _set_state(sim, state):
    f, ux, uy, T = state
    pond.pond_set_state(sim.ctx, 0, None, ux, uy, T, f)


class PondRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, nu, ux0, uy0, T0, steps: int, ckpt_every: int, overrides=None):
        if not rho0.is_cuda or rho0.dtype != torch.float64:
            raise TypeError("rho0 must be a CUDA float64 tensor")
        ny, nx = rho0.shape
        dev = rho0.device
        stream = torch.cuda.current_stream(dev).cuda_stream
        cfg = dict(overrides or {})
        precision = cfg.pop("precision", pond.POND_FP64)
        sim = pond.Sim(nx, ny, precision, stream=stream, nu=float(nu), **cfg)
        pond.pond_set_state(sim.ctx, 0, rho0.contiguous(), ux0.contiguous(), uy0.contiguous(),
                            T0.contiguous(), None)
        ckpts = []
        for t in range(steps):
            if t % ckpt_every == 0:
                ckpts.append(_get_state(sim, ny, nx, dev))
            pond.pond_step(sim.ctx, 1, want_stats=False)
        rho = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        pond.pond_moments(sim.ctx, 0, rho)
        ctx.final = _get_state(sim, ny, nx, dev)
        ctx.sim = sim
        ctx.ckpts = ckpts
        ctx.steps = steps
        ctx.ckpt_every = ckpt_every
        ctx.shape = (ny, nx)
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        sim = ctx.sim
        ny, nx = ctx.shape
        dev = grad_rho.device
        # rho = sum_q f_q  =>  fbar_q = rho_bar for every q
        fbar = grad_rho.contiguous().expand(sim.Q, ny, nx).contiguous()
        gbar = torch.zeros((3, ny, nx), dtype=torch.float64, device=dev)
        fbar_new = torch.empty_like(fbar)
        gbar_new = torch.empty_like(gbar)
        steps, every = ctx.steps, ctx.ckpt_every
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * every
            end = min(start + every, steps)
            states = [ctx.ckpts[seg]]
            _set_state(sim, ctx.ckpts[seg])
            for _ in range(start, end - 1):
                pond.pond_step(sim.ctx, 1, want_stats=False)
                states.append(_get_state(sim, ny, nx, dev))
            for t in reversed(range(start, end)):
                # the step's output state: recomputed, the next checkpoint, or final
                if t + 1 < end:
                    nxt = states[t + 1 - start]
                elif seg + 1 < len(ctx.ckpts):
                    nxt = ctx.ckpts[seg + 1]
                else:
                    nxt = ctx.final
                _set_state(sim, states[t - start])
                # the nu cotangent accumulates on the device: no wait per step
                pond.pond_adjoint_step_given(sim.ctx, nxt[1], nxt[2], nxt[3], fbar, gbar,
                                             fbar_new, gbar_new, nu_on_device=True)
                fbar, fbar_new = fbar_new, fbar
                gbar, gbar_new = gbar_new, gbar
            del states
        rho_bar = torch.empty((ny, nx), dtype=torch.float64, device=dev)
        pond.pond_adjoint_init(sim.ctx, fbar, rho_bar)
        nu_bar = pond.pond_adjoint_nu_bar(sim.ctx)
        torch.cuda.current_stream(dev).synchronize()
        sim.close()
        nu_grad = torch.tensor(nu_bar, dtype=torch.float64, device=dev)
        return rho_bar, nu_grad, None, None, None, None, None, None


def pond_rollout(rho0, nu, ux0, uy0, T0, steps: int, ckpt_every: int = 20, **overrides):
    """Final density after ``steps`` PonD steps (differentiable in rho0 and
    nu).  ``nu`` may be a float or a 0-d tensor; ``overrides`` are config
    fields (and ``precision``)."""
    if not torch.is_tensor(nu):
        nu = torch.tensor(float(nu), dtype=torch.float64, device=rho0.device)
    return PondRollout.apply(rho0, nu, ux0, uy0, T0, steps, ckpt_every, overrides or None)

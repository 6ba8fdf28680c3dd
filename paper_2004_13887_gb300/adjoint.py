"""Gradients through the time stepping: a torch.autograd.Function around the
library's steps and its step adjoint (sph_step_adjoint).

``Steps.apply(solver, dt, K, nsteps, *U0)`` advances the 5 fields U0 (CUDA float64
tensors, the layout of Solver.set_state) by nsteps steps of K Picard iterations
and returns U^N; its backward maps dJ/dU^N to dJ/dU0.  Memory: the forward keeps
the state every ceil(sqrt(nsteps)) steps (checkpoints); the backward re-runs each
stretch between checkpoints forwards, keeping its states, then walks it
backwards through the step adjoint -- about sqrt(nsteps) states held and one
extra forward pass in all.  Every step, forward and adjoint, runs in the
library's kernels; this module only orders the calls and keeps the checkpoints.
The solver must be an FP64 solver (the adjoint is the FP64 scheme's)."""
from __future__ import annotations

import math


def _clone(fields):
    return [f.clone() for f in fields]


def _steps_between(solver, dt, K, state, n):
    """the states after 0, 1, .., n-1 steps from `state` (n states)"""
    out = [_clone(state)]
    solver.set_state(state)
    for _ in range(n - 1):
        solver.step(dt, K)
        out.append(_clone(solver.get_state()))
    return out


def checkpoint_stride(nsteps: int) -> int:
    return max(1, int(math.ceil(math.sqrt(nsteps))))


def _make_function():
    import torch

    class Steps(torch.autograd.Function):
        @staticmethod
        def forward(ctx, solver, dt, K, nsteps, *U0):
            c = checkpoint_stride(nsteps)
            cps = []
            solver.set_state([u.detach().contiguous() for u in U0])
            for n in range(nsteps):
                if n % c == 0:
                    cps.append(_clone(solver.get_state()))
                solver.step(dt, K)
            ctx.solver, ctx.dt, ctx.K, ctx.nsteps, ctx.c = solver, dt, K, nsteps, c
            ctx.cps = cps
            return tuple(solver.get_state())

        @staticmethod
        def backward(ctx, *lam):
            solver, dt, K, nsteps, c = ctx.solver, ctx.dt, ctx.K, ctx.nsteps, ctx.c
            shapes = solver.shapes
            lam = [l.contiguous() if l is not None else torch.zeros(s, dtype=torch.float64, device="cuda")
                   for l, s in zip(lam, shapes)]
            for seg in range(len(ctx.cps) - 1, -1, -1):
                start = seg * c
                n = min(c, nsteps - start)
                states = _steps_between(solver, dt, K, ctx.cps[seg], n)
                for st in reversed(states):
                    solver.set_state(st)
                    lam = solver.step_adjoint(dt, K, lam)
            return (None, None, None, None) + tuple(lam)

    return Steps


_STEPS = None


def steps(solver, dt: float, K: int, nsteps: int, U0):
    """U^N from U0 (5 CUDA float64 tensors), differentiable in U0."""
    global _STEPS
    if _STEPS is None:
        _STEPS = _make_function()
    return list(_STEPS.apply(solver, float(dt), int(K), int(nsteps), *U0))


def kinetic_energy(U, grid, bg, par):
    """Kinetic energy 1/2 sum rho |u|^2 dV of a state (torch, differentiable):
    rho from the stiffened-gas EOS at the centres, the velocity components
    averaged from their faces to the centres, dV the exact cell volumes."""
    import torch
    dev = U[0].device
    bgp = torch.as_tensor(bg[0][1:-1], dtype=torch.float64, device=dev)[:, None, None]
    bgT = torch.as_tensor(bg[1][1:-1], dtype=torch.float64, device=dev)[:, None, None]
    Rg = par.cv * (par.gamma - 1.0)
    rho = (U[0] + bgp + par.pinf) / (Rg * (U[4] + bgT))
    ur = 0.5 * (U[1][1:] + U[1][:-1])
    ut = 0.5 * (U[2][:, 1:] + U[2][:, :-1])
    up = 0.5 * (U[3] + torch.roll(U[3], -1, dims=2)) if grid.periodic else 0.5 * (U[3][:, :, 1:] + U[3][:, :, :-1])
    rf = torch.as_tensor(grid.rf(), dtype=torch.float64, device=dev)
    tf = torch.as_tensor(grid.tf(), dtype=torch.float64, device=dev)
    V = ((rf[1:] ** 3 - rf[:-1] ** 3) / 3)[:, None, None] * (torch.cos(tf[:-1]) - torch.cos(tf[1:]))[None, :, None] \
        * grid.dph
    return 0.5 * torch.sum(rho * (ur * ur + ut * ut + up * up) * V)

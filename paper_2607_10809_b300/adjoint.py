"""Differentiable rollouts: a torch.autograd.Function over a number of
ADER-HWENO steps of the CUDA library, with the hand-written adjoint step of
the C ABI (hw_step_adjoint) and checkpointing every `every` steps.

The time steps are held fixed (they are inputs, not differentiated).  The
backward pass restores each checkpoint, recomputes the states of its segment
and runs the adjoint steps of the segment in reverse.  The last segment is
not recomputed: the forward pass keeps its states and edge-point data (the
backward pass starts with it)."""
from __future__ import annotations

import numpy as np
import torch

from . import hweno


class Rollout(torch.autograd.Function):
    """U_T = S_{dt_K} o ... o S_{dt_1} (U_0).  U_0, U_T: float64 CPU tensors
    [3, m, ntri] in the caller's numbering (cell averages of W, W_x, W_y)."""

    @staticmethod
    def forward(ctx, U0, solver, dts, every):
        s = solver
        buf = s.state_buffer()
        s.host_to_internal(np.asarray(U0.detach().cpu().numpy(), dtype=np.float64), buf)
        s.import_state(buf, 0.0)
        ckpts, times, t = [], [], 0.0
        last = (len(dts) - 1) // every * every if len(dts) else 0   # first step of the last segment
        states = [s.state_buffer() for _ in range(every)]
        pbs = [s.pb_buffer() for _ in range(every)]
        for k, dt in enumerate(dts):
            if k % every == 0:
                c = s.state_buffer()
                s.export_state(c)
                ckpts.append(c)
                times.append(t)
            if k >= last:   # keep the last segment's states and edge-point data
                s.export_state(states[k - last])
                s.step_keep(float(dt), pbs[k - last])
            else:
                s.step(float(dt))
            t += float(dt)
        UT = _host_tensor(U0.shape)
        s.get_state(out=UT.numpy())
        ctx.solver, ctx.dts, ctx.every, ctx.ckpts, ctx.times = s, list(dts), every, ckpts, times
        ctx.states, ctx.pbs = states, pbs
        return UT

    @staticmethod
    def backward(ctx, gUT):
        s, dts, every = ctx.solver, ctx.dts, ctx.every
        ub = s.state_buffer()
        s.host_to_internal(np.asarray(gUT.detach().cpu().numpy(), dtype=np.float64), ub)
        ubn = s.state_buffer()
        scratch = s.adjoint_scratch()
        states, pbs = ctx.states, ctx.pbs
        for seg in reversed(range(len(ctx.ckpts))):
            start, end = seg * every, min((seg + 1) * every, len(dts))
            if seg < len(ctx.ckpts) - 1:         # the last segment's data are still in the buffers
                s.import_state(ctx.ckpts[seg], ctx.times[seg])
                for k in range(start, end):      # recompute the segment's states and edge-point data
                    s.export_state(states[k - start])
                    s.step_keep(float(dts[k]), pbs[k - start])
            for k in reversed(range(start, end)):
                s.step_adjoint(float(dts[k]), states[k - start], ub, ubn, scratch, pbs[k - start])
                ub, ubn = ubn, ub
        g0 = _host_tensor(gUT.shape)
        s.internal_to_host(ub, out=g0.numpy())
        return g0, None, None, None


def _host_tensor(shape):
    """float64 CPU tensor in pinned memory (direct device-to-host copies)."""
    return torch.empty(tuple(shape), dtype=torch.float64, pin_memory=True)


def rollout(U0, solver, dts, every=10):
    """Differentiable map U0 -> U_T (see Rollout)."""
    return Rollout.apply(U0, solver, dts, every)


def cfl_steps(solver, U0, nsteps):
    """The CFL time steps of an unperturbed forward run (held fixed afterwards)."""
    solver.set_state(np.asarray(U0, dtype=np.float64), 0.0)
    dts = []
    for _ in range(nsteps):
        dts.append(solver.time()[1])
        solver.step()
    return dts

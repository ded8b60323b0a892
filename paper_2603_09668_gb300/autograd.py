"""torch.autograd wrappers of the MPM substep with checkpointing.

`mpm_frames` runs n_substeps substeps and returns the particle positions at
every `every`-th substep. Forward runs each segment of `every` substeps with
mpm_rollout and keeps only its starting state (a checkpoint); backward walks
the segments in reverse and calls mpm_segment_adjoint, which recomputes the
segment's intermediate states from its checkpoint into a tape and runs the
substep adjoints through them, so a rollout of S substeps holds S/every +
every states instead of S. Gradients flow to the wind-field values, Young's
modulus E and the initial state.
"""
from __future__ import annotations

import torch

from . import binding as B


class _MpmFrames(torch.autograd.Function):
    @staticmethod
    def forward(ctx, wind_values, E, x0, v0, C0, F0, cfg):
        mpm: B.MPM = cfg["mpm"]
        wind = B.WindField(wind_values.detach(), cfg["t_total"])
        mpm.set_material(float(E.detach()), mpm.nu)
        dt, every, S, t0 = mpm.dt, cfg["every"], cfg["n_substeps"], cfg["t0"]
        pinned = cfg.get("pinned")
        state = B.MpmState(x0.detach().clone(), v0.detach().clone(), C0.detach().clone(),
                           F0.detach().clone())
        ids = None
        if cfg.get("sort", True) and state.n > 0:
            # one sort by cell for the whole rollout (particles move far less
            # than a cell per checkpoint interval), undone on the outputs
            sorted_state = B.MpmState.empty_like(state)
            pin_s = torch.empty_like(pinned) if pinned is not None else None
            ids = torch.empty(state.n, dtype=torch.int32, device=state.x.device)
            mpm.sort(state, sorted_state, pinned, pin_s, None, ids)
            state, pinned = sorted_state, pin_s
        ckpts, frames = [], []
        for k0 in range(0, S, every):
            k1 = min(S, k0 + every)
            ckpts.append(state.clone())
            mpm.rollout(state, pinned, None, wind, t0 + k0 * dt, k1 - k0, 0)
            if k1 % every == 0:
                frames.append(state.x.clone())
        out = torch.stack(frames)
        if ids is not None:
            unsorted = torch.empty_like(out)
            unsorted[:, :, ids.long()] = out
            out = unsorted
        ctx.cfg = cfg
        ctx.ckpts = ckpts
        ctx.ids = ids
        ctx.pinned = pinned
        ctx.E = float(E.detach())
        ctx.save_for_backward(wind_values)
        return out

    @staticmethod
    def backward(ctx, g_frames):
        cfg = ctx.cfg
        mpm: B.MPM = cfg["mpm"]
        (wind_values,) = ctx.saved_tensors
        wind = B.WindField(wind_values.detach(), cfg["t_total"])
        mpm.set_material(ctx.E, mpm.nu)
        dt, every, S, t0 = mpm.dt, cfg["every"], cfg["n_substeps"], cfg["t0"]
        ids = ctx.ids.long() if ctx.ids is not None else None
        if ids is not None:
            g_frames = g_frames[:, :, ids]
        g = B.MpmState.zeros_like(ctx.ckpts[0])
        g_wind = torch.zeros_like(wind_values)
        g_E = torch.zeros(1, dtype=torch.float32, device=wind_values.device)
        n = g.n
        tape = torch.empty(max(every - 1, 1) * 24 * n, dtype=torch.float32, device=g.x.device)
        for seg in reversed(range(len(ctx.ckpts))):
            k0 = seg * every
            k1 = min(S, k0 + every)
            if (k1 % every == 0) and (k1 // every - 1) < g_frames.shape[0]:
                g.x.add_(g_frames[k1 // every - 1])
            mpm.segment_adjoint(ctx.ckpts[seg], tape, g, ctx.pinned, wind, t0 + k0 * dt, k1 - k0,
                                g_wind, g_E)
        ctx.ckpts = None
        out = [g.x, g.v, g.C, g.F]
        if ids is not None:
            for i, a in enumerate(out):
                u = torch.empty_like(a)
                u[:, ids] = a
                out[i] = u
        return (g_wind, g_E.reshape(()), *out, None)


def mpm_frames(mpm: B.MPM, state0: B.MpmState, wind_values: torch.Tensor, t_total: float,
               E: torch.Tensor, n_substeps: int, every: int, pinned=None, t0: float = 0.0,
               sort: bool = True):
    """Positions [n_substeps // every, 3, n] after every `every` substeps,
    differentiable with respect to wind_values, E and state0. With sort, the
    particles are ordered by cell once at the start (the outputs and
    gradients are in the caller's order)."""
    cfg = dict(mpm=mpm, t_total=t_total, n_substeps=n_substeps, every=every, pinned=pinned, t0=t0,
               sort=sort)
    return _MpmFrames.apply(wind_values, E, state0.x, state0.v, state0.C, state0.F, cfg)


class _LbmSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0, lbm, solid, steps, every):
        f = f0.detach().clone()
        ckpts = []
        done = 0
        while done < steps:
            k = min(every, steps - done)
            ckpts.append((f.clone(), k))
            lbm.step(f, solid, k)
            done += k
        ctx.lbm, ctx.solid, ctx.ckpts = lbm, solid, ckpts
        return f

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous().clone()
        for f_start, k in reversed(ctx.ckpts):
            ctx.lbm.step_adjoint(f_start, g, ctx.solid, k)
        ctx.ckpts = None
        return g, None, None, None, None


def lbm_steps(lbm: B.LBM, f0: torch.Tensor, solid, steps: int, every: int = 2):
    """Populations after `steps` lattice steps, differentiable with respect to
    f0; the adjoint recomputes each segment of `every` <= max_tape steps."""
    return _LbmSteps.apply(f0, lbm, solid, steps, every)

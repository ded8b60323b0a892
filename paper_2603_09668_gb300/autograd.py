"""torch.autograd wrappers of the MPM substep with checkpointing.

`mpm_frames` runs n_substeps substeps and returns the particle positions at
every `every`-th substep. Forward keeps only the state at the start of each
segment of `every` substeps (a checkpoint); backward walks the segments in
reverse, recomputes the segment's intermediate states from its checkpoint
and runs mpm_substep_adjoint through them, so a rollout of S substeps holds
S/every + every states instead of S. Gradients flow to the wind-field values,
Young's modulus E and the initial state.
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
        ckpts, frames = [], []
        for k in range(S):
            if k % every == 0:
                ckpts.append(state.clone())
            mpm.substep(state, state, pinned, wind, t0 + k * dt)
            if (k + 1) % every == 0:
                frames.append(state.x.clone())
        ctx.cfg = cfg
        ctx.ckpts = ckpts
        ctx.E = float(E.detach())
        ctx.save_for_backward(wind_values)
        return torch.stack(frames)

    @staticmethod
    def backward(ctx, g_frames):
        cfg = ctx.cfg
        mpm: B.MPM = cfg["mpm"]
        (wind_values,) = ctx.saved_tensors
        wind = B.WindField(wind_values.detach(), cfg["t_total"])
        mpm.set_material(ctx.E, mpm.nu)
        dt, every, S, t0 = mpm.dt, cfg["every"], cfg["n_substeps"], cfg["t0"]
        pinned = cfg.get("pinned")
        g = B.MpmState.zeros_like(ctx.ckpts[0])
        g_wind = torch.zeros_like(wind_values)
        g_E = torch.zeros(1, dtype=torch.float32, device=wind_values.device)
        n_seg = len(ctx.ckpts)
        for seg in reversed(range(n_seg)):
            k0 = seg * every
            k1 = min(S, k0 + every)
            if (k1 % every == 0) and (k1 // every - 1) < g_frames.shape[0]:
                g.x.add_(g_frames[k1 // every - 1])
            states = [ctx.ckpts[seg]]
            for k in range(k0, k1 - 1):
                s = states[-1].clone()
                mpm.substep(s, s, pinned, wind, t0 + k * dt)
                states.append(s)
            for j in reversed(range(k1 - k0)):
                mpm.substep_adjoint(states[j], g, g, pinned, wind, t0 + (k0 + j) * dt, g_wind, g_E)
        ctx.ckpts = None
        return g_wind, g_E.reshape(()), g.x, g.v, g.C, g.F, None


def mpm_frames(mpm: B.MPM, state0: B.MpmState, wind_values: torch.Tensor, t_total: float,
               E: torch.Tensor, n_substeps: int, every: int, pinned=None, t0: float = 0.0):
    """Positions [n_substeps // every, 3, n] after every `every` substeps,
    differentiable with respect to wind_values, E and state0."""
    cfg = dict(mpm=mpm, t_total=t_total, n_substeps=n_substeps, every=every, pinned=pinned, t0=t0)
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

"""Python binding of the libdiffwind C-ABI, one function per C entry point
with the same name. Arguments are torch CUDA tensors (float32 / uint8 /
int32, contiguous); the binding only checks and marshals them: every step of
the computation runs in the library's CUDA kernels.

Layouts follow include/diffwind.h: particle state x, v as [3, n], C, F as
[9, n]; wind values [n_frames, nf, nf, nf, 3]; LBM populations [19, nz, ny, nx]
(shifted, f - w); masks uint8 [nz, ny, nx].
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import NamedTuple, Optional

import numpy as np
import torch

from ._capi import (DiffWindError, DwCamera, DwBatchConfig, DwBatchTrial, DwLbmDesc, DwMpmDesc, DwMpmScene,
                    DwMpmState, DwWindField, check, lib)

__all__ = ["DiffWindError", "MpmState", "WindField", "wind_field_sample",
           "wind_field_sample_adjoint", "mpm_create", "mpm_destroy", "mpm_set_material",
           "mpm_substep", "mpm_substep_adjoint", "mpm_segment_adjoint", "mpm_sort", "mpm_device_status", "mpm_rollout",
           "mpm_profile_enable", "mpm_profile_read", "mpm_substep_noalloc", "lbm_create",
           "lbm_destroy", "lbm_step", "lbm_cache_mask", "fp32_peak", "lbm_step_adjoint", "lbm_macroscopic",
           "lbm_init_equilibrium", "lbm_home_init", "lbm_home_step", "lbm_home_macroscopic",
           "lbm_home_sample_velocity",
           "voxelize_particles", "lbm_sample_velocity", "wind_phys_loss",
           "adam_step", "wind_drag_force", "position_loss", "wind_field_scores", "vector_adam_step", "camera",
           "gs_covariance", "image_l1_loss", "image_dssim_loss", "GaussianRenderer", "MPM", "LBM", "surr_create",
           "surr_destroy", "surr_num_params", "surr_set_params", "surr_get_params",
           "surr_get_grads", "surr_zero_grads", "surr_features", "surr_set_features",
           "surr_get_features", "surr_forward", "surr_loss", "surr_set_output_grad",
           "surr_backward", "surr_device_status", "surr_adam", "surr_apply", "lbm_velocity_error", "Surrogate",
           "surr_features_fine", "surr_advance_fine", "surr_write_lattice",
           "surr_fine_velocity_error", "surr_set_correction", "surr_set_inlet", "mpm_batch_create", "mpm_batch_destroy",
           "mpm_batch_layout", "mpm_batch_rollout", "mpm_batch_set_config",
           "mpm_batch_get_config", "mpm_batch_tune", "mpm_batch_device_status", "mpm_batch_barrier_selftest",
           "mpm_batch_wind_layout", "mpm_batch_segment_adjoint", "MPMBatch"]

NEOHOOKEAN, FIXED_COROTATED = 0, 1
BATCH_PERSISTENT, BATCH_SPLIT, BATCH_PAIR = 0, 1, 2
P2G_AUTO, P2G_ATOMIC, P2G_WARP, P2G_TILE, P2G_PAIR = 0, 1, 2, 3, 4


def _dev(t: Optional[torch.Tensor], dtype=torch.float32, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (libdiffwind has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


class MpmState(NamedTuple):
    x: torch.Tensor  # [3, n]
    v: torch.Tensor  # [3, n]
    C: torch.Tensor  # [9, n]
    F: torch.Tensor  # [9, n]

    @property
    def n(self):
        return self.x.shape[1]

    def to_c(self):
        n = self.x.shape[1]
        for name, t, rows in (("x", self.x, 3), ("v", self.v, 3), ("C", self.C, 9), ("F", self.F, 9)):
            if t.dim() != 2 or t.shape[0] != rows or t.shape[1] != n:
                raise ValueError(f"state.{name} must have shape [{rows}, {n}], got {tuple(t.shape)}")
        return DwMpmState(_dev(self.x, name="x"), _dev(self.v, name="v"), _dev(self.C, name="C"),
                          _dev(self.F, name="F"), n)

    @staticmethod
    def empty_like(s: "MpmState") -> "MpmState":
        return MpmState(*(torch.empty_like(a) for a in s))

    @staticmethod
    def zeros_like(s: "MpmState") -> "MpmState":
        return MpmState(*(torch.zeros_like(a) for a in s))

    def clone(self) -> "MpmState":
        return MpmState(*(a.clone() for a in self))


class WindField(NamedTuple):
    values: torch.Tensor  # [n_frames, nf, nf, nf, 3]
    t_total: float

    @property
    def nf(self):
        return self.values.shape[1]

    @property
    def n_frames(self):
        return self.values.shape[0]

    def to_c(self):
        v = self.values
        if v.dim() != 5 or v.shape[4] != 3 or not (v.shape[1] == v.shape[2] == v.shape[3]):
            raise ValueError(f"wind values must be [n_frames, nf, nf, nf, 3], got {tuple(v.shape)}")
        return DwWindField(_dev(v, name="wind.values"), v.shape[1], v.shape[0], float(self.t_total))


# -------------------------------------------------------------------- wind --

def wind_field_sample(wind: WindField, pos: torch.Tensor, t: float, out=None, stream=None):
    n = pos.shape[1]
    if out is None:
        out = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    w = wind.to_c()
    check(lib().wind_field_sample(ct.byref(w), _dev(pos, name="pos"), n, t, _dev(out, name="out"),
                                  _stream(stream)))
    return out


def wind_field_sample_adjoint(wind: WindField, pos, t, g_out, g_values, stream=None):
    w = wind.to_c()
    check(lib().wind_field_sample_adjoint(ct.byref(w), _dev(pos, name="pos"), pos.shape[1], t,
                                          _dev(g_out, name="g_out"), _dev(g_values, name="g_values"),
                                          _stream(stream)))
    return g_values


# --------------------------------------------------------------------- MPM --

def mpm_create(n_grid, dt, gravity=(0.0, -9.8, 0.0), bc_band=3, material=NEOHOOKEAN, E=1e4,
               nu=0.3, p_mass=1.0, p_vol=1.0, max_particles=0, p2g_mode=P2G_AUTO):
    d = DwMpmDesc(int(n_grid), float(dt), (ct.c_float * 3)(*gravity), int(bc_band), int(material),
                  float(E), float(nu), float(p_mass), float(p_vol), int(max_particles), int(p2g_mode))
    h = ct.c_void_p()
    check(lib().mpm_create(ct.byref(d), ct.byref(h)))
    return h


def mpm_destroy(h):
    check(lib().mpm_destroy(h))


def mpm_set_material(h, E, nu):
    check(lib().mpm_set_material(h, float(E), float(nu)))


def _pin(pinned):
    return _dev(pinned, torch.uint8, "pinned") if pinned is not None else None


def mpm_substep(h, state_in: MpmState, state_out: MpmState, pinned, wind: WindField, t,
                stream=None):
    a, b, w = state_in.to_c(), state_out.to_c(), wind.to_c()
    check(lib().mpm_substep(h, ct.byref(a), ct.byref(b), _pin(pinned), ct.byref(w), float(t),
                            _stream(stream)))
    return state_out


def mpm_substep_adjoint(h, state_in: MpmState, g_out: MpmState, g_in: MpmState, pinned,
                        wind: WindField, t, g_wind=None, g_E=None, stream=None):
    a, go, gi, w = state_in.to_c(), g_out.to_c(), g_in.to_c(), wind.to_c()
    check(lib().mpm_substep_adjoint(h, ct.byref(a), ct.byref(go), ct.byref(gi), _pin(pinned),
                                    ct.byref(w), float(t), _dev(g_wind, name="g_wind"),
                                    _dev(g_E, name="g_E"), _stream(stream)))
    return g_in


def mpm_segment_adjoint(h, start: MpmState, tape, g: MpmState, pinned, wind: WindField, t0,
                        n_substeps, g_wind=None, g_E=None, stream=None):
    """Reverse mode of a segment of n_substeps substeps from `start`; tape is a
    device float32 tensor of at least (n_substeps - 1) * 24 * n elements."""
    a, gg, w = start.to_c(), g.to_c(), wind.to_c()
    tp = _dev(tape, name="tape") if tape is not None else None
    nt = tape.numel() if tape is not None else 0
    check(lib().mpm_segment_adjoint(h, ct.byref(a), tp, int(nt), ct.byref(gg), _pin(pinned),
                                    ct.byref(w), float(t0), int(n_substeps),
                                    _dev(g_wind, name="g_wind"), _dev(g_E, name="g_E"),
                                    _stream(stream)))
    return g


def mpm_sort(h, state_in: MpmState, state_out: MpmState, pinned_in, pinned_out, ids_in, ids_out,
             stream=None):
    a, b = state_in.to_c(), state_out.to_c()
    check(lib().mpm_sort(h, ct.byref(a), ct.byref(b), _pin(pinned_in), _pin(pinned_out),
                         _dev(ids_in, torch.int32, "ids_in"), _dev(ids_out, torch.int32, "ids_out"),
                         _stream(stream)))
    return state_out, pinned_out, ids_out


def mpm_device_status(h, stream=None):
    check(lib().mpm_device_status(h, _stream(stream)))


def mpm_rollout(h, state: MpmState, pinned, ids, wind: WindField, t0, n_substeps, sort_every,
                stream=None):
    a, w = state.to_c(), wind.to_c()
    check(lib().mpm_rollout(h, ct.byref(a), _pin(pinned), _dev(ids, torch.int32, "ids"),
                            ct.byref(w), float(t0), int(n_substeps), int(sort_every),
                            _stream(stream)))
    return state


def mpm_substep_noalloc(desc_params: dict, state_in: MpmState, state_out: MpmState, pinned,
                        wind: WindField, t, device_status=None, p2g_mode=P2G_AUTO, stream=None):
    """mpm_substep without a handle: the scratch grid is the library's fixed
    device array (n_grid <= 64), for callers that cannot allocate device
    memory at call time. desc_params holds the dw_mpm_desc fields (n_grid,
    dt, gravity, bc_band, material, E, nu, p_mass, p_vol); device_status is an
    optional device int32[1] that receives device-side error bits."""
    p = desc_params
    d = DwMpmDesc(int(p["n_grid"]), float(p["dt"]), (ct.c_float * 3)(*p["gravity"]),
                  int(p["bc_band"]), int(p["material"]), float(p["E"]), float(p["nu"]),
                  float(p["p_mass"]), float(p["p_vol"]), 0, int(p2g_mode))
    a, b, w = state_in.to_c(), state_out.to_c(), wind.to_c()
    check(lib().mpm_substep_noalloc(ct.byref(d), ct.byref(a), ct.byref(b), _pin(pinned),
                                    ct.byref(w), float(t),
                                    _dev(device_status, torch.int32, "device_status"),
                                    _stream(stream)))
    return state_out


def mpm_state_save(path, state: MpmState, pinned=None, ids=None, t=0.0, substep=0, stream=None):
    """Host checkpoint of a state (and pinned, ids when given) to `path`."""
    a = state.to_c()
    check(lib().mpm_state_save(os.fsencode(path), ct.byref(a), _pin(pinned),
                               _dev(ids, torch.int32, "ids"), float(t), int(substep),
                               _stream(stream)))


def mpm_state_peek(path):
    """Header of a checkpoint: dict(n, has_pinned, has_ids, t, substep)."""
    n, flags, t, k = ct.c_int64(), ct.c_int32(), ct.c_double(), ct.c_int64()
    check(lib().mpm_state_peek(os.fsencode(path), ct.byref(n), ct.byref(flags), ct.byref(t),
                               ct.byref(k)))
    return dict(n=n.value, has_pinned=bool(flags.value & 1), has_ids=bool(flags.value & 2),
                t=t.value, substep=k.value)


def mpm_state_load(path, state: MpmState, pinned=None, ids=None, stream=None):
    """Reads a checkpoint into `state` (and pinned, ids); returns (t, substep)."""
    a = state.to_c()
    t, k = ct.c_double(), ct.c_int64()
    check(lib().mpm_state_load(os.fsencode(path), ct.byref(a), _pin(pinned),
                               _dev(ids, torch.int32, "ids"), ct.byref(t), ct.byref(k),
                               _stream(stream)))
    return t.value, k.value


KERNEL_NAMES = ["p2g", "grid", "g2p", "rev_g2p", "rev_grid", "rev_p2g", "sort", "g2p2g"]


def mpm_profile_enable(h, max_records):
    check(lib().mpm_profile_enable(h, int(max_records)))


def mpm_profile_read(h):
    """{kernel name: (total device ms, launches)} since enable / the last read."""
    ms = (ct.c_double * len(KERNEL_NAMES))()
    cnt = (ct.c_int64 * len(KERNEL_NAMES))()
    check(lib().mpm_profile_read(h, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_NAMES)}


# ------------------------------------------------------------- batched MPM --

def _desc_of(p: dict, max_particles=0, p2g_mode=P2G_AUTO):
    return DwMpmDesc(int(p["n_grid"]), float(p["dt"]), (ct.c_float * 3)(*p["gravity"]),
                     int(p["bc_band"]), int(p["material"]), float(p["E"]), float(p["nu"]),
                     float(p["p_mass"]), float(p["p_vol"]), int(max_particles), int(p2g_mode))


def mpm_batch_create(scenes):
    """scenes: sequence of (params dict as for mpm_substep_noalloc, n_particles,
    WindField). The wind tensors must outlive the handle."""
    arr = (DwMpmScene * len(scenes))()
    for i, (params, n, wind) in enumerate(scenes):
        arr[i] = DwMpmScene(_desc_of(params), int(n), wind.to_c())
    h = ct.c_void_p()
    check(lib().mpm_batch_create(arr, len(scenes), ct.byref(h)))
    return h


def mpm_batch_destroy(h):
    check(lib().mpm_batch_destroy(h))


def mpm_batch_layout(h, n_scenes):
    """(total particle count, [off_0, ..., off_n_scenes])."""
    n = ct.c_int64()
    offs = (ct.c_int64 * (n_scenes + 1))()
    check(lib().mpm_batch_layout(h, ct.byref(n), offs))
    return n.value, list(offs)


def mpm_batch_rollout(h, state: MpmState, pinned, ids, t0, n_substeps, sort_every, stream=None):
    a = state.to_c()
    check(lib().mpm_batch_rollout(h, ct.byref(a), _pin(pinned), _dev(ids, torch.int32, "ids"),
                                  float(t0), int(n_substeps), int(sort_every), _stream(stream)))
    return state


def _config_dict(c: DwBatchConfig):
    return {"mode": c.mode, "threads": c.threads, "ctas_per_sm": c.ctas_per_sm,
            "use_graph": c.use_graph, "graph_active": c.graph_active}


def mpm_batch_set_config(h, mode, threads, ctas_per_sm, use_graph=1):
    c = DwBatchConfig(int(mode), int(threads), int(ctas_per_sm), int(use_graph), 0)
    check(lib().mpm_batch_set_config(h, ct.byref(c)))


def mpm_batch_get_config(h):
    c = DwBatchConfig()
    check(lib().mpm_batch_get_config(h, ct.byref(c)))
    return _config_dict(c)


def mpm_batch_tune(h, state: MpmState, pinned, n_trial_substeps, max_trials=64, stream=None):
    """(best configuration, [(configuration, ms per substep), ...])."""
    a = state.to_c()
    best = DwBatchConfig()
    trials = (DwBatchTrial * max_trials)()
    nt = ct.c_int32()
    check(lib().mpm_batch_tune(h, ct.byref(a), _pin(pinned), int(n_trial_substeps),
                               ct.byref(best), trials, int(max_trials), ct.byref(nt),
                               _stream(stream)))
    return _config_dict(best), [(_config_dict(trials[i].config), trials[i].ms_per_substep)
                                for i in range(nt.value)]


def mpm_batch_device_status(h, stream=None):
    check(lib().mpm_batch_device_status(h, _stream(stream)))


def mpm_batch_barrier_selftest(h, missing_ctas, stream=None):
    check(lib().mpm_batch_barrier_selftest(h, int(missing_ctas), _stream(stream)))


def mpm_batch_wind_layout(h, n_scenes):
    """(total floats of the concatenated wind gradient, [start of each scene's block, ..., total])."""
    n = ct.c_int64()
    offs = (ct.c_int64 * (n_scenes + 1))()
    check(lib().mpm_batch_wind_layout(h, ct.byref(n), offs))
    return n.value, list(offs)


def mpm_batch_segment_adjoint(h, start: MpmState, tape, g: MpmState, pinned, t0, n_substeps,
                              g_wind=None, g_E=None, stream=None):
    """Reverse mode of n_substeps batched substeps from `start` (all scenes);
    tape is a device float32 tensor of at least (n_substeps - 1) * 24 * n
    elements, g_wind the concatenated wind gradient, g_E float32[n_scenes]."""
    a, gg = start.to_c(), g.to_c()
    tp = _dev(tape, name="tape") if tape is not None else None
    nt = tape.numel() if tape is not None else 0
    check(lib().mpm_batch_segment_adjoint(h, ct.byref(a), tp, int(nt), ct.byref(gg), _pin(pinned),
                                          float(t0), int(n_substeps), _dev(g_wind, name="g_wind"),
                                          _dev(g_E, name="g_E"), _stream(stream)))
    return g


# --------------------------------------------------------------------- LBM --

def lbm_create(shape, tau, u_inlet=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0), bc_x=0, max_tape=2):
    nx, ny, nz = shape
    d = DwLbmDesc(int(nx), int(ny), int(nz), float(tau), (ct.c_float * 3)(*u_inlet),
                  (ct.c_float * 3)(*force), int(bc_x), int(max_tape))
    h = ct.c_void_p()
    check(lib().lbm_create(ct.byref(d), ct.byref(h)))
    return h


def lbm_destroy(h):
    check(lib().lbm_destroy(h))


def _mask(solid):
    return _dev(solid, torch.uint8, "solid") if solid is not None else None


def lbm_step(h, f, solid, steps, stream=None):
    check(lib().lbm_step(h, _dev(f, name="f"), _mask(solid), int(steps), _stream(stream)))
    return f


def fp32_peak(paired, iters=4096, blocks_per_sm=8, reps=3):
    """Measured FP32 throughput (FLOP/s) of the probe kernel: scalar FFMA
    (paired=False) or paired FFMA2 (paired=True), best of `reps` launches on
    the current stream, timed with CUDA events."""
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = blocks_per_sm * sms
    out = torch.zeros(blocks, dtype=torch.float32, device=f"cuda:{dev}")
    flops = ct.c_double(0.0)
    stream = torch.cuda.current_stream()
    best = None
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        check(lib().dw_fp32_probe(int(bool(paired)), int(iters), int(blocks), _dev(out, name="out"),
                                  ct.byref(flops), _stream(stream)))
        e1.record(stream)
        e1.synchronize()
        if r == 0:
            continue  # the first launch loads the module
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return flops.value / (best * 1e-3)


def lbm_cache_mask(h, solid, stream=None):
    """Registers `solid` so that calls with this tensor reuse its link words;
    the mask must not change while registered (None drops it)."""
    check(lib().lbm_cache_mask(h, _mask(solid), _stream(stream)))


def lbm_step_adjoint(h, f_in, g_f, solid, steps, stream=None):
    check(lib().lbm_step_adjoint(h, _dev(f_in, name="f_in"), _dev(g_f, name="g_f"), _mask(solid),
                                 int(steps), _stream(stream)))
    return g_f


def lbm_macroscopic(h, f, solid, rho=None, u=None, stream=None):
    check(lib().lbm_macroscopic(h, _dev(f, name="f"), _mask(solid), _dev(rho, name="rho"),
                                _dev(u, name="u"), _stream(stream)))
    return rho, u


def lbm_init_equilibrium(h, f, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
    arr = (ct.c_float * 3)(*u0)
    check(lib().lbm_init_equilibrium(h, _dev(f, name="f"), float(rho0), ct.byref(arr),
                                     _stream(stream)))
    return f


def lbm_home_init(h, m, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
    arr = (ct.c_float * 3)(*u0)
    check(lib().lbm_home_init(h, _dev(m, name="m"), float(rho0), ct.byref(arr), _stream(stream)))
    return m


def lbm_home_step(h, m, solid, steps, stream=None):
    check(lib().lbm_home_step(h, _dev(m, name="m"), _mask(solid), int(steps), _stream(stream)))
    return m


def lbm_home_macroscopic(h, m, solid, rho=None, u=None, stream=None):
    check(lib().lbm_home_macroscopic(h, _dev(m, name="m"), _mask(solid), _dev(rho, name="rho"),
                                     _dev(u, name="u"), _stream(stream)))
    return rho, u


def lbm_home_sample_velocity(h, m, solid, pos, u_out=None, stream=None):
    """u[3][n] of the HOME-LBM moments m at points pos[3][n] (unit cube)."""
    n = pos.shape[1]
    if u_out is None:
        u_out = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    check(lib().lbm_home_sample_velocity(h, _dev(m, name="m"), _mask(solid),
                                         _dev(pos, name="pos"), int(n),
                                         _dev(u_out, name="u_out"), _stream(stream)))
    return u_out


def lbm_sample_velocity(h, f, solid, pos, u_out=None, stream=None):
    """u[3][n] of the lattice f at points pos[3][n] (unit cube)."""
    n = pos.shape[1]
    if u_out is None:
        u_out = torch.empty((3, n), dtype=torch.float32, device=pos.device)
    check(lib().lbm_sample_velocity(h, _dev(f, name="f"), _mask(solid), _dev(pos, name="pos"),
                                    int(n), _dev(u_out, name="u_out"), _stream(stream)))
    return u_out


def wind_phys_loss(values, guide_u, loss, g_values=None, eps=1e-6, weight=1.0, stream=None):
    """loss += weight * L_phys of one keyframe (values [n][3], guide_u [3][n]);
    g_values += weight * its gradient (when given)."""
    n = guide_u.shape[1]
    check(lib().wind_phys_loss(_dev(values, name="values"), _dev(guide_u, name="guide_u"), int(n),
                               float(eps), float(weight), _dev(loss, name="loss"),
                               _dev(g_values, name="g_values"), _stream(stream)))
    return loss


def wind_field_scores(rec, gt, sums=None, eps=1e-12, stream=None):
    """sums[3] += (sum of unit-vector cosines, sum of squared unit-vector
    differences, count) over the locations of rec, gt [n][3] where both have a
    direction; CosSim = sums[0] / sums[2], NMSE = sums[1] / sums[2]."""
    if sums is None:
        sums = torch.zeros(3, dtype=torch.float32, device=rec.device)
    n = rec.numel() // 3
    check(lib().wind_field_scores(_dev(rec, name="rec"), _dev(gt, name="gt"), int(n), float(eps),
                                  _dev(sums, name="sums"), _stream(stream)))
    return sums


def wind_drag_force(u, scale, values=None, stream=None):
    """values[n][3] = scale |u| u for velocities u[3][n] (the drag relation)."""
    n = u.shape[1]
    if values is None:
        values = torch.empty((n, 3), dtype=torch.float32, device=u.device)
    check(lib().wind_drag_force(_dev(u, name="u"), int(n), float(scale),
                                _dev(values, name="values"), _stream(stream)))
    return values


def position_loss(x, x_target, loss, weight=1.0, g_x=None, stream=None):
    """loss += weight sum |x - x_target|^2 (x, x_target [3][n]); g_x += its gradient."""
    n = x.shape[1]
    check(lib().position_loss(_dev(x, name="x"), _dev(x_target, name="x_target"), int(n),
                              float(weight), _dev(loss, name="loss"), _dev(g_x, name="g_x"),
                              _stream(stream)))
    return loss


def adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(lib().adam_step(_dev(param, name="param"), _dev(grad, name="grad"), _dev(m, name="m"),
                          _dev(v, name="v"), int(param.numel()), float(lr), float(beta1),
                          float(beta2), float(eps), int(step), _stream(stream)))
    return param


def vector_adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """VectorAdam on param [n][3] (m [n][3], v [n])."""
    n = param.numel() // 3
    if m.numel() != 3 * n or v.numel() != n or grad.numel() != 3 * n:
        raise ValueError("vector_adam_step: param, grad, m must be [n][3] and v [n]")
    check(lib().vector_adam_step(_dev(param, name="param"), _dev(grad, name="grad"),
                                 _dev(m, name="m"), _dev(v, name="v"), int(n), float(lr),
                                 float(beta1), float(beta2), float(eps), int(step),
                                 _stream(stream)))
    return param


# ---------------------------------------------------- particle-bound Gaussians --

def camera(R, T, fx, fy, cx, cy, width, height, near=0.01) -> DwCamera:
    """A pinhole camera: t = R x + T, pixel = (fx t_x/t_z + cx, fy t_y/t_z + cy)."""
    R = [float(v) for v in np.asarray(R, np.float64).reshape(9)]
    T = [float(v) for v in np.asarray(T, np.float64).reshape(3)]
    return DwCamera((ct.c_float * 9)(*R), (ct.c_float * 3)(*T), float(fx), float(fy), float(cx),
                    float(cy), int(width), int(height), float(near))


def gs_covariance(F, sigma0, sigma=None, stream=None):
    """sigma [6][n] = F sigma0 F^T (F [9][n], sigma0 [6][n])."""
    n = F.shape[1]
    if sigma is None:
        sigma = torch.empty((6, n), dtype=torch.float32, device=F.device)
    check(lib().gs_covariance(_dev(F, name="F"), _dev(sigma0, name="sigma0"), int(n),
                              _dev(sigma, name="sigma"), _stream(stream)))
    return sigma


def image_l1_loss(image, target, loss, weight=1.0, g_image=None, stream=None):
    """loss += weight sum |image - target|; g_image += weight sign(image - target)."""
    check(lib().image_l1_loss(_dev(image, name="image"), _dev(target, name="target"),
                              int(image.numel()), float(weight), _dev(loss, name="loss"),
                              _dev(g_image, name="g_image"), _stream(stream)))
    return loss


def image_dssim_loss(image, target, loss, weight=1.0, g_image=None, workspace=None, stream=None):
    """loss += weight (1 - mean SSIM) of image against target ([C][H][W]);
    g_image += its gradient."""
    C, H, W = image.shape
    if workspace is None:
        workspace = torch.empty(10 * C * H * W, dtype=torch.float32, device=image.device)
    check(lib().image_dssim_loss(_dev(image, name="image"), _dev(target, name="target"), int(C),
                                 int(H), int(W), float(weight), _dev(loss, name="loss"),
                                 _dev(g_image, name="g_image"), _dev(workspace, name="workspace"),
                                 _stream(stream)))
    return loss


class GaussianRenderer:
    """Owns a gs handle: alpha-blended splatting of particle-bound Gaussians
    and its reverse mode (gs_render, gs_render_backward)."""

    def __init__(self, max_gaussians, width, height):
        self.width, self.height = int(width), int(height)
        h = ct.c_void_p()
        check(lib().gs_create(int(max_gaussians), self.width, self.height, ct.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None:
            lib().gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, cam, x, F, sigma0, color, opacity, image=None, stream=None):
        n = x.shape[1]
        if image is None:
            image = torch.empty((3, self.height, self.width), dtype=torch.float32, device=x.device)
        check(lib().gs_render(self.h, ct.byref(cam), _dev(x, name="x"), _dev(F, name="F"),
                              _dev(sigma0, name="sigma0"), _dev(color, name="color"),
                              _dev(opacity, name="opacity"), int(n), _dev(image, name="image"),
                              _stream(stream)))
        return image

    def backward(self, cam, x, F, sigma0, color, opacity, g_image, g_x, g_F, g_color=None,
                 g_opacity=None, stream=None):
        n = x.shape[1]
        check(lib().gs_render_backward(self.h, ct.byref(cam), _dev(x, name="x"),
                                       _dev(F, name="F"), _dev(sigma0, name="sigma0"),
                                       _dev(color, name="color"), _dev(opacity, name="opacity"),
                                       int(n), _dev(g_image, name="g_image"), _dev(g_x, name="g_x"),
                                       _dev(g_F, name="g_F"), _dev(g_color, name="g_color"),
                                       _dev(g_opacity, name="g_opacity"), _stream(stream)))
        return g_x, g_F


def voxelize_particles(pos, shape, dx, solid, stream=None):
    nx, ny, nz = shape
    check(lib().voxelize_particles(_dev(pos, name="pos"), pos.shape[1], int(nx), int(ny), int(nz),
                                   float(dx), _dev(solid, torch.uint8, "solid"), _stream(stream)))
    return solid


# ---------------------------------------------------------- owning handles --

class MPM:
    """Owns an MPM handle; the methods call the C-ABI functions above."""

    def __init__(self, n_grid, dt, *, gravity=(0.0, -9.8, 0.0), bc_band=3, material=NEOHOOKEAN,
                 E=1e4, nu=0.3, p_mass=1.0, p_vol=1.0, max_particles=0, p2g_mode=P2G_AUTO):
        self.n_grid, self.dt = n_grid, dt
        self.E, self.nu = E, nu
        self.p2g_mode = p2g_mode
        self.h = mpm_create(n_grid, dt, gravity, bc_band, material, E, nu, p_mass, p_vol,
                            max_particles, p2g_mode)

    @classmethod
    def from_params(cls, params: dict, max_particles: int, p2g_mode=P2G_AUTO):
        return cls(params["n_grid"], params["dt"], gravity=params["gravity"],
                   bc_band=params["bc_band"], material=params["material"], E=params["E"],
                   nu=params["nu"], p_mass=params["p_mass"], p_vol=params["p_vol"],
                   max_particles=max_particles, p2g_mode=p2g_mode)

    def close(self):
        if getattr(self, "h", None) is not None:
            mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_material(self, E, nu):
        mpm_set_material(self.h, E, nu)
        self.E, self.nu = E, nu

    def substep(self, state_in, state_out, pinned, wind, t, stream=None):
        return mpm_substep(self.h, state_in, state_out, pinned, wind, t, stream)

    def substep_adjoint(self, state_in, g_out, g_in, pinned, wind, t, g_wind=None, g_E=None,
                        stream=None):
        return mpm_substep_adjoint(self.h, state_in, g_out, g_in, pinned, wind, t, g_wind, g_E,
                                   stream)

    def segment_adjoint(self, start, tape, g, pinned, wind, t0, n_substeps, g_wind=None, g_E=None,
                        stream=None):
        return mpm_segment_adjoint(self.h, start, tape, g, pinned, wind, t0, n_substeps, g_wind,
                                   g_E, stream)

    def sort(self, state_in, state_out, pinned_in, pinned_out, ids_in, ids_out, stream=None):
        return mpm_sort(self.h, state_in, state_out, pinned_in, pinned_out, ids_in, ids_out, stream)

    def device_status(self, stream=None):
        mpm_device_status(self.h, stream)

    def rollout(self, state, pinned, ids, wind, t0, n_substeps, sort_every, stream=None):
        return mpm_rollout(self.h, state, pinned, ids, wind, t0, n_substeps, sort_every, stream)

    def profile_enable(self, max_records):
        mpm_profile_enable(self.h, max_records)

    def profile_read(self):
        return mpm_profile_read(self.h)


class MPMBatch:
    """Owns a batch of MPM scenes over one concatenated particle state.

    scenes: sequence of (params dict, n_particles, WindField); scene s owns
    the particles offsets[s]:offsets[s + 1] of the state."""

    def __init__(self, scenes):
        self._winds = [w for _, _, w in scenes]  # the handle reads them on every rollout
        self.n_scenes = len(scenes)
        self.h = mpm_batch_create(scenes)
        self.n, self.offsets = mpm_batch_layout(self.h, self.n_scenes)

    def close(self):
        if getattr(self, "h", None) is not None:
            mpm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rollout(self, state, pinned, ids, t0, n_substeps, sort_every, stream=None):
        return mpm_batch_rollout(self.h, state, pinned, ids, t0, n_substeps, sort_every, stream)

    def set_config(self, mode, threads, ctas_per_sm, use_graph=1):
        mpm_batch_set_config(self.h, mode, threads, ctas_per_sm, use_graph)

    def config(self):
        return mpm_batch_get_config(self.h)

    def tune(self, state, pinned, n_trial_substeps=10, stream=None):
        return mpm_batch_tune(self.h, state, pinned, n_trial_substeps, stream=stream)

    def device_status(self, stream=None):
        mpm_batch_device_status(self.h, stream)

    def barrier_selftest(self, missing_ctas, stream=None):
        mpm_batch_barrier_selftest(self.h, missing_ctas, stream)

    def scene_slice(self, s):
        return slice(self.offsets[s], self.offsets[s + 1])

    def wind_layout(self):
        return mpm_batch_wind_layout(self.h, self.n_scenes)

    def segment_adjoint(self, start, tape, g, pinned, t0, n_substeps, g_wind=None, g_E=None,
                        stream=None):
        return mpm_batch_segment_adjoint(self.h, start, tape, g, pinned, t0, n_substeps, g_wind,
                                         g_E, stream)


class LBM:
    """Owns an LBM handle; the methods call the C-ABI functions above."""

    def __init__(self, shape, tau, *, u_inlet=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0), bc_x=0,
                 max_tape=2):
        self.shape = tuple(shape)
        self.tau = tau
        self.force = force
        self.h = lbm_create(shape, tau, u_inlet, force, bc_x, max_tape)

    def close(self):
        if getattr(self, "h", None) is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lattice(self, device="cuda"):
        nx, ny, nz = self.shape
        return torch.zeros((19, nz, ny, nx), dtype=torch.float32, device=device)

    def step(self, f, solid, steps, stream=None):
        return lbm_step(self.h, f, solid, steps, stream)

    def step_adjoint(self, f_in, g_f, solid, steps, stream=None):
        return lbm_step_adjoint(self.h, f_in, g_f, solid, steps, stream)

    def cache_mask(self, solid, stream=None):
        return lbm_cache_mask(self.h, solid, stream)

    def sample_velocity(self, f, solid, pos, u_out=None, stream=None):
        return lbm_sample_velocity(self.h, f, solid, pos, u_out, stream)

    # HOME-LBM: ten moments per cell instead of nineteen populations
    def moments(self, device="cuda"):
        nx, ny, nz = self.shape
        return torch.zeros((10, nz, ny, nx), dtype=torch.float32, device=device)

    def home_init(self, m, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
        return lbm_home_init(self.h, m, rho0, u0, stream)

    def home_step(self, m, solid, steps, stream=None):
        return lbm_home_step(self.h, m, solid, steps, stream)

    def home_sample_velocity(self, m, solid, pos, u_out=None, stream=None):
        return lbm_home_sample_velocity(self.h, m, solid, pos, u_out, stream)

    def home_macroscopic(self, m, solid, stream=None):
        nx, ny, nz = self.shape
        rho = torch.empty((nz, ny, nx), dtype=torch.float32, device=m.device)
        u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=m.device)
        lbm_home_macroscopic(self.h, m, solid, rho, u, stream)
        return rho, u

    def macroscopic(self, f, solid, stream=None):
        nx, ny, nz = self.shape
        rho = torch.empty((nz, ny, nx), dtype=torch.float32, device=f.device)
        u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=f.device)
        lbm_macroscopic(self.h, f, solid, rho, u, stream)
        return rho, u

    def init_equilibrium(self, f, rho0=1.0, u0=(0.0, 0.0, 0.0), stream=None):
        return lbm_init_equilibrium(self.h, f, rho0, u0, stream)


# --------------------------------------------------------------- surrogate --

def surr_create(n):
    h = ct.c_void_p()
    check(lib().surr_create(int(n), ct.byref(h)))
    return h


def surr_destroy(h):
    check(lib().surr_destroy(h))


def surr_num_params(h):
    c = ct.c_int64()
    check(lib().surr_num_params(h, ct.byref(c)))
    return c.value


def surr_set_params(h, src, stream=None):
    check(lib().surr_set_params(h, _dev(src, name="params"), _stream(stream)))


def surr_get_params(h, dst, stream=None):
    check(lib().surr_get_params(h, _dev(dst, name="params"), _stream(stream)))
    return dst


def surr_get_grads(h, dst, stream=None):
    check(lib().surr_get_grads(h, _dev(dst, name="grads"), _stream(stream)))
    return dst


def surr_zero_grads(h, stream=None):
    check(lib().surr_zero_grads(h, _stream(stream)))


def surr_features(h, f, solid, in_scale=1.0, feats32=None, stream=None):
    check(lib().surr_features(h, _dev(f, name="f"), _mask(solid), float(in_scale),
                              _dev(feats32, name="feats32"), _stream(stream)))
    return feats32


def surr_set_features(h, feats, stream=None):
    check(lib().surr_set_features(h, _dev(feats, name="feats"), _stream(stream)))


def surr_get_features(h, feats_bf16, stream=None):
    check(lib().surr_get_features(h, _dev(feats_bf16, torch.bfloat16, "feats"), _stream(stream)))
    return feats_bf16


def surr_forward(h, out=None, keep_activations=True, stream=None):
    check(lib().surr_forward(h, _dev(out, name="out"), int(bool(keep_activations)), _stream(stream)))
    return out


def surr_features_fine(h, solid, in_scale=1.0, stream=None):
    check(lib().surr_features_fine(h, _mask(solid), float(in_scale), _stream(stream)))


def surr_advance_fine(h, out_scale, solid, in_scale=1.0, stream=None):
    check(lib().surr_advance_fine(h, float(out_scale), _mask(solid), float(in_scale),
                                  _stream(stream)))


def surr_write_lattice(h, solid, f, stream=None):
    check(lib().surr_write_lattice(h, _mask(solid), _dev(f, name="f"), _stream(stream)))
    return f


def surr_set_inlet(h, u):
    """Reference (inlet) velocity of the surrogate's features."""
    arr = (ct.c_float * 3)(*[float(a) for a in u])
    check(lib().surr_set_inlet(h, arr))


def surr_set_correction(h, f, solid, mode, stream=None):
    """Chained-mode defect correction: mode 1 sets corr = u(f) - u_fine, mode 2
    adds that difference, mode 0 stops using it."""
    check(lib().surr_set_correction(h, _dev(f, name="f") if f is not None else None, _mask(solid),
                                    int(mode), _stream(stream)))


def surr_fine_velocity_error(h, f, solid, sums, stream=None):
    check(lib().surr_fine_velocity_error(h, _dev(f, name="f"), _mask(solid),
                                         _dev(sums, torch.float64, "sums"), _stream(stream)))
    return sums


def surr_loss(h, target, loss=None, stream=None):
    check(lib().surr_loss(h, _dev(target, name="target"), _dev(loss, name="loss"), _stream(stream)))


def surr_set_output_grad(h, g_out, stream=None):
    check(lib().surr_set_output_grad(h, _dev(g_out, name="g_out"), _stream(stream)))


def surr_backward(h, stream=None):
    check(lib().surr_backward(h, _stream(stream)))


def surr_device_status(h, stream=None):
    check(lib().surr_device_status(h, _stream(stream)))


def surr_adam(h, lr, beta1, beta2, eps, step, stream=None):
    check(lib().surr_adam(h, float(lr), float(beta1), float(beta2), float(eps), int(step),
                          _stream(stream)))


def surr_apply(h, out, solid, f, out_scale=1.0, stream=None):
    check(lib().surr_apply(h, _dev(out, name="out"), float(out_scale), _mask(solid),
                           _dev(f, name="f"), _stream(stream)))
    return f


def lbm_velocity_error(fa, fb, solid, sums, stream=None):
    ncell = fa.numel() // 19
    check(lib().lbm_velocity_error(_dev(fa, name="fa"), _dev(fb, name="fb"), _mask(solid), ncell,
                                   _dev(sums, torch.float64, "sums"), _stream(stream)))
    return sums


class Surrogate:
    """Owns a surrogate handle (coarse grid n per axis)."""

    def __init__(self, n):
        self.n = n
        self.h = surr_create(n)
        self.nparams = surr_num_params(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            surr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        surr_set_params(self.h, p)

    def params(self, device="cuda"):
        return surr_get_params(self.h, torch.empty(self.nparams, dtype=torch.float32, device=device))

    def grads(self, device="cuda"):
        return surr_get_grads(self.h, torch.empty(self.nparams, dtype=torch.float32, device=device))

    def zero_grads(self):
        surr_zero_grads(self.h)

    def features(self, f, solid, in_scale=1.0, feats32=None):
        return surr_features(self.h, f, solid, in_scale, feats32)

    def set_features(self, feats):
        surr_set_features(self.h, feats)

    def get_features(self):
        out = torch.empty((self.n ** 3, 16), dtype=torch.bfloat16, device="cuda")
        return surr_get_features(self.h, out)

    def forward(self, out=None, keep_activations=True):
        return surr_forward(self.h, out, keep_activations)

    def features_fine(self, solid, in_scale=1.0):
        surr_features_fine(self.h, solid, in_scale)

    def advance_fine(self, out_scale, solid, in_scale=1.0):
        surr_advance_fine(self.h, out_scale, solid, in_scale)

    def write_lattice(self, solid, f):
        return surr_write_lattice(self.h, solid, f)

    def set_inlet(self, u):
        surr_set_inlet(self.h, u)

    def set_correction(self, f, solid, mode):
        surr_set_correction(self.h, f, solid, mode)

    def fine_velocity_error(self, f, solid, sums):
        return surr_fine_velocity_error(self.h, f, solid, sums)

    def loss(self, target, loss=None):
        surr_loss(self.h, target, loss)

    def set_output_grad(self, g):
        surr_set_output_grad(self.h, g)

    def backward(self):
        surr_backward(self.h)

    def weight_grad(self, cin, cout, x, g, gw, gb, impl=0, stream=None):
        """gw [27][cout][cin] += dW, gb [cout] += db of one layer from BF16
        planar volumes x (cin channels) and g (cout channels) of n^3 voxels
        (uint8 or bfloat16 tensors); impl 0 tcgen05, 1 mma.sync."""
        for t, name in ((x, "x"), (g, "g")):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CUDA tensor")
        check(lib().surr_weight_grad(self.h, int(cin), int(cout), x.data_ptr(), g.data_ptr(),
                                     _dev(gw, name="gw"), _dev(gb, name="gb"), int(impl),
                                     _stream(stream)))

    def device_status(self):
        surr_device_status(self.h)

    def adam(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        surr_adam(self.h, lr, beta1, beta2, eps, step)

    def apply(self, solid, f, out=None, out_scale=1.0):
        return surr_apply(self.h, out, solid, f, out_scale)

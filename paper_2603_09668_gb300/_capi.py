"""ctypes declarations of the libdiffwind C-ABI (include/diffwind.h).

Loading fails loudly when the library has not been built: there is no CPU
fallback for any call.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

from . import build as _build

c_float_p = ct.POINTER(ct.c_float)


class DwWindField(ct.Structure):
    _fields_ = [("values", ct.c_void_p), ("nf", ct.c_int32), ("n_frames", ct.c_int32),
                ("t_total", ct.c_float)]


class DwMpmDesc(ct.Structure):
    _fields_ = [("n_grid", ct.c_int32), ("dt", ct.c_float), ("gravity", ct.c_float * 3),
                ("bc_band", ct.c_int32), ("material", ct.c_int32), ("E", ct.c_float),
                ("nu", ct.c_float), ("p_mass", ct.c_float), ("p_vol", ct.c_float),
                ("max_particles", ct.c_int64), ("p2g_mode", ct.c_int32)]


class DwMpmState(ct.Structure):
    _fields_ = [("x", ct.c_void_p), ("v", ct.c_void_p), ("C", ct.c_void_p), ("F", ct.c_void_p),
                ("n", ct.c_int64)]


class DwMpmScene(ct.Structure):
    _fields_ = [("desc", DwMpmDesc), ("n_particles", ct.c_int64), ("wind", DwWindField)]


class DwBatchConfig(ct.Structure):
    _fields_ = [("mode", ct.c_int32), ("threads", ct.c_int32), ("ctas_per_sm", ct.c_int32),
                ("use_graph", ct.c_int32), ("graph_active", ct.c_int32)]


class DwBatchTrial(ct.Structure):
    _fields_ = [("config", DwBatchConfig), ("ms_per_substep", ct.c_float)]


class DwLbmDesc(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("tau", ct.c_float),
                ("u_inlet", ct.c_float * 3), ("force", ct.c_float * 3), ("bc_x", ct.c_int32),
                ("max_tape", ct.c_int32)]


class DwCamera(ct.Structure):
    _fields_ = [("R", ct.c_float * 9), ("T", ct.c_float * 3), ("fx", ct.c_float),
                ("fy", ct.c_float), ("cx", ct.c_float), ("cy", ct.c_float),
                ("width", ct.c_int32), ("height", ct.c_int32), ("near_z", ct.c_float)]


P = ct.POINTER
VP = ct.c_void_p
I32 = ct.c_int32
I64 = ct.c_int64
F32 = ct.c_float

# name -> (restype, argtypes); every function returns dw_status (int) unless noted
SIGNATURES = {
    "dw_last_error": (ct.c_char_p, []),
    "dw_version": (ct.c_char_p, []),
    "dw_fp32_probe": (I32, [I32, I32, I32, VP, P(ct.c_double), VP]),
    "wind_field_sample": (I32, [P(DwWindField), VP, I64, F32, VP, VP]),
    "wind_field_sample_adjoint": (I32, [P(DwWindField), VP, I64, F32, VP, VP, VP]),
    "mpm_create": (I32, [P(DwMpmDesc), P(VP)]),
    "mpm_destroy": (I32, [VP]),
    "mpm_set_material": (I32, [VP, F32, F32]),
    "mpm_substep": (I32, [VP, P(DwMpmState), P(DwMpmState), VP, P(DwWindField), F32, VP]),
    "mpm_substep_adjoint": (I32, [VP, P(DwMpmState), P(DwMpmState), P(DwMpmState), VP,
                                  P(DwWindField), F32, VP, VP, VP]),
    "mpm_sort": (I32, [VP, P(DwMpmState), P(DwMpmState), VP, VP, VP, VP, VP]),
    "mpm_segment_adjoint": (I32, [VP, P(DwMpmState), VP, I64, P(DwMpmState), VP, P(DwWindField),
                                  F32, I32, VP, VP, VP]),
    "mpm_device_status": (I32, [VP, VP]),
    "mpm_rollout": (I32, [VP, P(DwMpmState), VP, VP, P(DwWindField), F32, I32, I32, VP]),
    "mpm_profile_enable": (I32, [VP, I32]),
    "mpm_profile_read": (I32, [VP, P(ct.c_double), P(I64)]),
    "mpm_substep_noalloc": (I32, [P(DwMpmDesc), P(DwMpmState), P(DwMpmState), VP,
                                  P(DwWindField), F32, VP, VP]),
    "mpm_state_save": (I32, [ct.c_char_p, P(DwMpmState), VP, VP, ct.c_double, I64, VP]),
    "mpm_state_peek": (I32, [ct.c_char_p, P(I64), P(I32), P(ct.c_double), P(I64)]),
    "mpm_state_load": (I32, [ct.c_char_p, P(DwMpmState), VP, VP, P(ct.c_double), P(I64), VP]),
    "mpm_batch_create": (I32, [P(DwMpmScene), I32, P(VP)]),
    "mpm_batch_destroy": (I32, [VP]),
    "mpm_batch_layout": (I32, [VP, P(I64), P(I64)]),
    "mpm_batch_rollout": (I32, [VP, P(DwMpmState), VP, VP, F32, I32, I32, VP]),
    "mpm_batch_set_config": (I32, [VP, P(DwBatchConfig)]),
    "mpm_batch_get_config": (I32, [VP, P(DwBatchConfig)]),
    "mpm_batch_tune": (I32, [VP, P(DwMpmState), VP, I32, P(DwBatchConfig), P(DwBatchTrial), I32,
                             P(I32), VP]),
    "mpm_batch_device_status": (I32, [VP, VP]),
    "mpm_batch_barrier_selftest": (I32, [VP, I32, VP]),
    "mpm_batch_wind_layout": (I32, [VP, P(I64), P(I64)]),
    "mpm_batch_segment_adjoint": (I32, [VP, P(DwMpmState), VP, I64, P(DwMpmState), VP, F32, I32,
                                        VP, VP, VP]),
    "lbm_create": (I32, [P(DwLbmDesc), P(VP)]),
    "lbm_destroy": (I32, [VP]),
    "lbm_step": (I32, [VP, VP, VP, I32, VP]),
    "lbm_cache_mask": (I32, [VP, VP, VP]),
    "lbm_step_adjoint": (I32, [VP, VP, VP, VP, I32, VP]),
    "lbm_macroscopic": (I32, [VP, VP, VP, VP, VP, VP]),
    "lbm_init_equilibrium": (I32, [VP, VP, F32, P(F32 * 3), VP]),
    "voxelize_particles": (I32, [VP, I64, I32, I32, I32, F32, VP, VP]),
    "lbm_home_init": (I32, [VP, VP, F32, P(F32 * 3), VP]),
    "lbm_home_step": (I32, [VP, VP, VP, I32, VP]),
    "lbm_home_macroscopic": (I32, [VP, VP, VP, VP, VP, VP]),
    "lbm_home_sample_velocity": (I32, [VP, VP, VP, VP, I64, VP, VP]),
    "lbm_sample_velocity": (I32, [VP, VP, VP, VP, I64, VP, VP]),
    "wind_phys_loss": (I32, [VP, VP, I64, F32, F32, VP, VP, VP]),
    "wind_field_scores": (I32, [VP, VP, I64, F32, VP, VP]),
    "adam_step": (I32, [VP, VP, VP, VP, I64, F32, F32, F32, F32, I32, VP]),
    "wind_drag_force": (I32, [VP, I64, F32, VP, VP]),
    "gs_covariance": (I32, [VP, VP, I64, VP, VP]),
    "gs_create": (I32, [I64, I32, I32, P(VP)]),
    "gs_destroy": (I32, [VP]),
    "gs_render": (I32, [VP, P(DwCamera), VP, VP, VP, VP, VP, I64, VP, VP]),
    "gs_render_backward": (I32, [VP, P(DwCamera), VP, VP, VP, VP, VP, I64, VP, VP, VP, VP, VP,
                                 VP]),
    "image_l1_loss": (I32, [VP, VP, I64, F32, VP, VP, VP]),
    "image_dssim_loss": (I32, [VP, VP, I32, I32, I32, F32, VP, VP, VP, VP]),
    "vector_adam_step": (I32, [VP, VP, VP, VP, I64, F32, F32, F32, F32, I32, VP]),
    "position_loss": (I32, [VP, VP, I64, F32, VP, VP, VP]),
    "surr_create": (I32, [I32, P(VP)]),
    "surr_destroy": (I32, [VP]),
    "surr_num_params": (I32, [VP, P(I64)]),
    "surr_set_params": (I32, [VP, VP, VP]),
    "surr_get_params": (I32, [VP, VP, VP]),
    "surr_get_grads": (I32, [VP, VP, VP]),
    "surr_zero_grads": (I32, [VP, VP]),
    "surr_features": (I32, [VP, VP, VP, F32, VP, VP]),
    "surr_device_status": (I32, [VP, VP]),
    "surr_set_features": (I32, [VP, VP, VP]),
    "surr_get_features": (I32, [VP, VP, VP]),
    "surr_forward": (I32, [VP, VP, I32, VP]),
    "surr_features_fine": (I32, [VP, VP, F32, VP]),
    "surr_advance_fine": (I32, [VP, F32, VP, F32, VP]),
    "surr_write_lattice": (I32, [VP, VP, VP, VP]),
    "surr_set_inlet": (I32, [VP, P(F32)]),
    "surr_set_correction": (I32, [VP, VP, VP, I32, VP]),
    "surr_fine_velocity_error": (I32, [VP, VP, VP, VP, VP]),
    "surr_loss": (I32, [VP, VP, VP, VP]),
    "surr_set_output_grad": (I32, [VP, VP, VP]),
    "surr_backward": (I32, [VP, VP]),
    "surr_weight_grad": (I32, [VP, I32, I32, VP, VP, VP, VP, I32, VP]),
    "surr_adam": (I32, [VP, F32, F32, F32, F32, I32, VP]),
    "surr_apply": (I32, [VP, VP, F32, VP, VP, VP]),
    "lbm_velocity_error": (I32, [VP, VP, VP, I64, VP, VP]),
}

STATUS = {0: "DW_OK", 1: "DW_ERR_ARG", 2: "DW_ERR_CUDA", 3: "DW_ERR_OOM", 4: "DW_ERR_NONFINITE",
          5: "DW_ERR_DOMAIN", 6: "DW_ERR_TIMEOUT", 7: "DW_ERR_INVERTED", 8: "DW_ERR_IO"}

_lock = threading.Lock()
_lib = None


class DiffWindError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libdiffwind. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libdiffwind.so is not built ({path} missing); run "
                    "`python -c 'import __graft_entry__ as g; g.build()'` first")
            L = ct.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int):
    if status != 0:
        msg = lib().dw_last_error().decode(errors="replace")
        raise DiffWindError(status, msg)
    return status

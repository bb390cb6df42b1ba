"""ctypes binding of libtgs (include/tgs.h). Argument marshalling only: every step of the
rasterizer runs in the library's CUDA kernels. Importing this module loads the in-tree
library and raises if it is missing; there is no fallback of any kind."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtgs.so")

TGS_OK = 0
TGS_ERR_INVALID_ARG = 1
TGS_ERR_CUDA = 2
TGS_ERR_CAPACITY = 3
TGS_ERR_TIMEOUT = 4
TGS_ERR_OOM = 5
TGS_ERR_NOT_SUPPORTED = 6
TGS_ERR_SCRATCH_LIMIT = 7
TGS_ERR_INCONSISTENT = 8
TGS_NOALLOC_MAX_RECORDS = 131072
TGS_NOALLOC_MAX_KEYS = 524288
TGS_SUPPORT_BOX3 = 0
TGS_SUPPORT_ALPHA = 1
TGS_MAX_VIEWS = 64
TGS_MAX_STAGES = 8
TGS_ACCUMULATE = 1
TGS_NO_SH_REST_GRAD = 2
TGS_USE_GRAPH = 4
TGS_UNFUSED = 8
TGS_LOSS_DSSIM = 16
TGS_MASK_LOSS = 32
TGS_COMPACT_MASKED = 1
TGS_PARAM_F32 = 0
TGS_PARAM_F16 = 1

_fp = C.POINTER(C.c_float)
_vp = C.c_void_p


class tgs_config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("ppt", C.c_int32), ("support", C.c_int32),
                ("low_pass", C.c_float), ("eps_mask", C.c_float), ("eps_sh", C.c_float),
                ("near_plane", C.c_float), ("bg", C.c_float * 3), ("key_capacity", C.c_int64),
                ("spin_limit", C.c_int64), ("ssim_lambda", C.c_float), ("lambda_mask", C.c_float),
                ("lambda_sh_mask", C.c_float), ("batch", C.c_int32)]


class tgs_gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree_max", C.c_int32), ("param_dtype", C.c_int32),
                ("means", _vp), ("log_scales", _vp), ("quats", _vp), ("opacity_logits", _vp),
                ("sh_dc", _vp), ("sh_rest", _vp), ("sh_degree", _vp), ("mask_logits", _vp),
                ("sh_mask_logits", _vp)]


class tgs_camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("campos", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("low_pass", C.c_float)]


class tgs_view_out(C.Structure):
    _fields_ = [("image", _vp), ("T_final", _vp), ("last", _vp), ("n_examined", _vp),
                ("radii", _vp), ("n_contrib", _vp), ("n_eval", _vp)]


class tgs_grads(C.Structure):
    _fields_ = [(k, _vp) for k in ("means", "log_scales", "quats", "opacity_logits", "sh_dc",
                                   "sh_rest", "mask_logits", "sh_mask_logits")]


class tgs_stats(C.Structure):
    _fields_ = [("grad_norm_accum", _vp), ("vis_count", _vp), ("max_radius", _vp), ("hit_count", _vp)]


class tgs_peaks(C.Structure):
    _fields_ = [("fp32_fma_per_s", C.c_double), ("fp32x2_fma_per_s", C.c_double), ("ex2_per_s", C.c_double),
                ("rcp_per_s", C.c_double), ("sms", C.c_int32), ("ms", C.c_double)]


_ctx_p = C.c_void_p
_cfgp = C.POINTER(tgs_config)
class tgs_half_params(C.Structure):
    _fields_ = [(k, _vp) for k in ("means", "log_scales", "quats", "opacity_logits", "sh_dc", "sh_rest",
                                   "mask_logits", "sh_mask_logits")]


_gp = C.POINTER(tgs_gaussians)
_camp = C.POINTER(tgs_camera)
_outp = C.POINTER(tgs_view_out)
_gradp = C.POINTER(tgs_grads)
_statp = C.POINTER(tgs_stats)
_pp = C.POINTER(C.c_void_p)

# name -> (restype, argtypes)
SIGNATURES = {
    "tgs_default_config": (None, [_cfgp]),
    "tgs_create": (C.c_int32, [C.POINTER(_ctx_p), _cfgp]),
    "tgs_destroy": (None, [_ctx_p]),
    "tgs_get_config": (C.c_int32, [_ctx_p, _cfgp]),
    "tgs_set_config": (C.c_int32, [_ctx_p, _cfgp]),
    "tgs_status_string": (C.c_char_p, [C.c_int32]),
    "tgs_poll_status": (C.c_int32, [_ctx_p, _vp]),
    "tgs_forward": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _outp, C.c_uint32, _vp]),
    "tgs_backward": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _outp, _pp, _gradp, _statp,
                                 C.c_uint32, _vp]),
    "tgs_l1_loss": (C.c_int32, [_vp, _vp, C.c_int64, C.c_float, _vp, _vp, _vp]),
    "tgs_l1_dssim_loss": (C.c_int32, [_ctx_p, _camp, C.c_int32, _pp, _pp, C.c_float, _vp, _pp, _vp]),
    "tgs_params_to_half": (C.c_int32, [_gp, C.POINTER(tgs_half_params), _vp]),
    "tgs_compact": (C.c_int32, [_ctx_p, _gp, _vp, C.c_uint32, _gradp, _vp, _vp, C.POINTER(C.c_int64), _vp]),
    "tgs_mask_loss": (C.c_int32, [_ctx_p, _gp, _vp, _gradp, _vp]),
    "tgs_densify": (C.c_int32, [_ctx_p, _gp, _statp, _vp, C.c_float, C.c_float, _gradp, _vp, _vp, C.c_int64,
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp]),
    "tgs_plan": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, C.c_double, C.POINTER(C.c_int64)]),
    "tgs_train_step_batched": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _pp, _pp, _gradp,
                                           _statp, _vp, C.c_uint32, _vp]),
    "tgs_train_step_batched_host": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _pp, _gradp, _statp, _vp,
                                                C.c_uint32, _vp]),
    "tgs_render_batched": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _outp, C.c_uint32, _vp]),
    "tgs_autotune": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _pp, C.c_char_p, _vp]),
    "tgs_preprocess": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _vp, _vp, _vp]),
    "tgs_bin": (C.c_int32, [_ctx_p, _vp, _vp, C.c_int64, _camp, C.c_int32, _vp, _vp, _vp,
                            C.c_int64, C.POINTER(C.c_int64), _vp]),
    "tgs_blend_forward": (C.c_int32, [_ctx_p, _vp, _vp, _vp, _camp, C.c_int32, _outp, _vp]),
    "tgs_blend_backward": (C.c_int32, [_ctx_p, _vp, _vp, _vp, _camp, C.c_int32, _outp, _pp,
                                       _vp, _vp]),
    "tgs_preprocess_backward": (C.c_int32, [_ctx_p, _gp, _camp, C.c_int32, _vp, _vp, _gradp,
                                            _statp, C.c_uint32, _vp]),
    "tgs_bin_noalloc": (C.c_int32, [_vp, _vp, C.c_int64, _camp, C.c_int32, C.c_int32, _vp, _vp,
                                    _vp, C.c_int64, C.POINTER(C.c_int64), _vp]),
    "tgs_count_hits": (C.c_int32, [_ctx_p, C.POINTER(tgs_gaussians), _camp, C.c_int32, _vp, _vp]),
    "tgs_significance": (C.c_int32, [_ctx_p, C.POINTER(tgs_gaussians), _vp, C.c_double, _vp, _vp]),
    "tgs_prune_select": (C.c_int32, [_ctx_p, _vp, C.c_int64, C.c_double, _vp, _vp]),
    "tgs_prune_schedule": (C.c_int32, [C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_double)]),
    "tgs_set_profiling": (C.c_int32, [_ctx_p, C.c_int32]),
    "tgs_measure_peaks": (C.c_int32, [C.POINTER(tgs_peaks), _vp]),
    "tgs_stage_times": (C.c_int32, [_ctx_p, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_int32)]),
    "tgs_stage_name": (C.c_char_p, [_ctx_p, C.c_int32]),
    "tgs_kernels_per_step": (C.c_int64, [_ctx_p]),
    "tgs_arena_bytes": (C.c_size_t, [_ctx_p]),
    "tgs_num_tiles": (C.c_int64, [_ctx_p, _camp, C.c_int32]),
    "tgs_workspace_bytes": (C.c_size_t, [_ctx_p, C.c_int64, _camp, C.c_int32]),
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"libtgs is not built ({path}); run __graft_entry__.build() or "
                           "python -m paper_2501_14534_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class TgsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib.tgs_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def check(status, where):
    if status != TGS_OK:
        raise TgsError(status, where)

"""ctypes binding of the C ABI in include/gs.h (argument marshalling only).

Loads the in-tree ``libgs.so``; there is no fallback: if the library is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")

NOALLOC_MAX_GAUSSIANS = 4194304  # GS_NOALLOC_MAX_GAUSSIANS in include/gs.h
GS_OK, GS_ERR_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_TIMEOUT = range(6)
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
                4: "GS_ERR_OOM", 5: "GS_ERR_TIMEOUT"}

# every symbol include/gs.h declares
EXPORTS = (
    "gs_ctx_create", "gs_ctx_destroy", "gs_ctx_reserve", "gs_ctx_set_tile", "gs_ctx_set_sort_bits", "gs_ctx_set_sort_items", "gs_ctx_set_binning", "gs_ctx_set_raster_threads",
    "gs_ctx_set_raster_bwd_threads", "gs_ctx_get_tuning", "gs_ctx_set_wait_limit", "gs_ctx_set_wait_test",
    "gs_get_status", "gs_workspace_size", "gs_total_tiles", "gs_project", "gs_bin_sort",
    "gs_render_fwd", "gs_loss", "gs_raster_bwd", "gs_project_bwd", "gs_render_bwd",
    "gs_adam_step", "gs_extract_delta", "gs_render_batch", "gs_render_batch_sized", "gs_train_step",
    "gs_train_graph_capture", "gs_graph_launch", "gs_train_step_events",
    "gs_train_graph_capture_events", "gs_extract_delta_noalloc", "gs_autotune", "gs_tensor_record_bytes",
    "gs_extract_tensor_delta", "gs_apply_tensor_delta", "gs_apply_delta", "gs_cell_visibility",
    "gs_precull_workspace_size", "gs_light_depth_map", "gs_light_visibility",
)


class GsError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(code, code)}")
        self.code = code


class gs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float), ("_pad", C.c_float)]


class gs_dynamics(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("_pad", C.c_int32), ("group", C.c_void_p), ("poses", C.c_void_p),
                ("normals", C.c_void_p), ("light", C.c_void_p), ("ambient", C.c_float), ("diffuse", C.c_float)]


class gs_precull(C.Structure):
    _fields_ = [("cell_visible", C.c_void_p), ("origin", C.c_float * 3), ("cell_size", C.c_float),
                ("dims", C.c_int32 * 3), ("_pad", C.c_int32)]


class gs_lighting(C.Structure):
    _fields_ = [("light", C.c_void_p), ("visibility", C.c_void_p)]


class gs_light_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("origin", C.c_float * 3), ("texel", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("alpha_min", C.c_float), ("bias", C.c_float), ("_pad", C.c_float)]


class gs_scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("_pad", C.c_int32),
                ("params", C.c_void_p), ("dyn", C.POINTER(gs_dynamics)), ("precull", C.POINTER(gs_precull)),
                ("lighting", C.POINTER(gs_lighting))]


class gs_tune_entry(C.Structure):
    _fields_ = [("binning", C.c_int32), ("sort_bits", C.c_int32), ("sort_items", C.c_int32),
                ("raster_threads", C.c_int32), ("ms", C.c_float), ("ms_render_fwd", C.c_float),
                ("ms_render_bwd", C.c_float)]


class gs_adam_cfg(C.Structure):
    _fields_ = [("lr", C.c_float * 60), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("d_step", C.c_void_p), ("increment", C.c_int32),
                ("_pad", C.c_int32)]


class gs_train_io(C.Structure):
    _fields_ = [("params", C.c_void_p), ("grads", C.c_void_p), ("adam_m", C.c_void_p),
                ("adam_v", C.c_void_p), ("baseline", C.c_void_p), ("targets", C.c_void_p),
                ("image", C.c_void_p), ("d_loss", C.c_void_p), ("d_delta_idx", C.c_void_p),
                ("d_delta_records", C.c_void_p), ("d_delta_count", C.c_void_p), ("d_step", C.c_void_p),
                ("frozen", C.c_void_p)]


class gs_train_cfg(C.Structure):
    _fields_ = [("dyn", C.POINTER(gs_dynamics)), ("n", C.c_int64), ("sh_degree", C.c_int32), ("n_views", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("keys_cap", C.c_int64),
                ("w_l1", C.c_float), ("w_ssim", C.c_float), ("bg", C.c_float * 3),
                ("delta_thr", C.c_float), ("adam", gs_adam_cfg), ("n_frozen", C.c_int64),
                ("precull", C.POINTER(gs_precull)), ("lighting", C.POINTER(gs_lighting)),
                ("phases", C.c_int32), ("_pad2", C.c_int32)]


assert C.sizeof(gs_camera) == 80
assert C.sizeof(gs_light_camera) == 72

_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_F = C.c_float
_SIGS = {
    "gs_ctx_create": [C.POINTER(C.c_void_p), C.c_int, C.c_size_t],
    "gs_ctx_destroy": [_P],
    "gs_ctx_reserve": [_P, C.c_size_t],
    "gs_ctx_set_tile": [_P, _I32],
    "gs_ctx_set_sort_bits": [_P, _I32],
    "gs_ctx_set_sort_items": [_P, _I32],
    "gs_ctx_set_binning": [_P, _I32],
    "gs_ctx_set_raster_threads": [_P, _I32],
    "gs_ctx_set_raster_bwd_threads": [_P, _I32],
    "gs_ctx_set_wait_limit": [_P, _I64],
    "gs_ctx_set_wait_test": [_P, _I64],
    "gs_ctx_get_tuning": [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                          C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "gs_get_status": [_P, _P, C.POINTER(_I32), C.POINTER(_I64)],
    "gs_project": [_P, C.POINTER(gs_scene), _P, _I32, _P, _P],
    "gs_bin_sort": [_P, _P, _P, _I32, _I64, _I64, _I64, _P, _P, _P, _P, _P],
    "gs_render_fwd": [_P, _P, _P, _I32, _I64, _I64, _P, _P, _P, _P, _P, _P, _P],
    "gs_loss": [_P, _P, _P, _I32, _I32, _I32, _F, _F, _P, _P, _P],
    "gs_raster_bwd": [_P, _P, _P, _I32, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P],
    "gs_project_bwd": [_P, C.POINTER(gs_scene), _P, _I32, _P, _P, _P, _I32, _P],
    "gs_render_bwd": [_P, C.POINTER(gs_scene), _P, _I32, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "gs_adam_step": [_P, _P, _P, _P, _P, _I64, C.POINTER(gs_adam_cfg), _P],
    "gs_extract_delta": [_P, _P, _P, _I64, _F, _P, _P, _P, _P],
    "gs_extract_delta_noalloc": [_P, _P, _I64, _F, _P, _P, _P, _P],
    "gs_render_batch": [_P, C.POINTER(gs_scene), _P, _I32, _I64, _I64, _P, _P, _P],
    "gs_render_batch_sized": [_P, C.POINTER(gs_scene), _P, C.POINTER(gs_camera), _I32, _I64, _P, _P, _P],
    "gs_train_step": [_P, _P, C.POINTER(gs_train_io), C.POINTER(gs_train_cfg), _P],
    "gs_train_graph_capture": [_P, _P, C.POINTER(gs_train_io), C.POINTER(gs_train_cfg), _P],
    "gs_graph_launch": [_P, _P],
    "gs_train_step_events": [_P, _P, C.POINTER(gs_train_io), C.POINTER(gs_train_cfg), C.POINTER(_P), _P],
    "gs_train_graph_capture_events": [_P, _P, C.POINTER(gs_train_io), C.POINTER(gs_train_cfg), C.POINTER(_P), _P],
    "gs_autotune": [_P, C.POINTER(gs_scene), _P, C.POINTER(gs_camera), _I32, _I64, _I32, C.POINTER(gs_tune_entry),
                    _I32, C.POINTER(_I32), _P],
    "gs_tensor_record_bytes": [_I32],
    "gs_extract_tensor_delta": [_P, _P, _P, _I64, _I32, _F, _P, _P, _P, _P],
    "gs_apply_tensor_delta": [_P, _P, _I64, _I32, _P, _P, _P, _P],
    "gs_apply_delta": [_P, _P, _I64, _P, _P, _P],
    "gs_cell_visibility": [_P, _P, C.POINTER(gs_camera), _I32, _P, C.POINTER(gs_precull), _P, _P],
    "gs_precull_workspace_size": [C.POINTER(gs_camera), _I32],
    "gs_light_depth_map": [_P, C.POINTER(gs_scene), C.POINTER(gs_light_camera), _P, _I32, _P],
    "gs_light_visibility": [_P, C.POINTER(gs_scene), C.POINTER(gs_light_camera), _P, _P, _P],
}
TRAIN_PHASE_EVENTS = 11
TRAIN_GRADIENT, TRAIN_UPDATE, TRAIN_ALL = 1, 2, 3  # GS_TRAIN_* in include/gs.h
TRAIN_PHASES = ("project", "depth_sort", "emit", "tile_sort", "render_fwd", "loss", "raster_bwd", "project_bwd",
                "adam", "delta")
_RESTYPES = {"gs_workspace_size": C.c_size_t, "gs_total_tiles": C.c_int64, "gs_tensor_record_bytes": C.c_int32,
             "gs_precull_workspace_size": C.c_size_t}
_SIGS["gs_workspace_size"] = [_P, C.POINTER(gs_camera), _I32, _I64, _I64]
_SIGS["gs_total_tiles"] = [_P, C.POINTER(gs_camera), _I32]

_lib = None


def lib():
    """The loaded libgs.so; raises if it is missing (no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2604_02851_b300/build.py)")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, C.c_int)
        _lib = L
    return _lib


def check(fn: str, code: int) -> None:
    if code != GS_OK:
        raise GsError(fn, code)

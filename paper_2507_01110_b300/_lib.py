"""ctypes declarations of liblodgs.so (include/lodgs.h).  Marshalling only.

The library is loaded from this package's folder; if it is missing or fails to
load, every call raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LODGS_LIBRARY", os.path.join(_HERE, "liblodgs.so"))

LODGS_OK = 0
LODGS_E_INVALID = -1
LODGS_E_OOM = -2
LODGS_E_CUDA = -3
LODGS_E_TIMEOUT = -4
LODGS_E_STATE = -5
LODGS_E_CAPACITY = -6
LODGS_SELECT_BATCH_MAX = 8       # views per lodgs_select_lod_batch call
STAGES = ("select", "project", "count", "emit", "tile_sort", "blend", "blend_bwd", "project_bwd")
_NAMES = {-1: "INVALID", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "STATE", -6: "CAPACITY"}


class LodgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"lodgs error {code} ({_NAMES.get(code, '?')}): {msg}")
        self.code = code


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("pos", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("tau", C.c_float), ("znear", C.c_float), ("spt_scale", C.c_float)]


class BuildParams(C.Structure):
    _fields_ = [("spt_volume", C.c_float), ("kappa", C.c_float)]


class SceneInfo(C.Structure):
    _fields_ = [("n_leaves", C.c_int64), ("n_nodes", C.c_int64), ("n_upper", C.c_int64),
                ("n_upper_rows", C.c_int64), ("n_spt", C.c_int64), ("sh_degree", C.c_int32),
                ("stride", C.c_int32), ("d_rows", C.c_void_p), ("root", C.c_int64), ("layout_version", C.c_int64)]


class DensifyOp(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("target", C.c_int64), ("dead", C.c_int64)]


DENSIFY_SPAWN, DENSIFY_RESPAWN = 0, 1
FAULT_STREAM, FAULT_ALLOC, FAULT_RENDER = 1, 2, 3


class CacheParams(C.Structure):
    _fields_ = [("capacity_bytes", C.c_int64), ("d_min", C.c_float), ("d_max", C.c_float),
                ("release_scene_rows", C.c_int32), ("train", C.c_int32)]


class StreamStats(C.Structure):
    _fields_ = [("spt_hits", C.c_int64), ("spt_resident", C.c_int64), ("spt_loaded", C.c_int64),
                ("bytes_streamed", C.c_int64), ("evictions", C.c_int64), ("cached_spts", C.c_int64),
                ("cached_records", C.c_int64), ("bytes_written_back", C.c_int64)]


class FrameStats(C.Structure):
    _fields_ = [("n_selected", C.c_int64), ("n_upper_selected", C.c_int64), ("n_spt_cut", C.c_int64),
                ("n_spt_scanned", C.c_int64), ("n_visible", C.c_int64), ("n_pairs", C.c_int64),
                ("status", C.c_int32), ("width", C.c_int32), ("height", C.c_int32)]


_lib = None

_P = C.c_void_p
_SIGS = {
    "lodgs_last_error": (C.c_char_p, []),
    "lodgs_version": (C.c_char_p, []),
    "lodgs_kernel_launches": (C.c_uint64, []),
    "lodgs_build_hierarchy": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, C.POINTER(BuildParams), C.POINTER(_P)]),
    "lodgs_scene_free": (None, [_P]),
    "lodgs_scene_get_info": (C.c_int, [_P, C.POINTER(SceneInfo)]),
    "lodgs_scene_export": (C.c_int, [_P] + [_P] * 13),
    "lodgs_scene_densify": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64]),
    "lodgs_scene_save": (C.c_int, [_P, C.c_char_p]),
    "lodgs_debug_inject_fault": (C.c_int, [C.c_int, C.c_int64]),
    "lodgs_scene_load": (C.c_int, [C.c_char_p, C.POINTER(_P)]),
    "lodgs_densify_plan": (C.c_int, [_P, _P, _P, _P, C.c_float, C.c_float, C.c_int64, _P, C.c_int64,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P]),
    "lodgs_gather_rows": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int64, C.c_int32, _P]),
    "lodgs_frame_create": (C.c_int, [_P, C.POINTER(_P)]),
    "lodgs_frame_free": (None, [_P]),
    "lodgs_select_lod": (C.c_int, [_P, C.POINTER(Camera), _P, _P]),
    "lodgs_frame_set_view": (C.c_int, [_P, C.POINTER(Camera), _P, _P]),
    "lodgs_select_lod_noalloc": (C.c_int, [_P, C.POINTER(Camera), _P, C.c_int64, _P, _P]),
    "lodgs_frame_selection": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_int64)]),
    "lodgs_cache_create": (C.c_int, [_P, C.POINTER(CacheParams), C.POINTER(_P)]),
    "lodgs_cache_free": (None, [_P]),
    "lodgs_cache_records": (C.c_int, [_P, C.POINTER(_P)]),
    "lodgs_cache_flush": (C.c_int, [_P]),
    "lodgs_cache_adam_step": (C.c_int, [_P, _P, _P, C.c_int64, _P, C.c_float, C.c_float, C.c_float, _P]),
    "lodgs_cache_writeback": (C.c_int, [_P, _P]),
    "lodgs_cache_written_bytes": (C.c_int, [_P, C.POINTER(C.c_int64)]),
    "lodgs_cache_host_state": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), C.POINTER(_P)]),
    "lodgs_stream_nodes": (C.c_int, [_P, _P, C.POINTER(Camera), _P, _P, _P, C.POINTER(StreamStats)]),
    "lodgs_render": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "lodgs_render_backward": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_int64, C.c_int, _P]),
    "lodgs_render_backward_blend": (C.c_int, [_P, _P, _P, _P, _P]),
    "lodgs_render_backward_blend_l1": (C.c_int, [_P, _P, _P, _P, C.c_float, _P, _P]),
    "lodgs_render_backward_blend_l1_u8": (C.c_int, [_P, _P, _P, _P, C.c_float, _P, _P]),
    "lodgs_render_backward_project": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int, _P]),
    "lodgs_frame_get_stats": (C.c_int, [_P, C.POINTER(FrameStats)]),
    "lodgs_frame_set_ordering": (C.c_int, [_P, C.c_int]),
    "lodgs_frame_memory": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "lodgs_select_lod_batch": (C.c_int, [_P, _P, _P, C.c_int, _P]),
    "lodgs_frame_reserve": (C.c_int, [_P, C.c_int64, C.c_int64]),
    "lodgs_adam_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, C.c_int64, _P, C.c_float, C.c_float, C.c_float,
                                  _P]),
    "lodgs_frame_screen_grad_max": (C.c_int, [_P, _P, _P]),
    "lodgs_frame_device_count": (C.c_int, [_P, C.POINTER(_P)]),
    "lodgs_accumulate_grads": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, C.c_int64, _P, _P]),
    "lodgs_l1_loss_grad": (C.c_int, [_P, _P, C.c_int64, C.c_float, _P, _P, _P]),
    "lodgs_frame_export": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    "lodgs_frame_set_profiling": (C.c_int, [_P, C.c_int]),
    "lodgs_frame_work": (C.c_int, [_P, _P]),
    "lodgs_frame_stage_ms": (C.c_int, [_P, _P]),
}

# every symbol include/lodgs.h declares
EXPORTED = tuple(_SIGS.keys())


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LodgsError(LODGS_E_STATE, f"{LIB_PATH} is missing: build it with "
                             "`python -m paper_2507_01110_b300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != LODGS_OK:
        raise LodgsError(rc, lib().lodgs_last_error().decode(errors="replace"))

"""ctypes binding of include/lodge.h (argument marshalling only).

Every entry point of the C ABI is declared here with the same name.  The
library is loaded from this package's _build/ directory; if it is missing the
import of any entry point raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblodge.so")

LODGE_OK = 0
STATUS_NAMES = {0: "LODGE_OK", 1: "LODGE_E_INVALID", 2: "LODGE_E_OOM", 3: "LODGE_E_CUDA",
                4: "LODGE_E_NOT_RESIDENT", 5: "LODGE_E_TIMEOUT", 6: "LODGE_E_BUDGET",
                7: "LODGE_E_OVERFLOW"}
FULL, LOD, CHUNK, CHUNK_BLEND = 0, 1, 2, 3


class LodgeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class lodge_level_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p),
                ("filter_var", C.c_float), ("pad_", C.c_float)]


RESIDENT, STREAMED = 0, 1


class lodge_scene_desc(C.Structure):
    _fields_ = [("num_levels", C.c_int32), ("sh_degree", C.c_int32), ("levels", C.c_void_p),
                ("d_thresholds", C.c_void_p), ("num_chunks", C.c_int32), ("residency", C.c_int32),
                ("chunk_centers", C.c_void_p), ("filter2d", C.c_int32), ("pad_", C.c_int32)]


class lodge_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("pad_", C.c_float), ("center", C.c_double * 3)]


class lodge_selection(C.Structure):
    _fields_ = [("chunk_a", C.c_int32), ("chunk_b", C.c_int32), ("t_a", C.c_double),
                ("t_b", C.c_double), ("n_active", C.c_int64)]


NUM_STAGES = 8
STAGE_NAMES = ["select", "union", "project", "depth_sort", "emit", "tile_sort", "ranges", "blend"]


class lodge_profile(C.Structure):
    _fields_ = [("ms", C.c_double * NUM_STAGES), ("launches", C.c_int64 * NUM_STAGES),
                ("frames", C.c_int64), ("keys", C.c_int64), ("visible", C.c_int64),
                ("active", C.c_int64), ("packed_keys", C.c_int64), ("bin_keys", C.c_int64),
                ("bin_sort_passes", C.c_int64), ("blend_pairs", C.c_int64),
                ("blend_pairs_used", C.c_int64), ("redone", C.c_int64), ("host_ms", C.c_double)]


class lodge_frame_stats(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_visible", C.c_int64), ("n_keys", C.c_int64),
                ("n_tiles", C.c_int64), ("chunk_a", C.c_int32), ("chunk_b", C.c_int32),
                ("t_a", C.c_double), ("t_b", C.c_double)]


class lodge_request(C.Structure):
    _fields_ = [("scene", C.c_int32), ("mode", C.c_int32), ("cam", lodge_camera),
                ("arrival_s", C.c_double)]


class lodge_request_result(C.Structure):
    _fields_ = [("start_s", C.c_double), ("finish_s", C.c_double), ("status", C.c_int32),
                ("slot", C.c_int32), ("stats", lodge_frame_stats), ("uploads", C.c_int32),
                ("step_frames", C.c_int32)]


class lodge_serve_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("realtime", C.c_int32), ("h_images", C.c_void_p),
                ("wait_limit_s", C.c_double), ("batch", C.c_int32), ("pad_", C.c_int32)]


class lodge_residency(C.Structure):
    _fields_ = [("resident_blocks", C.c_int64), ("block_hits", C.c_int64),
                ("block_uploads", C.c_int64), ("block_evictions", C.c_int64),
                ("upload_bytes", C.c_int64), ("failed_uploads", C.c_int64),
                ("hbm_used", C.c_int64), ("hbm_budget", C.c_int64)]


P = C.c_void_p
_SIGS = {
    "lodge_create": [C.c_int, C.c_size_t, C.POINTER(P)],
    "lodge_destroy": [P],
    "lodge_load_scene": [P, C.POINTER(lodge_scene_desc), C.POINTER(C.c_int32)],
    "lodge_unload_scene": [P, C.c_int32],
    "lodge_upload_chunks": [P, C.c_int32, P, C.c_int32, C.c_int],
    "lodge_select_lod": [P, C.c_int32, C.c_int, P, C.c_int32, P, P, C.c_int64, P],
    "lodge_select_thresholds": [P, C.c_int32, P, C.c_int32, P, C.c_int32, P, P, P],
    "lodge_num_clusters": [P, C.c_int32, C.c_double, P],
    "lodge_kmeans_centers": [P, C.c_int32, C.c_int32, P, C.c_int32, P, P, P],
    "lodge_importance": [P, C.c_int32, C.c_int, C.c_int32, P, C.c_int32, P, P],
    "lodge_render_lod": [P, C.c_int32, P, C.c_int32, P, P, P, P],
    "lodge_render_params_lod": [P, C.c_int32, P, P, P, P, P, P, C.c_int32, P, P, P, P, P,
                                C.c_int32, P, C.c_int32, C.POINTER(C.c_int64), P],
    "lodge_render_batch": [P, C.c_int32, P, P, P, P, P, P, P],
    "lodge_filter_chunk": [P, C.c_int32, C.c_int32, P, C.c_float, C.POINTER(C.c_int64), P],
    "lodge_render": [P, C.c_int32, C.c_int, P, C.c_int32, P, P, C.c_int32,
                     C.POINTER(C.c_int64), P],
    "lodge_render_host": [P, C.c_int32, C.c_int, P, C.c_int32, P, P, P],
    "lodge_render_params": [P, C.c_int64, P, P, P, P, P, C.c_int32, C.c_float, P, P, P,
                            C.c_int32, C.POINTER(C.c_int64), P],
    "lodge_render_backward": [P, C.c_int64, P, P, P, P, P, P, P],
    "lodge_release": [P, C.c_int64],
    "lodge_debug_keys": [P, C.c_int64, P, P, C.c_int64, C.POINTER(C.c_int64), P],
    "lodge_debug_records": [P, C.c_int64, P, P, P, P, P, P, P, C.c_int64,
                            C.POINTER(C.c_int64), P],
    "lodge_sort_pairs": [P, P, P, C.c_int64, C.c_int32, P],
    "lodge_sort_pairs_noalloc": [P, P, C.c_int64, C.c_int32, P],
    "lodge_debug_lookback": [C.c_int32, C.c_int32, C.c_uint32, P, P],
    "lodge_serve": [P, P, C.c_int32, C.POINTER(lodge_serve_opts), P],
    "lodge_residency_stats": [P, C.POINTER(lodge_residency)],
    "lodge_inject_upload_failures": [P, C.c_int32],
    "lodge_set_bin_size": [P, C.c_int32],
    "lodge_profile_enable": [P, C.c_int],
    "lodge_profile_read": [P, C.POINTER(lodge_profile)],
}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded liblodge.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2505_23158_gb300.build.build() "
                    "(there is no CPU fallback)")
            L = C.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.lodge_last_error.argtypes = []
            L.lodge_last_error.restype = C.c_char_p
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS) + ["lodge_last_error"]


def check(status: int):
    if status != LODGE_OK:
        msg = lib().lodge_last_error().decode(errors="replace")
        raise LodgeError(status, msg)


def call(name: str, *args):
    check(getattr(lib(), name)(*args))

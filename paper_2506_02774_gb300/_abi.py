"""ctypes mirror of include/vgr.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import re

from . import _build

c_u32, c_u64, c_f32, c_i32, c_vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float, ctypes.c_int32, ctypes.c_void_p

VGR_OK, VGR_E_INVALID, VGR_E_NOMEM, VGR_E_CUDA, VGR_E_TIMEOUT, VGR_E_NONMONOTONE, VGR_E_OVERFLOW = range(7)
STATUS_NAMES = {0: "VGR_OK", 1: "VGR_E_INVALID", 2: "VGR_E_NOMEM", 3: "VGR_E_CUDA", 4: "VGR_E_TIMEOUT",
                5: "VGR_E_NONMONOTONE", 6: "VGR_E_OVERFLOW"}
STORE_FP32, STORE_HALF = 0, 1
FILTER_PREEMPTIVE, FILTER_CANONICAL = 0, 1
EXP_EXACT, EXP_LUT = 0, 1
STAGES = ["lod", "compact", "preprocess", "depth_sort", "color", "emit", "tile_sort", "ranges", "blend"]


class SceneDesc(ctypes.Structure):
    _fields_ = [("n_nodes", c_u32), ("sh_degree", c_u32), ("parent", c_vp), ("first_child", c_vp),
                ("n_child", c_vp), ("mean", c_vp), ("cov6", c_vp), ("opacity", c_vp), ("sh", c_vp),
                ("radius2", c_vp), ("storage", c_i32), ("bbox", c_vp)]


class Camera(ctypes.Structure):
    _fields_ = [("R", c_f32 * 9), ("pos", c_f32 * 3), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32),
                ("cy", c_f32), ("width", c_u32), ("height", c_u32), ("z_near", c_f32)]


class ViewOpts(ctypes.Structure):
    _fields_ = [("stream", c_vp), ("filter", c_u32), ("exp_mode", c_u32), ("lut_size", c_u32),
                ("temporal", c_u32), ("timing", c_u32), ("use_graph", c_u32), ("cut_capacity", c_u64),
                ("pair_capacity", c_u64), ("lod_budget", c_u32), ("grid_wide", c_u32), ("grid_scan", c_u32),
                ("test_hooks", c_u32), ("lod_frustum", c_u32), ("lod_frustum_guard", c_f32),
                ("lod_interp", c_u32), ("blend_depth", c_u32), ("tile_size", c_u32)]


class FrameStats(ctypes.Structure):
    _fields_ = [("cut_count", c_u32), ("front_count", c_u32), ("visible_count", c_u32), ("pair_count", c_u64),
                ("candidate_pairs", c_u64), ("nodes_evaluated", c_u64), ("lod_from_scratch", c_u32),
                ("replays", c_u32), ("kernels", c_u32), ("pixel_pair_evals", c_u64),
                ("pixel_pair_contribs", c_u64), ("stage_ms", c_f32 * 9),
                ("frame_ms", c_f32)]


class Frame(ctypes.Structure):
    _fields_ = [("image", c_vp), ("cut", c_vp), ("cut_count", c_u32), ("width", c_u32), ("height", c_u32),
                ("stats", FrameStats)]


class DebugBuffers(ctypes.Structure):
    _fields_ = [("n_cut", c_u32), ("n_front", c_u32), ("n_visible", c_u32), ("n_pairs", c_u64), ("tiles_x", c_u32),
                ("tiles_y", c_u32), ("cut", c_vp), ("vis_node", c_vp), ("vis_depth", c_vp),
                ("vis_ntile", c_vp), ("vis_rect", c_vp), ("vis_recA", c_vp), ("vis_recB", c_vp),
                ("vis_rgb", c_vp), ("depth_order", c_vp), ("pair_tile", c_vp), ("pair_val", c_vp),
                ("tile_range", c_vp), ("tile_size", c_u32)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("n_clients", c_u32), ("max_inflight", c_u32), ("host_images", c_u32), ("hbm_reserve", c_u64),
                ("view", ViewOpts), ("evict_idle", c_u32)]


class Request(ctypes.Structure):
    _fields_ = [("client", c_u32), ("tau", c_f32), ("arrival_s", ctypes.c_double), ("cam", Camera),
                ("host_rgb", c_vp)]


class RequestResult(ctypes.Structure):
    _fields_ = [("start_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("status", c_i32),
                ("cut_count", c_u32), ("visible_count", c_u32), ("pair_count", c_u64), ("replays", c_u32),
                ("lod_from_scratch", c_u32), ("admission_waits", c_u32), ("views_released", c_u32)]


_PROTOS = {
    "vgr_default_view_opts": (None, [ctypes.POINTER(ViewOpts)]),
    "vgr_load_hierarchy": (c_i32, [ctypes.POINTER(SceneDesc), ctypes.POINTER(c_vp)]),
    "vgr_free_hierarchy": (c_i32, [c_vp]),
    "vgr_hierarchy_info": (c_i32, [c_vp, ctypes.POINTER(c_u64), ctypes.POINTER(c_u32)]),
    "vgr_create_view": (c_i32, [c_vp, ctypes.POINTER(ViewOpts), ctypes.POINTER(c_vp)]),
    "vgr_destroy_view": (c_i32, [c_vp]),
    "vgr_reset_view": (c_i32, [c_vp]),
    "vgr_view_set_tuning": (c_i32, [c_vp, c_u32, c_u32, c_u32, c_u32]),
    "vgr_view_device_bytes": (c_i32, [c_vp, ctypes.POINTER(c_u64)]),
    "vgr_render_frame": (c_i32, [c_vp, ctypes.POINTER(Camera), c_f32, ctypes.POINTER(Frame)]),
    "vgr_render_frame_host": (c_i32, [c_vp, ctypes.POINTER(Camera), c_f32, c_vp, ctypes.POINTER(Frame)]),
    "vgr_render_frame_pipelined": (c_i32, [c_vp, ctypes.POINTER(Camera), c_f32, c_vp, ctypes.POINTER(Frame)]),
    "vgr_wait_host_images": (c_i32, [c_vp]),
    "vgr_view_debug": (c_i32, [c_vp, ctypes.POINTER(DebugBuffers)]),
    "vgr_set_batch_chains": (c_i32, [c_u32]),
    "vgr_sort_pairs": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_u32, c_vp]),
    "vgr_sort_pairs_noalloc": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_u32, c_vp]),
    "vgr_last_error": (ctypes.c_char_p, []),
    "vgr_submit_frame": (c_i32, [c_vp, ctypes.POINTER(Camera), c_f32, c_vp]),
    "vgr_frame_done": (c_i32, [c_vp, ctypes.POINTER(c_i32)]),
    "vgr_finish_frame": (c_i32, [c_vp, ctypes.POINTER(Frame)]),
    "vgr_render_batch": (c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(Camera), ctypes.POINTER(c_f32),
                                 ctypes.POINTER(c_vp), c_u32, ctypes.POINTER(Frame)]),
    "vgr_view_bytes_estimate": (c_i32, [c_vp, ctypes.POINTER(ViewOpts), c_u32, c_u32, ctypes.POINTER(c_u64)]),
    "vgr_default_serve_opts": (None, [ctypes.POINTER(ServeOpts)]),
    "vgr_create_server": (c_i32, [c_vp, ctypes.POINTER(ServeOpts), ctypes.POINTER(c_vp)]),
    "vgr_destroy_server": (c_i32, [c_vp]),
    "vgr_serve_trace": (c_i32, [c_vp, ctypes.POINTER(Request), c_u32, ctypes.POINTER(RequestResult)]),
    "vgr_server_client_view": (c_i32, [c_vp, c_u32, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp)]),
}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/vgr.h."""
    src = open(os.path.join(_build.INCLUDE, "vgr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:vgr_status|void|const char\*)\s+(vgr_\w+)\s*\(", src, re.M)))


def load(build: bool = True):
    """Load libvgr.so (building it in-tree first if it is missing or stale).

    There is no fallback: if the library cannot be built or loaded this
    raises, so nothing silently runs without the CUDA path.
    """
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libvgr.so is missing; run paper_2506_02774_gb300._build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class VgrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def check(status: int):
    if status != VGR_OK:
        raise VgrError(status, _lib.vgr_last_error().decode(errors="replace"))

"""GB300 frame path of a city-scale Gaussian-splatting renderer (arXiv
2506.02774): temporal-aware LoD cut update, projection with preemptive
alpha filtering, tile binning, radix sort and front-to-back blending.

This package is the thin Python binding of the C ABI in ``include/vgr.h``
(``libvgr.so``, hand-written CUDA for sm_103a).  It only marshals arguments;
every step of a frame runs in the library's kernels.  PyTorch is used to
view the library's device buffers as tensors and for streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (EXP_EXACT, EXP_LUT, FILTER_CANONICAL, FILTER_PREEMPTIVE, STAGES, STORE_FP32, STORE_HALF,
                   VgrError)

__all__ = ["Renderer", "Hierarchy", "View", "FrameResult", "Server", "render_batch", "camera_struct", "sort_pairs", "VgrError", "view_bytes_estimate",
           "load_library", "STORE_FP32",
           "STORE_HALF", "FILTER_PREEMPTIVE", "FILTER_CANONICAL", "EXP_EXACT", "EXP_LUT", "STAGES"]


def load_library(build: bool = True):
    return _abi.load(build)


def _require(ok: bool, msg: str, exc=ValueError):
    """Argument check that survives python -O (unlike assert)."""
    if not ok:
        raise exc(msg)


def _host_image_ok(a, cam, what: str):
    _require(isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"],
             "%s must be a C-contiguous float32 numpy array" % what, TypeError)
    _require(a.shape == (int(cam["height"]), int(cam["width"]), 3),
             "%s has shape %s, the camera needs (%d, %d, 3)" % (what, a.shape, int(cam["height"]), int(cam["width"])))


def _ptr(a: np.ndarray):
    _require(a.flags["C_CONTIGUOUS"], "array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


class _CudaArray:
    """__cuda_array_interface__ wrapper of a device pointer owned by the library."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_tensor(ptr: int, shape, dtype: str):
    """A torch view (no copy) of library-owned device memory."""
    import torch
    n = int(np.prod(shape)) if len(shape) else 1
    if n == 0 or not ptr:
        return torch.empty(tuple(shape), dtype=getattr(torch, dtype), device="cuda")
    typestr = {"float32": "<f4", "int32": "<i4", "uint8": "|u1"}[dtype if dtype != "uint32" else "int32"]
    t = torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")
    return t


def camera_struct(cam: dict) -> _abi.Camera:
    c = _abi.Camera()
    R = np.asarray(cam["R"], np.float32).reshape(9)
    for i in range(9):
        c.R[i] = float(R[i])
    p = np.asarray(cam["pos"], np.float32)
    for i in range(3):
        c.pos[i] = float(p[i])
    c.fx, c.fy = float(cam["fx"]), float(cam["fy"])
    c.cx, c.cy = float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.z_near = float(cam.get("z_near", 0.2))
    return c


def sort_pairs(keys, vals, key_bits: int = 32, stream=None):
    """Stable radix sort of int32 CUDA tensors (u32 bit patterns) via
    vgr_sort_pairs; returns new (keys, values) tensors."""
    import torch
    _require(keys.is_cuda and vals.is_cuda and keys.dtype == torch.int32 and vals.dtype == torch.int32,
             "keys and values must be int32 CUDA tensors", TypeError)
    _require(keys.is_contiguous() and vals.is_contiguous() and keys.numel() == vals.numel(),
             "keys and values must be contiguous and of equal length")
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    s = torch.cuda.current_stream().cuda_stream if stream is None else int(stream)
    _abi.check(_abi.load().vgr_sort_pairs(keys.data_ptr(), vals.data_ptr(), ko.data_ptr(), vo.data_ptr(),
                                          keys.numel(), int(key_bits), ctypes.c_void_p(s)))
    return ko, vo


class Hierarchy:
    """A LoD tree uploaded to the GPU (``vgr_load_hierarchy``)."""

    def __init__(self, scene: dict, storage: int = STORE_FP32):
        lib = _abi.load()
        self._keep = [np.ascontiguousarray(scene[k]) for k in
                      ("parent", "first_child", "n_child", "mean", "cov6", "opacity", "sh", "radius2")]
        a = self._keep
        _require(a[0].dtype == np.uint32 and a[1].dtype == np.uint32 and a[2].dtype == np.uint8,
                 "parent and first_child must be uint32, n_child uint8", TypeError)
        for name, x in zip(("mean", "cov6", "opacity", "sh", "radius2"), a[3:]):
            _require(x.dtype == np.float32, "%s must be float32" % name, TypeError)
        box = scene.get("bbox")
        if box is not None:
            box = np.ascontiguousarray(box, np.float32)
            _require(box.shape == (int(scene["n_nodes"]), 6), "bbox must have shape (n_nodes, 6)")
            self._keep.append(box)
        d = _abi.SceneDesc(int(scene["n_nodes"]), int(scene["sh_degree"]), *[_ptr(x) for x in a[:8]], int(storage),
                           _ptr(box) if box is not None else None)
        h = ctypes.c_void_p()
        _abi.check(lib.vgr_load_hierarchy(ctypes.byref(d), ctypes.byref(h)))
        self._keep = None  # the library copied everything
        self.handle = h
        self.n_nodes = int(scene["n_nodes"])
        self.sh_degree = int(scene["sh_degree"])
        self.storage = storage
        b, dep = ctypes.c_uint64(), ctypes.c_uint32()
        _abi.check(lib.vgr_hierarchy_info(h, ctypes.byref(b), ctypes.byref(dep)))
        self.device_bytes, self.max_depth = int(b.value), int(dep.value)

    def close(self):
        if self.handle:
            _abi.check(_abi.load().vgr_free_hierarchy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FrameResult:
    """Result of one frame: device image/cut views plus statistics."""

    def __init__(self, fr: _abi.Frame):
        self.raw = fr
        self.width, self.height = int(fr.width), int(fr.height)
        self.cut_count = int(fr.cut_count)
        s = fr.stats
        self.stats = dict(cut_count=int(s.cut_count), front_count=int(s.front_count),
                          visible_count=int(s.visible_count),
                          pair_count=int(s.pair_count), candidate_pairs=int(s.candidate_pairs),
                          nodes_evaluated=int(s.nodes_evaluated), lod_from_scratch=int(s.lod_from_scratch),
                          replays=int(s.replays), kernels=int(s.kernels),
                          pixel_pair_evals=int(s.pixel_pair_evals),
                          pixel_pair_contribs=int(s.pixel_pair_contribs),
                          stage_ms={n: float(s.stage_ms[i]) for i, n in enumerate(STAGES)},
                          frame_ms=float(s.frame_ms))

    def image(self):
        """H x W x 3 float32 CUDA tensor viewing the view's image buffer."""
        return device_tensor(self.raw.image, (self.height, self.width, 3), "float32")

    def cut(self):
        """Ascending node ids (int32 view of the u32 ids) on the device."""
        return device_tensor(self.raw.cut, (self.cut_count,), "int32")


class View:
    """One client's render state (``vgr_create_view``)."""

    def __init__(self, hier: Hierarchy, *, filter: int = FILTER_PREEMPTIVE, exp_mode: int = EXP_EXACT,
                 lut_size: int = 32, temporal: bool = True, timing: bool = False, use_graph: bool = False,
                 cut_capacity: int = 0, pair_capacity: int = 0, lod_budget: int = 0, grid_wide: int = 0,
                 grid_scan: int = 0, test_hooks: int = 0, lod_frustum: bool = False,
                 lod_frustum_guard: float = 2.0, lod_interp: bool = False, blend_depth: int = 0,
                 tile_size: int = 0, stream=None):
        lib = _abi.load()
        o = _abi.ViewOpts()
        lib.vgr_default_view_opts(ctypes.byref(o))
        o.filter, o.exp_mode, o.lut_size = filter, exp_mode, lut_size
        o.temporal, o.timing, o.use_graph = int(temporal), int(timing), int(use_graph)
        o.cut_capacity, o.pair_capacity = cut_capacity, pair_capacity
        if lod_budget:
            o.lod_budget = lod_budget
        o.grid_wide, o.grid_scan = int(grid_wide), int(grid_scan)
        o.test_hooks = int(test_hooks)
        o.lod_frustum, o.lod_frustum_guard = int(lod_frustum), float(lod_frustum_guard)
        o.lod_interp = int(lod_interp)
        if blend_depth:
            o.blend_depth = int(blend_depth)
        if tile_size:
            o.tile_size = int(tile_size)
        if stream is not None:
            o.stream = ctypes.c_void_p(int(stream))
        v = ctypes.c_void_p()
        _abi.check(lib.vgr_create_view(hier.handle, ctypes.byref(o), ctypes.byref(v)))
        self.handle = v
        self.hier = hier
        self._pipelined_hosts = []  # host arrays of copies not yet waited for

    def render(self, cam: dict, tau: float) -> FrameResult:
        fr = _abi.Frame()
        c = camera_struct(cam)
        _abi.check(_abi.load().vgr_render_frame(self.handle, ctypes.byref(c), float(tau), ctypes.byref(fr)))
        return FrameResult(fr)

    def render_host(self, cam: dict, tau: float, out: np.ndarray) -> FrameResult:
        """Render and copy the image into the float32 H x W x 3 host array ``out``."""
        _host_image_ok(out, cam, "out")
        fr = _abi.Frame()
        c = camera_struct(cam)
        _abi.check(_abi.load().vgr_render_frame_host(self.handle, ctypes.byref(c), float(tau),
                                                     ctypes.c_void_p(out.ctypes.data), ctypes.byref(fr)))
        return FrameResult(fr)

    def render_host_ptr(self, cam_struct: _abi.Camera, tau: float, host_ptr: int, fr: _abi.Frame) -> int:
        """Lowest-overhead form of render_host (pre-built structs); returns the status."""
        return _abi.load().vgr_render_frame_host(self.handle, ctypes.byref(cam_struct), float(tau),
                                                 ctypes.c_void_p(host_ptr), ctypes.byref(fr))

    def render_pipelined(self, cam: dict, tau: float, out: np.ndarray) -> FrameResult:
        """Render, with the copy of the image into the float32 H x W x 3 host
        array ``out`` overlapping the next frame (``vgr_render_frame_pipelined``):
        ``out`` holds the image once ``wait_host_images`` returns, and is kept
        alive until then."""
        _host_image_ok(out, cam, "out")
        fr = _abi.Frame()
        c = camera_struct(cam)
        self._pipelined_hosts.append(out)
        _abi.check(_abi.load().vgr_render_frame_pipelined(self.handle, ctypes.byref(c), float(tau),
                                                          ctypes.c_void_p(out.ctypes.data), ctypes.byref(fr)))
        return FrameResult(fr)

    def render_pipelined_ptr(self, cam_struct: _abi.Camera, tau: float, host_ptr: int, fr: _abi.Frame) -> int:
        """Lowest-overhead form of render_pipelined (pre-built structs, the
        caller keeps the host buffer alive); returns the status."""
        return _abi.load().vgr_render_frame_pipelined(self.handle, ctypes.byref(cam_struct), float(tau),
                                                      ctypes.c_void_p(host_ptr), ctypes.byref(fr))

    def wait_host_images(self) -> None:
        """Wait until every pipelined image copy of this view has landed."""
        _abi.check(_abi.load().vgr_wait_host_images(self.handle))
        self._pipelined_hosts = []

    def submit(self, cam: dict, tau: float, host_out: np.ndarray | None = None):
        """Enqueue a frame without waiting (``vgr_submit_frame``); ``host_out``
        (float32 H x W x 3, kept alive until finish) receives the image."""
        c = camera_struct(cam)
        ptr = None
        if host_out is not None:
            _host_image_ok(host_out, cam, "host_out")
            ptr = ctypes.c_void_p(host_out.ctypes.data)
        self._pending_host = host_out
        _abi.check(_abi.load().vgr_submit_frame(self.handle, ctypes.byref(c), float(tau), ptr))

    def done(self) -> bool:
        d = ctypes.c_int32()
        _abi.check(_abi.load().vgr_frame_done(self.handle, ctypes.byref(d)))
        return bool(d.value)

    def finish(self) -> FrameResult:
        fr = _abi.Frame()
        try:
            _abi.check(_abi.load().vgr_finish_frame(self.handle, ctypes.byref(fr)))
        finally:
            self._pending_host = None
        return FrameResult(fr)

    def reset(self):
        _abi.check(_abi.load().vgr_reset_view(self.handle))

    def set_tuning(self, grid_wide: int = 0, grid_scan: int = 0, blend_depth: int = 0, tile_size: int = 0):
        """Change the launch geometry, the blend's staging depth and the tile
        size (0 keeps a value; ``vgr_view_set_tuning``)."""
        _abi.check(_abi.load().vgr_view_set_tuning(self.handle, int(grid_wide), int(grid_scan), int(blend_depth),
                                                   int(tile_size)))

    def device_bytes(self) -> int:
        b = ctypes.c_uint64()
        _abi.check(_abi.load().vgr_view_device_bytes(self.handle, ctypes.byref(b)))
        return int(b.value)

    def debug(self) -> dict:
        """Copies of the last frame's intermediate buffers (numpy).  The
        per-Gaussian arrays are returned for the visible Gaussians only, in
        ascending node order, and depth_order indexes them."""
        d = _abi.DebugBuffers()
        _abi.check(_abi.load().vgr_view_debug(self.handle, ctypes.byref(d)))
        nf, nv, nc, npairs = int(d.n_front), int(d.n_visible), int(d.n_cut), int(d.n_pairs)
        T = int(d.tiles_x) * int(d.tiles_y)

        def u32(ptr, n):
            return device_tensor(ptr, (n,), "int32").cpu().numpy().view(np.uint32).copy()

        def f32(ptr, shape):
            return device_tensor(ptr, shape, "float32").cpu().numpy().copy()

        ntile = u32(d.vis_ntile, nf)
        vis = ntile > 0
        compact = np.cumsum(vis) - 1
        order = u32(d.depth_order, nf)[:nv]
        pval = u32(d.pair_val, npairs)
        rank_of_front = np.full(max(nf, 1), 0xFFFFFFFF, np.int64)  # in-front index -> depth rank
        rank_of_front[order] = np.arange(nv)
        assert vis[order].all(), "the first n_visible depth ranks must be visible entries"
        return dict(n_cut=nc, n_front=nf, n_visible=nv, n_pairs=npairs, tiles=(int(d.tiles_x), int(d.tiles_y)),
                    cut=u32(d.cut, nc), vis_node=u32(d.vis_node, nf)[vis], vis_depth=u32(d.vis_depth, nf)[vis],
                    vis_ntile=ntile[vis], vis_rect=u32(d.vis_rect, 2 * nf).reshape(nf, 2)[vis],
                    vis_recA=f32(d.vis_recA, (nf, 4))[vis], vis_recB=f32(d.vis_recB, (nf, 4))[vis],
                    vis_rgb=f32(d.vis_rgb, (nf, 4))[vis], depth_order=compact[order].astype(np.uint32),
                    pair_tile=u32(d.pair_tile, npairs), pair_rank=rank_of_front[pval >> 8], pair_rowmask=pval & 0xFF,
                    tile_range=u32(d.tile_range, 2 * T).reshape(T, 2), tile_size=int(d.tile_size))

    def close(self):
        if self.handle:
            _abi.check(_abi.load().vgr_destroy_view(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render_batch(views, cams, taus, host_outs=None):
    """One frame on each of several distinct views (``vgr_render_batch``):
    all submitted, then all finished.  Returns one FrameResult per view."""
    n = len(views)
    _require(len(cams) == n and len(taus) == n, "views, cams and taus must have the same length")
    if n == 0:
        return []
    hv = (ctypes.c_void_p * n)(*[v.handle.value for v in views])
    cs = (_abi.Camera * n)(*[camera_struct(c) for c in cams])
    ts = (ctypes.c_float * n)(*[float(t) for t in taus])
    hp = None
    if host_outs is not None:
        for a, c in zip(host_outs, cams):
            if a is not None:
                _host_image_ok(a, c, "host_outs[i]")
        hp = (ctypes.c_void_p * n)(*[(a.ctypes.data if a is not None else None) for a in host_outs])
    frs = (_abi.Frame * n)()
    _abi.check(_abi.load().vgr_render_batch(hv, cs, ts, hp, n, frs))
    return [FrameResult(frs[i]) for i in range(n)]


class Renderer:
    """One scene and one view in a single object: ``vgr_load_hierarchy``,
    then ``vgr_create_view`` with the given view options (the keyword
    arguments of :class:`View`), then ``vgr_render_frame`` per call.  Frames
    rendered in sequence reuse the previous cut (the temporal update)."""

    def __init__(self, scene: dict, storage: int = STORE_FP32, **view_opts):
        self.hierarchy = Hierarchy(scene, storage)
        try:
            self.view = View(self.hierarchy, **view_opts)
        except BaseException:
            self.hierarchy.close()
            raise

    def render(self, cam: dict, tau: float) -> FrameResult:
        return self.view.render(cam, tau)

    def render_host(self, cam: dict, tau: float, out: np.ndarray) -> FrameResult:
        return self.view.render_host(cam, tau, out)

    def render_pipelined(self, cam: dict, tau: float, out: np.ndarray) -> FrameResult:
        return self.view.render_pipelined(cam, tau, out)

    def wait_host_images(self) -> None:
        self.view.wait_host_images()

    def reset(self):
        self.view.reset()

    def close(self):
        self.view.close()
        self.hierarchy.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def set_batch_chains(chains: int) -> None:
    """How many views of a captured batch run at once (``vgr_set_batch_chains``):
    ``chains`` parallel chains, largest image first to the least-loaded chain;
    0 runs every view as its own branch.  Results do not depend on it."""
    _abi.check(_abi.load().vgr_set_batch_chains(int(chains)))


def view_bytes_estimate(hier: Hierarchy, width: int, height: int, **view_kw) -> int:
    """Device bytes a view with these options holds after its first frame at
    width x height (``vgr_view_bytes_estimate``)."""
    lib = _abi.load()
    o = _abi.ViewOpts()
    lib.vgr_default_view_opts(ctypes.byref(o))
    for k, val in view_kw.items():
        setattr(o, k, val)
    b = ctypes.c_uint64()
    _abi.check(lib.vgr_view_bytes_estimate(hier.handle, ctypes.byref(o), int(width), int(height), ctypes.byref(b)))
    return int(b.value)


class Server:
    """Continuous-batching frame server over one hierarchy (``vgr_create_server``)."""

    def __init__(self, hier: Hierarchy, n_clients: int, *, max_inflight: int | None = None,
                 host_images: bool = False, hbm_reserve: int | None = None, use_graph: bool = True,
                 evict_idle: bool = True, **view_kw):
        lib = _abi.load()
        o = _abi.ServeOpts()
        lib.vgr_default_serve_opts(ctypes.byref(o))
        o.n_clients, o.host_images = int(n_clients), int(host_images)
        if max_inflight is not None:  # else the library's default (2)
            o.max_inflight = int(max_inflight)
        o.evict_idle = int(bool(evict_idle))
        if hbm_reserve is not None:
            o.hbm_reserve = int(hbm_reserve)
        o.view.use_graph = int(use_graph)
        for k, val in view_kw.items():
            setattr(o.view, k, val)
        s = ctypes.c_void_p()
        _abi.check(lib.vgr_create_server(hier.handle, ctypes.byref(o), ctypes.byref(s)))
        self.handle = s
        self.hier = hier
        self.n_clients = int(n_clients)

    def serve(self, requests, images: bool = False):
        """Serve a trace in real time.  ``requests``: list of dicts with client,
        arrival_s, cam, tau (arrival_s non-decreasing).  Returns a numpy record
        array with start_s, finish_s, status, counts per request; with
        ``images`` also a list of every request's image (pinned host buffers
        the blend writes directly, one per request)."""
        n = len(requests)
        rq = (_abi.Request * max(1, n))()
        bufs = []
        if images:
            import torch
        for i, r in enumerate(requests):
            rq[i].client = int(r["client"])
            rq[i].tau = float(r["tau"])
            rq[i].arrival_s = float(r["arrival_s"])
            rq[i].cam = camera_struct(r["cam"])
            if images:
                b = torch.zeros((int(r["cam"]["height"]), int(r["cam"]["width"]), 3), dtype=torch.float32,
                                pin_memory=True)
                bufs.append(b)
                rq[i].host_rgb = b.data_ptr()
        rs = (_abi.RequestResult * max(1, n))()
        _abi.check(_abi.load().vgr_serve_trace(self.handle, rq, n, rs))
        out = np.zeros(n, dtype=[("client", "u4"), ("arrival_s", "f8"), ("start_s", "f8"), ("finish_s", "f8"),
                                 ("status", "i4"), ("cut_count", "u4"), ("visible_count", "u4"),
                                 ("pair_count", "u8"), ("replays", "u4"), ("lod_from_scratch", "u4"),
                                 ("admission_waits", "u4"), ("views_released", "u4")])
        for i in range(n):
            x = rs[i]
            out[i] = (rq[i].client, rq[i].arrival_s, x.start_s, x.finish_s, x.status, x.cut_count, x.visible_count,
                      x.pair_count, x.replays, x.lod_from_scratch, x.admission_waits, x.views_released)
        if images:
            return out, [b.numpy().copy() for b in bufs]
        return out

    def client_host_image(self, client: int, height: int, width: int):
        """A copy of the client's last image from its pinned host buffer
        (servers created with host_images=True); None before admission."""
        v, hp = ctypes.c_void_p(), ctypes.c_void_p()
        _abi.check(_abi.load().vgr_server_client_view(self.handle, int(client), ctypes.byref(v), ctypes.byref(hp)))
        if not hp.value:
            return None
        n = int(height) * int(width) * 3
        return np.ctypeslib.as_array((ctypes.c_float * n).from_address(hp.value)).reshape(height, width, 3).copy()

    def close(self):
        if self.handle:
            _abi.check(_abi.load().vgr_destroy_server(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

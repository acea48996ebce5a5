"""Seeded synthetic inputs: leaf Gaussians, their LoD tree, camera paths.

This module is input infrastructure shared by the CPU oracle tests and the
GPU renderer's tests and bench.  It contains none of the per-frame method
(cut finding, projection, binning, sorting, blending); it draws the scenes
and the camera poses the method is run on, and builds the LoD tree of
paper Sec. 3.1 (one Gaussian per node, variable fan-out, finer Gaussians
lower in the tree) with opacity-weighted moment-matched parents.

The heavy lifting is in ``scenegen.c`` (compiled on first use with gcc).

Workloads (the paper's city datasets are not available; these synthetic
scenes stand in for them with the same scale and structure):

* ``tiny``  -- 4,096 leaves uniform in a 20x20x5 m box, log-scales
  N(-3, 0.5), opacity sigmoid(N(0, 1.5)), SH degree 0 with DC ~ N(0, 0.3);
  128x128, fx = fy = 120, tau = 3 px, 16 frames at 30 fps, 1 m/s.
* ``m1``    -- 1M leaves in a 200x200x30 m box, same distributions but SH
  degree 3 (DC ~ N(0, 0.3), bands 1-3 ~ N(0, 0.1)); 1920x1080,
  fx = fy = 1100, tau = 3 px, 300 frames, 1.2 m/s, yaw rate <= 20 deg/s.
* ``city``  -- 18M leaves on a 1.5 x 1.5 km street grid: 80 % on 38 x- and
  38 y-streets 40 m apart (lateral offset U[-15, 15] m, height U[0, 40] m),
  20 % on the ground (z = |N(0, 0.2)|); log-scales N(-2.5, 0.7), SH degree 3;
  1080p, fx = fy = 1100, tau = 3 px, 600-frame walk at 1.7 m height, 1.4 m/s.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scenegen.c")
_LIB = os.path.join(_HERE, "libscenegen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile scenegen.c into libscenegen.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
        ("box", ctypes.c_double * 6),
        ("logscale_mu", ctypes.c_double), ("logscale_sigma", ctypes.c_double),
        ("opacity_sigma", ctypes.c_double),
        ("dc_sigma", ctypes.c_double), ("band_sigma", ctypes.c_double),
        ("city_extent", ctypes.c_double), ("street_spacing", ctypes.c_double),
        ("n_streets", ctypes.c_int32), ("street_halfwidth", ctypes.c_double),
        ("street_height", ctypes.c_double), ("street_frac", ctypes.c_double),
        ("ground_sigma", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.sg_gen_leaves.argtypes = [ctypes.POINTER(_Params), ctypes.c_uint64, ctypes.c_uint64,
                                          P, P, P, P, P]
            lib.sg_gen_leaves.restype = ctypes.c_int
            lib.sg_tree_build.argtypes = [ctypes.c_uint64, P]
            lib.sg_tree_build.restype = P
            lib.sg_tree_nodes.argtypes = [P]
            lib.sg_tree_nodes.restype = ctypes.c_uint64
            lib.sg_tree_depth.argtypes = [P]
            lib.sg_tree_depth.restype = ctypes.c_uint32
            lib.sg_tree_fill.argtypes = [P, ctypes.c_int] + [P] * 13
            lib.sg_tree_fill.restype = ctypes.c_int
            lib.sg_tree_boxes.argtypes = [ctypes.c_uint64, P, P, P, P, P]
            lib.sg_tree_boxes.restype = ctypes.c_int
            lib.sg_tree_free.argtypes = [P]
            lib.sg_tree_free.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ----------------------------------------------------------------- leaves
def gen_leaves(n: int, seed: int, *, kind: str = "box", sh_degree: int = 0,
               box=(0.0, 20.0, 0.0, 20.0, 0.0, 5.0), logscale=(-3.0, 0.5),
               opacity_sigma: float = 1.5, dc_sigma: float = 0.3, band_sigma: float = 0.1,
               city_extent: float = 1500.0, street_spacing: float = 40.0, n_streets: int = 38,
               street_halfwidth: float = 15.0, street_height: float = 40.0,
               street_frac: float = 0.8, ground_sigma: float = 0.2) -> dict:
    """Draw ``n`` leaf Gaussians (FP32 arrays, see scenegen.c for the recipe)."""
    lib = _load()
    p = _Params()
    p.kind = 0 if kind == "box" else 1
    p.sh_degree = sh_degree
    for i, v in enumerate(box):
        p.box[i] = v
    p.logscale_mu, p.logscale_sigma = logscale
    p.opacity_sigma = opacity_sigma
    p.dc_sigma, p.band_sigma = dc_sigma, band_sigma
    p.city_extent, p.street_spacing, p.n_streets = city_extent, street_spacing, n_streets
    p.street_halfwidth, p.street_height = street_halfwidth, street_height
    p.street_frac, p.ground_sigma = street_frac, ground_sigma
    K = (sh_degree + 1) ** 2
    out = dict(mean=np.empty((n, 3), np.float32), cov6=np.empty((n, 6), np.float32),
               opacity=np.empty(n, np.float32), sh=np.empty((n, K, 3), np.float32),
               rad2=np.empty(n, np.float32))
    rc = lib.sg_gen_leaves(ctypes.byref(p), n, seed, _ptr(out["mean"]), _ptr(out["cov6"]),
                           _ptr(out["opacity"]), _ptr(out["sh"]), _ptr(out["rad2"]))
    if rc != 0:
        raise RuntimeError("sg_gen_leaves failed")
    out["sh_degree"] = sh_degree
    return out


def leaf_rad2(scales: np.ndarray) -> np.ndarray:
    """radius^2 of a leaf with the given axis scales: (3 max scale)^2 rounded up to FP32."""
    r = 3.0 * np.max(np.asarray(scales, np.float64), axis=-1)
    r2 = r * r
    f = r2.astype(np.float32)
    low = f.astype(np.float64) < r2
    f[low] = np.nextafter(f[low], np.float32(np.inf))
    return f


# ------------------------------------------------------------------- tree
def build_tree(leaves: dict) -> dict:
    """Build the BFS-ordered, moment-matched LoD tree over ``leaves``.

    Returns a scene dict: parent (u32, root = 0xFFFFFFFF), first_child (u32),
    n_child (u8), mean (N,3), cov6 (N,6: xx xy xz yy yz zz), opacity (N),
    sh (N, (deg+1)^2, 3), radius2 (N), plus sh_degree, n_nodes, n_leaves,
    max_depth.
    """
    lib = _load()
    mean = np.ascontiguousarray(leaves["mean"], np.float32)
    n = mean.shape[0]
    t = lib.sg_tree_build(n, _ptr(mean))
    if not t:
        raise RuntimeError("sg_tree_build failed")
    try:
        N = int(lib.sg_tree_nodes(t))
        depth = int(lib.sg_tree_depth(t))
        K = (leaves["sh_degree"] + 1) ** 2
        sc = dict(parent=np.empty(N, np.uint32), first_child=np.empty(N, np.uint32),
                  n_child=np.empty(N, np.uint8), mean=np.empty((N, 3), np.float32),
                  cov6=np.empty((N, 6), np.float32), opacity=np.empty(N, np.float32),
                  sh=np.empty((N, K, 3), np.float32), radius2=np.empty(N, np.float32))
        lc = np.ascontiguousarray(leaves["cov6"], np.float32)
        lo = np.ascontiguousarray(leaves["opacity"], np.float32)
        ls = np.ascontiguousarray(leaves["sh"], np.float32)
        lr = np.ascontiguousarray(leaves["rad2"], np.float32)
        rc = lib.sg_tree_fill(t, 3 * K, _ptr(mean), _ptr(lc), _ptr(lo), _ptr(ls), _ptr(lr),
                              _ptr(sc["parent"]), _ptr(sc["first_child"]), _ptr(sc["n_child"]),
                              _ptr(sc["mean"]), _ptr(sc["cov6"]), _ptr(sc["opacity"]),
                              _ptr(sc["sh"]), _ptr(sc["radius2"]))
        if rc != 0:
            raise RuntimeError("sg_tree_fill failed")
    finally:
        lib.sg_tree_free(t)
    sc.update(sh_degree=leaves["sh_degree"], n_nodes=N, n_leaves=n, max_depth=depth)
    sc["bbox"] = tree_boxes(sc)
    return sc


def tree_boxes(sc: dict) -> np.ndarray:
    """Nested axis-aligned node boxes (N, 6: lo xyz, hi xyz), FP32 rounded
    outward: a node's box holds mu +- 3.34 sqrt(diag Sigma) of its own
    Gaussian and its children's boxes."""
    lib = _load()
    N = int(sc["n_nodes"])
    box = np.empty((N, 6), np.float32)
    fc = np.ascontiguousarray(sc["first_child"], np.uint32)
    nc = np.ascontiguousarray(sc["n_child"], np.uint8)
    mean = np.ascontiguousarray(sc["mean"], np.float32)
    cov = np.ascontiguousarray(sc["cov6"], np.float32)
    if lib.sg_tree_boxes(N, _ptr(fc), _ptr(nc), _ptr(mean), _ptr(cov), _ptr(box)) != 0:
        raise RuntimeError("sg_tree_boxes failed")
    return box


def single_node_scene(mean, cov6, opacity, sh, sh_degree: int = 0) -> dict:
    """A one-node tree (the root is the only Gaussian and is a leaf)."""
    K = (sh_degree + 1) ** 2
    return dict(parent=np.array([0xFFFFFFFF], np.uint32), first_child=np.zeros(1, np.uint32),
                n_child=np.zeros(1, np.uint8), mean=np.asarray(mean, np.float32).reshape(1, 3),
                cov6=np.asarray(cov6, np.float32).reshape(1, 6),
                opacity=np.asarray([opacity], np.float32),
                sh=np.asarray(sh, np.float32).reshape(1, K, 3),
                radius2=np.ones(1, np.float32), sh_degree=sh_degree, n_nodes=1, n_leaves=1,
                max_depth=0)


def cov6_from_scale_rot(scale, R) -> np.ndarray:
    """Sigma = R diag(scale^2) R^T packed as xx xy xz yy yz zz (FP32)."""
    R = np.asarray(R, np.float64)
    S = R @ np.diag(np.asarray(scale, np.float64) ** 2) @ R.T
    return np.array([S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]], np.float32)


# --------------------------------------------------------------- workloads
CONFIGS = {
    "tiny": dict(n_leaves=4096, seed=1, leaves=dict(kind="box", sh_degree=0,
                 box=(0.0, 20.0, 0.0, 20.0, 0.0, 5.0), logscale=(-3.0, 0.5)),
                 width=128, height=128, focal=120.0, tau=3.0, frames=16, fps=30.0,
                 start=(2.0, 10.0, 2.5), speed=1.0, yaw_amp_deg=5.0, yaw_period=2.0),
    "m1": dict(n_leaves=1_000_000, seed=2, leaves=dict(kind="box", sh_degree=3,
               box=(0.0, 200.0, 0.0, 200.0, 0.0, 30.0), logscale=(-3.0, 0.5)),
               width=1920, height=1080, focal=1100.0, tau=3.0, frames=300, fps=30.0,
               start=(20.0, 100.0, 10.0), speed=1.2, yaw_amp_deg=30.0, yaw_period=10.0),
    "city": dict(n_leaves=18_000_000, seed=3, leaves=dict(kind="city", sh_degree=3,
                 logscale=(-2.5, 0.7)),
                 width=1920, height=1080, focal=1100.0, tau=3.0, frames=600, fps=30.0,
                 start=(100.0, 720.0, 1.7), speed=1.4, yaw_amp_deg=30.0, yaw_period=10.0),
}


# image sizes of the multi-view and serving workloads
RESOLUTIONS = {"360p": (640, 360), "720p": (1280, 720), "1080p": (1920, 1080), "1440p": (2560, 1440)}


def street_trajectory(name: str, seed: int, frame: int, width: int, height: int) -> dict:
    """Camera of ``frame`` on a street walk of its own (one per view or
    client, chosen by ``seed``): a street of the city grid (x- or y-street,
    index 1..36 of the 40 m grid), a direction and a starting point drawn from
    ``seed``; the workload's height, speed and yaw law; focal length scaled
    with the image width (fx = focal * width / the workload's width)."""
    c = CONFIGS[name]
    rng = np.random.default_rng(seed)
    along_x = bool(rng.random() < 0.5)
    k = int(rng.integers(1, 37))
    forward = bool(rng.random() < 0.5)
    s0 = float(rng.uniform(200.0, 1300.0))
    z = c["start"][2]
    if along_x:
        start, heading = (s0, 40.0 * k, z), (0.0 if forward else math.pi)
    else:
        start, heading = (40.0 * k, s0, z), (0.5 * math.pi if forward else -0.5 * math.pi)
    t = frame / c["fps"]
    pos = np.asarray(start) + c["speed"] * t * np.array([math.cos(heading), math.sin(heading), 0.0])
    yaw = heading + math.radians(c["yaw_amp_deg"]) * math.sin(2.0 * math.pi * t / c["yaw_period"])
    return camera(pos, yaw, width, height, c["focal"] * width / c["width"])


def make_scene(name: str, n_leaves: int | None = None, seed: int | None = None) -> dict:
    """Generate the named workload's scene (optionally with fewer leaves)."""
    c = CONFIGS[name]
    n = c["n_leaves"] if n_leaves is None else n_leaves
    leaves = gen_leaves(n, c["seed"] if seed is None else seed, **c["leaves"])
    sc = build_tree(leaves)
    del leaves
    sc["config"] = name
    return sc


def look_rotation(yaw: float, pitch: float = 0.0) -> np.ndarray:
    """World->camera rotation (rows: right, down, forward) in a z-up world.

    The camera looks along (cos yaw cos pitch, sin yaw cos pitch, sin pitch);
    camera axes follow OpenCV: x right, y down, z forward.
    """
    f = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return np.stack([r, d, f])


def camera(pos, yaw: float, width: int, height: int, focal: float, pitch: float = 0.0,
           z_near: float = 0.2) -> dict:
    """Pinhole camera: p_cam = R (p - pos); pixel = (fx x/z + cx, fy y/z + cy)."""
    return dict(R=look_rotation(yaw, pitch).astype(np.float32), pos=np.asarray(pos, np.float32),
                fx=np.float32(focal), fy=np.float32(focal), cx=np.float32(width / 2.0),
                cy=np.float32(height / 2.0), width=int(width), height=int(height),
                z_near=np.float32(z_near))


def trajectory(name: str, frame: int, heading: float = 0.0, start=None) -> dict:
    """Camera of ``frame`` on the workload's walk.

    The position advances along ``heading`` at the workload's speed; the view
    yaw swings as heading + A sin(2 pi t / period) (t = frame / fps), which
    keeps |d yaw / dt| <= 2 pi A / period (18.9 deg/s for A = 30 deg, 10 s).
    """
    c = CONFIGS[name]
    t = frame / c["fps"]
    s = np.asarray(c["start"] if start is None else start, np.float64)
    pos = s + c["speed"] * t * np.array([math.cos(heading), math.sin(heading), 0.0])
    yaw = heading + math.radians(c["yaw_amp_deg"]) * math.sin(2.0 * math.pi * t / c["yaw_period"])
    return camera(pos, yaw, c["width"], c["height"], c["focal"])

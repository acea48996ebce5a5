"""FP64 CPU oracle of the per-frame path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA renderer; the
two meet only in the seeded inputs of ``scenegen``.

``oracle.c`` holds the arithmetic (each step cites the paper section it
follows); this module compiles it with gcc on first use and returns numpy
arrays.  The environment variable ``ORACLE_LIB`` names another build of
``oracle.c`` to load instead (the planted-mistake test loads mutated copies
this way).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALPHA_MIN = 1.0 / 255.0
T_MIN = 1e-4
TILE = 16


def build(force: bool = False) -> str:
    """Compile oracle.c (FP64, no FMA contraction, OpenMP) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint32), ("sh_degree", ctypes.c_uint32),
                ("parent", ctypes.c_void_p), ("first_child", ctypes.c_void_p),
                ("n_child", ctypes.c_void_p), ("mean", ctypes.c_void_p),
                ("cov6", ctypes.c_void_p), ("opacity", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("radius2", ctypes.c_void_p), ("bbox", ctypes.c_void_p)]


class _Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("pos", ctypes.c_float * 3),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("z_near", ctypes.c_float)]


class _Frame(ctypes.Structure):
    _fields_ = [("n_cut", ctypes.c_int64), ("cut", ctypes.c_void_p), ("proj", ctypes.c_void_p),
                ("n_cand", ctypes.c_int64), ("cand_tile", ctypes.c_void_p),
                ("cand_idx", ctypes.c_void_p), ("cand_margin", ctypes.c_void_p),
                ("n_pairs", ctypes.c_int64), ("pair_tile", ctypes.c_void_p),
                ("pair_idx", ctypes.c_void_p), ("tile_start", ctypes.c_void_p),
                ("n_tiles", ctypes.c_int64), ("image", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("n_eval", ctypes.c_void_p),
                ("n_contrib", ctypes.c_void_p), ("n_visible", ctypes.c_int64),
                ("n_eval_total", ctypes.c_int64)]


PROJ_DTYPE = np.dtype([("valid", np.int32), ("visible", np.int32), ("zkey", np.float32),
                       ("z", np.float64), ("u", np.float64), ("v", np.float64),
                       ("cov", np.float64, 3), ("conic", np.float64, 3), ("rgb", np.float64, 3),
                       ("theta", np.float64), ("thr", np.float64), ("rect", np.int32, 4),
                       ("ntile", np.int32)], align=True)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(os.environ.get("ORACLE_LIB") or build())
            P = ctypes.c_void_p
            lib.orc_lod_k.argtypes = [ctypes.c_float, ctypes.c_float]
            lib.orc_lod_k.restype = ctypes.c_float
            lib.orc_expand_node.argtypes = [ctypes.POINTER(_Scene), ctypes.c_uint32, P, ctypes.c_float, P]
            lib.orc_expand_node.restype = ctypes.c_int
            for fn in (lib.orc_cut_topdown, lib.orc_cut_bruteforce):
                fn.argtypes = [ctypes.POINTER(_Scene), P, ctypes.c_float, P, P]
                fn.restype = ctypes.c_int64
            lib.orc_frustum_planes.argtypes = [ctypes.POINTER(_Camera), ctypes.c_float, P]
            lib.orc_frustum_planes.restype = None
            lib.orc_box_meets.argtypes = [P, P]
            lib.orc_box_meets.restype = ctypes.c_int
            lib.orc_sh_basis.argtypes = [ctypes.c_int, P, P]
            lib.orc_sh_basis.restype = None
            lib.orc_rho_max_rect.argtypes = [P] + [ctypes.c_double] * 6
            lib.orc_rho_max_rect.restype = ctypes.c_double
            lib.orc_render.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera), ctypes.c_float,
                                       P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_float,
                                       ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32]
            lib.orc_interp_weight.argtypes = [ctypes.POINTER(_Scene), ctypes.c_uint32, P, ctypes.c_float]
            lib.orc_interp_weight.restype = ctypes.c_float
            lib.orc_render.restype = ctypes.POINTER(_Frame)
            lib.orc_frame_free.argtypes = [ctypes.POINTER(_Frame)]
            lib.orc_frame_free.restype = None
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            lib.orc_proj_size.restype = ctypes.c_size_t
            assert lib.orc_proj_size() == PROJ_DTYPE.itemsize, "orc_proj layout mismatch"
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class _SceneRef:
    """Keeps the numpy arrays alive while C holds pointers into them."""

    def __init__(self, sc: dict):
        self.arrays = [np.ascontiguousarray(sc[k]) for k in
                       ("parent", "first_child", "n_child", "mean", "cov6", "opacity", "sh", "radius2")]
        a = self.arrays
        assert a[0].dtype == np.uint32 and a[1].dtype == np.uint32 and a[2].dtype == np.uint8
        for x in a[3:]:
            assert x.dtype == np.float32
        box = sc.get("bbox")
        if box is not None:
            box = np.ascontiguousarray(box, np.float32)
            self.arrays.append(box)
        self.s = _Scene(int(sc["n_nodes"]), int(sc["sh_degree"]), *[_ptr(x) for x in a[:8]],
                        _ptr(box) if box is not None else None)


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    R = np.asarray(cam["R"], np.float32).reshape(9)
    for i in range(9):
        c.R[i] = float(R[i])
    pos = np.asarray(cam["pos"], np.float32)
    for i in range(3):
        c.pos[i] = float(pos[i])
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.z_near = float(cam.get("z_near", 0.2))
    return c


def set_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def lod_k(tau: float, f: float) -> np.float32:
    """k = fl(fl(tau / f)^2), the squared size ratio of the granularity test."""
    return np.float32(_load().orc_lod_k(float(np.float32(tau)), float(np.float32(f))))


def frustum_planes(cam: dict, guard: float) -> np.ndarray:
    """The five (w0, w1, w2, o) planes of the frustum-aware test (5 x 4 float32)."""
    c = _camera(cam)
    out = np.zeros((5, 4), np.float32)
    _load().orc_frustum_planes(ctypes.byref(c), float(np.float32(guard)), _ptr(out))
    return out


def box_meets(box6, planes) -> bool:
    """Does the box (lo xyz, hi xyz) meet all five half-spaces?"""
    b = np.ascontiguousarray(box6, np.float32)
    pl = np.ascontiguousarray(planes, np.float32)
    return bool(_load().orc_box_meets(_ptr(b), _ptr(pl)))


def _planes_arg(planes):
    if planes is None:
        return None, None
    pl = np.ascontiguousarray(planes, np.float32).reshape(20)
    return pl, _ptr(pl)


def expand(sc: dict, node: int, cam_pos, k, planes=None) -> bool:
    """The granularity test (with the frustum-aware box test when ``planes`` is given)."""
    ref = _SceneRef(sc)
    p = np.asarray(cam_pos, np.float32)
    keep, pp = _planes_arg(planes)
    return bool(_load().orc_expand_node(ctypes.byref(ref.s), node, _ptr(p), float(np.float32(k)), pp))


def cut(sc: dict, cam_pos, k, bruteforce: bool = False, planes=None) -> np.ndarray:
    """Ascending node ids of the cut for camera position ``cam_pos`` and ``k``
    (frustum-aware when ``planes``, from :func:`frustum_planes`, is given)."""
    lib = _load()
    ref = _SceneRef(sc)
    p = np.ascontiguousarray(cam_pos, np.float32)
    out = np.empty(max(1, int(sc["n_nodes"])), np.uint32)
    fn = lib.orc_cut_bruteforce if bruteforce else lib.orc_cut_topdown
    keep, pp = _planes_arg(planes)
    n = fn(ctypes.byref(ref.s), _ptr(p), float(np.float32(k)), pp, _ptr(out))
    if n < 0:
        raise MemoryError("oracle cut")
    return out[:n].copy()


def interp_weight(sc: dict, node: int, cam_pos, t) -> np.float32:
    """Parent weight of cut node ``node`` in the interpolated Gaussian
    (FP32), with t = fl(tau / f)."""
    ref = _SceneRef(sc)
    p = np.ascontiguousarray(cam_pos, np.float32)
    return np.float32(_load().orc_interp_weight(ctypes.byref(ref.s), int(node), _ptr(p), float(np.float32(t))))


def sh_basis(degree: int, d) -> np.ndarray:
    """Real orthonormal SH basis values (index l*l + l + m) at unit vector d."""
    d = np.ascontiguousarray(d, np.float64)
    Y = np.zeros(16, np.float64)
    _load().orc_sh_basis(int(degree), _ptr(d), _ptr(Y))
    return Y[:(degree + 1) ** 2].copy()


def rho_max_rect(conic, u, v, x0, x1, y0, y1) -> float:
    c = np.ascontiguousarray(conic, np.float64)
    return float(_load().orc_rho_max_rect(_ptr(c), u, v, x0, x1, y0, y1))


def _arr(ptr, dtype, n):
    if n <= 0:
        return np.zeros(0, dtype)
    dt = np.dtype(dtype)
    buf = (ctypes.c_char * (dt.itemsize * n)).from_address(ptr)
    return np.frombuffer(buf, dtype=dt, count=n).copy()


def render(sc: dict, cam: dict, tau: float, *, tile_mask=None, band: float = 2e-3, t_flag: float = 0.05,
           exhaustive: bool = False, frustum_guard: float | None = None, interp: bool = False,
           lut_m: int = 0, tile: int = TILE) -> dict:
    """Render one frame; returns the cut, per-cut projection, pairs and image.

    ``tile_mask`` (bool per tile, row-major) restricts binning and blending
    to those tiles.  A pixel is flagged when some Gaussian's rho lies within
    ``band`` (nats) of ln alpha* - ln theta while the transmittance is still
    >= ``t_flag``: there an FP32 renderer may take the other side of the
    alpha >= alpha* test and move the pixel by up to ~alpha* T max(rgb).
    ``frustum_guard`` (pixels; needs ``sc["bbox"]``) selects the
    frustum-aware cut; ``interp`` renders the cut's Gaussians interpolated
    with their parents; ``lut_m`` > 0 blends with the Eq. 5 lookup table of
    that many intervals; ``tile`` is the side of a tile in pixels (binning,
    pair lists and ``tile_mask`` are per tile of that size).
    """
    if int(lut_m) < 0:
        raise ValueError("lut_m must be >= 0")
    if int(tile) < 1:
        raise ValueError("tile must be >= 1")
    lib = _load()
    ref = _SceneRef(sc)
    c = _camera(cam)
    W, H = c.width, c.height
    TW, TH = (W + tile - 1) // tile, (H + tile - 1) // tile
    mask = None
    if tile_mask is not None:
        mask = np.ascontiguousarray(np.asarray(tile_mask, bool).reshape(TW * TH).astype(np.uint8))
    fp = lib.orc_render(ctypes.byref(ref.s), ctypes.byref(c), float(np.float32(tau)),
                        _ptr(mask) if mask is not None else None, float(band), float(t_flag),
                        int(bool(exhaustive)), float(-1.0 if frustum_guard is None else frustum_guard),
                        int(bool(interp)), int(lut_m), int(tile))
    if not fp:
        raise MemoryError("oracle render")
    try:
        F = fp.contents
        nc = int(F.n_cut)
        out = dict(cut=_arr(F.cut, np.uint32, nc), proj=_arr(F.proj, PROJ_DTYPE, nc),
                   image=_arr(F.image, np.float64, W * H * 3).reshape(H, W, 3),
                   flags=_arr(F.flags, np.uint8, W * H).reshape(H, W),
                   n_eval=_arr(F.n_eval, np.uint32, W * H).reshape(H, W),
                   n_contrib=_arr(F.n_contrib, np.uint32, W * H).reshape(H, W),
                   n_eval_total=int(F.n_eval_total), n_tiles=int(F.n_tiles), tiles=(TW, TH), tile=int(tile))
        if not exhaustive:
            ncand, np_ = int(F.n_cand), int(F.n_pairs)
            out.update(cand_tile=_arr(F.cand_tile, np.uint32, ncand),
                       cand_idx=_arr(F.cand_idx, np.uint32, ncand),
                       cand_margin=_arr(F.cand_margin, np.float64, ncand),
                       pair_tile=_arr(F.pair_tile, np.uint32, np_),
                       pair_idx=_arr(F.pair_idx, np.uint32, np_),
                       tile_start=_arr(F.tile_start, np.int64, int(F.n_tiles) + 1),
                       n_visible=int(F.n_visible), n_pairs=np_, n_cand=ncand)
        return out
    finally:
        lib.orc_frame_free(fp)

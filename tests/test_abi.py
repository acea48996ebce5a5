"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/vgr.h declares, and rejects malformed hierarchies and
arguments before touching the GPU."""
import ctypes

import numpy as np
import pytest

import scenegen
from paper_2506_02774_gb300 import _abi


@pytest.fixture(scope="module")
def lib():
    return _abi.load()


def test_exports_every_declared_function(lib):
    names = _abi.header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_default_opts(lib):
    o = _abi.ViewOpts()
    lib.vgr_default_view_opts(ctypes.byref(o))
    assert o.filter == _abi.FILTER_PREEMPTIVE and o.temporal == 1 and o.lut_size == 32 and o.lod_budget == 4096


def _desc(sc, **over):
    keep = {k: np.ascontiguousarray(sc[k]) for k in
            ("parent", "first_child", "n_child", "mean", "cov6", "opacity", "sh", "radius2")}
    keep.update(over)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    d = _abi.SceneDesc(int(sc["n_nodes"]), int(sc["sh_degree"]), p(keep["parent"]), p(keep["first_child"]),
                       p(keep["n_child"]), p(keep["mean"]), p(keep["cov6"]), p(keep["opacity"]), p(keep["sh"]),
                       p(keep["radius2"]), 0)
    return d, keep


def _load_status(lib, sc, **over):
    d, keep = _desc(sc, **over)
    h = ctypes.c_void_p()
    st = lib.vgr_load_hierarchy(ctypes.byref(d), ctypes.byref(h))
    return st, lib.vgr_last_error().decode()


def test_rejects_malformed_trees(lib, tiny_scene):
    sc = tiny_scene
    par = sc["parent"].copy()
    par[5] = 3  # wrong parent link
    assert _load_status(lib, sc, parent=par)[0] == _abi.VGR_E_INVALID
    fc = sc["first_child"].copy()
    fc[0] += 1  # children not the next BFS block
    assert _load_status(lib, sc, first_child=fc)[0] == _abi.VGR_E_INVALID
    r2 = sc["radius2"].copy()
    r2[0] = r2[1] * 0.5  # root radius no longer contains its child
    st, msg = _load_status(lib, sc, radius2=r2)
    assert st == _abi.VGR_E_INVALID and "nesting" in msg
    op = sc["opacity"].copy()
    op[7] = 1.5
    assert _load_status(lib, sc, opacity=op)[0] == _abi.VGR_E_INVALID
    m = sc["mean"].copy()
    m[9, 1] = np.nan
    assert _load_status(lib, sc, mean=m)[0] == _abi.VGR_E_INVALID
    nch = sc["n_child"].copy()
    nch[0] = 9
    assert _load_status(lib, sc, n_child=nch)[0] == _abi.VGR_E_INVALID


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.vgr_load_hierarchy(None, ctypes.byref(h)) == _abi.VGR_E_INVALID
    assert lib.vgr_free_hierarchy(None) == _abi.VGR_E_INVALID
    assert lib.vgr_destroy_view(None) == _abi.VGR_E_INVALID
    assert lib.vgr_render_frame(None, None, 3.0, None) == _abi.VGR_E_INVALID

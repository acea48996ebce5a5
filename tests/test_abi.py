"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/vgr.h declares, and rejects malformed hierarchies and
arguments before touching the GPU."""
import ctypes
import os

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
    assert o.lod_frustum == 0 and o.lod_frustum_guard == 2.0


def _desc(sc, **over):
    keep = {k: np.ascontiguousarray(sc[k]) for k in
            ("parent", "first_child", "n_child", "mean", "cov6", "opacity", "sh", "radius2")}
    keep.update(over)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    box = keep.get("bbox")
    d = _abi.SceneDesc(int(sc["n_nodes"]), int(sc["sh_degree"]), p(keep["parent"]), p(keep["first_child"]),
                       p(keep["n_child"]), p(keep["mean"]), p(keep["cov6"]), p(keep["opacity"]), p(keep["sh"]),
                       p(keep["radius2"]), 0, p(box) if box is not None else None)
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
    box = sc["bbox"].copy()
    c = int(sc["first_child"][0])
    box[c, 3] = box[0, 3] + 1.0  # a child's box pokes out of the root's
    st, msg = _load_status(lib, sc, bbox=box)
    assert st == _abi.VGR_E_INVALID and "box" in msg and "nesting" in msg
    box = sc["bbox"].copy()
    box[c, 0], box[c, 3] = box[c, 3], box[c, 0]  # lo > hi
    st, msg = _load_status(lib, sc, bbox=box)
    assert st == _abi.VGR_E_INVALID and "box" in msg


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.vgr_load_hierarchy(None, ctypes.byref(h)) == _abi.VGR_E_INVALID
    assert lib.vgr_free_hierarchy(None) == _abi.VGR_E_INVALID
    assert lib.vgr_destroy_view(None) == _abi.VGR_E_INVALID
    assert lib.vgr_render_frame(None, None, 3.0, None) == _abi.VGR_E_INVALID


def test_ctypes_layout_matches_header(tmp_path):
    """Every ctypes mirror has the size and field offsets the C compiler
    gives the structs of include/vgr.h."""
    import subprocess
    from paper_2506_02774_gb300 import _build
    structs = {"vgr_scene_desc": _abi.SceneDesc, "vgr_camera": _abi.Camera, "vgr_view_opts": _abi.ViewOpts,
               "vgr_frame_stats": _abi.FrameStats, "vgr_frame": _abi.Frame, "vgr_debug_buffers": _abi.DebugBuffers,
               "vgr_serve_opts": _abi.ServeOpts, "vgr_request": _abi.Request, "vgr_request_result": _abi.RequestResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vgr.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", _build.INCLUDE, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert int(got["%s.%s" % (cname, f[0])]) == getattr(py, f[0]).offset, (cname, f[0])


def test_async_and_server_argument_errors(lib):
    assert lib.vgr_submit_frame(None, None, 3.0, None) == _abi.VGR_E_INVALID
    d = ctypes.c_int32()
    assert lib.vgr_frame_done(None, ctypes.byref(d)) == _abi.VGR_E_INVALID
    assert lib.vgr_finish_frame(None, None) == _abi.VGR_E_INVALID
    assert lib.vgr_render_batch(None, None, None, None, 0, None) == _abi.VGR_OK  # nothing to do
    assert lib.vgr_render_batch(None, None, None, None, 2, None) == _abi.VGR_E_INVALID
    o = _abi.ServeOpts()
    lib.vgr_default_serve_opts(ctypes.byref(o))
    assert o.n_clients == 1 and o.view.use_graph == 1 and o.view.temporal == 1
    s = ctypes.c_void_p()
    assert lib.vgr_create_server(None, ctypes.byref(o), ctypes.byref(s)) == _abi.VGR_E_INVALID
    assert lib.vgr_destroy_server(None) == _abi.VGR_E_INVALID
    assert lib.vgr_serve_trace(None, None, 0, None) == _abi.VGR_E_INVALID


def test_renderer_fails_loudly_without_a_gpu(tiny_scene):
    """No CPU fallback: on a machine without a CUDA device the library
    validates the scene, then reports the missing device as an error."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2506_02774_gb300 as vgr
    with pytest.raises(vgr.VgrError):
        vgr.Renderer(tiny_scene)


def test_binding_argument_checks_survive_optimised_python(tiny_scene):
    """The binding's own checks raise real exceptions (not asserts, which
    python -O removes) before anything reaches the library."""
    import paper_2506_02774_gb300 as vgr
    bad = dict(tiny_scene)
    bad["parent"] = tiny_scene["parent"].astype(np.int64)
    with pytest.raises(TypeError, match="uint32"):
        vgr.Hierarchy(bad)
    bad = dict(tiny_scene)
    bad["opacity"] = tiny_scene["opacity"].astype(np.float64)
    with pytest.raises(TypeError, match="opacity"):
        vgr.Hierarchy(bad)
    bad = dict(tiny_scene)
    bad["bbox"] = tiny_scene["bbox"][:-1]
    with pytest.raises(ValueError, match="bbox"):
        vgr.Hierarchy(bad)
    cam = scenegen.trajectory("tiny", 0)
    with pytest.raises(ValueError, match="same length"):
        vgr.render_batch([object()], [cam, cam], [3.0])
    with pytest.raises(TypeError, match="float32"):
        vgr._host_image_ok(np.zeros((128, 128, 3)), cam, "out")
    with pytest.raises(ValueError, match="shape"):
        vgr._host_image_ok(np.zeros((64, 128, 3), np.float32), cam, "out")
    vgr._host_image_ok(np.zeros((128, 128, 3), np.float32), cam, "out")


def test_ctypes_prototypes_match_header_arity():
    """Every function the binding declares to ctypes has the header's number
    of parameters and a matching return kind (status, void or string)."""
    import re
    from paper_2506_02774_gb300 import _build
    src = open(os.path.join(_build.INCLUDE, "vgr.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    protos = {}
    for ret, name, params in re.findall(r"(vgr_status|void|const char\s*\*)\s*(vgr_\w+)\s*\(([^)]*)\)\s*;", src):
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        protos[name] = (ret.replace(" ", ""), n)
    assert len(protos) >= 20
    for name, (res, args) in _abi._PROTOS.items():
        assert name in protos, name
        ret, n = protos[name]
        assert len(args) == n, (name, len(args), n)
        want = {"vgr_status": ctypes.c_int32, "void": None, "constchar*": ctypes.c_char_p}[ret]
        assert res is want, (name, res, ret)

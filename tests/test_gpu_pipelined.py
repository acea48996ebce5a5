"""Pipelined host images (``vgr_render_frame_pipelined``): each frame's image
is copied into host memory on the view's copy stream while the next frame
runs, into the view's other device image.  Every copied image equals the same
frame rendered synchronously (and the last one the oracle's), with pinned and
pageable host buffers, graph replay, an overflow replay, a resize between
frames and plain frames mixed in."""
import numpy as np
import pytest

import oracle
import scenegen
from parity import check_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402


def _walk(n, W=328, H=250):
    return [scenegen.camera((2.0 + 0.05 * k, 15.0, 3.0), 0.2 + 0.01 * k, W, H, 260.0) for k in range(n)]


def _reference(h, cams, tau=3.0):
    v = vgr.View(h)
    imgs = [v.render(c, tau).image().cpu().numpy().copy() for c in cams]
    v.close()
    return imgs


def _host(cam, pinned):
    shape = (cam["height"], cam["width"], 3)
    if pinned:
        return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()
    return np.empty(shape, np.float32)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("kw", [dict(), dict(use_graph=True), dict(pair_capacity=64, use_graph=True)])
def test_pipelined_walk_equals_synchronous(small_sh3_scene, pinned, kw):
    h = vgr.Hierarchy(small_sh3_scene)
    cams = _walk(6)
    ref = _reference(h, cams)
    v = vgr.View(h, **kw)
    outs = [_host(c, pinned) for c in cams]
    for c, o in zip(cams, outs):
        o.fill(-1.0)
        r = v.render_pipelined(c, 3.0, o)
        assert r.cut_count > 0
    dev_last = r.image().cpu().numpy()
    v.wait_host_images()
    for k, (o, e) in enumerate(zip(outs, ref)):
        assert np.array_equal(o, e), "frame %d" % k
    assert np.array_equal(dev_last, ref[-1])
    check_image(outs[-1], oracle.render(small_sh3_scene, cams[-1], 3.0))
    v.close()
    h.close()


def test_pipelined_mixed_with_plain_and_resize(small_sh3_scene):
    """Plain frames between pipelined ones, and an image size that grows (the
    device images are reallocated while a copy may still read the old ones)."""
    h = vgr.Hierarchy(small_sh3_scene)
    cams = _walk(3) + _walk(3, 200, 120)[:1] + _walk(3, 480, 300)
    ref = _reference(h, cams)
    v = vgr.View(h, use_graph=True)
    outs = [_host(c, True) for c in cams]
    plain = {2, 4}
    for k, (c, o) in enumerate(zip(cams, outs)):
        if k in plain:
            r = v.render_host(c, 3.0, o)
            assert np.array_equal(o, ref[k]), "plain frame %d" % k  # lands before the call returns
        else:
            v.render_pipelined(c, 3.0, o)
    v.wait_host_images()
    for k, (o, e) in enumerate(zip(outs, ref)):
        assert np.array_equal(o, e), "frame %d" % k
    v.wait_host_images()  # nothing pending: returns at once
    v.close()
    h.close()


def test_pipelined_bad_arguments(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    v = vgr.View(h)
    cam = _walk(1)[0]
    fr = vgr._abi.Frame()
    assert v.render_pipelined_ptr(vgr.camera_struct(cam), 3.0, 0, fr) == vgr._abi.VGR_E_INVALID
    with pytest.raises(ValueError):
        v.render_pipelined(cam, 3.0, np.empty((10, 10, 3), np.float32))
    o = _host(cam, True)
    v.render_pipelined(cam, 3.0, o)  # the view still works
    v.wait_host_images()
    assert np.array_equal(o, _reference(h, [cam])[0])
    v.close()
    h.close()

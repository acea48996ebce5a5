"""GPU parity of parent-child weight interpolation (Sec. 3.1 'Weight
Interpolation') against the FP64 oracle: the cut unchanged and bit-exact, the
interpolated means' FP32 depth keys bit-exact, records, pairs and images
within the parity bar; FP32 and the FP16/BF16 store; SH degree 0 and 3."""
import numpy as np
import pytest

import oracle
import scenegen
from parity import check_image, check_stages, image_report, quantize_scene

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402


# the interpolated opacity is computed in FP32 (a few roundings of expm1,
# log1p and one fma) against the oracle's FP64
THETA_RTOL = 2e-6


def _cut(res):
    return res.cut().cpu().numpy().view(np.uint32).copy()


def _img(res):
    return res.image().cpu().numpy().copy()


def test_tiny_walk_every_frame(tiny_scene):
    h = vgr.Hierarchy(tiny_scene)
    v = vgr.View(h, lod_interp=True)
    vs = vgr.View(h, lod_interp=True, temporal=False)
    vp = vgr.View(h)
    tau = scenegen.CONFIGS["tiny"]["tau"]
    moved = 0
    for fr in range(scenegen.CONFIGS["tiny"]["frames"]):
        cam = scenegen.trajectory("tiny", fr)
        res = v.render(cam, tau)
        ref = oracle.render(tiny_scene, cam, tau, interp=True)
        np.testing.assert_array_equal(_cut(res), ref["cut"])
        check_image(_img(res), ref)
        check_stages(v.debug(), ref, theta_rtol=THETA_RTOL)
        rs = vs.render(cam, tau)
        assert np.array_equal(_img(rs), _img(res))
        rp = vp.render(cam, tau)
        np.testing.assert_array_equal(_cut(rp), _cut(res))  # the cut does not change
        moved += float(np.abs(_img(rp) - _img(res)).max()) > 1e-3
    assert moved > 0
    for x in (v, vs, vp):
        x.close()
    h.close()


def test_sh3_ragged_tiles(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    v = vgr.View(h, lod_interp=True)
    for fr in range(4):
        cam = scenegen.camera((2.0 + 0.05 * fr, 15.0, 3.0), 0.2 + 0.02 * fr, 328, 250, 260.0)
        res = v.render(cam, 3.0)
        ref = oracle.render(small_sh3_scene, cam, 3.0, interp=True)
        np.testing.assert_array_equal(_cut(res), ref["cut"])
        r = check_image(_img(res), ref)
        s = check_stages(v.debug(), ref, theta_rtol=THETA_RTOL)
        print("interp frame", fr, r, s)
    v.close()
    h.close()


def test_half_storage(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene, storage=vgr.STORE_HALF)
    v = vgr.View(h, lod_interp=True)
    cam = scenegen.camera((2.0, 15.0, 3.0), 0.2, 328, 250, 260.0)
    r = v.render(cam, 3.0)
    refq = oracle.render(quantize_scene(small_sh3_scene), cam, 3.0, interp=True)
    np.testing.assert_array_equal(_cut(r), refq["cut"])
    check_image(_img(r), refq)
    print("interp, half store vs FP32-scene oracle:",
          image_report(_img(r), oracle.render(small_sh3_scene, cam, 3.0, interp=True)))
    v.close()
    h.close()


def test_collapse_is_smooth_on_the_gpu():
    """A root and two coincident children: across the distance where the
    root collapses, the interpolated centre pixel does not jump."""
    n = 3
    sc = dict(parent=np.array([0xFFFFFFFF, 0, 0], np.uint32), first_child=np.array([1, 0, 0], np.uint32),
              n_child=np.array([2, 0, 0], np.uint8), mean=np.zeros((n, 3), np.float32),
              cov6=np.tile(np.array([0.01, 0, 0, 0.01, 0, 0.01], np.float32), (n, 1)),
              opacity=np.full(n, 0.6, np.float32), sh=np.tile(np.array([[[0.6, 0.2, -0.1]]], np.float32), (n, 1, 1)),
              radius2=np.array([0.36, 0.09, 0.09], np.float32), sh_degree=0, n_nodes=n)
    h = vgr.Hierarchy(sc)
    vi, vp = vgr.View(h, lod_interp=True), vgr.View(h)
    tau, f = 30.0, 120.0
    t = float(np.float32(np.float32(tau) / np.float32(f)))
    px = {}
    for side, s in (("inside", 1 - 1e-5), ("outside", 1 + 1e-5)):
        cam = dict(R=np.eye(3, dtype=np.float32), pos=np.array([0, 0, -0.6 / t * s], np.float32), fx=f, fy=f,
                   cx=32.5, cy=32.5, width=64, height=64, z_near=0.2)
        ri, rp = vi.render(cam, tau), vp.render(cam, tau)
        assert _cut(ri).tolist() == ([1, 2] if side == "inside" else [0])
        px[side] = _img(ri)[32, 32]
        px["plain_" + side] = _img(rp)[32, 32]
    np.testing.assert_allclose(px["inside"], px["outside"], rtol=1e-3, atol=1e-5)
    assert np.abs(px["plain_inside"] - px["plain_outside"]).max() > 0.05
    vi.close()
    vp.close()
    h.close()

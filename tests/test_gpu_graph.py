"""Frames replayed as captured CUDA graphs (``use_graph``) against the plain
launch sequence: the same kernels on the same buffers, so cut, image and
counters must be bit-identical, through temporal updates, top-down
fallbacks, buffer growth (which drops and re-captures the graphs) and a
change of image size.  The first frames are also checked against the oracle.
"""
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

COUNTS = ("cut_count", "front_count", "visible_count", "pair_count", "candidate_pairs", "nodes_evaluated",
          "lod_from_scratch", "pixel_pair_evals", "pixel_pair_contribs", "kernels")


def _same(a, b):
    np.testing.assert_array_equal(a.cut().cpu().numpy(), b.cut().cpu().numpy())
    assert np.array_equal(a.image().cpu().numpy(), b.image().cpu().numpy())
    for k in COUNTS:
        assert a.stats[k] == b.stats[k], k


def test_graph_equals_plain_walk(tiny_scene):
    h = vgr.Hierarchy(tiny_scene)
    vg = vgr.View(h, use_graph=True)
    vp = vgr.View(h)
    tau = scenegen.CONFIGS["tiny"]["tau"]
    for fr in range(scenegen.CONFIGS["tiny"]["frames"]):
        cam = scenegen.trajectory("tiny", fr)
        a, b = vg.render(cam, tau), vp.render(cam, tau)
        _same(a, b)
        if fr < 3:
            ref = oracle.render(tiny_scene, cam, tau)
            np.testing.assert_array_equal(a.cut().cpu().numpy().view(np.uint32), ref["cut"])
            check_image(a.image().cpu().numpy(), ref)
    vg.close(); vp.close(); h.close()


def test_graph_growth_fallback_and_resize(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    kw = dict(cut_capacity=64, pair_capacity=16, lod_budget=2)
    vg = vgr.View(h, use_graph=True, **kw)
    vp = vgr.View(h, **kw)
    cams = [scenegen.camera((2.0, 15.0, 3.0), 0.2, 328, 250, 260.0),
            scenegen.camera((2.1, 15.0, 3.0), 0.22, 328, 250, 260.0),
            scenegen.camera((30.0, 5.0, 8.0), 2.0, 328, 250, 260.0),     # teleport: budget fallback
            scenegen.camera((30.1, 5.0, 8.0), 2.0, 200, 120, 160.0),     # new size and focal length
            scenegen.camera((30.2, 5.0, 8.0), 2.02, 200, 120, 160.0)]
    for i, cam in enumerate(cams):
        a, b = vg.render(cam, 3.0), vp.render(cam, 3.0)
        _same(a, b)
        assert a.stats["replays"] == b.stats["replays"]
        if i in (0, 3):
            ref = oracle.render(small_sh3_scene, cam, 3.0)
            np.testing.assert_array_equal(a.cut().cpu().numpy().view(np.uint32), ref["cut"])
            check_image(a.image().cpu().numpy(), ref)
    vg.close(); vp.close(); h.close()


def test_renderer_equals_hierarchy_and_view(tiny_scene):
    tau = scenegen.CONFIGS["tiny"]["tau"]
    h = vgr.Hierarchy(tiny_scene)
    v = vgr.View(h, use_graph=True)
    with vgr.Renderer(tiny_scene, use_graph=True) as r:
        for fr in range(4):
            cam = scenegen.trajectory("tiny", fr)
            _same(r.render(cam, tau), v.render(cam, tau))
    v.close()
    h.close()

"""Parity at the bench's full sizes and launch configuration (default view
options): the 1M-leaf box scene and the 18M-leaf city, both at 1920x1080.

The cut is compared with the oracle's top-down cut in full, bit for bit.
Images and pair lists are compared on sampled tiles (corners, the ragged
last tile row, the heaviest tiles and random ones), which the oracle bins
and blends alone; projected records, depth keys and the depth order are
compared for every visible Gaussian.  Over a longer stretch of the walk the
temporal cut is compared with a from-scratch cut at every frame.
"""
import numpy as np
import pytest

import oracle
import scenegen
from parity import check_image, check_stages

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402


def _tile_mask(dbg, seed, n_random=48, n_heavy=8):
    TW, TH = dbg["tiles"]
    T = TW * TH
    m = np.zeros(T, bool)
    m[[0, TW - 1, T - TW, T - 1]] = True          # corners
    m[(TH - 1) * TW + np.arange(0, TW, 7)] = True  # ragged last row (1080 = 67.5 tiles)
    cnt = dbg["tile_range"][:, 1].astype(np.int64) - dbg["tile_range"][:, 0]
    m[np.argsort(cnt)[-n_heavy:]] = True           # the heaviest tiles
    m[np.random.default_rng(seed).choice(T, n_random, replace=False)] = True
    return m.reshape(TH, TW)


def _frame_check(sc, view, cam, tau, seed):
    res = view.render(cam, tau)
    dbg = view.debug()
    mask = _tile_mask(dbg, seed)
    ref = oracle.render(sc, cam, tau, tile_mask=mask)
    np.testing.assert_array_equal(res.cut().cpu().numpy().view(np.uint32), ref["cut"])
    img = res.image().cpu().numpy()
    r = check_image(img, ref, tile_mask=mask)
    s = check_stages(dbg, ref, tile_mask=mask)
    return res, r, s


@pytest.fixture(scope="module")
def m1_scene():
    return scenegen.make_scene("m1")


def test_m1_1080p_sampled_tiles(m1_scene):
    h = vgr.Hierarchy(m1_scene)
    v = vgr.View(h)
    tau = scenegen.CONFIGS["m1"]["tau"]
    for fr in (0, 1, 2, 45):
        if fr == 45:
            for k in range(3, 45):  # advance the temporal state along the walk
                v.render(scenegen.trajectory("m1", k), tau)
        res, r, s = _frame_check(m1_scene, v, scenegen.trajectory("m1", fr), tau, fr)
        assert res.stats["lod_from_scratch"] == (1 if fr == 0 else 0)
        print("m1 frame", fr, res.stats["cut_count"], res.stats["pair_count"], r, s)
    v.close()
    h.close()


def test_m1_temporal_equals_scratch_60_frames(m1_scene):
    h = vgr.Hierarchy(m1_scene)
    vt, vs = vgr.View(h), vgr.View(h, temporal=False)
    tau = scenegen.CONFIGS["m1"]["tau"]
    for fr in range(60):
        cam = scenegen.trajectory("m1", fr)
        a = vt.render(cam, tau)
        ca = a.cut().cpu().numpy().view(np.uint32).copy()
        ia = a.image().cpu().numpy().copy()
        b = vs.render(cam, tau)
        np.testing.assert_array_equal(ca, b.cut().cpu().numpy().view(np.uint32))
        assert np.array_equal(ia, b.image().cpu().numpy())
        if fr % 20 == 19:
            k = oracle.lod_k(tau, float(cam["fx"]))
            np.testing.assert_array_equal(ca, oracle.cut(m1_scene, cam["pos"], k))
    vt.close()
    vs.close()
    h.close()


def test_city_1080p_sampled_tiles():
    sc = scenegen.make_scene("city")
    h = vgr.Hierarchy(sc)
    v = vgr.View(h)
    tau = scenegen.CONFIGS["city"]["tau"]
    for fr in (0, 1, 20):
        if fr == 20:
            for k in range(2, 20):
                v.render(scenegen.trajectory("city", k), tau)
        res, r, s = _frame_check(sc, v, scenegen.trajectory("city", fr), tau, 100 + fr)
        print("city frame", fr, res.stats["cut_count"], res.stats["visible_count"], res.stats["pair_count"], r, s)
    v.close()
    h.close()


def test_city_half_storage_sampled_tiles():
    """FP16 SH + BF16 covariance store on the full city: the cut is the FP32
    one (centres and radii stay FP32); sampled tiles within the image bar of
    the oracle run on the quantized scene; the error against the FP32 scene
    is reported."""
    from parity import image_report, quantize_scene
    sc = scenegen.make_scene("city")
    h = vgr.Hierarchy(sc, storage=vgr.STORE_HALF)
    v = vgr.View(h)
    tau = scenegen.CONFIGS["city"]["tau"]
    q = quantize_scene(sc)
    for fr in (0, 1):
        cam = scenegen.trajectory("city", fr)
        res = v.render(cam, tau)
        mask = _tile_mask(v.debug(), 200 + fr)
        refq = oracle.render(q, cam, tau, tile_mask=mask)
        np.testing.assert_array_equal(res.cut().cpu().numpy().view(np.uint32), refq["cut"])
        img = res.image().cpu().numpy()
        r = check_image(img, refq, tile_mask=mask)
        ref = oracle.render(sc, cam, tau, tile_mask=mask)
        print("city half store frame", fr, "vs quantized-scene oracle", r, "vs FP32-scene oracle",
              image_report(img, ref, mask))
    v.close()
    h.close()

"""The autotuner: results do not depend on the launch geometry or the blend's
staging depth it picks, its choice is cached per (device, hierarchy, image
size) in JSON and reused, and a batch's blend depth is tuned on the batch."""
import json

import numpy as np
import pytest

import scenegen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402
from paper_2506_02774_gb300 import autotune  # noqa: E402


def test_geometry_does_not_change_results(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    cams = [scenegen.camera((2.0 + 0.05 * k, 15.0, 3.0), 0.2 + 0.01 * k, 328, 250, 260.0) for k in range(3)]
    views = [vgr.View(h), vgr.View(h, grid_wide=1, grid_scan=1), vgr.View(h, grid_wide=7, grid_scan=5, use_graph=True),
             vgr.View(h, blend_depth=16), vgr.View(h, blend_depth=48, use_graph=True)]
    for cam in cams:
        res = [v.render(cam, 3.0) for v in views]
        for r in res[1:]:
            np.testing.assert_array_equal(r.cut().cpu().numpy(), res[0].cut().cpu().numpy())
            assert np.array_equal(r.image().cpu().numpy(), res[0].image().cpu().numpy())
            assert r.stats["pair_count"] == res[0].stats["pair_count"]
    for v in views:
        v.close()
    h.close()


def test_tune_and_cache(small_sh3_scene, tmp_path):
    h = vgr.Hierarchy(small_sh3_scene)
    cams = [scenegen.camera((2.0 + 0.05 * k, 15.0, 3.0), 0.2, 200, 120, 160.0) for k in range(6)]
    path = str(tmp_path / "tune.json")
    e = autotune.tune(h, cams, 3.0, cache_path=path, wide=(2, 8), scan=(2, 4))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert e["grid_wide"] in (2 * sms, 8 * sms) and e["grid_scan"] in (2 * sms, 4 * sms)
    assert e["blend_depth"] in (16, 32, 48) and e["tile_size"] in (8, 16, 32)
    assert len(e["candidates"]) == 4 + 7 and e["ms"] == min(c["ms"] for c in e["candidates"])
    cache = json.load(open(path))
    assert autotune.cache_key(h, 200, 120) in cache
    assert autotune.tune(h, cams, 3.0, cache_path=path) == cache[autotune.cache_key(h, 200, 120)]  # reused
    h.close()


def test_set_tuning_between_frames_keeps_results(small_sh3_scene):
    """Changing the geometry and staging depth of a view between frames (its
    captured frames are dropped) leaves the cut and image of every frame as a
    fresh view renders them; a bad depth is refused."""
    h = vgr.Hierarchy(small_sh3_scene)
    v, ref = vgr.View(h, use_graph=True), vgr.View(h)
    cams = [scenegen.camera((2.0 + 0.05 * k, 15.0, 3.0), 0.2 + 0.01 * k, 328, 250, 260.0) for k in range(4)]
    for k, cam in enumerate(cams):
        v.set_tuning(grid_wide=(k + 1) * 100, grid_scan=0, blend_depth=(16, 32, 48, 32)[k],
                     tile_size=(16, 8, 32, 16)[k])
        a, b = v.render(cam, 3.0), ref.render(cam, 3.0)
        np.testing.assert_array_equal(a.cut().cpu().numpy(), b.cut().cpu().numpy())
        assert np.array_equal(a.image().cpu().numpy(), b.image().cpu().numpy())
        assert a.stats["lod_from_scratch"] == (1 if k == 0 else 0)  # the temporal state survives
    with pytest.raises(vgr.VgrError):
        v.set_tuning(blend_depth=24)
    with pytest.raises(vgr.VgrError):
        v.set_tuning(tile_size=8, blend_depth=48)
    v.close()
    ref.close()
    h.close()


def test_tune_batch(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    views = [vgr.View(h, use_graph=True) for _ in range(3)]
    sizes = [(200, 120), (328, 250), (64, 48)]
    steps = [[scenegen.camera((2.0 + 0.05 * k + i, 15.0, 3.0), 0.2, W, H, 160.0) for i, (W, H) in enumerate(sizes)]
             for k in range(4)]
    r = autotune.tune_batch(views, steps, [3.0] * 3)
    assert r["blend_depth"] in (16, 32, 48) and r["tile_size"] in (8, 16, 32)
    assert len(r["candidates"]) == 3 + 7  # chains 0 (= 3), 1, 2; then the other (tile, depth) pairs
    assert r["chains"] in (0, 1, 2) and r["ms_per_batch"] == min(c["ms_per_batch"] for c in r["candidates"])
    res = vgr.render_batch(views, steps[-1], [3.0] * 3)
    for i, v in enumerate(views):
        alone = vgr.View(h)
        solo = alone.render(steps[-1][i], 3.0)
        assert np.array_equal(res[i].image().cpu().numpy(), solo.image().cpu().numpy())
        alone.close()
        v.close()
    h.close()

"""The launch-geometry autotuner: results do not depend on the geometry it
picks, its choice is cached per (device, hierarchy, image size) in JSON and
reused."""
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
    views = [vgr.View(h), vgr.View(h, grid_wide=1, grid_scan=1), vgr.View(h, grid_wide=7, grid_scan=5, use_graph=True)]
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
    assert len(e["candidates"]) == 4 and e["ms"] == min(c["ms"] for c in e["candidates"])
    cache = json.load(open(path))
    assert autotune.cache_key(h, 200, 120) in cache
    assert autotune.tune(h, cams, 3.0, cache_path=path) == cache[autotune.cache_key(h, 200, 120)]  # reused
    h.close()

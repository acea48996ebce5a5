"""Failure paths on the GPU without a fault: a bounded device wait that
runs out reports VGR_E_TIMEOUT and the device stays usable; an allocation
the device cannot satisfy reports VGR_E_NOMEM and nothing is left behind."""
import time

import numpy as np
import pytest

import oracle
import scenegen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2506_02774_gb300 as vgr  # noqa: E402
from paper_2506_02774_gb300 import _abi  # noqa: E402


def test_lookback_wait_runs_out(small_sh3_scene):
    h = vgr.Hierarchy(small_sh3_scene)
    cam = scenegen.camera((2.0, 15.0, 3.0), 0.2, 328, 250, 260.0)  # thousands of visible Gaussians
    bad = vgr.View(h, test_hooks=1)  # VGR_HOOK_WITHHOLD_LOOKBACK
    t = time.time()
    with pytest.raises(vgr.VgrError) as e:
        bad.render(cam, 3.0)
    assert e.value.status == _abi.VGR_E_TIMEOUT
    assert time.time() - t < 60.0  # the waits are bounded
    bad.close()
    # the device and the hierarchy are still usable, and the result is right
    v = vgr.View(h)
    r = v.render(cam, 3.0)
    assert r.stats["visible_count"] > 2048  # several emission tiles waited on the silent one
    ref = oracle.render(small_sh3_scene, cam, 3.0)
    np.testing.assert_array_equal(r.cut().cpu().numpy().view(np.uint32), ref["cut"])
    v.close()
    h.close()


def test_allocation_failure_is_reported(tiny_scene):
    h = vgr.Hierarchy(tiny_scene)
    with pytest.raises(vgr.VgrError) as e:
        vgr.View(h, pair_capacity=1 << 42)  # 64 TB of pair buffers
    assert e.value.status == _abi.VGR_E_NOMEM
    v = vgr.View(h)
    assert v.render(scenegen.trajectory("tiny", 1), 3.0).cut_count > 0
    v.close()
    h.close()

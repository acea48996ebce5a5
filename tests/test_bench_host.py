"""Host-side helpers of bench.py (CPU): the code hash that keys the committed
DRAM-traffic record, the rule that a record taken on other code is not
reported, the CPU baseline's two timings, the whole-frame roofline
arithmetic, the serving leg's request trace and the autotuner's cache."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_and_spacing(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n    return x + 1;  // one more\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("// a new header line\nint f(int  x) {\n\n        return x + 1;\n}  // end\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.code_sha256(str(a)) == bench.code_sha256(str(b))
    assert bench.code_sha256(str(a)) != bench.code_sha256(str(c))


def test_traffic_record_only_for_the_code_it_was_taken_on(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2506_02774_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "k_blend.cu"
    src.write_text("__global__ void k() {}\n")
    rec = {"k_blend": {"code_sha256": bench.code_sha256(str(src)), "dram_bytes_per_launch": 123456,
                       "units_per_launch": 1000}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("k_blend", "k_blend.cu", 1000.0) == 123456
    assert bench._traffic("k_blend", "k_blend.cu", 3000.0) == 3 * 123456  # scaled by the units of the launch
    src.write_text("// comment only\n__global__ void k() {}\n")
    assert bench._traffic("k_blend", "k_blend.cu", 1000.0) == 123456
    src.write_text("__global__ void k() { int x = 0; }\n")
    assert bench._traffic("k_blend", "k_blend.cu", 1.0) is None
    assert bench._traffic("k_emit", "k_emit.cu", 1.0) is None


def test_reference_arm_times_every_step_it_reports():
    """The reference arm's line reports the steps and warm-up frames it ran,
    all of them timed, on the GPU arm's config dict."""
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
           "--steps", "3", "--warmup", "4"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert d["steps"] == 3 and d["warmup"] == 4
    assert d["cpu_baseline"]["sample"].startswith("all 3 timed frames 4..6")
    assert abs(d["ms_per_step"] * d["value"] - 1000.0) < 1.0
    assert d["config"]["frames"] == "4..6 of the 16-frame walk" and d["config"]["workload"] == "box-4096-leaves-128px"
    assert set(d["config"]) == {"workload", "leaves", "nodes", "width", "height", "tau", "storage", "frames", "l2",
                                "parallelism"}



def test_cpu_baseline_reports_all_cores_and_one_thread(tiny_scene):
    import oracle
    import scenegen
    n = oracle.num_threads()
    cams = [scenegen.trajectory("tiny", f) for f in range(3)]
    r = bench.cpu_baseline(tiny_scene, cams, 3.0, budget_s=0.05)
    assert r["kind"] == "oracle" and r["unit"] == "frames/s" and r["cores"] == n and r["value"] > 0
    st = r["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and st["unit"] == "frames/s"
    assert oracle.num_threads() == n  # the thread count is restored
    assert "single_thread" not in bench.cpu_baseline(tiny_scene, cams, 3.0, budget_s=0.05, single_thread=False)


def test_frame_roofline_arithmetic():
    fb = {"lod": 2e8, "blend": 6e8, "emit": 2e8}
    ms = {"lod": 0.1, "blend": 0.3, "emit": 0.0}
    r = bench.frame_roofline(fb, ms, 1.0, 8000.0)
    assert r["algorithmic_bytes"] == 10 ** 9
    assert r["hbm_roofline_ms"] == 0.125            # 1 GB at 8 TB/s
    assert r["frac"] == 0.125                       # of a 1 ms frame
    assert r["stage_frac"] == {"lod": 0.25, "blend": 0.25}  # 2 GB/ms = 2 TB/s of 8; emit untimed


def test_serving_trace_is_the_poisson_recipe():
    """32 clients at 8 req/s each for 10 s: arrivals sorted inside the window,
    about 2560 requests in all (Poisson, 3 sigma), each client's requests
    walking consecutive frames of its own street at its own image size, and
    the same trace for the same seed."""
    import scenegen
    names = ["720p", "1080p", "1440p"]
    pick = [names[i % 3] for i in range(32)]
    tr = bench._serve_trace(32, 8.0, 10.0, 5, pick, 2)
    t = np.array([r["arrival_s"] for r in tr])
    assert np.all(np.diff(t) >= 0) and t[0] > 0 and t[-1] <= 10.0
    assert abs(len(tr) - 2560) <= 3 * np.sqrt(2560)
    for c in (0, 7, 31):
        mine = [r for r in tr if r["client"] == c]
        W, H = scenegen.RESOLUTIONS[pick[c]]
        assert all(r["cam"]["width"] == W and r["cam"]["height"] == H for r in mine)
        ref = [scenegen.street_trajectory("city", 300 + c, 2 + k, W, H)["pos"] for k in range(len(mine))]
        np.testing.assert_array_equal(np.array([r["cam"]["pos"] for r in mine]), np.array(ref))
    # gaps are exponential with mean 1/8 s (mean within 5 %)
    gaps = np.concatenate([np.diff([0.0] + [r["arrival_s"] for r in tr if r["client"] == c]) for c in range(32)])
    assert abs(gaps.mean() - 0.125) < 0.00625
    tr2 = bench._serve_trace(32, 8.0, 10.0, 5, pick, 2)
    assert [r["arrival_s"] for r in tr2] == list(t)


def test_autotune_cache_is_reused_and_sizes_must_agree(tmp_path, monkeypatch):
    """A cached launch geometry is returned without timing anything; a
    tuning walk of mixed image sizes is refused."""
    import pytest
    from paper_2506_02774_gb300 import autotune
    path = str(tmp_path / "geom.json")
    entry = {"grid_wide": 1216, "grid_scan": 608, "ms": 1.0, "default_ms": 1.1, "candidates": []}
    autotune.save_cache(path, {"dev|64x32": entry})
    assert autotune.load_cache(path) == {"dev|64x32": entry}
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
    monkeypatch.setattr(autotune, "cache_key", lambda h, W, H: "dev|%dx%d" % (W, H))
    timed = []
    monkeypatch.setattr(autotune, "_time_walk", lambda *a, **k: timed.append(k) or 1.0)
    cams = [dict(width=64, height=32)] * 3
    assert autotune.tune(None, cams, 3.0, cache_path=path) == entry
    assert not timed
    with pytest.raises(ValueError, match="same image size"):
        autotune.tune(None, [dict(width=64, height=32), dict(width=32, height=32)], 3.0, cache_path=path)

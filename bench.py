"""Frame-rate bench of the GB300 frame path (one JSON line on stdout).

Default workload: the 18M-leaf synthetic city (about 26.5M LoD nodes, SH
degree 3, FP32 storage) at 1920x1080, tau = 3 px, frames W .. W+K-1 of its
600-frame street walk.  A step is one frame: temporal LoD cut update, cut
compaction, preprocess, depth sort, pair emission, tile sort, ranges and
blend, plus the end-of-frame status read.

value    frames/s with the scene resident in HBM (device-clock time of the K
         frames, CUDA events on the view's stream, max over ranks)
e2e      the same through vgr_render_frame_host: camera from host memory and
         the 1080p image copied back to pinned host memory every frame
roofline the dominant kernel against MEASURED_PEAKS.json
cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload

--impl reference times the oracle alone (the reference arm of this project:
there is no released code of the paper).  Under torchrun each rank renders
its own view of its own scene replica (no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "1080p frames/s on 18M-Gaussian scene (LoD+raster ms); served p50/p99 ms"
WORKLOADS = {
    "city": dict(scene="city", label="city-18M-leaves-1080p"),
    "m1": dict(scene="m1", label="box-1M-leaves-1080p"),
    "tiny": dict(scene="tiny", label="box-4096-leaves-128px"),
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured", sm_max_mhz=float(d.get("sm_max_mhz", 2070)))
    return dict(hbm_gbs=6800.0, source="fallback", sm_max_mhz=2070.0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


OPS_PER_EVAL = 9      # 2 FADD (dx, dy), 4 FMUL + 2 FFMA (rho), 1 compare (Eq. 4)
OPS_PER_CONTRIB = 10  # FMUL (exp argument), FMUL (theta e^rho), min, 1 - alpha, T', compare, alpha T, 3 FFMA, + 1 MUFU


def code_sha256(path: str) -> str:
    """SHA-256 of a source file's code: // comments and blank space removed,
    so an edit of comments alone keeps the hash."""
    import hashlib
    import re
    lines = []
    for line in open(path).read().splitlines():
        code = re.sub(r"//.*$", "", line).strip()
        if code:
            lines.append(" ".join(code.split()))
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def _traffic(kernel: str, source: str, units: float):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json), used only while the kernel's code is the one the
    counters were taken on (code_sha256 of csrc/<source>); else None.  The
    counters come from a smaller case of the same workload (one kernel, a few
    launches); they are scaled to this launch by its units (the count named
    in the record: visible Gaussians or pairs)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2506_02774_gb300", "csrc", source)
    if not os.path.exists(p) or not os.path.exists(src):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("code_sha256") != code_sha256(src) or not d.get("units_per_launch"):
        return None
    per_unit = float(d["dram_bytes_per_launch"]) / float(d["units_per_launch"])
    return int(round(per_unit * units))


def rank_walk(cfg: dict, rank: int):
    """(heading, start) of rank's walk: rank 0 the workload's own walk, rank r
    the parallel street 40 r m over (replicas: every rank renders its own
    frames of its own scene copy)."""
    if rank == 0:
        return 0.0, None
    start = list(cfg["start"])
    start[1] += 40.0 * rank
    return 0.0, start


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The job's time: the maximum of x over the ranks (no-op for one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _frame_bytes(sc: dict, st: dict, W: int, H: int, tile_passes: int) -> dict:
    """Algorithmic bytes per frame and stage (FP32 store), from the counters."""
    C, V, P, E = st["cut_count"], st["visible_count"], st["pair_count"], st["nodes_evaluated"]
    N = int(sc["n_nodes"])
    K3 = 3 * (int(sc["sh_degree"]) + 1) ** 2
    shb = 4 * ((K3 + 3) // 4 * 4)
    P0 = st.get("candidate_pairs", P)
    F = st.get("front_count", V)
    return dict(
        lod=16 * E + 4 * C + 4 * C + 2 * N / 8,      # node and parent tests, lmax, prev cut read, two bitmaps set
        compact=2 * (N / 8 * 2) + 4 * C + 4 * F,     # two bitmaps read + cleared, cut and in-front ids written
        # ids, centre, covariance + opacity, records out; SH in and rgb out (visible)
        preprocess=(4 + 16 + 32 + 48) * F + (shb + 16) * V,
        depth_sort=4 * 2 * 8 * F + 4 * F,            # 4 passes x (key+value) read+write, histogram read
        color=0,                                     # evaluated in preprocess
        emit=(4 + 4 + 8 + 32) * V + 8 * P0,          # order, count, rect, record halves; slots
        tile_sort=tile_passes * 2 * 8 * P0,
        ranges=4 * P + 8 * (W // 16 + 1) * (H // 16 + 1),
        blend=(4 + 48) * P + 12 * W * H,
    )


def frame_roofline(fb: dict, stage_ms: dict, frame_ms: float, hbm_gbs: float) -> dict:
    """HBM roofline of the whole frame: the algorithmic bytes of every stage
    at the measured copy bandwidth, as a share of the measured frame time,
    and each stage's achieved bandwidth as a share of that peak."""
    total = float(sum(fb.values()))
    roof_ms = total / (hbm_gbs * 1e9) * 1e3
    per_stage = {k: round(fb[k] / (stage_ms[k] * 1e-3) / 1e9 / hbm_gbs, 4)
                 for k in fb if stage_ms.get(k, 0.0) > 0}
    return dict(algorithmic_bytes=int(total), hbm_roofline_ms=round(roof_ms, 4), frame_ms=round(frame_ms, 4),
                frac=round(roof_ms / frame_ms, 4), stage_frac=per_stage)


def blend_roofline(mean: dict, blend_ms: float, sms: int, peaks: dict, blend_bytes: float, blend_gbs: float) -> dict:
    """The blend (the kernel with the largest share of the frame) against its
    plain-ALU roofline: FP32 lane-instructions the method needs per evaluated
    pixel-pair (dx, dy, rho, Eq. 4 test) and per blended one (exp argument,
    alpha, T update, test, weight, 3 colour FMAs), against the device's SMs x
    128 FP32 lanes x the maximum SM clock."""
    X, K = mean["pixel_pair_evals"], mean["pixel_pair_contribs"]
    ops = OPS_PER_EVAL * X + OPS_PER_CONTRIB * K
    t = blend_ms * 1e-3
    peak_t = sms * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12
    units = mean["pair_count"]
    return dict(bound="alu", stage="blend", kernel="k_blend", achieved=round(ops / t / 1e12, 3),
                peak=round(peak_t, 2), unit="TFLOP/s", frac=round(ops / t / 1e12 / peak_t, 4),
                traffic=_traffic("k_blend", "k_blend.cu", units),
                peak_source="%d SMs x 128 FP32 lanes x %.0f MHz (sm_max_mhz, %s), one op per FP32 "
                            "lane-instruction" % (sms, peaks["sm_max_mhz"], peaks["source"]),
                ops_per_launch=int(ops), kernel_ms=round(blend_ms, 4), algorithmic_bytes=int(blend_bytes),
                hbm_frac=round(blend_gbs / peaks["hbm_gbs"], 4))


def hbm_roofline(stage: str, kernel: str, source: str, alg_bytes: float, ms: float, peaks: dict, units: float) -> dict:
    """An HBM-bound stage: algorithmic bytes per launch over its mean stage time
    against the measured copy bandwidth."""
    gbs = alg_bytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return dict(bound="hbm", stage=stage, kernel=kernel, achieved=round(gbs, 1), peak=peaks["hbm_gbs"], unit="GB/s",
                frac=round(gbs / peaks["hbm_gbs"], 4), traffic=_traffic(kernel, source, units),
                peak_source=peaks["source"] + " hbm_gbs (MEASURED_PEAKS.json)", algorithmic_bytes=int(alg_bytes),
                kernel_ms=round(ms, 4))


def workload_label(wl: dict, leaves: int) -> dict:
    """The workload with its label naming an overridden leaf count."""
    if not leaves:
        return wl
    return dict(wl, label="%s (%d leaves)" % (wl["label"].replace("18M-leaves-", ""), leaves))


def workload_config(wl: dict, sc: dict, cfg: dict, args, ws: int) -> dict:
    """The `config` of the JSON line; identical for both arms of a run."""
    nbytes = sum(int(np.asarray(sc[k]).nbytes) for k in
                 ("parent", "first_child", "n_child", "mean", "cov6", "opacity", "sh", "radius2", "bbox")
                 if sc.get(k) is not None)
    return dict(workload=wl["label"], leaves=int(sc["n_leaves"]), nodes=int(sc["n_nodes"]),
                width=cfg["width"], height=cfg["height"], tau=cfg["tau"], storage=args.storage,
                frames="%d..%d of the %d-frame walk" % (args.warmup, args.warmup + args.steps - 1, cfg["frames"]),
                l2="inputs larger than L2 (scene arrays %.1f GB)" % (nbytes / 1e9),
                parallelism="replicas" if ws > 1 else "single")


def run_ours(args) -> dict:
    import torch

    import scenegen
    import paper_2506_02774_gb300 as vgr

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    wl = WORKLOADS[args.config]
    cfg = scenegen.CONFIGS[wl["scene"]]
    t0 = time.time()
    sc = scenegen.make_scene(wl["scene"], n_leaves=args.leaves or None)
    wl = workload_label(wl, args.leaves)
    t_gen = time.time() - t0
    t0 = time.time()
    h = vgr.Hierarchy(sc, storage=vgr.STORE_HALF if args.storage == "half" else vgr.STORE_FP32)
    t_up = time.time() - t0
    stream = torch.cuda.Stream()
    view = vgr.View(h, stream=stream.cuda_stream, timing=False, use_graph=not args.no_graph)
    view_loop = vgr.View(h, stream=stream.cuda_stream, timing=False, use_graph=False)
    tau = cfg["tau"]
    nfr = cfg["frames"]
    W, H = cfg["width"], cfg["height"]
    # each rank walks its own street (replicas: no data-path collective)
    heading, start = rank_walk(cfg, rank)
    cams = [scenegen.trajectory(wl["scene"], f % nfr, heading, start) for f in range(args.warmup + args.steps)]
    structs = [vgr.camera_struct(c) for c in cams]

    def timed(v):
        """Warm-up frames (frame 0 finds its cut top-down, then temporal
        updates), then K timed frames on the view's stream, max over ranks."""
        v.reset()
        for i in range(args.warmup):
            v.render(cams[i], tau)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lat, stats, kernels = [], [], 0
        ev0.record(stream)
        for i in range(args.warmup, args.warmup + args.steps):
            t = time.perf_counter()
            r = v.render(cams[i], tau)
            lat.append(time.perf_counter() - t)
            stats.append(r.stats)
            kernels += r.stats["kernels"]
        ev1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), ws)
        return ms, lat, stats, kernels

    # ---- timed regions: the plain launch loop, then the headline view
    # (each frame one captured CUDA graph unless --no-graph)
    clk = ClockSampler(dev)
    clk.start()
    ms_loop, _, _, _ = timed(view_loop)
    ms, lat, stats, kernels = timed(view)
    clocks = clk.stop()
    view_loop.close()
    frames = args.steps * ws
    value = frames / (ms / 1e3)
    value_loop = frames / (ms_loop / 1e3)

    # ---- per-stage device times (a second pass over the same frames with stage events)
    view_t = vgr.View(h, stream=stream.cuda_stream, timing=True)
    for i in range(args.warmup):
        view_t.render(cams[i], tau)
    stage_ms = np.zeros(len(vgr.STAGES))
    n_t = 0
    for i in range(args.warmup, args.warmup + args.steps):
        r = view_t.render(cams[i], tau)
        stage_ms += np.array([r.stats["stage_ms"][s] for s in vgr.STAGES])
        n_t += 1
    stage_ms /= max(1, n_t)
    view_t.close()

    # ---- the same walk with the reduced-precision store (FP16 SH + BF16
    # covariance, FP32 arithmetic): second run of the city configuration
    half_store = None
    if args.config == "city" and not args.leaves and args.storage == "fp32" and not args.no_half:
        h16 = vgr.Hierarchy(sc, storage=vgr.STORE_HALF)
        v16 = vgr.View(h16, stream=stream.cuda_stream, use_graph=not args.no_graph)
        ms16, _, st16, _ = timed(v16)
        half_store = dict(value=round(frames / (ms16 / 1e3), 2), unit="frames/s", ms_per_step=round(ms16 / args.steps, 4),
                          scene_device_gb=round(h16.device_bytes / 1e9, 2),
                          pairs=round(float(np.mean([s["pair_count"] for s in st16])), 1))
        v16.close()
        h16.close()

    # ---- cut reuse between consecutive frames (the motivation of the
    # temporal update, Sec. 4.1): overlap of the cuts of two consecutive
    # frames and the nodes each LoD form evaluates for the same frame
    lod_reuse = None
    if (ws == 1 or rank == 0) and not args.no_lod_reuse:
        vr = vgr.View(h, stream=stream.cuda_stream, timing=True)
        vs = vgr.View(h, stream=stream.cuda_stream, temporal=False, timing=True)
        i0 = args.warmup + args.steps // 2
        for i in range(max(0, i0 - 3), i0):
            vr.render(cams[i], tau)
        a = vr.render(cams[i0], tau)
        ca = a.cut().cpu().numpy().copy()
        lod_t, lod_s, ev_t, ev_s = [], [], [], []
        for i in range(i0 + 1, min(len(cams), i0 + 6)):
            b = vr.render(cams[i], tau)
            if i == i0 + 1:
                cb = b.cut().cpu().numpy().copy()
            s_ = vs.render(cams[i], tau)
            lod_t.append(b.stats["stage_ms"]["lod"])
            lod_s.append(s_.stats["stage_ms"]["lod"])
            ev_t.append(b.stats["nodes_evaluated"])
            ev_s.append(s_.stats["nodes_evaluated"])
        common = int(np.intersect1d(ca, cb, assume_unique=True).size)
        lod_reuse = dict(frames="%d, %d" % (i0, i0 + 1), cut=int(cb.size), common_with_previous=common,
                         overlap=round(common / max(1, cb.size), 5),
                         nodes_evaluated_temporal=int(np.mean(ev_t)), nodes_evaluated_top_down=int(np.mean(ev_s)),
                         lod_ms_temporal=round(float(np.mean(lod_t)), 4),
                         lod_ms_top_down=round(float(np.mean(lod_s)), 4))
        vr.close()
        vs.close()
        # across granularities (Sec. 2 motivation): the share of an exhaustive
        # pass over all nodes that the top-down traversal never needs, and the
        # cut overlap between consecutive frames
        levels = []
        for tau_l in (1.5, 3.0, 6.0, 12.0, 24.0):
            vr = vgr.View(h, stream=stream.cuda_stream, timing=True)
            vs = vgr.View(h, stream=stream.cuda_stream, temporal=False, timing=True)
            ia, ib = min(i0, len(cams) - 2), min(i0, len(cams) - 2) + 1
            for i in range(max(0, ia - 2), ia):
                vr.render(cams[i], tau_l)
            ca = vr.render(cams[ia], tau_l).cut().cpu().numpy().copy()
            b = vr.render(cams[ib], tau_l)
            cb = b.cut().cpu().numpy().copy()
            s_ = vs.render(cams[ib], tau_l)
            common = int(np.intersect1d(ca, cb, assume_unique=True).size)
            levels.append(dict(tau=tau_l, cut=int(cb.size), overlap=round(common / max(1, cb.size), 5),
                               exhaustive_redundant=round(1.0 - s_.stats["nodes_evaluated"] / h.n_nodes, 4),
                               nodes_evaluated_temporal=b.stats["nodes_evaluated"],
                               nodes_evaluated_top_down=s_.stats["nodes_evaluated"],
                               lod_ms_temporal=round(b.stats["stage_ms"]["lod"], 4),
                               lod_ms_top_down=round(s_.stats["stage_ms"]["lod"], 4)))
            vr.close()
            vs.close()
        lod_reuse.update(nodes=h.n_nodes, by_tau=levels)

    # ---- frustum-aware granularity test (node boxes against the view
    # frustum widened by 2 pixels): the same walk, timed like the headline
    frustum_lod = None
    if sc.get("bbox") is not None and not args.no_frustum:
        vf = vgr.View(h, stream=stream.cuda_stream, use_graph=not args.no_graph, lod_frustum=True)
        msf, _, stf, _ = timed(vf)
        vf.close()
        vft = vgr.View(h, stream=stream.cuda_stream, timing=True, lod_frustum=True)
        vd = vgr.View(h, stream=stream.cuda_stream)
        for i in range(args.warmup):
            vft.render(cams[i], tau)
        st_ms, n_st = np.zeros(3), min(args.steps, 50)
        for i in range(args.warmup, args.warmup + n_st):
            r_f = vft.render(cams[i], tau)
            st_ms += np.array([r_f.stats["stage_ms"][k] for k in ("lod", "compact", "preprocess")])
        st_ms /= n_st
        i1 = args.warmup + n_st - 1  # the last frame above, against the distance-only cut
        vd.render(cams[i1 - 1], tau)
        r_d = vd.render(cams[i1], tau)
        img_f, img_d = r_f.image().double(), r_d.image().double()
        mse = float(((img_f - img_d) ** 2).mean())
        frustum_lod = dict(value=round(frames / (msf / 1e3), 2), unit="frames/s",
                           ms_per_step=round(msf / args.steps, 4), guard_px=2.0,
                           cut=round(float(np.mean([x["cut_count"] for x in stf])), 1),
                           front=round(float(np.mean([x["front_count"] for x in stf])), 1),
                           visible=round(float(np.mean([x["visible_count"] for x in stf])), 1),
                           replays=int(sum(x["replays"] for x in stf)),
                           stage_ms=dict(lod=round(st_ms[0], 4), compact=round(st_ms[1], 4),
                                         preprocess=round(st_ms[2], 4)),
                           psnr_vs_distance_only_db=round(10 * math.log10(1.0 / mse), 2) if mse > 0 else None,
                           max_abs_vs_distance_only=round(float((img_f - img_d).abs().max()), 5))
        vft.close()
        vd.close()

    # ---- parent-child weight interpolation of the cut's Gaussians: the same
    # walk, timed like the headline
    weight_interp = None
    if not args.no_interp:
        vi = vgr.View(h, stream=stream.cuda_stream, use_graph=not args.no_graph, lod_interp=True)
        msi, _, sti, _ = timed(vi)
        vi.close()
        vit = vgr.View(h, stream=stream.cuda_stream, timing=True, lod_interp=True)
        vd = vgr.View(h, stream=stream.cuda_stream)
        for i in range(args.warmup):
            vit.render(cams[i], tau)
        st_ms, n_st = np.zeros(2), min(args.steps, 50)
        for i in range(args.warmup, args.warmup + n_st):
            r_i = vit.render(cams[i], tau)
            st_ms += np.array([r_i.stats["stage_ms"][k] for k in ("lod", "preprocess")])
        st_ms /= n_st
        i1 = args.warmup + n_st - 1
        vd.render(cams[i1 - 1], tau)
        r_d = vd.render(cams[i1], tau)
        img_i, img_d = r_i.image().double(), r_d.image().double()
        mse = float(((img_i - img_d) ** 2).mean())
        weight_interp = dict(value=round(frames / (msi / 1e3), 2), unit="frames/s",
                             ms_per_step=round(msi / args.steps, 4),
                             front=round(float(np.mean([x["front_count"] for x in sti])), 1),
                             visible=round(float(np.mean([x["visible_count"] for x in sti])), 1),
                             stage_ms=dict(lod=round(st_ms[0], 4), preprocess=round(st_ms[1], 4)),
                             psnr_vs_plain_db=round(10 * math.log10(1.0 / mse), 2) if mse > 0 else None)
        vit.close()
        vd.close()

    # ---- the Eq. 5 lookup table (m = 32) in place of the exponential: the
    # same walk, timed like the headline, and the blend stage on its own
    exp_lut = None
    if not args.no_lut:
        try:
            vl = vgr.View(h, stream=stream.cuda_stream, use_graph=not args.no_graph, exp_mode=vgr.EXP_LUT,
                          lut_size=32)
            msl, _, _, _ = timed(vl)
            vl.close()
            vlt = vgr.View(h, stream=stream.cuda_stream, timing=True, exp_mode=vgr.EXP_LUT, lut_size=32)
            for i in range(args.warmup):
                vlt.render(cams[i], tau)
            bl, n_st = 0.0, min(args.steps, 50)
            for i in range(args.warmup, args.warmup + n_st):
                bl += vlt.render(cams[i], tau).stats["stage_ms"]["blend"]
            vlt.close()
            exp_lut = dict(m=32, value=round(frames / (msl / 1e3), 2), unit="frames/s",
                           ms_per_step=round(msl / args.steps, 4), blend_ms=round(bl / n_st, 4))
        except vgr.VgrError as e:
            exp_lut = dict(error=str(e))

    # ---- without the preemptive filter (Sec. 4.2): 3-sigma square footprints,
    # every tile of the box kept, alpha computed before the alpha* test at every
    # pixel of every pair; the same walk, timed like the headline, and the image
    # difference from the filtered render of the same frame
    canonical = None
    if not args.no_canonical:
        vc = vgr.View(h, stream=stream.cuda_stream, use_graph=not args.no_graph, filter=vgr.FILTER_CANONICAL)
        msc, _, stc, _ = timed(vc)
        vc.close()
        vct = vgr.View(h, stream=stream.cuda_stream, timing=True, filter=vgr.FILTER_CANONICAL)
        vd = vgr.View(h, stream=stream.cuda_stream)
        for i in range(args.warmup):
            vct.render(cams[i], tau)
        st_ms, n_st = np.zeros(3), min(args.steps, 50)
        for i in range(args.warmup, args.warmup + n_st):
            r_c = vct.render(cams[i], tau)
            st_ms += np.array([r_c.stats["stage_ms"][k] for k in ("emit", "tile_sort", "blend")])
        st_ms /= n_st
        i1 = args.warmup + n_st - 1  # the last frame above, filtered
        vd.render(cams[i1 - 1], tau)
        r_d = vd.render(cams[i1], tau)
        img_c, img_d = r_c.image().double(), r_d.image().double()
        mse = float(((img_c - img_d) ** 2).mean())
        value_c = frames / (msc / 1e3)
        canonical = dict(value=round(value_c, 2), unit="frames/s", ms_per_step=round(msc / args.steps, 4),
                         filter_speedup=round(value / value_c, 3),
                         pairs=round(float(np.mean([x["pair_count"] for x in stc])), 1),
                         pixel_pair_evals=round(float(np.mean([x["pixel_pair_evals"] for x in stc])), 1),
                         stage_ms=dict(emit=round(st_ms[0], 4), tile_sort=round(st_ms[1], 4),
                                       blend=round(st_ms[2], 4)),
                         psnr_vs_filtered_db=round(10 * math.log10(1.0 / mse), 2) if mse > 0 else None,
                         max_abs_vs_filtered=round(float((img_c - img_d).abs().max()), 6))
        vct.close()
        vd.close()

    # ---- end to end through the host-buffer entry points: the pipelined one
    # (each frame's image copied into pinned host memory while the next frame
    # runs; two host buffers in turn; the last copy awaited inside the timed
    # region) and the synchronous one (the image in host memory when the call
    # returns)
    host_imgs = [torch.empty((H, W, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    hps = [a.data_ptr() for a in host_imgs]
    from paper_2506_02774_gb300 import _abi
    fr = _abi.Frame()
    e2e_val = {}
    for mode, call in (("synchronous", view.render_host_ptr), ("pipelined", view.render_pipelined_ptr)):
        view.reset()
        for i in range(args.warmup):
            _abi.check(call(structs[i], tau, hps[i & 1], fr))
        view.wait_host_images()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for i in range(args.warmup, args.warmup + args.steps):
            _abi.check(call(structs[i], tau, hps[i & 1], fr))
        view.wait_host_images()
        e2e_val[mode] = args.steps / (time.perf_counter() - t)
    e2e = dict(value=e2e_val["pipelined"], unit="frames/s", h2d_bytes_per_step=int(128 + 4),
               d2h_bytes_per_step=int(W * H * 3 * 4 + 48 + 8), value_synchronous=e2e_val["synchronous"])

    # ---- roofline of the dominant kernel
    mean = {k: float(np.mean([s[k] for s in stats])) for k in
            ("cut_count", "front_count", "visible_count", "pair_count", "nodes_evaluated", "candidate_pairs",
             "pixel_pair_evals", "pixel_pair_contribs")}
    n_tiles = ((W + 15) // 16) * ((H + 15) // 16)
    tp = max(1, (int(math.ceil(math.log2(max(2, n_tiles)))) + 7) // 8)
    fb = _frame_bytes(sc, mean, W, H, tp)
    peaks = _peaks()
    shares = {s: float(stage_ms[i]) for i, s in enumerate(vgr.STAGES)}
    hbm_stages = {s: fb[s] / (shares[s] * 1e-3) / 1e9 for s in vgr.STAGES if shares[s] > 0}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof_blend = blend_roofline(mean, shares["blend"], sms, peaks, fb["blend"], hbm_stages.get("blend", 0.0))
    roof_pre = hbm_roofline("preprocess", "k_preprocess", "k_preprocess.cu", fb["preprocess"], shares["preprocess"],
                            peaks, mean["front_count"])
    out = dict(metric=METRIC, value=round(value, 2), unit="frames/s", n_gpus=ws, steps=args.steps,
               warmup=args.warmup, ms_per_step=round(ms / args.steps, 4), higher_is_better=True,
               scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
               config=workload_config(wl, sc, cfg, args, ws),
               e2e=dict(value=round(e2e["value"], 2), unit=e2e["unit"],
                        h2d_bytes_per_step=e2e["h2d_bytes_per_step"], d2h_bytes_per_step=e2e["d2h_bytes_per_step"],
                        mode="vgr_render_frame_pipelined: each image copied to pinned host memory during the "
                             "next frame, the last copy awaited in the timed region",
                        value_synchronous=round(e2e["value_synchronous"], 2)),
               gpu_launches=int(kernels),
               launch_mode="cuda-graph replay per frame" if not args.no_graph else "plain launch loop",
               value_plain_loop=round(value_loop, 2),
               roofline=roof_blend, roofline_blend=roof_blend, roofline_preprocess=roof_pre, clocks=clocks,
               frame_latency_ms=dict(p50=round(1e3 * float(np.percentile(lat, 50)), 4),
                                     p99=round(1e3 * float(np.percentile(lat, 99)), 4)),
               stage_ms={k: round(v, 4) for k, v in shares.items()},
               stage_gbs={k: round(v, 1) for k, v in hbm_stages.items()},
               frame_hbm=frame_roofline(fb, shares, ms / args.steps, peaks["hbm_gbs"]),
               counts={k: round(v, 1) for k, v in mean.items()},
               lod_reuse=lod_reuse,
               half_store=half_store,
               frustum_lod=frustum_lod,
               weight_interp=weight_interp,
               exp_lut=exp_lut,
               canonical_filter=canonical,
               setup_s=dict(generate=round(t_gen, 1), upload=round(t_up, 1)))
    view.close()
    if args.config == "city" and not args.leaves and not args.no_served:
        out["served"] = run_served(sc, h, args.serve_clients, args.serve_rate, args.serve_seconds,
                                   [float(x) for x in args.serve_sweep.split(",") if x], args.sweep_seconds,
                                   args.p99_bound)
        out["p50_ms"], out["p99_ms"] = out["served"]["continuous"]["p50_ms"], out["served"]["continuous"]["p99_ms"]
    h.close()
    if args.config == "city" and not args.leaves and not args.no_batched:
        out["batched"] = run_batched(sc, args.batch_views, args.batch_steps, 4)
    if ws > 1:
        torch.distributed.destroy_process_group()
    out["_scene"] = sc if rank == 0 else None
    out["_cams"] = cams
    out["_rank"] = rank
    return out


def run_batched(sc, n_views: int, steps: int, warmup: int, seed: int = 4) -> dict:
    """Multi-view batch: n_views views of the city (FP16 SH + BF16 covariance
    storage), each at frames 300.. of its own street walk at a size drawn
    uniformly from 360p/720p/1080p/1440p (fx scaled with the width); one
    vgr_render_batch per step, against the same frames rendered one view
    after another.  Wall-clock throughput (views/s)."""
    import torch
    import scenegen
    import paper_2506_02774_gb300 as vgr
    rng = np.random.default_rng(seed)
    names = ["360p", "720p", "1080p", "1440p"]
    pick = [names[i] for i in rng.integers(0, 4, n_views)]
    sizes = [scenegen.RESOLUTIONS[n] for n in pick]
    tau = scenegen.CONFIGS["city"]["tau"]
    h = vgr.Hierarchy(sc, storage=vgr.STORE_HALF)
    # launch geometry per image size from the autotuner (a 13-frame walk of
    # the first view of each size, frames 287..299)
    from paper_2506_02774_gb300 import autotune
    geom = {}
    for name in names:
        if name in pick:
            i = pick.index(name)
            walk = [scenegen.street_trajectory("city", 200 + i, fr, *sizes[i]) for fr in range(287, 300)]
            geom[name] = autotune.tune(h, walk, tau)
    views = [vgr.View(h, use_graph=True, grid_wide=geom[pick[i]]["grid_wide"], grid_scan=geom[pick[i]]["grid_scan"])
             for i in range(n_views)]
    frames = list(range(300 - warmup, 300 + steps))
    cams = {fr: [scenegen.street_trajectory("city", 200 + i, fr, *sizes[i]) for i in range(n_views)] for fr in frames}
    taus = [tau] * n_views
    # the single blend launch of the batch: its tile size and staging depth
    # tuned on the batch itself (frames 290..295 of every view's walk), then left set
    tune_steps = [[scenegen.street_trajectory("city", 200 + i, fr, *sizes[i]) for i in range(n_views)]
                  for fr in range(290, 296)]
    batch_tuned = autotune.tune_batch(views, tune_steps, taus)
    out = {}
    for mode in ("sequential", "batched"):
        for v in views:
            v.reset()
        pix = 0
        for fr in frames:
            if fr == 300:
                torch.cuda.synchronize()
                t = time.perf_counter()
            if mode == "batched":
                res = vgr.render_batch(views, cams[fr], taus)
            else:
                res = [v.render(c, tau) for v, c in zip(views, cams[fr])]
            if fr >= 300:
                pix += sum(r.width * r.height for r in res)
        dt = time.perf_counter() - t
        out[mode] = dict(views_per_s=round(n_views * steps / dt, 1), ms_per_step=round(1e3 * dt / steps, 3),
                         mpix_per_s=round(pix / dt / 1e6, 1))
    dev_bytes = sum(v.device_bytes() for v in views)
    for v in views:
        v.close()
    h.close()
    counts = {n: pick.count(n) for n in names}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    tuned = {n: dict(grid_wide_per_sm=g["grid_wide"] // sms, grid_scan_per_sm=g["grid_scan"] // sms,
                     tile_size_alone=g["tile_size"], blend_depth_alone=g["blend_depth"], ms=g["ms"],
                     default_ms=g["default_ms"])
             for n, g in geom.items()}
    return dict(views=n_views, sizes=counts, frames="300..%d of each view's own street walk" % (300 + steps - 1),
                autotuned=tuned, batch_tuned=batch_tuned,
                launch="every view's frame a branch of one captured graph up to its tile order; one launch "
                       "orders all views' tiles, one persistent blend shades them",
                storage="fp16 SH + bf16 covariance", views_device_gb=round(dev_bytes / 1e9, 1),
                speedup=round(out["batched"]["views_per_s"] / out["sequential"]["views_per_s"], 3), **out)


def _serve_trace(n_clients: int, rate: float, seconds: float, seed: int, pick, frame0: int):
    """Poisson arrivals (rate req/s per client) over `seconds`; client c's
    k-th request renders frame frame0 + k of its own street walk."""
    import scenegen
    rng = np.random.default_rng(seed)
    tau = scenegen.CONFIGS["city"]["tau"]
    trace = []
    for c in range(n_clients):
        W, H = scenegen.RESOLUTIONS[pick[c]]
        t, k = 0.0, frame0
        while True:
            t += float(rng.exponential(1.0 / rate))
            if t > seconds:
                break
            trace.append(dict(client=c, arrival_s=t, tau=tau, cam=scenegen.street_trajectory("city", 300 + c, k, W, H)))
            k += 1
    trace.sort(key=lambda r: r["arrival_s"])
    return trace


def _serve_once(h, n_clients, inflight, pick, trace):
    import scenegen
    import paper_2506_02774_gb300 as vgr
    tau = scenegen.CONFIGS["city"]["tau"]
    warm = [dict(client=c, arrival_s=0.0, tau=tau, cam=scenegen.street_trajectory("city", 300 + c, k, *scenegen.RESOLUTIONS[pick[c]]))
            for c in range(n_clients) for k in range(2)]
    sv = vgr.Server(h, n_clients, max_inflight=inflight, host_images=True)
    sv.serve(warm)
    r = sv.serve(trace)
    sv.close()
    ok = r["status"] == 0
    lat = 1e3 * (r["finish_s"] - r["arrival_s"])[ok]
    span = float(r["finish_s"].max() - r["arrival_s"].min())
    svc = 1e3 * (r["finish_s"] - r["start_s"])[ok]
    arr = r["arrival_s"][ok]
    slow = np.argsort(lat)[::-1][:5]
    return dict(p50_ms=round(float(np.percentile(lat, 50)), 3), p99_ms=round(float(np.percentile(lat, 99)), 3),
                mean_ms=round(float(lat.mean()), 3), completed=int(ok.sum()), refused=int((r["status"] == 2).sum()),
                frames_per_s=round(float(ok.sum()) / span, 1),
                service_p99_ms=round(float(np.percentile(svc, 99)), 3),
                slowest=[dict(arrival_s=round(float(arr[i]), 4), latency_ms=round(float(lat[i]), 3),
                              service_ms=round(float(svc[i]), 3)) for i in slow])


def run_served(sc, h, n_clients: int, rate: float, seconds: float, sweep, sweep_seconds: float,
               p99_bound_ms: float, seed: int = 5, modes=(("continuous", 2), ("one_at_a_time", 1))) -> dict:
    """Serving: n_clients clients with Poisson arrivals (rate req/s each) for
    `seconds`, image sizes uniform over 720p/1080p/1440p, each client on its
    own street walk (one frame step per request), images copied to pinned
    host memory.  Latency = completion - arrival.  Continuous batching (up
    to two clients' frames in flight, the server's default) against one
    frame at a time; then a
    sweep of the offered load, reporting for each mode the highest
    throughput whose p99 stays within p99_bound_ms."""
    rng = np.random.default_rng(seed)
    names = ["720p", "1080p", "1440p"]
    pick = [names[i] for i in rng.integers(0, 3, n_clients)]
    trace = _serve_trace(n_clients, rate, seconds, seed, pick, 2)
    out = {m: _serve_once(h, n_clients, inf, pick, trace) for m, inf in modes}
    pts = {m: [] for m, _ in modes}
    for r in sweep:
        tr = _serve_trace(n_clients, r, sweep_seconds, seed + int(r), pick, 2)
        for m, inf in modes:
            x = _serve_once(h, n_clients, inf, pick, tr)
            pts[m].append(dict(rate_per_client=r, offered=round(n_clients * r, 1), frames_per_s=x["frames_per_s"],
                               p50_ms=x["p50_ms"], p99_ms=x["p99_ms"]))
    best = {m: max([p["frames_per_s"] for p in pts[m] if p["p99_ms"] <= p99_bound_ms] or [0.0]) for m, _ in modes}
    saturated = {m: pts[m][-1]["frames_per_s"] if pts[m] else None for m, _ in modes}
    return dict(clients=n_clients, rate_per_client=rate, seconds=seconds, requests=len(trace),
                sizes={n: pick.count(n) for n in names}, host_images=True,
                max_inflight={m: inf for m, inf in modes}, **out,
                sweep=dict(seconds=sweep_seconds, p99_bound_ms=p99_bound_ms, points=pts,
                           max_frames_per_s_within_bound=best, frames_per_s_at_highest_load=saturated))


def cpu_baseline(sc, cams, tau, budget_s: float = 20.0, single_thread: bool = True) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    whole frames of the same walk until ~budget_s of CPU time on every host
    core, then (single_thread) the first of those frames again on one
    thread."""
    import oracle
    n_thr = oracle.num_threads()
    done, t_total = 0, 0.0
    for cam in cams:
        t = time.perf_counter()
        oracle.render(sc, cam, tau)
        t_total += time.perf_counter() - t
        done += 1
        if t_total >= budget_s:
            break
    out = dict(value=round(done / t_total, 4), unit="frames/s", cores=n_thr, kind="oracle",
               sample="%d full frame(s) of the same walk (FP64 oracle, %d OpenMP threads), %.1f s"
                      % (done, n_thr, t_total))
    if single_thread and cams:
        oracle.set_threads(1)
        try:
            t = time.perf_counter()
            oracle.render(sc, cams[0], tau)
            t1 = time.perf_counter() - t
        finally:
            oracle.set_threads(n_thr)
        out["single_thread"] = dict(value=round(1.0 / t1, 4), unit="frames/s", cores=1,
                                    sample="the first of those frames on one thread, %.1f s" % t1)
    return out


def run_reference(args) -> dict:
    """The reference arm: the FP64 oracle (the paper released no code) on the
    host cores, on the same walk, config, metric and unit as the GPU arm.
    Every step is one whole frame of the walk: W untimed warm-up frames, then
    the K timed ones (about 1.7 s each on 16 Arm cores for the city)."""
    import oracle
    import scenegen
    ws, rank, _ = _dist()
    wl = WORKLOADS[args.config]
    cfg = scenegen.CONFIGS[wl["scene"]]
    if rank != 0:
        return None
    sc = scenegen.make_scene(wl["scene"], n_leaves=args.leaves or None)
    wl = workload_label(wl, args.leaves)
    cams = [scenegen.trajectory(wl["scene"], f % cfg["frames"]) for f in range(args.warmup + args.steps)]
    n_thr = oracle.num_threads()
    for cam in cams[:args.warmup]:
        oracle.render(sc, cam, cfg["tau"])
    t = time.perf_counter()
    for cam in cams[args.warmup:]:
        oracle.render(sc, cam, cfg["tau"])
    dt = time.perf_counter() - t
    value = args.steps / dt
    desc = "all %d timed frames %d..%d of the walk after %d warm-up frames, FP64 oracle, %d OpenMP threads, %.1f s" % (
        args.steps, args.warmup, args.warmup + args.steps - 1, args.warmup, n_thr, dt)
    return dict(impl="reference", metric=METRIC, value=round(value, 4), unit="frames/s", n_gpus=ws,
                steps=args.steps, warmup=args.warmup, ms_per_step=round(1e3 * dt / args.steps, 2),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=workload_config(wl, sc, cfg, args, ws),
                cpu_baseline=dict(value=round(value, 4), unit="frames/s", cores=n_thr, kind="oracle", sample=desc),
                e2e=dict(value=round(value, 4), unit="frames/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed frames (default 300; 20 for --impl reference, whose frames take seconds)")
    ap.add_argument("--warmup", type=int, default=None, help="untimed frames before them (default 10; 3 for the reference)")
    ap.add_argument("--no-graph", action="store_true", help="headline view without CUDA graph replay")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-view batch leg")
    ap.add_argument("--no-half", action="store_true", help="skip the FP16/BF16-store run of the walk")
    ap.add_argument("--no-lod-reuse", action="store_true", help="skip the cut-reuse statistics")
    ap.add_argument("--no-frustum", action="store_true", help="skip the frustum-aware LoD run of the walk")
    ap.add_argument("--no-interp", action="store_true", help="skip the weight-interpolation run of the walk")
    ap.add_argument("--no-lut", action="store_true", help="skip the Eq. 5 lookup-table run of the walk")
    ap.add_argument("--no-canonical", action="store_true",
                    help="skip the run of the walk without the preemptive filter (3-sigma binning)")
    ap.add_argument("--no-served", action="store_true", help="skip the serving leg")
    ap.add_argument("--batch-views", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--serve-clients", type=int, default=32)
    ap.add_argument("--serve-rate", type=float, default=8.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-sweep", default="12,16,20,24,28,32,40,48", help="per-client request rates of the load sweep")
    ap.add_argument("--sweep-seconds", type=float, default=4.0)
    ap.add_argument("--p99-bound", type=float, default=25.0, help="p99 latency bound (ms) of the load sweep")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="city", choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default="fp32", choices=["fp32", "half"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-single", action="store_true", help="skip the single-threaded oracle frame")
    ap.add_argument("--leaves", type=int, default=0, help="override the workload's leaf count (smaller profiling cases)")
    args = ap.parse_args()
    ref = args.impl == "reference"
    if args.steps is None:
        args.steps = 20 if ref else 300
    if args.warmup is None:
        args.warmup = 3 if ref else 10
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out = run_ours(args)
    sc, cams, rank = out.pop("_scene"), out.pop("_cams"), out.pop("_rank")
    if rank == 0:
        if args.no_cpu_baseline or out["n_gpus"] > 1:
            out["cpu_baseline"] = None
        else:
            tau = 3.0
            out["cpu_baseline"] = cpu_baseline(sc, cams[args.warmup:], tau, args.cpu_budget,
                                               single_thread=not args.no_cpu_single)
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

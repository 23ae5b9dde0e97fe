#!/usr/bin/env python
"""Benchmark of the 2DGS rasterizer hot path: frame-to-map tracking on the
tracking-scale workload (200k-surfel synthetic room, 640x480, fx = fy = 525,
target RGB-D rendered at ground truth with 1 mm depth noise, 100 pose-only
iterations from a 2 cm / 1 degree perturbation).

One step = one tracking frame = 100 iterations of project -> bin_sort ->
render_fwd -> tracking loss -> render_bwd (pose) -> AdamW + retraction, all
in one gs2d_track_step call.  The metric is 2DGS fwd+bwd Mpix/s
(iterations x 640 x 480 / time); the tracking time to reach 1 cm / 0.5
degree is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (the path has no cross-GPU exchange), one
rank per GPU under torch.distributed.run; rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on a bounded pixel sample of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "2DGS fwd+bwd Mpix/s; tracking ms/frame to 1 cm/0.5° error vs plain loop"
UNIT = "Mpix/s"
N_SURFELS = 200_000
N_ITER = 100
WORKLOAD = ("tracking-scale room: 200k surfels on a 5x4x3 m room with 20 boxes/spheres, 640x480, "
            "fx=fy=525, target at ground truth + N(0, 1 mm) depth noise, 100 pose-only iterations "
            "from a 2 cm / 1 deg perturbation")
ORACLE_CROP = 64          # reference arm: a 64x64 pixel crop per step (~1 s of host work)
CPU_SAMPLE_CROP = 192       # cpu_baseline: one 192x192 crop (~10 s of host work)
L2_FLUSH_BYTES = 256 << 20
TIMED_EVERY = 10          # fused-kernel launches bracketed by events: every 10th iteration
# DRAM bytes per launch of the roofline kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of the fused tracking kernel on
# this workload); None while the kernel has changed since the capture.
TRAFFIC_BYTES = {"track_tile": 6610432}
# batched workloads reported beside the tracking line
MAP_SURFELS, MAP_VIEWS = 1_000_000, 8
UNEVEN_SURFELS, UNEVEN_VIEWS = 2_000_000, 32
MAP_W_D, MAP_W_N = 0.5, 0.02
# learned proposal: training pairs, AdamW steps at batch 256 (about 12 s of training), held-out
# frames
PROP_PAIRS, PROP_STEPS, PROP_EVAL_FRAMES = 100_000, 9000, 256
# the network refines its own proposal once (two passes of proposal + acceptance test)
PROP_PASSES = 2
PROP_TRACK_FRAMES = 32    # tracking-workload frames for the proposal at tracking scale
# its network is trained on starts up to 3 cm / 1.5 deg (the tracking frames start 2 cm / 1 deg
# off); one pass: at full resolution a loop iteration costs a third of a proposal pass
PROP_TRACK_MAX, PROP_TRACK_PASSES = (0.03, 1.5), 1


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    return ap.parse_args()


def _dist():
    from paper_2506_00970_gb300 import replicas
    return replicas.init("nccl")


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# workload
# --------------------------------------------------------------------------
def make_frames(n_frames: int, rank: int):
    """Seeded frames: ground-truth pose, start pose (2 cm / 1 deg off) and the
    observed RGB-D frame rendered on the GPU at ground truth (+1 mm noise)."""
    import torch
    from paper_2506_00970_gb300 import gs2d, replicas, scenes
    s = scenes.room_scene(0, N_SURFELS)
    cam = scenes.tracking_camera()
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, ds.n)
    frames = []
    kmax = 0
    for f in range(n_frames):
        seed = replicas.seed_base(rank) + f
        gt = scenes.room_pose(100 + seed)
        start = scenes.perturb_pose(gt, 0.02, 1.0, seed=5000 + seed)
        out = r.forward(ds, gs2d.pose_tensor(gt))
        noise = np.random.default_rng(9000 + seed).normal(0.0, 1e-3, (cam.height, cam.width))
        obs_d = (out["depth"] / out["opacity"].clamp_min(1e-6)).cpu().numpy() + noise
        obs_d = torch.tensor(obs_d.astype(np.float32), device="cuda")
        frames.append(dict(gt=gt, start=start, obs_rgb=out["rgb"].clone(), obs_depth=obs_d,
                           start_t=gs2d.pose_tensor(start)))
        r.forward(ds, gs2d.pose_tensor(start))
        kmax = max(kmax, int(r.n_isect.item()))
    torch.cuda.synchronize()
    return s, cam, ds, r, frames, kmax


def first_below(ph, gt, tcm=0.01, tdeg=0.5):
    for it in range(ph.shape[0]):
        et, er = _pose_err_np(ph[it], gt)
        if et < tcm and er < tdeg:
            return it + 1
    return None


def _pose_err_np(row, gt):
    R = row[:9].reshape(3, 3)
    t = row[9:]
    c = -R.T @ t
    cg = -gt.R.T @ gt.t
    from paper_2506_00970_gb300.proposal import rotation_angle_deg
    return float(np.linalg.norm(c - cg)), rotation_angle_deg(R @ gt.R.T)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_mhz: float) -> float:
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA per clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# FP32 operations per (pixel, surfel) pair of the compositing loop, counted
# from the arithmetic the method needs (FMA = 2; MUFU rcp/exp not counted):
#  every evaluated pair: the linear map p (6 FMA = 12), u, v (2), u^2 + v^2
#  (FMA + mul = 3) -> 17; pairs inside the cutoff radius add z, the exp
#  argument, alpha G and the clamp -> 4; blended pairs add 1 - a, T (1 - a),
#  w, colour, depth and normal accumulation (3 + 6 + 2 + 6) -> 17.  The
#  pose-only backward adds per replayed blended pair ~80 (transmittance
#  recovery, dL/da, the chain through G, q, beta, Gv, X x Gv, t_nc x g and
#  the 6-vector accumulation); it evaluates the pairs up to each pixel's
#  last blended one (gs2d_render_count's replayed counts).
FLOPS_EVAL, FLOPS_IN, FLOPS_BLEND, FLOPS_BWD_BLEND = 17, 4, 17, 80
FLOPS_LOSS_PIXEL = 20   # masks, three colour and one depth difference, signs


def run_ours(args):
    import torch
    from paper_2506_00970_gb300 import replicas
    from paper_2506_00970_gb300 import build as _b
    _b.build()
    from paper_2506_00970_gb300 import gs2d, scenes
    ws_n, rank, local = _dist()
    torch.cuda.set_device(local)
    W_ = max(args.warmup, 3)
    K = args.steps
    n_frames = min(max(K, 4), 20)
    s, cam, ds, r, frames, kmax = make_frames(n_frames, rank)
    ccam, cfg = gs2d.camera(cam), gs2d.default_config()
    prm = gs2d.default_track_params(stop_tol=0.0)     # always the full 100 iterations
    cap = int(kmax * 1.5) + 4096
    ws = torch.empty(gs2d.gs2d_track_workspace(ds.n, cap, ccam, cfg), dtype=torch.uint8, device="cuda")
    lh = torch.zeros(N_ITER, device="cuda")
    ph = torch.zeros(N_ITER, 12, device="cuda")
    pose = torch.empty(12, device="cuda")
    obs_rgb = torch.empty_like(frames[0]["obs_rgb"])
    obs_d = torch.empty_like(frames[0]["obs_depth"])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def load(f):
        fr = frames[f % n_frames]
        pose.copy_(fr["start_t"])
        obs_rgb.copy_(fr["obs_rgb"])
        obs_d.copy_(fr["obs_depth"])

    def track():
        gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, N_ITER, cap, lh, ph, ws)

    # one direct call, then capture a whole frame (reset + 100 x 2 kernels)
    # into a CUDA graph; the fused tile kernel's launches of every
    # TIMED_EVERY-th iteration are bracketed by event-record nodes inside the
    # graph (live timing inside the timed region; a node pair costs about
    # 11 us, so bracketing all 100 launches would add ~8% to a frame)
    load(0)
    track()
    torch.cuda.synchronize()
    n_timed = (N_ITER + TIMED_EVERY - 1) // TIMED_EVERY
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(n_timed)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(n_timed)]
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        load(0)
    torch.cuda.current_stream().wait_stream(side)
    gs2d.gs2d_profile_track_kernel(k0, k1)
    gs2d.gs2d_profile_track_kernel_every(TIMED_EVERY)
    with torch.cuda.graph(graph):
        track()
    gs2d.gs2d_profile_track_kernel([], [])
    gs2d.gs2d_profile_track_kernel_every(1)
    stream = torch.cuda.current_stream()

    for i in range(W_):
        load(i)
        graph.replay()
    torch.cuda.synchronize()
    st = int(gs2d.gs2d_track_status(ws).item())
    if st not in (0, gs2d.CONVERGED):
        raise RuntimeError(f"track status {st}")

    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    hist, fused = [], []
    replicas.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(K):
            load(i)
            flush.zero_()
            e0[i].record(stream)
            graph.replay()
            e1[i].record(stream)
            e1[i].synchronize()
            fused.extend(a.elapsed_time(b) for a, b in zip(k0, k1))
            hist.append(ph.clone())
        torch.cuda.synchronize()
    replicas.barrier()
    wall = time.perf_counter() - t_wall
    fused_ms = float(np.mean(fused))
    st = int(gs2d.gs2d_track_status(ws).item())
    if st not in (0, gs2d.CONVERGED):
        raise RuntimeError(f"track status {st}")
    step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    tot_ms = replicas.max_over_ranks(sum(step_ms), device="cuda")
    P = cam.width * cam.height
    value = replicas.weak_scaling_value(ws_n, K * N_ITER * P, tot_ms) / 1e6
    ms_step = tot_ms / K

    # tracking accuracy and time to 1 cm / 0.5 deg
    its, fin = [], []
    for i, h in enumerate(hist):
        fr = frames[i % n_frames]
        h = h.cpu().numpy().astype(np.float64)
        it = first_below(h, fr["gt"])
        its.append(it if it is not None else np.nan)
        fin.append(_pose_err_np(h[-1], fr["gt"]))
    ms_iter = ms_step / N_ITER
    it_med = float(np.nanmedian(its)) if np.isfinite(its).any() else None
    tracking = {
        "ms_per_frame_100_iters": ms_step,
        "ms_per_iter": ms_iter,
        "iters_to_1cm_0.5deg_median": it_med,
        "ms_to_1cm_0.5deg_median": None if it_med is None else it_med * ms_iter,
        "frames_reaching_threshold": int(np.isfinite(its).sum()),
        "frames": len(its),
        "final_err_cm_median": float(np.median([e[0] for e in fin]) * 100),
        "final_err_deg_median": float(np.median([e[1] for e in fin])),
        "learned_proposal": None,
    }

    # end to end through the C ABI from pinned host buffers: each step copies
    # the observed frame and the start pose in, replays the captured frame
    # and reads the final pose and loss back
    h_rgb = [frames[f]["obs_rgb"].cpu().pin_memory() for f in range(n_frames)]
    h_d = [frames[f]["obs_depth"].cpu().pin_memory() for f in range(n_frames)]
    h_pose = [frames[f]["start_t"].cpu().pin_memory() for f in range(n_frames)]
    out_pose = torch.empty(12).pin_memory()
    out_loss = torch.empty(1).pin_memory()

    def step_e2e(f):
        f = f % n_frames
        obs_rgb.copy_(h_rgb[f], non_blocking=True)
        obs_d.copy_(h_d[f], non_blocking=True)
        pose.copy_(h_pose[f], non_blocking=True)
        graph.replay()
        out_pose.copy_(pose, non_blocking=True)
        out_loss.copy_(lh[-1:], non_blocking=True)

    for i in range(2):
        step_e2e(i)
    torch.cuda.synchronize()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee1 = torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for i in range(K):
        flush.zero_()
        ee0.record(stream)
        step_e2e(i)
        ee1.record(stream)
        ee1.synchronize()
        e2e_ms += ee0.elapsed_time(ee1)
    e2e_ms = replicas.max_over_ranks(e2e_ms, device="cuda")
    e2e_value = replicas.weak_scaling_value(ws_n, K * N_ITER * P, e2e_ms) / 1e6
    h2d = h_rgb[0].numel() * 4 + h_d[0].numel() * 4 + 12 * 4
    d2h = 12 * 4 + 4

    roof = roofline(r, ds, frames, cam, cfg, stream, ms_iter, fused_ms)
    del graph
    batch = batch_workloads(K, W_, flush)
    batch["slab_single_view"] = slab_render(K, W_, flush)
    maint = map_maintenance(flush)
    tracking["learned_proposal"] = learned_proposal(flush)
    tracking["learned_proposal_tracking_scale"] = tracking_scale_proposal(rank)

    if rank == 0:
        clocks = clk.summary()
        pk, src = peaks()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": K,
            "warmup": W_, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "surfels": N_SURFELS, "width": cam.width,
                       "height": cam.height, "iterations_per_step": N_ITER, "frames": n_frames,
                       "tile": "16x16", "l2": "256 MB buffer written between steps",
                       "launch": "one CUDA graph per frame (reset + 100 x 2 kernels)",
                       "parallelism": f"replicas x{ws_n}"},
            "tracking": tracking,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / K},
            "gpu_launches": K * (1 + N_ITER * LAUNCHES_PER_ITER),
            "roofline": roof["main"],
            "roofline_other": roof["other"],
            **batch,
            **maint,
            "wall_s": wall,
            "peak_source": src,
        }
        line["cpu_baseline"] = cpu_baseline(s, cam, frames[0])
        print(json.dumps(line))
    replicas.finish()


# kernels per tracking iteration at 640x480 (1200 tiles): the projection
# with the tile counts, the tile scan and the scatter of the pairs (one
# cooperative launch; the counters are zeroed by the previous iteration's
# fused kernel) 1; the fused tile kernel (per-tile depth sort, render, loss,
# pose backward, and the reduction + AdamW + retraction in its last block) 1.
# Plus one reset per frame.
LAUNCHES_PER_ITER = 2


def roofline(r, ds, frames, cam, cfg, stream, ms_iter, fused_ms):
    """The fused tile kernel (render + loss + pose backward, the largest share
    of a tracking iteration), timed live in the timed region, and the
    standalone forward and pose-backward kernels timed here on the same start
    poses (CUDA events around each launch on the launching stream).  Work is
    the algorithmic FP32 flops from the pair counts, against the FP32 peak."""
    import torch
    from paper_2506_00970_gb300 import gs2d
    pk, src = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak = fp32_peak_tflops(sm_mhz)
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    g_rgb = torch.zeros(cam.height, cam.width, 3, device="cuda")
    g_d = torch.zeros(cam.height, cam.width, device="cuda")
    g_o = torch.zeros(cam.height, cam.width, device="cuda")
    loss = torch.zeros(1, device="cuda")
    lws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    prm = gs2d.default_track_params()
    fwd_ms, bwd_ms, work_f, work_b, pairs = [], [], [], [], []
    R = 10
    for fr in frames[:4]:
        pt = fr["start_t"]
        r.forward(ds, pt)
        gs2d.gs2d_tracking_loss(r.rgb, r.depth, r.normal, r.opacity, fr["obs_rgb"], fr["obs_depth"],
                                r.cam, prm, g_rgb, g_d, g_o, loss, lws)
        gs2d.gs2d_render_count(r.proj, r.bins, r.cam, r.cfg, counts)
        torch.cuda.synchronize()
        E, Ein, B, Eb, Ebin = (int(x) for x in counts.cpu().numpy())
        work_f.append(FLOPS_EVAL * E + FLOPS_IN * Ein + FLOPS_BLEND * B)
        work_b.append(FLOPS_EVAL * Eb + FLOPS_IN * Ebin + FLOPS_BWD_BLEND * B)
        pairs.append((E, Ein, B, Eb, Ebin))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * R)]
        for k in range(R):
            ev[2 * k].record(stream)
            gs2d.gs2d_render_fwd(r.proj, r.bins, r.cam, r.cfg, r.rgb, r.depth, r.normal, r.opacity,
                                 r.t_final, r.n_last)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        fwd_ms.append(np.mean([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(R)]))
        for k in range(R):
            ev[2 * k].record(stream)
            r.backward(ds, pt, g_rgb, g_d, None, g_o, full=False)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        bwd_ms.append(np.mean([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(R)]))
    tf = np.mean(fwd_ms) / 1e3
    tb = np.mean(bwd_ms) / 1e3
    P = cam.width * cam.height
    work_fused = np.mean(work_f) + np.mean(work_b) + FLOPS_LOSS_PIXEL * P
    tfu = fused_ms / 1e3
    afu = work_fused / tfu / 1e12
    fused = {"kernel": "track_tile_kernel (render + tracking loss + pose backward)", "bound": "alu",
             "achieved": afu, "peak": peak, "unit": "TFLOP/s", "frac": afu / peak,
             "traffic": TRAFFIC_BYTES["track_tile"],
             "traffic_note": "ncu capture of one launch on the first of the timed frames "
                             "(the lightest); the other frames read their own records",
             "launch_ms": fused_ms,
             "launch_timing": f"CUDA events around the launches of every {TIMED_EVERY}th "
                              "iteration inside each timed frame graph",
             "share_of_iter": fused_ms / ms_iter, "flop_per_launch": work_fused,
             "pairs_per_launch": dict(zip(("evaluated", "inside_cutoff", "blended",
                                           "replayed_evaluated", "replayed_inside_cutoff"),
                                          (float(x) for x in np.mean(pairs, axis=0)))),
             "flop_per_pair": {"evaluated": FLOPS_EVAL, "inside_cutoff": FLOPS_IN,
                               "blended_fwd": FLOPS_BLEND, "blended_bwd": FLOPS_BWD_BLEND,
                               "loss_per_pixel": FLOPS_LOSS_PIXEL},
             "peak_note": f"FP32 152 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz (of measured max clock)"}
    af = np.mean(work_f) / tf / 1e12
    ab = np.mean(work_b) / tb / 1e12
    fwd = {"kernel": "render_fwd_kernel", "bound": "alu", "achieved": af, "peak": peak,
           "unit": "TFLOP/s", "frac": af / peak, "launch_ms": tf * 1e3}
    bwd = {"kernel": "render_bwd_kernel<pose> + pose_reduce", "bound": "alu", "achieved": ab,
           "peak": peak, "unit": "TFLOP/s", "frac": ab / peak, "launch_ms": tb * 1e3}
    return {"main": fused, "other": [fwd, bwd]}


def _perturbed_map(s, seed):
    """The map being optimised: the true map with centres moved by N(0, 3 mm)
    and colours by N(0, 0.05), so every loss term has a gradient."""
    from paper_2506_00970_gb300 import scenes
    rng = np.random.default_rng(seed)
    return scenes.Surfels(s.mu + rng.normal(0, 3e-3, s.mu.shape), s.quat, s.scale, s.opacity,
                          np.clip(s.rgb + rng.normal(0, 0.05, s.rgb.shape), 0, 1))


def measure_batch(name, s_true, cams, poses, actives, K, W_, flush, seed):
    """One batched mapping step over all views: project, bin_sort, forward
    (one persistent launch), the mapping loss of every view in one launch
    (colour L1 + 0.5 depth L1 + 0.02 normal consistency, each view's mean over
    its pixels) and backward (one persistent launch + the
    per-surfel reductions), gradients to every surfel parameter.  Tile shapes
    come from the autotuner per resolution class.  Timed as direct calls
    (per phase) and as one CUDA graph replay per step."""
    import torch
    from paper_2506_00970_gb300 import autotune, gs2d
    stream = torch.cuda.current_stream()
    ds_true = gs2d.DeviceSurfels(s_true)
    ds = gs2d.DeviceSurfels(_perturbed_map(s_true, seed))
    t0 = time.perf_counter()
    px, tiles, sweep = autotune.tune(ds, cams, poses, actives)
    tune_s = time.perf_counter() - t0
    br = gs2d.BatchRasterizer(cams, ds.n, actives=actives, tiles=tiles, px=px)
    br.set_poses(poses)
    br.fit(ds_true)
    br.forward(ds_true)
    obs = []
    for v, b in enumerate(br.keep):
        noise = torch.randn(b["depth"].shape, generator=torch.Generator("cuda").manual_seed(seed + v),
                            device="cuda") * 1e-3
        obs.append((b["rgb"].clone(), b["depth"] / b["opacity"].clamp_min(1e-6) + noise))
    del ds_true
    kv = br.fit(ds)
    loss = torch.zeros(len(cams), device="cuda")
    lviews = gs2d.loss_views([(b["ccam"], b["rgb"], b["depth"], b["normal"], b["opacity"],
                               obs[v][0], obs[v][1], b["d_rgb"], b["d_depth"], b["d_normal"],
                               b["d_opacity"]) for v, b in enumerate(br.keep)])
    lws = torch.empty(gs2d.gs2d_mapping_loss_batch_workspace(lviews), dtype=torch.uint8,
                      device="cuda")

    def losses():
        gs2d.gs2d_mapping_loss_batch(lviews, MAP_W_D, MAP_W_N, loss, lws)

    def step():
        br.forward(ds, check_status=False)
        losses()
        br.backward(ds)

    # direct calls, per phase
    phases = ("project", "bin_sort", "render_fwd", "loss", "render_bwd")
    per = {k: [] for k in phases}
    direct = []
    for i in range(W_ + K):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        for b in br.keep:
            b["status"].zero_()
        ev[0].record(stream)
        gs2d.gs2d_project_batch(ds, br.views)
        ev[1].record(stream)
        gs2d.gs2d_bin_sort_batch(br.views, br.n, br.sort_ws)
        ev[2].record(stream)
        gs2d.gs2d_render_fwd_batch(br.views, br.render_ws)
        ev[3].record(stream)
        losses()
        ev[4].record(stream)
        br.backward(ds)
        ev[5].record(stream)
        ev[5].synchronize()
        if i >= W_:
            for j, k in enumerate(phases):
                per[k].append(ev[j].elapsed_time(ev[j + 1]))
            direct.append(ev[0].elapsed_time(ev[5]))
    st = [int(b["status"].item()) for b in br.keep]
    if any(st):
        raise RuntimeError(f"{name}: batch status {st}")
    # one CUDA graph per step
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(W_):
        graph.replay()
    torch.cuda.synchronize()
    gms = []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        gms.append(e0.elapsed_time(e1))
    st = [int(b["status"].item()) for b in br.keep]
    if any(st):
        raise RuntimeError(f"{name}: batch status {st}")
    # algorithmic FP32 work of the two compositing launches from pair counts
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    E = np.zeros(5)
    for b in br.keep:
        gs2d.gs2d_render_count(b["proj"], b["bins"], b["ccam"], b["cfg"], counts)
        torch.cuda.synchronize()
        E += counts.cpu().numpy()
    pk, src = peaks()
    peak = fp32_peak_tflops(float(pk.get("sm_max_mhz", 2070.0)))
    w_f = FLOPS_EVAL * E[0] + FLOPS_IN * E[1] + FLOPS_BLEND * E[2]
    w_b = FLOPS_EVAL * E[3] + FLOPS_IN * E[4] + FLOPS_BWD_BLEND * E[2]
    tf, tb = np.median(per["render_fwd"]) / 1e3, np.median(per["render_bwd"]) / 1e3
    P = sum(int(c.width) * int(c.height) for c in cams)
    g_ms = float(np.median(gms))
    out = {
        "value": P / (g_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": g_ms,
        "ms_per_step_direct": float(np.median(direct)),
        "mpix_per_s_direct": P / (np.median(direct) / 1e3) / 1e6,
        "phase_ms": {k: float(np.median(v)) for k, v in per.items()},
        "views": len(cams), "pixels": P, "surfels": int(ds.n),
        "active_sizes": [int(b["m"]) for b in br.keep], "intersections": [int(k) for k in kv],
        "resolutions": sorted({f"{c.width}x{c.height}" for c in cams}),
        "px_per_thread": px, "tiles": [f"{t[0]}x{t[1]}" for t in tiles],
        "autotune_ms_per_view": sweep,
        "autotune_s": tune_s, "loss": [float(x) for x in loss.cpu().numpy()],
        "pairs": {"evaluated": int(E[0]), "inside_cutoff": int(E[1]), "blended": int(E[2]),
                  "replayed_evaluated": int(E[3]), "replayed_inside_cutoff": int(E[4])},
        "roofline": [
            {"kernel": "fwd_batch_kernel (persistent)", "bound": "alu",
             "achieved": w_f / tf / 1e12, "peak": peak, "unit": "TFLOP/s",
             "frac": w_f / tf / 1e12 / peak, "launch_ms": tf * 1e3},
            {"kernel": "bwd_batch_kernel (persistent) + per-view surfel reductions",
             "bound": "alu", "achieved": w_b / tb / 1e12, "peak": peak, "unit": "TFLOP/s",
             "frac": w_b / tb / 1e12 / peak, "launch_ms": tb * 1e3,
             "note": "flops count the pose-chain work per blended pair only (a lower bound)"}],
        "launch": "one CUDA graph per step",
        "peak_mem_gb": torch.cuda.max_memory_allocated() / 1e9,
    }
    del graph, br, ds
    torch.cuda.empty_cache()
    return out


def slab_render(K, W_, flush):
    """The plain single-view workload: 4,096 surfels, centres uniform in a
    2 x 2 m slab 1-3 m in front of a 160x120 camera (fx = fy = 150),
    log-uniform 1-5 cm scales, random rotations, sigmoid(N(0,1)) opacity,
    random colours; L1 colour + L1 depth (on D/O, lambda_d = 1) against a
    target rendered at a pose 2 cm / 1 deg away; one step = project,
    bin_sort, render_fwd, the loss and the full render_bwd (gradients to
    every surfel parameter and the pose), timed as direct calls and as one
    CUDA graph replay (L2 flushed before each).  The FP64 oracle runs the
    same step on the full image."""
    import torch
    from paper_2506_00970_gb300 import gs2d, scenes
    import oracle
    stream = torch.cuda.current_stream()
    s, cam = scenes.slab_scene(0), scenes.slab_camera()
    pose = scenes.identity_pose()
    target = scenes.perturb_pose(pose, 0.02, 1.0, seed=11)
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, ds.n, capacity=64 * ds.n)
    out = r.forward(ds, gs2d.pose_tensor(target))
    obs_rgb = out["rgb"].clone()
    obs_d = out["depth"] / out["opacity"].clamp_min(1e-6)
    pose_t = gs2d.pose_tensor(pose)
    r.forward(ds, pose_t)
    torch.cuda.synchronize()
    H, W, n = cam.height, cam.width, ds.n
    f = dict(dtype=torch.float32, device="cuda")
    g = [torch.empty(H, W, 3, **f), torch.empty(H, W, **f), torch.empty(H, W, 3, **f),
         torch.empty(H, W, **f)]
    loss = torch.empty(1, **f)
    lws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    grads = [torch.empty(n, 3, **f), torch.empty(n, 4, **f), torch.empty(n, 2, **f),
             torch.empty(n, **f), torch.empty(n, 3, **f), torch.empty(6, **f)]

    def project():
        gs2d.gs2d_project(ds, r.cam, pose_t, r.cfg, r.proj, r.tiles)

    def bin_sort():
        gs2d.gs2d_bin_sort(r.proj, r.tiles, r.n, r.cam, r.cfg, r.sort_ws, r.bins)

    def render_fwd():
        r.render_fwd()

    def loss_fn():
        gs2d.gs2d_mapping_loss(r.rgb, r.depth, r.normal, r.opacity, obs_rgb, obs_d, r.cam, 1.0, 0.0,
                               *g, loss, lws)

    def render_bwd():
        gs2d.gs2d_render_bwd(r.proj, r.bins, r.tiles, ds, pose_t, r.cam, r.cfg, r.t_final, r.n_last,
                             g[0], g[1], g[2], g[3], *grads, r.bwd_ws)

    phases = (("project", project), ("bin_sort", bin_sort), ("render_fwd", render_fwd),
              ("loss", loss_fn), ("render_bwd", render_bwd))

    def step():
        for _, fn in phases:
            fn()

    per = {k: [] for k, _ in phases}
    direct = []
    for i in range(W_ + K):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(phases) + 1)]
        ev[0].record(stream)
        for j, (_, fn) in enumerate(phases):
            fn()
            ev[j + 1].record(stream)
        ev[-1].synchronize()
        if i >= W_:
            for j, (k, _) in enumerate(phases):
                per[k].append(ev[j].elapsed_time(ev[j + 1]))
            direct.append(ev[0].elapsed_time(ev[-1]))
    if int(r.status.item()) != 0:
        raise RuntimeError(f"slab status {int(r.status.item())}")
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(W_):
        graph.replay()
    gms = []
    for _ in range(K):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        gms.append(e0.elapsed_time(e1))
    if int(r.status.item()) != 0:
        raise RuntimeError(f"slab status {int(r.status.item())}")
    counts = torch.zeros(5, dtype=torch.int64, device="cuda")
    gs2d.gs2d_render_count(r.proj, r.bins, r.cam, r.cfg, counts)
    torch.cuda.synchronize()
    E = counts.cpu().numpy().astype(np.float64)
    w_f = FLOPS_EVAL * E[0] + FLOPS_IN * E[1] + FLOPS_BLEND * E[2]
    w_b = FLOPS_EVAL * E[3] + FLOPS_IN * E[4] + FLOPS_BWD_BLEND * E[2]
    pk, src = peaks()
    peak = fp32_peak_tflops(float(pk.get("sm_max_mhz", 2070.0)))
    tf, tb = np.median(per["render_fwd"]) / 1e3, np.median(per["render_bwd"]) / 1e3
    g_ms = float(np.median(gms))
    P = H * W
    # the oracle on the full image: forward, the same loss, full backward
    cores = oracle.default_threads()
    ot = oracle.render(s, cam, target, n_threads=cores)
    o_rgb, o_d = ot["rgb"], ot["depth"] / np.maximum(ot["opacity"], 1e-6)
    t0 = time.perf_counter()
    o = oracle.render(s, cam, pose, n_threads=cores)
    img = {k: o[k] for k in ("rgb", "depth", "normal", "opacity")}
    _, og = oracle.mapping_loss(img, o_rgb, o_d, cam, w_d=1.0, w_n=0.0)
    oracle.render_bwd(s, cam, pose, og["rgb"], og["depth"], og["normal"], og["opacity"],
                      n_threads=cores)
    dt = time.perf_counter() - t0
    return {
        "workload": (f"plain single view: {n} surfels in a 2x2 m slab 1-3 m ahead, 160x120, "
                     "fx=fy=150, L1 colour + L1 depth against a target 2 cm / 1 deg away, "
                     "gradients to all surfel parameters and the pose"),
        "value": P / (g_ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": g_ms,
        "ms_per_step_direct": float(np.median(direct)),
        "mpix_per_s_direct": P / (np.median(direct) / 1e3) / 1e6,
        "phases_ms": {k: float(np.median(v)) for k, v in per.items()},
        "launch": "one CUDA graph per step (project, bin_sort 5 kernels, render_fwd, loss, "
                  "render_bwd 2 kernels); L2 flushed before each",
        "pairs": {"evaluated": int(E[0]), "inside_cutoff": int(E[1]), "blended": int(E[2]),
                  "replayed_evaluated": int(E[3]), "replayed_inside_cutoff": int(E[4])},
        "roofline": {"kernel": "render_fwd_kernel + render_bwd_kernel<full> + surfel_grad_kernel",
                     "bound": "alu", "unit": "TFLOP/s", "peak": peak,
                     "fwd_achieved": w_f / tf / 1e12, "fwd_frac": w_f / tf / 1e12 / peak,
                     "bwd_achieved": w_b / tb / 1e12, "bwd_frac": w_b / tb / 1e12 / peak,
                     "note": "a 160x120 view has 80 tiles on 152 SMs: launch- and "
                             "latency-bound, not throughput-bound"},
        "cpu_baseline": {"value": P / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "the full step on the full 160x120 image (FP64 forward, "
                                   "loss, full backward)", "seconds": dt},
    }


def batch_workloads(K, W_, flush):
    """The mapping window (1M surfels, 8 keyframes at 1200x680 on a smooth
    trajectory) and the uneven batch (32 views of a 2M-surfel room, mixed
    resolutions, active subsets of 50k-1M surfels)."""
    from paper_2506_00970_gb300 import scenes
    s1 = scenes.room_scene(1, MAP_SURFELS)
    cams = [scenes.mapping_camera()] * MAP_VIEWS
    poses = scenes.room_trajectory(2, MAP_VIEWS)
    mw = measure_batch("mapping window", s1, cams, poses, None, K, W_, flush, 31)
    mw["workload"] = (f"mapping window: {MAP_SURFELS} surfels, {MAP_VIEWS} keyframes 1200x680 "
                      f"fx=fy=600 on a smooth trajectory, colour L1 + {MAP_W_D} depth L1 + "
                      f"{MAP_W_N} normal consistency, gradients to all surfel parameters")
    del s1
    s2 = scenes.room_scene(3, UNEVEN_SURFELS)
    cams, poses, actives = scenes.uneven_batch(4, s2, UNEVEN_VIEWS)
    ub = measure_batch("uneven batch", s2, cams, poses, actives, K, W_, flush, 47)
    ub["workload"] = (f"uneven batch: {UNEVEN_VIEWS} views of a {UNEVEN_SURFELS}-surfel room, "
                      "resolutions from {320x240, 640x480, 1200x680}, active subsets of "
                      "50k-1M surfels (log-uniform), same loss as the mapping window")
    return {"mapping_window": mw, "uneven_batch": ub}


# FP32 operations per pair of the contribution pass: the forward's
# evaluation (17 + 4 inside the cutoff) plus, per blended pair, T (1 - a)
# and w += a T (4), and one add per evaluated pair in the per-warp sums.
FLOPS_CONTRIB_BLEND = 4
# Algorithmic bytes per surfel of the map-state passes (each array read or
# written once): observe reads contrib, mu and the state (4 + 12 + 13) and
# writes the state (13); correct reads t_c, mu, quat (32) and writes mu, quat
# (28); prune reads contrib, t_c (8) and writes keep (1); compact reads keep
# twice, the parameters and the state (2 + 52 + 13) and writes them and the
# new index (65 + 4).
MAP_BYTES = {"observe": 42, "correct": 60, "prune": 9, "compact": 136}
# FP32 operations per pixel of the SSIM term with its gradient (3 channels):
# five moment maps filtered separably (2 x 11 FMA each = 44 flops, plus 8
# to form the products and the difference), the SSIM value and its partials
# (~40), three partial maps filtered back (3 x 44) and the combination (4):
# 3 x (5 x 44 + 8 + 40 + 132 + 4) = 1212, halo work not counted.
SSIM_FLOPS_PER_PX = 1212


def _timed_ms(fn, reps, flush, stream):
    """Median device time of fn over reps calls, L2 flushed before each."""
    import torch
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms))


def map_maintenance(flush, reps=10):
    """Keyframe bookkeeping of Sec. III-D / III-F / IV-C on the GPU.
    (a) keyframe test of a tracking frame (200k-surfel room, 640x480):
    projection, binning, per-surfel contributions (gs2d_render_contrib) and
    the covisibility score + keyframe rule against the last keyframe's
    contributions; the contribution kernel's FP32 roofline from the pair
    counts.  (b) the map-state passes on a 2M-surfel map with the
    contributions of a 1200x680 keyframe view: state update, correction by
    64 keyframe increments, pruning and compaction, each against HBM."""
    import torch
    from paper_2506_00970_gb300 import gs2d, scenes
    stream = torch.cuda.current_stream()
    pk, _ = peaks()
    peak_f = fp32_peak_tflops(float(pk.get("sm_max_mhz", 2070.0)))
    hbm = float(pk["hbm_gbs"])
    out = {}
    # (a)
    s = scenes.room_scene(0, N_SURFELS)
    cam = scenes.tracking_camera()
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, ds.n)
    kf_pose = gs2d.pose_tensor(scenes.room_pose(1))
    cur_pose = gs2d.pose_tensor(scenes.perturb_pose(scenes.room_pose(1), 0.05, 2.0, seed=3))
    r.forward(ds, kf_pose)
    c_kf = r.contribution().clone()
    r.forward(ds, cur_pose)
    c_cur = torch.empty(ds.n, device="cuda")
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    score = torch.zeros(1, device="cuda")
    is_kf = torch.zeros(1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(5, dtype=torch.int64, device="cuda")
    gs2d.gs2d_render_count(r.proj, r.bins, r.cam, r.cfg, cnt)
    torch.cuda.synchronize()
    E, Ein, B = (int(x) for x in cnt.cpu().numpy()[:3])
    work = (FLOPS_EVAL + 1) * E + FLOPS_IN * Ein + FLOPS_CONTRIB_BLEND * B

    def keyframe_test():
        r.project(ds, cur_pose)
        r.bin_sort(grow=False)
        r.contribution(out=c_cur)
        gs2d.gs2d_covisibility(c_cur, c_kf, ds.n, 0.5, cur_pose, kf_pose, 0.9, 0.15, counts, score,
                               is_kf)

    keyframe_test()
    t_all = _timed_ms(keyframe_test, reps, flush, stream)
    t_c = _timed_ms(lambda: r.contribution(out=c_cur), reps, flush, stream)
    a = work / (t_c / 1e3) / 1e12
    out["keyframe_test"] = {
        "workload": f"tracking frame: {N_SURFELS} surfels, 640x480",
        "ms": t_all, "contrib_ms": t_c, "mpix_s": cam.width * cam.height / t_c / 1e3,
        "covisibility": float(score.item()), "is_keyframe": int(is_kf.item()),
        "roofline": {"kernel": "contrib_tile_kernel + contrib_reduce_kernel", "bound": "alu",
                     "achieved": a, "peak": peak_f, "unit": "TFLOP/s", "frac": a / peak_f,
                     "flop_per_launch": work}}
    del r, ds, s
    # (b)
    n = UNEVEN_SURFELS
    s = scenes.room_scene(3, n)
    ds = gs2d.DeviceSurfels(s)
    kcam = scenes.mapping_camera()
    r = gs2d.Rasterizer(kcam, n)
    r.forward(ds, gs2d.pose_tensor(scenes.room_pose(5)))
    contrib = r.contribution().clone()
    del r
    rng = np.random.default_rng(11)
    n_kf = 64
    st0 = {"delta": torch.ones(n, dtype=torch.uint8, device="cuda"),
           "t_c": torch.tensor(rng.integers(0, n_kf, n).astype(np.int32), device="cuda"),
           "d_c": torch.full((n,), 2.5, device="cuda"),
           "t_l": torch.tensor(rng.integers(40, n_kf, n).astype(np.int32), device="cuda")}
    st = gs2d.DeviceMapState.from_tensors(*(v.clone() for v in st0.values()))
    prm = gs2d.StateParams(0.5, 20, 0, -1)
    mcount = torch.zeros(4, dtype=torch.int32, device="cuda")
    poses_old = torch.tensor(np.concatenate([np.r_[np.eye(3).ravel(), rng.normal(size=3)]
                                             for _ in range(n_kf)]).astype(np.float32), device="cuda")
    poses_new = poses_old + 1e-3
    cws = torch.empty(gs2d.gs2d_map_correct_workspace(n_kf), dtype=torch.uint8, device="cuda")
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    outs = gs2d.DeviceSurfels.from_tensors(torch.empty_like(ds.mu), torch.empty_like(ds.quat),
                                           torch.empty_like(ds.scale), torch.empty_like(ds.opacity),
                                           torch.empty_like(ds.rgb))
    st_o = gs2d.DeviceMapState.from_tensors(*(torch.empty_like(v) for v in st0.values()))
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    new_index = torch.empty(n, dtype=torch.int32, device="cuda")
    kws = torch.empty(gs2d.gs2d_map_compact_workspace(n), dtype=torch.uint8, device="cuda")
    kp = gs2d.pose_tensor(scenes.room_pose(5))
    ops = {
        "observe": lambda: gs2d.gs2d_map_observe(contrib, ds.mu, n, kp, n_kf, prm, st, mcount),
        "correct": lambda: gs2d.gs2d_map_correct(ds.mu, ds.quat, st.t_c, n, poses_old, poses_new,
                                                 n_kf, cws),
        "prune": lambda: gs2d.gs2d_map_prune(contrib, st.t_c, n, 7, 0.5, keep),
        "compact": lambda: gs2d.gs2d_map_compact(keep, n, ds, st, outs, st_o, new_index, n_out,
                                                 kws),
    }
    res = {}
    for name, fn in ops.items():
        fn()
        t = _timed_ms(fn, reps, flush, stream)
        gbs = MAP_BYTES[name] * n / (t / 1e3) / 1e9
        res[name] = {"ms": t, "bytes_per_surfel": MAP_BYTES[name], "achieved_gbs": gbs,
                     "frac_of_hbm": gbs / hbm}
    torch.cuda.synchronize()
    res["visible_active"] = int(mcount[0].item())
    res["kept"] = int(n_out.item())
    out["map_state"] = {"workload": f"{n}-surfel map, contributions of a 1200x680 keyframe view, "
                                    f"{n_kf} keyframe increments", "passes": res}
    del ds, outs, st, st_o, contrib
    # (d) map expansion of a 1200x680 keyframe against the active map's voxel
    # table (rebuilt from the active flags first, as after a state change)
    cam_k = scenes.Camera(600.0, 600.0, 600.0, 340.0, 1200, 680)
    rgb_k, dep_k = scenes.rgbd_frame(21, cam_k)
    rng2 = np.random.default_rng(21)
    T_ = lambda a: torch.tensor(a, device="cuda")
    rgb_d, dep_d = T_(rgb_k), T_(dep_k)
    u_keep = T_(rng2.uniform(size=dep_k.shape).astype(np.float32))
    u_ang = T_(rng2.uniform(size=dep_k.shape).astype(np.float32))
    pose_k = gs2d.pose_tensor(scenes.identity_pose())
    ex_ratio = 0.04
    n_act = 1_000_000
    act_pts = T_(np.random.default_rng(22).uniform([-2.1, -1.4, 0.3], [2.1, 1.3, 3.2],
                                                    (n_act, 3)).astype(np.float32))
    table = gs2d.DeviceVoxelTable(1 << 22, 0.02)
    cap_m = n_act + dep_k.size
    f32 = dict(dtype=torch.float32, device="cuda")
    new_s = gs2d.DeviceSurfels.from_tensors(torch.empty(cap_m, 3, **f32), torch.empty(cap_m, 4, **f32),
                                            torch.empty(cap_m, 2, **f32), torch.empty(cap_m, **f32),
                                            torch.empty(cap_m, 3, **f32))
    new_st = gs2d.DeviceMapState(cap_m)
    n_new = torch.zeros(1, dtype=torch.int32, device="cuda")
    ews = torch.empty(gs2d.gs2d_expand_workspace(gs2d.camera(cam_k)), dtype=torch.uint8,
                      device="cuda")
    eprm = gs2d.ExpandParams(ex_ratio, 0.99, 0.05, 9, 0)

    def rebuild():
        table.clear()
        table.insert(act_pts)

    def expand():
        gs2d.gs2d_expand(rgb_d, dep_d, gs2d.camera(cam_k), pose_k, u_keep, u_ang, table, eprm,
                         n_act, cap_m, new_s, new_st, n_new, ews)

    rebuild()
    expand()
    t_rb = _timed_ms(rebuild, reps, flush, stream)
    t_ex = _timed_ms(expand, reps, flush, stream)
    m_ps = int(((dep_k > 0) & (u_keep.cpu().numpy() < ex_ratio)).sum())
    out["map_expansion"] = {
        "workload": (f"1200x680 RGB-D keyframe, random downsampling {ex_ratio}, voxel table of "
                     f"{n_act} active surfels (2 cm voxels)"),
        "table_rebuild_ms": t_rb, "expand_ms": t_ex, "points_ps": m_ps,
        "new_surfels": int(n_new.item()),
        "nearest_pairs": m_ps * m_ps}
    del table, new_s, new_st, act_pts
    # (c) the SSIM term of the full mapping loss (Table I weight) on one
    # 1200x680 keyframe image: loss and gradient in one fused pass
    h, w = kcam.height, kcam.width
    yy = torch.rand(h, w, 3, generator=torch.Generator(device="cuda").manual_seed(1),
                    device="cuda")
    xx = (yy + 0.1 * torch.randn_like(yy)).clamp(0, 1)
    gx = torch.zeros_like(xx)
    lo = torch.zeros(1, device="cuda")
    sws = torch.empty(gs2d.gs2d_ssim_workspace(h, w), dtype=torch.uint8, device="cuda")
    fn = lambda: gs2d.gs2d_ssim_loss(xx, yy, h, w, 0.125, gx, lo, sws)
    fn()
    t = _timed_ms(fn, reps, flush, stream)
    flops = SSIM_FLOPS_PER_PX * h * w
    a = flops / (t / 1e3) / 1e12
    out["ssim_term"] = {"workload": f"SSIM term + gradient, one {w}x{h} RGB image", "ms": t,
                        "mpix_s": h * w / t / 1e3,
                        "roofline": {"kernel": "ssim_kernel + ssim_sum_kernel", "bound": "alu",
                                     "achieved": a, "peak": peak_f, "unit": "TFLOP/s",
                                     "frac": a / peak_f, "flop_per_launch": flops}}
    return out


def net_flops_per_sample():
    """Algorithmic FLOPs of the proposal network per sample (2 per
    multiply-add): forward; training = forward + weight gradients (same
    products) + data gradients (all but the first layer's)."""
    hw = [(120, 160), (60, 80), (30, 40), (15, 20), (8, 10), (4, 5), (2, 3)]
    ch = [8, 32, 64, 128, 256, 256, 256]
    conv = [2 * hw[l + 1][0] * hw[l + 1][1] * ch[l + 1] * 9 * ch[l] for l in range(6)]
    fc = [2 * 1536 * 256, 2 * 256 * 6]
    fwd = sum(conv) + sum(fc)
    return fwd, fwd + fwd + (fwd - conv[0])


def learned_proposal(flush):
    """Train the proposal network on self-rendered pairs (4 rooms, 160x120,
    perturbations up to 5 cm / 3 deg) and compare tracking from the proposal
    with the plain loop on frames of a held-out room."""
    import torch
    from paper_2506_00970_gb300 import gs2d, proposal, scenes
    t0 = time.perf_counter()
    rooms = [scenes.room_scene(100 + r, N_SURFELS) for r in range(4)]
    X, Y = proposal.make_pairs(rooms, PROP_PAIRS, seed=1)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    tr = proposal.Trainer(seed=0, batch=256)
    t0 = time.perf_counter()
    hist = tr.fit(X, Y, PROP_STEPS, lr=1e-3, log_every=PROP_STEPS // 4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    # tensor-core throughput of the network kernels (batch 256)
    stream = torch.cuda.current_stream()
    y = torch.empty(256, 6, device="cuda")
    fwd_ms, step_ms, prep_ms = [], [], []
    # inference with the bfloat16 weights cast once (as the proposal runs it)
    pws = torch.empty(gs2d.gs2d_net_workspace(256), dtype=torch.uint8, device="cuda")
    gs2d.gs2d_net_prepare(tr.params, 256, pws)
    for k in range(8):
        sl = slice(256 * k, 256 * (k + 1))
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e[0].record(stream)
        gs2d.gs2d_net_forward(tr.params, X[sl], y, tr.ws)
        e[1].record(stream)
        gs2d.gs2d_net_grad(tr.params, X[sl], Y[sl], tr.loss, tr.grad, tr.ws)
        gs2d.gs2d_net_adamw(tr.params, tr.grad, tr.m, tr.v, tr.step + 1, lr=0.0)
        e[2].record(stream)
        flush.zero_()
        e[3].record(stream)
        gs2d.gs2d_net_forward_prepared(tr.params, X[sl], y, pws)
        e[4].record(stream)
        e[4].synchronize()
        if k >= 2:
            fwd_ms.append(e[0].elapsed_time(e[1]))
            step_ms.append(e[1].elapsed_time(e[2]))
            prep_ms.append(e[3].elapsed_time(e[4]))
    del pws
    del X, Y
    torch.cuda.empty_cache()
    held_out = scenes.room_scene(200, N_SURFELS)
    ev = proposal.evaluate(held_out, tr.params, PROP_EVAL_FRAMES, seed=3, passes=PROP_PASSES)
    one = proposal.evaluate(held_out, tr.params, PROP_EVAL_FRAMES, seed=3, passes=1)
    fl_f, fl_t = net_flops_per_sample()
    pk, _ = peaks()
    peak = float(pk.get("bf16_tflops", 1900.0))
    f_ms, s_ms = float(np.median(fwd_ms)), float(np.median(step_ms))
    p_ms = float(np.median(prep_ms))
    ev.update({
        "train_pairs": PROP_PAIRS, "train_steps": PROP_STEPS, "batch": 256,
        "pair_gen_s": gen_s, "train_s": train_s, "train_loss": hist,
        "held_out_room": "room seed 200 (training rooms 100-103)",
        "proposal_passes": PROP_PASSES,
        "single_pass": {"learned_ms_median": one["learned"]["ms_to_1cm_0.5deg_median"],
                        "learned_iters_median": one["learned"]["iters_median"],
                        "proposal_ms": one["proposal_ms"],
                        "proposal_err_median_cm_deg": one["proposal_err_median_cm_deg"],
                        "speedup_median": one["speedup_median"]},
        "net": {"fwd_batch256_ms": p_ms, "fwd_batch256_with_weight_cast_ms": f_ms,
                "train_step_batch256_ms": s_ms,
                "fwd_gflop_per_batch": fl_f * 256 / 1e9, "train_gflop_per_batch": fl_t * 256 / 1e9,
                "roofline": {"kernel": "network forward with the bfloat16 weights cast once "
                                       "(gs2d_net_forward_prepared, as the proposal runs it): "
                                       "conv_s2_kernel (direct, mma.sync bf16) for the first "
                                       "convolution, conv_tma_kernel (tcgen05 + TMEM, operands by "
                                       "tiled TMA with element strides and 64/128-byte swizzle) for "
                                       "layers 2-6 (layers 5-6: whole images per 128-row tile), "
                                       "gemm_tc_kernel (tcgen05 split-K) for the FC products; "
                                       "training adds gemm_tc_kernel for the split-K weight "
                                       "gradients and gemm_kernel (mma.sync) for the data gradients",
                             "bound": "tensor",
                             "achieved": fl_f * 256 / (p_ms / 1e3) / 1e12, "peak": peak,
                             "unit": "TFLOP/s", "frac": fl_f * 256 / (p_ms / 1e3) / 1e12 / peak,
                             "with_weight_cast_frac": fl_f * 256 / (f_ms / 1e3) / 1e12 / peak,
                             "train_achieved": fl_t * 256 / (s_ms / 1e3) / 1e12,
                             "peak_note": "dense bf16, of measured (cuBLAS burst)"}},
    })
    return ev


def tracking_scale_proposal(rank):
    """The learned proposal on the tracking workload itself: a network for the
    tracking camera's 160x120 view (640x480 / 4, fx = fy = 131.25) trained on
    self-rendered pairs of rooms 100-103 with starts up to 3 cm / 1.5 deg,
    then frames of the tracking room (seed 0, 2 cm / 1 deg starts): proposal
    at 160x120 from the box-downsampled observation, the full-resolution
    plain loop from the kept pose, against the plain loop from the usual
    start."""
    import torch
    from paper_2506_00970_gb300 import proposal, scenes
    _, cam, ds, _, frames, _ = make_frames(PROP_TRACK_FRAMES, rank)
    lo = proposal.low_res_camera(cam, 4)
    t0 = time.perf_counter()
    rooms = [scenes.room_scene(100 + r, N_SURFELS) for r in range(4)]
    X, Y = proposal.make_pairs(rooms, PROP_PAIRS, seed=11, cam=lo, max_t=PROP_TRACK_MAX[0],
                               max_deg=PROP_TRACK_MAX[1])
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    tr = proposal.Trainer(seed=0, batch=256)
    t0 = time.perf_counter()
    tr.fit(X, Y, PROP_STEPS, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del X, Y
    torch.cuda.empty_cache()
    ev = proposal.evaluate_full_res(ds, tr.params, cam, frames, passes=PROP_TRACK_PASSES)
    ev.update({"train_pairs": PROP_PAIRS, "train_steps": PROP_STEPS, "pair_gen_s": gen_s,
               "train_s": train_s, "train_rooms": "room seeds 100-103",
               "train_starts": f"magnitudes uniform in [0, {PROP_TRACK_MAX[0] * 100:.0f} cm] x "
                               f"[0, {PROP_TRACK_MAX[1]} deg], random directions",
               "frames_room": "room seed 0 (the tracking frames' room, not in training)"})
    return ev


def _oracle_sample(s, cam, fr, crop, n_threads):
    """Seconds of the FP64 oracle's forward + pose backward (tracking-loss
    gradient, Eq. tracking_loss) on a crop x crop pixel sample of one frame."""
    import oracle
    y0, x0 = cam.height // 2 - crop // 2, cam.width // 2 - crop // 2
    ys, xs = np.mgrid[y0:y0 + crop, x0:x0 + crop]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    obs_rgb = fr["obs_rgb"].cpu().numpy()[ys, xs].reshape(-1, 3)
    obs_d = fr["obs_depth"].cpu().numpy()[ys, xs].reshape(-1)
    t0 = time.perf_counter()
    img = oracle.render(s, cam, fr["start"], pixels=pix, n_threads=n_threads)
    Dh = img["depth"] / np.maximum(img["opacity"], 1e-6)
    m = (img["opacity"] > 0.95).astype(float)
    g_rgb = np.sign(img["rgb"] - obs_rgb) * m[:, None]
    g_d = np.sign(Dh - obs_d) * m / np.maximum(img["opacity"], 1e-6)
    oracle.render_bwd(s, cam, fr["start"], g_rgb, g_d, np.zeros_like(g_rgb), np.zeros_like(g_d),
                      pixels=pix, n_threads=n_threads)
    return len(pix), time.perf_counter() - t0


def cpu_baseline(s, cam, fr):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    forward + pose backward of a 192x192 pixel crop of one frame against all
    200k surfels on every host core (OpenMP), and of a 48x48 crop on one."""
    import oracle
    cores = oracle.default_threads()
    n, dt = _oracle_sample(s, cam, fr, CPU_SAMPLE_CROP, cores)
    n1, dt1 = _oracle_sample(s, cam, fr, CPU_SAMPLE_CROP // 4, 1)
    return {"value": n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 fwd + pose bwd of a {CPU_SAMPLE_CROP}x{CPU_SAMPLE_CROP} crop of one "
                      f"640x480 frame, all {N_SURFELS} surfels", "seconds": dt,
            "single_thread": {"value": n1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                              "sample": f"a {CPU_SAMPLE_CROP // 4}x{CPU_SAMPLE_CROP // 4} crop",
                              "seconds": dt1}}


def run_reference(args):
    """The oracle as the reference arm: each step is the bounded sample of the
    workload (see cpu_baseline), timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2506_00970_gb300 import scenes
    import oracle
    s = scenes.room_scene(0, N_SURFELS)
    cam = scenes.tracking_camera()
    gt = scenes.room_pose(100)
    start = scenes.perturb_pose(gt, 0.02, 1.0, seed=5000)
    y0, x0 = cam.height // 2 - ORACLE_CROP // 2, cam.width // 2 - ORACLE_CROP // 2
    ys, xs = np.mgrid[y0:y0 + ORACLE_CROP, x0:x0 + ORACLE_CROP]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    tgt = oracle.render(s, cam, gt, pixels=pix)
    obs_rgb = tgt["rgb"]
    obs_d = tgt["depth"] / np.maximum(tgt["opacity"], 1e-6)

    def one():
        img = oracle.render(s, cam, start, pixels=pix)
        Dh = img["depth"] / np.maximum(img["opacity"], 1e-6)
        m = (img["opacity"] > 0.95).astype(float)
        g_rgb = np.sign(img["rgb"] - obs_rgb) * m[:, None]
        g_d = np.sign(Dh - obs_d) * m / np.maximum(img["opacity"], 1e-6)
        oracle.render_bwd(s, cam, start, g_rgb, g_d, np.zeros_like(g_rgb), np.zeros_like(g_d),
                          pixels=pix)

    for _ in range(max(args.warmup, 1)):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = args.steps * len(pix) / dt / 1e6
    cores = oracle.default_threads()
    sample = (f"FP64 fwd + pose bwd of a {ORACLE_CROP}x{ORACLE_CROP} crop per step, all "
              f"{N_SURFELS} surfels")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)

"""Learned tracking-pose proposal (not in the paper): self-rendered training
pairs, training on the BF16 tensor-core network kernels of gs2d_net.h, and
frame tracking that starts the plain loop of Sec. III-D from the proposal --
or, when the proposal raises the tracking loss (Eq. tracking_loss), from the
usual starting pose.

Workload: rooms of the synthetic room generator rendered at 160x120,
fx = fy = 150; starting poses perturbed from ground truth by up to 5 cm and
3 degrees (magnitudes uniform, directions random); the observed frame is the
ground-truth render with expected depth D/O + N(0, 1 mm), 0 where the
rendered opacity is at most 0.5.  Everything runs through the C ABI; torch
only holds device memory, draws the sensor noise and captures CUDA graphs.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gs2d, scenes

CAM = scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120)
MAX_T, MAX_DEG = 0.05, 3.0
VIEWS = 32


def poses_tensor(poses, device="cuda"):
    return torch.stack([gs2d.pose_tensor(p, device) for p in poses])


def rotation_angle_deg(Rd) -> float:
    """Angle of a rotation matrix in degrees, atan2(|vee(R - R^T)| / 2,
    (tr R - 1) / 2): unlike acos of the trace alone it keeps small angles
    of an FP32 rotation (acos loses everything below ~0.03 degrees)."""
    Rd = np.asarray(Rd, np.float64)
    w = np.array([Rd[2, 1] - Rd[1, 2], Rd[0, 2] - Rd[2, 0], Rd[1, 0] - Rd[0, 1]])
    return math.degrees(math.atan2(0.5 * float(np.linalg.norm(w)), 0.5 * (np.trace(Rd) - 1.0)))


def pose_error(P12, gt) -> tuple[float, float]:
    """Camera-centre distance (m) and geodesic rotation angle (degrees)
    between a pose given as 12 floats and a ground-truth Pose."""
    P = np.asarray(P12, np.float64)
    R, t = P[:9].reshape(3, 3), P[9:]
    c = -R.T @ t
    cg = -gt.R.T @ gt.t
    return float(np.linalg.norm(c - cg)), rotation_angle_deg(R @ gt.R.T)


def first_below(pose_hist, gt, tcm=0.01, tdeg=0.5):
    """1-based index of the first iteration whose pose is within tcm metres
    and tdeg degrees of gt, 0 if the starting pose already is, or None."""
    for it in range(pose_hist.shape[0]):
        et, er = pose_error(pose_hist[it], gt)
        if et < tcm and er < tdeg:
            return it + 1
    return None


def observed_depth(depth, opacity, gen, sigma=1e-3):
    """Synthetic sensor depth from a render: D/O + N(0, sigma), 0 where the
    opacity is at most 0.5."""
    noise = torch.randn(depth.shape, generator=gen, device=depth.device) * sigma
    return torch.where(opacity > 0.5, depth / opacity.clamp_min(1e-6) + noise,
                       torch.zeros_like(depth))


class ViewRenderer:
    """Forward renders of up to VIEWS poses of a 160x120 camera (CAM by
    default) per batched call."""

    def __init__(self, surf: gs2d.DeviceSurfels, views: int = VIEWS, cam=CAM):
        self.surf = surf
        self.views = views
        self.br = gs2d.BatchRasterizer([cam] * views, surf.n, capacities=[3 * surf.n] * views)

    def render(self, poses_t):
        n = poses_t.shape[0]
        pad = [poses_t[min(i, n - 1)] for i in range(self.views)]
        self.br.set_poses(pad)
        self.br.forward(self.surf)
        return self.br.stacked


def make_pairs(rooms, n_pairs: int, seed: int, device="cuda", cam=CAM, max_t: float = MAX_T,
               max_deg: float = MAX_DEG, fixed: bool = False):
    """Training pairs over the given rooms (Surfels): x [n, 120, 160, 8]
    bfloat16 (rendered at the perturbed pose + observed at ground truth) and
    the target y* [n, 6]; ``cam``: the network's 160x120 camera; start poses
    perturbed by magnitudes uniform in [0, max_t] and [0, max_deg], or by
    exactly max_t and max_deg (``fixed``), in random directions."""
    X = torch.empty(n_pairs, 120, 160, 8, dtype=torch.bfloat16, device=device)
    Y = torch.empty(n_pairs, 6, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    per_room = -(-n_pairs // len(rooms))
    i = 0
    for r, s in enumerate(rooms):
        ds = gs2d.DeviceSurfels(s)
        vr = ViewRenderer(ds, cam=cam)
        obs_rgb = torch.empty(VIEWS, 120, 160, 3, device=device)
        obs_d = torch.empty(VIEWS, 120, 160, device=device)
        c0 = 0
        while c0 < per_room and i < n_pairs:
            cnt = min(VIEWS, n_pairs - i, per_room - c0)
            k = seed * 10_000_000 + r * 1_000_000 + c0
            gts = [scenes.room_pose(k + j) for j in range(cnt)]
            inits = [scenes.perturb_pose(g, max_t, max_deg, seed=k + j + 7_000_000) if fixed
                     else scenes.perturb_uniform(g, max_t, max_deg, k + j)
                     for j, g in enumerate(gts)]
            G, I = poses_tensor(gts, device), poses_tensor(inits, device)
            img = vr.render(G)
            obs_rgb.copy_(img["rgb"])
            obs_d.copy_(observed_depth(img["depth"], img["opacity"], gen))
            img = vr.render(I)
            gs2d.gs2d_net_pack_input(img["rgb"][:cnt], img["depth"][:cnt], img["opacity"][:cnt],
                                     obs_rgb[:cnt], obs_d[:cnt], X[i:i + cnt])
            gs2d.gs2d_net_target(I, G, Y[i:i + cnt])
            i += cnt
            c0 += cnt
        del vr, ds
    return X[:i], Y[:i]


class Trainer:
    """AdamW on FP32 master weights; every step is one gs2d_net_grad (forward,
    loss, backward) and one gs2d_net_adamw on a contiguous batch."""

    def __init__(self, seed: int = 0, batch: int = 256, device="cuda"):
        self.batch = batch
        self.params = torch.tensor(scenes.net_init(seed, gs2d.net_init_blocks()), device=device)
        n = self.params.numel()
        self.m = torch.zeros(n, device=device)
        self.v = torch.zeros(n, device=device)
        self.grad = torch.empty(n, device=device)
        self.loss = torch.empty(1, device=device)
        self.ws = torch.empty(gs2d.gs2d_net_workspace(batch), dtype=torch.uint8, device=device)
        self.step = 0

    def fit(self, X, Y, steps: int, lr=1e-3, lr_min=1e-5, wd=1e-4, log_every=0):
        B = self.batch
        nb = X.shape[0] // B
        hist = []
        for k in range(steps):
            j = k % nb
            self.step += 1
            lr_t = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * k / max(steps, 1)))
            gs2d.gs2d_net_grad(self.params, X[j * B:(j + 1) * B], Y[j * B:(j + 1) * B], self.loss,
                               self.grad, self.ws)
            gs2d.gs2d_net_adamw(self.params, self.grad, self.m, self.v, self.step, lr=lr_t, wd=wd)
            if log_every and (k % log_every == 0 or k == steps - 1):
                hist.append((k, float(self.loss.item())))
        return hist

    def state_dict(self) -> dict:
        """Everything a resumed training needs: FP32 master weights, AdamW
        moments and the step count (host copies)."""
        return {"params": self.params.detach().cpu(), "m": self.m.detach().cpu(),
                "v": self.v.detach().cpu(), "step": int(self.step), "batch": int(self.batch)}

    def load_state_dict(self, d: dict):
        if d["params"].numel() != self.params.numel():
            raise ValueError("checkpoint of a different network")
        self.params.copy_(d["params"])
        self.m.copy_(d["m"])
        self.v.copy_(d["v"])
        self.step = int(d["step"])

    def save(self, path: str):
        torch.save(self.state_dict(), path)

    def load(self, path: str):
        self.load_state_dict(torch.load(path, map_location="cpu"))

    def eval_loss(self, X, Y):
        """Mean loss over contiguous batches of (X, Y) (no update)."""
        B = self.batch
        tot, nb = 0.0, X.shape[0] // B
        for j in range(nb):
            gs2d.gs2d_net_grad(self.params, X[j * B:(j + 1) * B], Y[j * B:(j + 1) * B], self.loss,
                               self.grad, self.ws)
            tot += float(self.loss.item())
        return tot / max(nb, 1)


class Proposer:
    """One frame's proposal as a fixed launch sequence (capturable in a CUDA
    graph, no host round trip): render at the current pose, tracking loss
    there, pack with the observation, network forward, apply, render at the
    proposal, tracking loss there, keep the better pose.  With passes > 1 the
    sequence repeats from the kept pose (the network refines its own
    proposal); the kept pose's images and loss are kept with it
    (gs2d_net_accept_keep), so later passes render only their proposal."""

    def __init__(self, surf: gs2d.DeviceSurfels, params, capacity: int, device="cuda",
                 passes: int = 1, cam=CAM):
        self.surf = surf
        self.params = params
        self.passes = int(passes)
        # r renders the current (kept) pose, rp the proposals
        self.r = gs2d.Rasterizer(cam, surf.n, capacity=capacity, device=device)
        self.rp = gs2d.Rasterizer(cam, surf.n, capacity=capacity, device=device) \
            if self.passes > 1 else self.r
        f = dict(dtype=torch.float32, device=device)
        self.pose = torch.empty(1, 12, **f)
        self.prop = torch.empty(1, 12, **f)
        self.obs_rgb = torch.empty(120, 160, 3, **f)
        self.obs_d = torch.empty(120, 160, **f)
        self.x = torch.empty(1, 120, 160, 8, dtype=torch.bfloat16, device=device)
        self.y = torch.empty(1, 6, **f)
        self.ws = torch.empty(gs2d.gs2d_net_workspace(1), dtype=torch.uint8, device=device)
        gs2d.gs2d_net_prepare(params, 1, self.ws)      # the bfloat16 weights, cast once
        self.g = [torch.empty(120, 160, 3, **f), torch.empty(120, 160, **f), torch.empty(120, 160, **f)]
        self.loss_init = torch.empty(1, **f)
        self.loss_prop = torch.empty(1, **f)
        self.lws = torch.empty(1 << 16, dtype=torch.uint8, device=device)
        self.accepted = torch.zeros(1, dtype=torch.int32, device=device)
        self.prm = gs2d.default_track_params()

    def _render(self, pose_row, r):
        r.status.zero_()
        r.project(self.surf, pose_row)
        fwd_bins = gs2d.Bins(r.bins.keys, r.bins.vals, None, None, r.bins.tile_ranges,
                             r.bins.n_isect, r.bins.status, r.bins.capacity)
        gs2d.gs2d_bin_sort(r.proj, r.tiles, r.n, r.cam, r.cfg, r.sort_ws, fwd_bins)
        r.render_fwd()

    def _loss(self, out, r):
        gs2d.gs2d_tracking_loss(r.rgb, r.depth, r.normal, r.opacity, self.obs_rgb, self.obs_d, r.cam,
                                self.prm, self.g[0], self.g[1], self.g[2], out, self.lws)

    def run(self):
        r, rp = self.r, self.rp
        self._render(self.pose[0], r)
        self._loss(self.loss_init, r)
        for p in range(self.passes):
            gs2d.gs2d_net_pack_input(r.rgb[None], r.depth[None], r.opacity[None],
                                     self.obs_rgb[None], self.obs_d[None], self.x)
            gs2d.gs2d_net_forward_prepared(self.params, self.x, self.y, self.ws)
            self.prop.copy_(self.pose)
            gs2d.gs2d_net_apply(self.y, self.prop)
            self._render(self.prop[0], rp)
            self._loss(self.loss_prop, rp)
            if p + 1 < self.passes:
                gs2d.gs2d_net_accept_keep(self.loss_prop, self.loss_init, self.prop, self.pose,
                                          (rp.rgb, rp.depth, rp.opacity),
                                          (r.rgb, r.depth, r.opacity), self.accepted)
            else:
                gs2d.gs2d_net_accept(self.loss_prop, self.loss_init, self.prop, self.pose,
                                     self.accepted)

    def status(self) -> int:
        return max(int(self.r.status.item()), int(self.rp.status.item()))


def capture(fn, warm: int = 1):
    """fn's launches as a CUDA graph (after warm-up calls on a side stream)."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warm):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def timed_replays(graph, reps: int, before=None) -> list[float]:
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        if before is not None:
            before()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        graph.replay()
        e1.record(st)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def timed_ms(fn) -> float:
    """Device time of fn's launches on the current stream (CUDA events)."""
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    fn()
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1)


# The plain loop's limits under the stop rule of Sec. III-D: n_iter of
# Table I and the step-size reading |tau| < 1e-5.
STOP_ITERS, STOP_TOL = 120, 1e-5


class LoopGraphs:
    """The plain tracking loop on fixed buffers (pose, observation, a
    caller-owned AdamW state zeroed at the start of every frame) as CUDA
    graphs, one per (iterations, stop tolerance), captured on first use."""

    def __init__(self, surf, cam, capacity: int, obs_rgb, obs_d, device="cuda"):
        self.surf, self.obs_rgb, self.obs_d = surf, obs_rgb, obs_d
        self.ccam, self.cfg = gs2d.camera(cam), gs2d.default_config()
        self.cap = capacity
        self.pose = torch.empty(12, device=device)
        self.adam = torch.zeros(16, device=device)
        self.ws = torch.empty(gs2d.gs2d_track_workspace(surf.n, capacity, self.ccam, self.cfg),
                              dtype=torch.uint8, device=device)
        self.device = device
        self._graphs, self.hist = {}, {}

    def graph(self, n_iter: int, stop_tol: float = 0.0):
        key = (int(n_iter), float(stop_tol))
        if key not in self._graphs:
            prm = gs2d.default_track_params(stop_tol=stop_tol)
            lh = torch.zeros(n_iter, device=self.device)
            ph = torch.zeros(n_iter, 12, device=self.device)

            def frame():
                self.adam.zero_()
                gs2d.gs2d_track_step(self.surf, self.ccam, self.cfg, prm, self.pose, self.obs_rgb,
                                     self.obs_d, n_iter, self.cap, lh, ph, self.ws,
                                     adam_state=self.adam)

            saved = self.pose.clone()
            self._graphs[key] = capture(frame)
            self.pose.copy_(saved)
            self.hist[key] = (lh, ph)
        return self._graphs[key]

    def status(self) -> int:
        return int(gs2d.gs2d_track_status(self.ws).item())

    def iterations_run(self) -> int:
        """AdamW steps of the last frame: the iterations before the stop."""
        return int(self.adam[12].item())


def compare_frames(loops: LoopGraphs, propose, proposal_pose, frames, n_iter: int):
    """Plain loop vs proposal + loop, frame by frame.  ``frames``: (gt, load)
    with load(target) writing the frame's observation and its usual start
    pose into the proposer's and the loop's buffers (target 'loop' or
    'proposal'); ``propose``: the proposal's captured graph, whose kept pose
    ends in ``proposal_pose`` [12].
    Per frame:
      * untimed passes find the iteration where the pose first comes within
        1 cm / 0.5 degrees of gt, from the usual start and from the proposal;
      * timed end to end (CUDA events around everything the frame runs):
        the loop cut at that iteration, and the proposal + acceptance + the
        loop cut at its iteration (frames already within the threshold after
        the proposal run no loop);
      * timed under the stop rule (|tau| < STOP_TOL or STOP_ITERS
        iterations): both arms, with the iterations run and the error at
        the stop.
    The GT-based cut needs the untimed pass; the stop-rule frames are what a
    tracker without ground truth runs."""
    g_full = loops.graph(n_iter)
    g_stop = loops.graph(STOP_ITERS, STOP_TOL)
    ph_full = loops.hist[(n_iter, 0.0)][1]
    res = {k: [] for k in ("plain_it", "learned_it", "prop", "accepted", "plain_ms", "learned_ms",
                           "prop_ms", "iter_ms", "stop_plain_ms", "stop_learned_ms",
                           "stop_plain_it", "stop_learned_it", "stop_plain_err",
                           "stop_learned_err")}
    for gt, load, accepted in frames:
        # untimed: iterations to the threshold from both starts
        load("loop")
        res["iter_ms"].append(timed_ms(g_full.replay) / n_iter)
        if loops.status() not in (0, gs2d.CONVERGED):
            raise gs2d.Gs2dError("tracking status")
        k_plain = first_below(ph_full.cpu().numpy(), gt)
        load("proposal")
        res["prop_ms"].append(timed_ms(propose.replay))
        res["accepted"].append(int(accepted().item()))
        start = proposal_pose.clone()
        e = pose_error(start.cpu().numpy(), gt)
        res["prop"].append(e)
        if e[0] < 0.01 and e[1] < 0.5:
            k_learned = 0
        else:
            loops.pose.copy_(start)
            g_full.replay()
            k_learned = first_below(ph_full.cpu().numpy(), gt)
        res["plain_it"].append(k_plain)
        res["learned_it"].append(k_learned)
        # timed end to end: the loop cut where it reaches the threshold
        kp = n_iter if k_plain is None else k_plain
        kl = n_iter if k_learned is None else k_learned
        gp = loops.graph(kp) if kp > 0 else None
        gl = loops.graph(kl) if kl > 0 else None
        load("loop")
        res["plain_ms"].append(timed_ms(gp.replay) if gp is not None else 0.0)
        load("proposal")

        def learned():
            propose.replay()
            if gl is not None:
                loops.pose.copy_(proposal_pose)
                gl.replay()

        res["learned_ms"].append(timed_ms(learned))
        # timed under the stop rule
        load("loop")
        res["stop_plain_ms"].append(timed_ms(g_stop.replay))
        res["stop_plain_it"].append(loops.iterations_run())
        res["stop_plain_err"].append(pose_error(loops.pose.cpu().numpy(), gt))
        load("proposal")

        def learned_stop():
            propose.replay()
            loops.pose.copy_(proposal_pose)
            g_stop.replay()

        res["stop_learned_ms"].append(timed_ms(learned_stop))
        res["stop_learned_it"].append(loops.iterations_run())
        res["stop_learned_err"].append(pose_error(loops.pose.cpu().numpy(), gt))
        if loops.status() not in (0, gs2d.CONVERGED):
            raise gs2d.Gs2dError("tracking status")
    return res


def summarize_frames(res, n_iter: int) -> dict:
    """Medians of compare_frames: the timed frames are the primary numbers;
    the composite (median proposal time + iterations x median iteration
    time) is kept beside them."""
    cap_it = lambda v: n_iter if v is None else v
    ms_iter = float(np.median(res["iter_ms"]))
    ms_prop = float(np.median(res["prop_ms"]))
    plain_c = np.array([cap_it(v) * ms_iter for v in res["plain_it"]])
    learned_c = np.array([ms_prop + cap_it(v) * ms_iter for v in res["learned_it"]])
    pm, lm = np.array(res["plain_ms"]), np.array(res["learned_ms"])
    pp = np.array(res["prop"])
    sp, sl = np.array(res["stop_plain_err"]), np.array(res["stop_learned_err"])
    reach = lambda e: int(np.sum((e[:, 0] < 0.01) & (e[:, 1] < 0.5)))
    return {
        "frames": len(pm),
        "ms_per_iter": ms_iter,
        "proposal_ms": ms_prop,
        "timing": "each frame timed end to end on the device (CUDA events around the proposal "
                  "graph, the acceptance and the loop graph cut at the iteration an untimed pass "
                  "found within 1 cm / 0.5 deg of ground truth)",
        "plain": {"ms_to_1cm_0.5deg_median": float(np.median(pm)), "ms_mean": float(np.mean(pm)),
                  "iters_median": float(np.median([cap_it(v) for v in res["plain_it"]])),
                  "reached": int(sum(v is not None for v in res["plain_it"]))},
        "learned": {"ms_to_1cm_0.5deg_median": float(np.median(lm)), "ms_mean": float(np.mean(lm)),
                    "iters_median": float(np.median([cap_it(v) for v in res["learned_it"]])),
                    "reached": int(sum(v is not None for v in res["learned_it"])),
                    "accepted_frac": float(np.mean(res["accepted"]))},
        "speedup_median": float(np.median(pm) / max(np.median(lm), 1e-9)),
        "composite": {"plain_ms_median": float(np.median(plain_c)),
                      "learned_ms_median": float(np.median(learned_c)),
                      "note": "proposal median + iterations x median iteration time"},
        "stop_rule": {"n_iter": STOP_ITERS, "stop_tol": STOP_TOL,
                      "plain": {"ms_median": float(np.median(res["stop_plain_ms"])),
                                "iters_median": float(np.median(res["stop_plain_it"])),
                                "err_cm_median": float(np.median(sp[:, 0]) * 100),
                                "err_deg_median": float(np.median(sp[:, 1])),
                                "within_1cm_0.5deg": reach(sp)},
                      "learned": {"ms_median": float(np.median(res["stop_learned_ms"])),
                                  "iters_median": float(np.median(res["stop_learned_it"])),
                                  "err_cm_median": float(np.median(sl[:, 0]) * 100),
                                  "err_deg_median": float(np.median(sl[:, 1])),
                                  "within_1cm_0.5deg": reach(sl)}},
        "proposal_err_median_cm_deg": [float(np.median(pp[:, 0]) * 100), float(np.median(pp[:, 1]))],
    }


def evaluate(scene, params, n_frames: int, seed: int, n_iter: int = 100, device="cuda",
             passes: int = 1):
    """Plain loop vs proposal + loop on held-out frames of one room
    (compare_frames): per frame the iterations and the end-to-end device
    time to 1 cm / 0.5 degrees, the frames under the stop rule, and the
    proposal's own error."""
    ds = gs2d.DeviceSurfels(scene)
    vr = ViewRenderer(ds)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    gts, inits = [], []
    obs_rgb = torch.empty(n_frames, 120, 160, 3, device=device)
    obs_d = torch.empty(n_frames, 120, 160, device=device)
    kmax = 0
    for c0 in range(0, n_frames, VIEWS):
        cnt = min(VIEWS, n_frames - c0)
        k = seed * 10_000_000 + c0
        g = [scenes.room_pose(k + j) for j in range(cnt)]
        it = [scenes.perturb_uniform(p, MAX_T, MAX_DEG, k + j) for j, p in enumerate(g)]
        img = vr.render(poses_tensor(g, device))
        obs_rgb[c0:c0 + cnt] = img["rgb"][:cnt]
        obs_d[c0:c0 + cnt] = observed_depth(img["depth"][:cnt], img["opacity"][:cnt], gen)
        vr.render(poses_tensor(it, device))
        kmax = max([kmax] + [int(b["n_isect"].item()) for b in vr.br.keep])
        gts += g
        inits += it
    del vr
    cap = 4 * kmax + 4096
    # the proposal, one frame per replay
    pr = Proposer(ds, params, cap, device, passes=passes)
    pr.pose.copy_(poses_tensor(inits[:1], device))
    pr.obs_rgb.copy_(obs_rgb[0])
    pr.obs_d.copy_(obs_d[0])
    pg = capture(pr.run)
    # the plain loop, one frame per replay
    t_rgb = torch.empty(120, 160, 3, device=device)
    t_d = torch.empty(120, 160, device=device)
    loops = LoopGraphs(ds, CAM, cap, t_rgb, t_d, device)
    init_t = poses_tensor(inits, device)
    st = np.array([pose_error(init_t[f].cpu().numpy(), gts[f]) for f in range(n_frames)])

    def frame(f):
        def load(target):
            t_rgb.copy_(obs_rgb[f])
            t_d.copy_(obs_d[f])
            pr.obs_rgb.copy_(obs_rgb[f])
            pr.obs_d.copy_(obs_d[f])
            if target == "loop":
                loops.pose.copy_(init_t[f])
            else:
                pr.pose.copy_(init_t[f:f + 1])
        return gts[f], load, lambda: pr.accepted

    res = compare_frames(loops, pg, pr.pose[0], (frame(f) for f in range(n_frames)), n_iter)
    if pr.status() != 0:
        raise gs2d.Gs2dError(f"proposal render status {pr.status()}")
    out = summarize_frames(res, n_iter)
    out["start_err_median_cm_deg"] = [float(np.median(st[:, 0]) * 100), float(np.median(st[:, 1]))]
    out["proposal_passes"] = passes
    return out


def low_res_camera(cam, factor: int):
    """The network's camera for a full-resolution one: intrinsics and size
    divided by ``factor`` (the pixel grid of gs2d_net_downsample_rgbd)."""
    return scenes.Camera(cam.fx / factor, cam.fy / factor, cam.cx / factor, cam.cy / factor,
                         cam.width // factor, cam.height // factor)


def evaluate_full_res(surf: gs2d.DeviceSurfels, params, cam, frames, passes: int = 2,
                      n_iter: int = 100, device="cuda"):
    """Tracking at full resolution from the network's proposal: per frame the
    observation (full-resolution RGB-D) is box-downsampled to the network's
    160x120 view, the proposal (``passes`` passes with the acceptance test)
    runs at that resolution, and the full-resolution plain loop refines the
    kept pose; against the plain loop from the usual start.  ``frames``:
    dicts with gt (Pose), start_t [12], obs_rgb [H, W, 3], obs_depth [H, W]
    on the device.  Reports what compare_frames measures."""
    factor = cam.width // 160
    lo = low_res_camera(cam, factor)
    cap = 8 * surf.n
    pr = Proposer(surf, params, cap, device, passes=passes, cam=lo)
    obs_rgb = torch.empty(cam.height, cam.width, 3, device=device)
    obs_d = torch.empty(cam.height, cam.width, device=device)

    def propose():
        gs2d.gs2d_net_downsample_rgbd(obs_rgb, obs_d, factor, pr.obs_rgb, pr.obs_d)
        pr.run()

    pr.pose.copy_(frames[0]["start_t"][None])
    obs_rgb.copy_(frames[0]["obs_rgb"])
    obs_d.copy_(frames[0]["obs_depth"])
    pg = capture(propose)
    loops = LoopGraphs(surf, cam, cap, obs_rgb, obs_d, device)

    def frame(fr):
        def load(target):
            obs_rgb.copy_(fr["obs_rgb"])
            obs_d.copy_(fr["obs_depth"])
            if target == "loop":
                loops.pose.copy_(fr["start_t"])
            else:
                pr.pose.copy_(fr["start_t"][None])
        return fr["gt"], load, lambda: pr.accepted

    res = compare_frames(loops, pg, pr.pose[0], (frame(fr) for fr in frames), n_iter)
    if pr.status() != 0:
        raise gs2d.Gs2dError(f"proposal render status {pr.status()}")
    out = summarize_frames(res, n_iter)
    out["proposal_passes"] = passes
    out["network_camera"] = [lo.fx, lo.fy, lo.cx, lo.cy, lo.width, lo.height]
    return out

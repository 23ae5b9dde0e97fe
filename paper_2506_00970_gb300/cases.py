"""Small fixed workloads of the hot path, one per command, for profilers
(ncu) and quick timing:  python -m paper_2506_00970_gb300.cases <case> [reps]

  track    tracking frames: 200k-surfel room, 640x480, 10 iterations each
  track_small  tracking frames of the learned-proposal workload: 200k-surfel
           room, 160x120, fx=fy=150, 10 iterations each
  mapping  a batched mapping step: 300k-surfel room, 4 keyframes at 1200x680
           (project, bin_sort, persistent forward, mapping loss, persistent
           backward + per-surfel reductions)
  uneven   a batched step over 8 views of mixed resolution with active
           subsets of a 1M-surfel room
  uneven32 the same over 32 views of a 2M-surfel room (active subsets of
           50k-1M surfels: more views than side streams, so the binning runs
           one launch per stage over all views)
  net      the proposal network at batch 256: forward, then forward + loss +
           backward (gs2d_net_grad) + AdamW
  sort     bin_sort of a 200k-surfel room at 160x120 (long tile segments)
  contrib  per-surfel contributions (gs2d_render_contrib) of a 200k-surfel room
           at 640x480
  ssim     the SSIM term with its gradient (gs2d_ssim_loss) at 1200x680
  proposal one frame's learned pose proposal at 160x120 (two passes: render,
           tracking loss, network at batch 1, render at the proposal, loss,
           acceptance), replayed as a CUDA graph; random network weights
  map      map-state passes on a 2M-surfel map (state update, correction by 64
           keyframe increments, pruning, compaction) and the expansion of a
           1200x680 RGB-D keyframe (downsampling 0.04) against a voxel table

Each case runs ``reps`` times (default 3) after one warm-up and prints the
mean device time per repetition (CUDA events).  An optional third argument
sets the pixels per thread of the rendering cases (1, 2 or 4; the tile is the
first shape of that count).
"""
from __future__ import annotations

import sys

import numpy as np
import torch

from . import build as _build
from . import gs2d, scenes


def _timed(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def case_track(reps, px=1, cam=None):
    s = scenes.room_scene(0, 200_000)
    cam = cam or scenes.tracking_camera()
    ds = gs2d.DeviceSurfels(s)
    tile = gs2d.TILE_SHAPES[px][0]
    r = gs2d.Rasterizer(cam, ds.n, tile=tile, px=px)
    gt = scenes.room_pose(100)
    out = r.forward(ds, gs2d.pose_tensor(gt))
    obs_rgb = out["rgb"].clone()
    obs_d = out["depth"] / out["opacity"].clamp_min(1e-6)
    start = gs2d.pose_tensor(scenes.perturb_pose(gt, 0.02, 1.0, seed=5))
    ccam, cfg = gs2d.camera(cam), gs2d.default_config(tile, px)
    prm = gs2d.default_track_params(stop_tol=0.0)
    cap = 8 * ds.n
    ws = torch.empty(gs2d.gs2d_track_workspace(ds.n, cap, ccam, cfg), dtype=torch.uint8, device="cuda")
    pose = torch.empty(12, device="cuda")

    def run():
        pose.copy_(start)
        gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, 10, cap, None, None, ws)

    return _timed(run, reps)


def _batch(s, cams, poses, actives, reps, px=1):
    ds = gs2d.DeviceSurfels(s)
    br = gs2d.BatchRasterizer(cams, ds.n, actives=actives, px=px)
    br.set_poses(poses)
    br.fit(ds)
    br.forward(ds)
    obs = [(b["rgb"].clone(), b["depth"] / b["opacity"].clamp_min(1e-6) + 0.01) for b in br.keep]
    loss = torch.zeros(len(cams), device="cuda")
    lviews = gs2d.loss_views([(b["ccam"], b["rgb"], b["depth"], b["normal"], b["opacity"],
                               obs[v][0], obs[v][1], b["d_rgb"], b["d_depth"], b["d_normal"],
                               b["d_opacity"]) for v, b in enumerate(br.keep)])
    lws = torch.empty(gs2d.gs2d_mapping_loss_batch_workspace(lviews), dtype=torch.uint8,
                      device="cuda")

    def run():
        br.forward(ds, check_status=False)
        gs2d.gs2d_mapping_loss_batch(lviews, 0.5, 0.02, loss, lws)
        br.backward(ds)

    return _timed(run, reps)


def case_mapping(reps, px=1):
    s = scenes.room_scene(1, 300_000)
    poses = scenes.room_trajectory(2, 4)
    return _batch(s, [scenes.mapping_camera()] * 4, poses, None, reps, px)


def case_uneven(reps, px=1):
    s = scenes.room_scene(3, 1_000_000)
    cams, poses, actives = scenes.uneven_batch(4, s, 8, sizes=(50_000, 500_000))
    return _batch(s, cams, poses, actives, reps, px)


def case_uneven32(reps, px=1):
    s = scenes.room_scene(3, 2_000_000)
    cams, poses, actives = scenes.uneven_batch(4, s, 32)
    return _batch(s, cams, poses, actives, reps, px)


def case_net(reps, px=1):
    B = 256
    params = torch.tensor(scenes.net_init(0, gs2d.net_init_blocks()), device="cuda")
    n = params.numel()
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.uniform(-1, 1, (B, 120, 160, 8)), dtype=torch.float32,
                     device="cuda").to(torch.bfloat16)
    t = torch.tensor(rng.normal(0, 1, (B, 6)), dtype=torch.float32, device="cuda")
    ws = torch.empty(gs2d.gs2d_net_workspace(B), dtype=torch.uint8, device="cuda")
    y = torch.empty(B, 6, device="cuda")
    grad = torch.empty(n, device="cuda")
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    loss = torch.empty(1, device="cuda")
    step = [0]

    def run():
        gs2d.gs2d_net_forward(params, x, y, ws)
        gs2d.gs2d_net_grad(params, x, t, loss, grad, ws)
        step[0] += 1
        gs2d.gs2d_net_adamw(params, grad, m, v, step[0], lr=1e-4)

    return _timed(run, reps)


def case_sort(reps, px=1):
    s = scenes.room_scene(100, 200_000)
    cam = scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120)
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, ds.n, capacity=4 * ds.n)
    r.project(ds, gs2d.pose_tensor(scenes.room_pose(3)))
    return _timed(lambda: r.bin_sort(grow=False), reps)


def case_contrib(reps, px=1):
    s = scenes.room_scene(0, 200_000)
    cam = scenes.tracking_camera()
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, ds.n, tile=gs2d.TILE_SHAPES[px][0], px=px)
    r.forward(ds, gs2d.pose_tensor(scenes.room_pose(1)))
    out = torch.empty(ds.n, device="cuda")
    return _timed(lambda: r.contribution(out=out), reps)


def case_ssim(reps, px=1):
    rng = np.random.default_rng(0)
    h, w = 680, 1200
    y = torch.tensor(rng.uniform(size=(h, w, 3)), dtype=torch.float32, device="cuda")
    x = (y + 0.1 * torch.randn_like(y)).clamp(0, 1)
    g = torch.zeros_like(x)
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(gs2d.gs2d_ssim_workspace(h, w), dtype=torch.uint8, device="cuda")
    return _timed(lambda: gs2d.gs2d_ssim_loss(x, y, h, w, 0.125, g, loss, ws), reps)


def case_track_small(reps, px=1):
    return case_track(reps, px, scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120))


def case_map(reps, px=1):
    n, n_kf = 2_000_000, 64
    rng = np.random.default_rng(0)
    f = dict(dtype=torch.float32, device="cuda")
    T = lambda a: torch.tensor(a, device="cuda")
    mu = T(rng.uniform([-2.5, -2.0, 0.0], [2.5, 2.0, 3.0], (n, 3)).astype(np.float32))
    ds = gs2d.DeviceSurfels.from_tensors(mu, T(rng.normal(size=(n, 4)).astype(np.float32)),
                                         torch.full((n, 2), 0.02, **f), torch.full((n,), 0.9, **f),
                                         torch.rand(n, 3, **f))
    contrib = T(rng.choice(np.float32([0.0, 0.3, 0.7, 2.0]), n))
    st = gs2d.DeviceMapState.from_tensors(torch.ones(n, dtype=torch.uint8, device="cuda"),
                                          T(rng.integers(0, n_kf, n).astype(np.int32)),
                                          torch.full((n,), 2.5, **f),
                                          T(rng.integers(40, n_kf, n).astype(np.int32)))
    out = gs2d.DeviceSurfels.from_tensors(*(torch.empty_like(t) for t in (
        ds.mu, ds.quat, ds.scale, ds.opacity, ds.rgb)))
    st_o = gs2d.DeviceMapState.from_tensors(*(torch.empty_like(t) for t in (
        st.delta, st.t_c, st.d_c, st.t_l)))
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    kws = torch.empty(gs2d.gs2d_map_compact_workspace(n), dtype=torch.uint8, device="cuda")
    po = T(np.concatenate([np.r_[np.eye(3).ravel(), rng.normal(size=3)]
                           for _ in range(n_kf)]).astype(np.float32))
    pn = po + 1e-3
    cws = torch.empty(gs2d.gs2d_map_correct_workspace(n_kf), dtype=torch.uint8, device="cuda")
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    prm = gs2d.StateParams(0.5, 20, 0, -1)
    pose = gs2d.pose_tensor(scenes.identity_pose())
    cam = scenes.Camera(600.0, 600.0, 600.0, 340.0, 1200, 680)
    rgb, dep = scenes.rgbd_frame(21, cam)
    rgb, dep = T(rgb), T(dep)
    u_keep, u_ang = torch.rand(680, 1200, **f), torch.rand(680, 1200, **f)
    table = gs2d.DeviceVoxelTable(1 << 22, 0.02)
    table.insert(mu[:1_000_000])
    new_s = gs2d.DeviceSurfels.from_tensors(torch.empty(cam.width * cam.height, 3, **f),
                                            torch.empty(cam.width * cam.height, 4, **f),
                                            torch.empty(cam.width * cam.height, 2, **f),
                                            torch.empty(cam.width * cam.height, **f),
                                            torch.empty(cam.width * cam.height, 3, **f))
    n_new = torch.zeros(1, dtype=torch.int32, device="cuda")
    ews = torch.empty(gs2d.gs2d_expand_workspace(gs2d.camera(cam)), dtype=torch.uint8,
                      device="cuda")
    eprm = gs2d.ExpandParams(0.04, 0.99, 0.05, 9, 0)

    def run():
        gs2d.gs2d_map_observe(contrib, ds.mu, n, pose, n_kf, prm, st, counts)
        gs2d.gs2d_map_correct(ds.mu, ds.quat, st.t_c, n, po, pn, n_kf, cws)
        gs2d.gs2d_map_prune(contrib, st.t_c, n, 7, 0.5, keep)
        gs2d.gs2d_map_compact(keep, n, ds, st, out, st_o, None, n_out, kws)
        gs2d.gs2d_expand(rgb, dep, gs2d.camera(cam), pose, u_keep, u_ang, table, eprm, 0,
                         cam.width * cam.height, new_s, None, n_new, ews)

    return _timed(run, reps)


def case_proposal(reps, px=1):
    from . import proposal
    s = scenes.room_scene(200, 200_000)
    ds = gs2d.DeviceSurfels(s)
    params = torch.tensor(scenes.net_init(0, gs2d.net_init_blocks()), device="cuda")
    pr = proposal.Proposer(ds, params, 8 * ds.n, passes=2)
    gt = scenes.room_pose(5)
    pr.pose.copy_(proposal.poses_tensor([scenes.perturb_pose(gt, 0.03, 2.0, seed=1)]))
    img = proposal.ViewRenderer(ds).render(proposal.poses_tensor([gt]))
    pr.obs_rgb.copy_(img["rgb"][0])
    pr.obs_d.copy_(img["depth"][0] / img["opacity"][0].clamp_min(1e-6))
    g = proposal.capture(pr.run)
    return _timed(g.replay, reps)


CASES = {"track": case_track, "track_small": case_track_small, "mapping": case_mapping, "uneven": case_uneven,
         "uneven32": case_uneven32, "net": case_net,
         "sort": case_sort, "contrib": case_contrib,
         "ssim": case_ssim, "map": case_map, "proposal": case_proposal}


def main(argv):
    if len(argv) < 1 or argv[0] not in CASES:
        print(__doc__)
        return 2
    reps = int(argv[1]) if len(argv) > 1 else 3
    px = int(argv[2]) if len(argv) > 2 else 1
    _build.build()
    ms = CASES[argv[0]](reps, px)
    print(f"{argv[0]} (px {px}): {ms:.3f} ms per repetition")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))

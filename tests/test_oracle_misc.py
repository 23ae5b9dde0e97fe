"""Pins of the oracle's binning/sorting, SE(3) maps, AdamW, losses and the
tracking loop (no GPU).

* bin_sort: a brute-force per-tile list, sorted by (depth, id), "sorts them
  by depth" (Sec. III-A);
* tile_rects: every pixel a surfel touches lies in its rectangle;
* se3_exp / se3_log: the 4x4 matrix exponential (scipy.linalg.expm) and the
  round trip (Sec. III-B manifold derivative);
* adamw_step: torch.optim.AdamW, the optimiser named in Sec. III-D;
* tracking_loss / mapping_loss: closed forms on constant images
  (Eq. tracking_loss, normal_mask, opacity_mask; Sec. III-E);
* normal_from_depth: a plane's normal (Eq. normal_fromD);
* tracking loop: zero loss and gradient at ground truth; convergence from a
  2 cm / 1 degree perturbation to 1 cm / 0.5 degree (Sec. III-D).
"""

import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes


def test_bin_sort_matches_per_tile_lists(orc):
    tx, ty = 7, 5
    rect, depth, count = scenes.random_tile_records(3, 400, tx, ty)
    keys, vals, ranges = orc.bin_sort(rect, depth, tx, ty)
    assert len(vals) == count.sum()
    bits = depth.view(np.uint32)
    for t in range(tx * ty):
        cx, cy = t % tx, t // tx
        ids = [i for i in range(len(rect)) if rect[i, 0] <= cx <= rect[i, 2] and rect[i, 1] <= cy <= rect[i, 3]]
        ids.sort(key=lambda i: (float(depth[i]), i))
        s, e = ranges[t]
        assert list(vals[s:e]) == ids
        assert all(int(k) >> 32 == t for k in keys[s:e])
        assert all(int(k) & 0xFFFFFFFF == bits[i] for k, i in zip(keys[s:e], ids))


def test_bin_sort_ties_keep_id_order(orc):
    rect = np.array([[0, 0, 1, 0]] * 4, np.int32)
    depth = np.array([2.0, 1.0, 2.0, 1.0], np.float32)
    _, vals, ranges = orc.bin_sort(rect, depth, 2, 1)
    assert list(vals) == [1, 3, 0, 2, 1, 3, 0, 2]
    assert ranges.tolist() == [[0, 4], [4, 8]]


def test_tile_rects_cover_every_touched_pixel(orc):
    s = scenes.slab_scene(9, 120)
    s.scale *= 3
    cam = scenes.Camera(60.0, 60.0, 40.0, 30.0, 80, 60)
    rule = orc.Rule()
    tile = (16, 16)
    rect, depth = orc.tile_rects(s, cam, scenes.identity_pose(), rule, tile)
    touched = 0
    for i in range(s.n):
        out = orc.render(s.subset(np.array([i])), cam, scenes.identity_pose(), rule)
        ys, xs = np.nonzero(out["opacity"] > 0)
        if len(xs) == 0:
            continue
        touched += 1
        r = rect[i]
        assert r[0] <= r[2] and r[1] <= r[3]
        assert np.all(xs // tile[0] >= r[0]) and np.all(xs // tile[0] <= r[2])
        assert np.all(ys // tile[1] >= r[1]) and np.all(ys // tile[1] <= r[3])
        # tight: the rectangle is at most one tile larger than the touched set on each side
        assert r[0] >= xs.min() // tile[0] - 1 and r[2] <= xs.max() // tile[0] + 1
    assert touched > 60
    np.testing.assert_allclose(depth, s.mu[:, 2])


def test_se3_exp_matches_matrix_exponential(orc):
    from scipy.linalg import expm
    rng = np.random.default_rng(0)
    for scale in (1e-7, 1e-3, 0.3, 2.0):
        tau = rng.normal(size=6) * scale
        X = np.zeros((4, 4))
        X[:3, :3] = orc.hat(tau[3:])
        X[:3, 3] = tau[:3]
        E = expm(X)
        R, t = orc.se3_exp(tau)
        np.testing.assert_allclose(R, E[:3, :3], atol=1e-13)
        np.testing.assert_allclose(t, E[:3, 3], atol=1e-13)
        np.testing.assert_allclose(orc.se3_log(R, t), tau, atol=1e-10, rtol=1e-9)


def test_adamw_matches_torch(orc):
    import torch
    rng = np.random.default_rng(1)
    p = rng.normal(size=6)
    tp = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.AdamW([tp], lr=3e-3, betas=(0.8, 0.99), eps=1e-7, weight_decay=0.05)
    st = orc.AdamState(np.zeros(6), np.zeros(6))
    for _ in range(7):
        g = rng.normal(size=6)
        tp.grad = torch.tensor(g)
        opt.step()
        p = orc.adamw_step(p, g, st, lr=3e-3, betas=(0.8, 0.99), eps=1e-7, wd=0.05)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def _const_images(h, w, rgb, depth, normal, opacity):
    return dict(rgb=np.full((h, w, 3), rgb), depth=np.full((h, w), depth * opacity),
                normal=np.tile(np.asarray(normal, float), (h, w, 1)), opacity=np.full((h, w), opacity))


def test_tracking_loss_closed_forms(orc):
    cam = scenes.Camera(50.0, 50.0, 6.0, 4.0, 12, 8)
    h, w = cam.height, cam.width
    I = np.full((h, w, 3), 0.3)
    D = np.full((h, w), 2.0)
    img = _const_images(h, w, 0.5, 2.5, (0, 0, 1), 0.98)
    L, g = orc.tracking_loss(img, I, D, cam, lambda_d=0.7)
    assert L == pytest.approx(3 * 0.2 + 0.7 * 0.5, rel=1e-12)
    np.testing.assert_allclose(g["rgb"], 1.0 / (h * w))
    # D_hat = D / O: d/dD = 1/O, d/dO = -D/O^2
    np.testing.assert_allclose(g["depth"], 0.7 / 0.98 / (h * w), rtol=1e-12)
    np.testing.assert_allclose(g["opacity"], -0.7 * 2.5 * 0.98 / 0.98 ** 2 / (h * w), rtol=1e-12)
    np.testing.assert_allclose(g["normal"], 0.0)
    # opacity mask: O <= 0.95 contributes nothing
    L, g = orc.tracking_loss(_const_images(h, w, 0.5, 2.5, (0, 0, 1), 0.95), I, D, cam)
    assert L == 0 and np.all(g["rgb"] == 0)
    # normal mask: a normal facing the camera (N . r < 0) contributes nothing
    L, _ = orc.tracking_loss(_const_images(h, w, 0.5, 2.5, (0, 0, -1), 0.99), I, D, cam)
    assert L == 0
    # literal depth mode (no division by O)
    L, g = orc.tracking_loss(img, I, D, cam, lambda_d=1.0, depth_mode=0)
    assert L == pytest.approx(3 * 0.2 + abs(2.5 * 0.98 - 2.0), rel=1e-12)


def test_normal_from_depth_of_plane(orc):
    cam = scenes.Camera(40.0, 45.0, 10.0, 8.0, 20, 16)
    n = np.array([0.2, -0.3, 1.0])
    n /= np.linalg.norm(n)
    x = np.arange(cam.width) + 0.5
    y = np.arange(cam.height) + 0.5
    X, Y = np.meshgrid(x, y)
    r = np.stack([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, np.ones_like(X)], -1)
    depth = 2.0 / (r @ n)            # plane n . X = 2 (the camera looks at its back)
    ND, valid = orc.normal_from_depth(depth, cam)
    ND = ND.numpy()
    valid = valid.numpy()
    assert valid[1:-1, 1:-1].all() and not valid[0].any() and not valid[:, -1].any()
    np.testing.assert_allclose(ND[valid], np.broadcast_to(n, ND[valid].shape), atol=1e-12)


def test_mapping_loss_of_consistent_plane(orc):
    cam = scenes.Camera(40.0, 40.0, 8.0, 6.0, 16, 12)
    n = np.array([0.0, 0.2, 1.0])
    n /= np.linalg.norm(n)
    x = np.arange(cam.width) + 0.5
    y = np.arange(cam.height) + 0.5
    X, Y = np.meshgrid(x, y)
    r = np.stack([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, np.ones_like(X)], -1)
    depth = 1.5 / (r @ n)
    img = dict(rgb=np.full((12, 16, 3), 0.4), depth=depth, normal=np.tile(n, (12, 16, 1)),
               opacity=np.ones((12, 16)))
    L, g = orc.mapping_loss(img, np.full((12, 16, 3), 0.4), depth, cam)
    assert L == pytest.approx(0.0, abs=1e-12)
    # misaligned normal: L_n = 1 - n'.n on the 10x14 interior
    img["normal"] = np.tile(np.array([0.0, 0.0, 1.0]), (12, 16, 1))
    L, _ = orc.mapping_loss(img, np.full((12, 16, 3), 0.4), depth, cam, w_d=0.5, w_n=0.02)
    assert L == pytest.approx(0.02 * (1 - n[2]) * 10 * 14 / (12 * 16), rel=1e-10)


def test_mapping_loss_gradient_fd(orc):
    rng = np.random.default_rng(2)
    cam = scenes.Camera(30.0, 30.0, 5.0, 4.0, 10, 8)
    img = dict(rgb=rng.uniform(size=(8, 10, 3)), depth=rng.uniform(1.5, 1.6, (8, 10)),
               normal=rng.normal(size=(8, 10, 3)), opacity=rng.uniform(0.7, 1.0, (8, 10)))
    I = rng.uniform(size=(8, 10, 3))
    D = rng.uniform(1.0, 2.0, (8, 10))
    _, g = orc.mapping_loss(img, I, D, cam)
    h = 1e-7
    for key in ("depth", "normal", "opacity"):
        arr = img[key]
        for idx in [(3, 4), (1, 1), (6, 8)]:
            idx = idx + ((1,) if arr.ndim == 3 else ())
            old = arr[idx]
            arr[idx] = old + h
            lp, _ = orc.mapping_loss(img, I, D, cam)
            arr[idx] = old - h
            lm, _ = orc.mapping_loss(img, I, D, cam)
            arr[idx] = old
            assert g[key][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def _small_room(seed=0):
    s = scenes.room_scene(seed, n=6000, scale_cm=(4.0, 7.0))
    cam = scenes.Camera(60.0, 60.0, 32.0, 24.0, 64, 48)
    gt = scenes.room_pose(seed + 1)
    return s, cam, gt


def test_tracking_zero_at_ground_truth(orc):
    s, cam, gt = _small_room()
    img = orc.render(s, cam, gt)
    L, g = orc.tracking_loss(img, img["rgb"], img["depth"] / np.maximum(img["opacity"], 1e-6), cam)
    assert L == 0.0
    gr = orc.render_bwd(s, cam, gt, g["rgb"], g["depth"], g["normal"], g["opacity"])
    assert np.all(gr["pose6"] == 0.0)


@pytest.mark.slow
def test_tracking_converges_from_perturbation(orc):
    s, cam, gt = _small_room()
    img = orc.render(s, cam, gt)
    obs_d = img["depth"] / np.maximum(img["opacity"], 1e-6)
    start = scenes.perturb_pose(gt, 0.02, 1.0, seed=5)
    e0 = orc.pose_error(start, gt)
    assert e0[0] > 0.015 and e0[1] > 0.9
    pose, losses = orc.track(s, cam, start, img["rgb"], obs_d, n_iter=100, lr=1e-3)
    et, er = orc.pose_error(pose, gt)
    assert et < 0.01 and er < 0.5, (e0, (et, er), losses[:3], losses[-3:])


def test_tile_rects_cover_surfels_reaching_past_the_camera_plane(orc):
    """Large surfels beside the camera whose discs reach behind it: the
    clipped-disc footprint still covers every pixel they touch, and is far
    smaller than the image."""
    rng = np.random.default_rng(4)
    n = 40
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.3, 0.3, n), rng.uniform(0.06, 0.2, n)], 1)
    q = rng.normal(size=(n, 4))
    s = scenes.Surfels(mu, q, rng.uniform(0.05, 0.15, (n, 2)), rng.uniform(0.5, 0.95, n),
                       rng.uniform(size=(n, 3)))
    cam = scenes.Camera(60.0, 60.0, 40.0, 30.0, 80, 60)
    rect, _ = orc.tile_rects(s, cam, scenes.identity_pose(), orc.Rule(), (8, 8))
    covered = 0
    for i in range(n):
        out = orc.render(s.subset(np.array([i])), cam, scenes.identity_pose())
        ys, xs = np.nonzero(out["opacity"] > 0)
        if len(xs) == 0:
            continue
        covered += 1
        r = rect[i]
        assert r[0] <= xs.min() // 8 and r[2] >= xs.max() // 8
        assert r[1] <= ys.min() // 8 and r[3] >= ys.max() // 8
    assert covered > 10


def test_active_subset_is_the_nearest_ball():
    """The active-map subset of a view holds exactly the requested number of
    surfels, sorted, and every chosen surfel is at least as close to the
    point ahead of the camera as every surfel left out."""
    s = scenes.room_scene(5, 20_000)
    pose = scenes.room_pose(7)
    ids = scenes.active_subset(s, pose, 3000, reach=1.5)
    assert ids.dtype == np.int32 and len(ids) == 3000 and np.all(np.diff(ids) > 0)
    eye = -pose.R.T @ pose.t
    ahead = eye + 1.5 * pose.R[2]
    d = np.linalg.norm(s.mu - ahead, axis=1)
    out = np.setdiff1d(np.arange(s.n), ids)
    assert d[ids].max() <= d[out].min()
    cams, poses, acts = scenes.uneven_batch(1, s, n_views=6, sizes=(500, 5000))
    assert len(cams) == len(poses) == len(acts) == 6
    assert all(500 <= len(a) <= 5000 for a in acts)
    assert {(c.width, c.height) for c in cams} <= {(320, 240), (640, 480), (1200, 680)}

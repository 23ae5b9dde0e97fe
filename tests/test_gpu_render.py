"""GPU parity of the CUDA rasterizer (through the C ABI) against the FP64 oracle.

* gs2d_bin_sort: bit-exact keys, surfel order and tile ranges against the
  oracle's library stable sort, on synthetic tile records (empty, one,
  ragged multi-chunk, two-pass tile ids, large);
* gs2d_project: tile rectangles against the oracle's FP64 footprint (equal
  up to tile-boundary ties) and the centre depth;
* gs2d_render_fwd: images within 1e-4 abs (colour, opacity) and 1e-4 rel
  (depth, normal) on the 4,096-surfel slab (full image, several tiles and a
  ragged last tile row) and on sampled pixels of the 200k-surfel room at
  640x480;
* gs2d_render_bwd: surfel and pose gradients within 1e-3 relative, full
  and tracking (pose-only) modes, deterministic across runs: every element
  of every surfel that the oracle does not flag (a candidate at a pixel with
  a threshold decision within rounding, or seen within ~3 degrees of
  edge-on) within 1e-3 relative plus 2^-17 of the array's scale, no
  exceptions; every surfel within 1e-3 of the array's scale.
"""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes
from gpu_helpers import (assert_grads_close, assert_images_close, gpu_render, grad_rows_ok,
                         records_to_proj, to_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


# ---------------------------------------------------------------------------
# binning / sort
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,tiles_x,tiles_y,seed", [
    (0, 5, 4, 0), (1, 5, 4, 1), (7, 3, 2, 2), (4097, 10, 8, 3),
    (20000, 40, 30, 4), (150_000, 75, 43, 5),
    # a tile grid whose scatter histograms need more than the default
    # 48 KB of shared memory per block (5440 tiles: 1280x1080 at 16x16)
    (30000, 80, 68, 9),
    # long tile segments: ~6k keys (one shared-memory chunk of the long
    # path) and ~40k keys (three chunks, two merge passes) per tile
    (9000, 2, 2, 6), (60000, 2, 2, 7)])
def test_bin_sort_bit_exact(torch_cuda, orc, n, tiles_x, tiles_y, seed):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    if n:
        rect, depth, count = scenes.random_tile_records(seed, n, tiles_x, tiles_y)
    else:
        rect = np.zeros((0, 4), np.int32)
        depth = np.zeros(0, np.float32)
        count = np.zeros(0, np.int32)
    proj, tiles = records_to_proj(torch, rect, depth, count)
    cam = scenes.Camera(100.0, 100.0, 8.0, 8.0, tiles_x * 16 - 5, tiles_y * 16 - 3)
    r = gs2d.Rasterizer(cam, n, capacity=int(count.sum()) + 17, keys=True)
    r.proj.copy_(proj[: r.proj.numel()]) if n else None
    if n:
        r.tiles.copy_(tiles)
    r.bin_sort()
    torch.cuda.synchronize()
    K = int(r.n_isect.item())
    ok, ov, orng = orc.bin_sort(rect, depth, tiles_x, tiles_y) if n else (
        np.zeros(0, np.uint64), np.zeros(0, np.uint32), np.zeros((tiles_x * tiles_y, 2), np.int32))
    assert K == len(ov)
    np.testing.assert_array_equal(r.vals[:K].cpu().numpy().astype(np.uint32), ov)
    np.testing.assert_array_equal(r.keys[:K].cpu().numpy().view(np.uint64), ok)
    # non-empty tiles: identical ranges; an empty tile may sit anywhere (start == end)
    grng = r.ranges.cpu().numpy().reshape(-1, 2)
    nonempty = orng[:, 1] > orng[:, 0]
    np.testing.assert_array_equal(grng[nonempty], orng[nonempty])
    assert np.all(grng[~nonempty, 0] == grng[~nonempty, 1])
    # emission indices: a permutation; each surfel's block is contiguous
    emit = r.emit[:K].cpu().numpy()
    assert np.array_equal(np.sort(emit), np.arange(K))
    off = r.surfel_off.cpu().numpy()
    vals = r.vals[:K].cpu().numpy()
    if K:
        assert np.all(emit >= off[vals]) and np.all(emit < off[vals] + count[vals])


def test_bin_sort_capacity_overflow_reports_needed(torch_cuda, orc):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    rect, depth, count = scenes.random_tile_records(9, 3000, 12, 9)
    proj, tiles = records_to_proj(torch, rect, depth, count)
    cam = scenes.Camera(100.0, 100.0, 8.0, 8.0, 12 * 16, 9 * 16)
    r = gs2d.Rasterizer(cam, 3000, capacity=100)
    r.proj.copy_(proj)
    r.tiles.copy_(tiles)
    r.status.zero_()
    gs2d.gs2d_bin_sort(r.proj, r.tiles, r.n, r.cam, r.cfg, r.sort_ws, r.bins)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 3
    assert int(r.n_isect.item()) == int(count.sum())
    r.bin_sort(grow=True)        # grows the capacity and redoes the sort
    _, ov, _ = orc.bin_sort(rect, depth, 12, 9)
    np.testing.assert_array_equal(r.vals[: len(ov)].cpu().numpy().astype(np.uint32), ov)


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["slab", "room"])
def test_project_rects_and_depth(torch_cuda, orc, which):
    if which == "slab":
        s, cam, pose = scenes.slab_scene(0), scenes.slab_camera(), scenes.identity_pose()
    else:
        s, cam, pose = scenes.room_scene(1, 50_000), scenes.tracking_camera(), scenes.room_pose(2)
    r, ds, pose_t, _ = gpu_render(s, cam, pose)
    proj = r.proj.cpu().numpy().reshape(-1, 32)[: s.n]
    r01 = proj[:, 28].view(np.uint32)
    r23 = proj[:, 29].view(np.uint32)
    g = np.stack([r01 & 0xFFFF, r01 >> 16, r23 & 0xFFFF, r23 >> 16], 1).astype(np.int64)
    o, depth = orc.tile_rects(s, cam, pose)
    g_cull = g[:, 0] > g[:, 2]
    o_cull = o[:, 0] > o[:, 2]
    both = ~g_cull & ~o_cull
    diff = np.abs(g[both] - o[both]).max(1) if both.any() else np.zeros(0)
    # equal except at tile-boundary ties, where they differ by one tile
    assert np.all(diff <= 1)
    assert (diff > 0).sum() <= max(3, 0.005 * both.sum())
    assert (g_cull != o_cull).sum() <= max(3, 0.005 * s.n)
    np.testing.assert_allclose(proj[:, 26], depth, rtol=2e-6, atol=1e-6)
    k = r.tiles.cpu().numpy()[: s.n]
    area = np.where(g_cull, 0, (g[:, 2] - g[:, 0] + 1) * (g[:, 3] - g[:, 1] + 1))
    np.testing.assert_array_equal(k, area)


# ---------------------------------------------------------------------------
# forward
# ---------------------------------------------------------------------------
# tile shapes with 1, 2 and 4 pixels per thread
TILE_PX = [((16, 16), 1), ((16, 32), 2), ((32, 16), 2), ((64, 8), 2), ((32, 24), 3), ((64, 12), 3),
           ((32, 32), 4), ((16, 64), 4)]


@pytest.mark.parametrize("tile,px", TILE_PX)
def test_render_fwd_slab_full_image(torch_cuda, orc, tile, px):
    s, cam, pose = scenes.slab_scene(0), scenes.slab_camera(), scenes.identity_pose()
    _, _, _, g = gpu_render(s, cam, pose, tile=tile, px=px)
    o = orc.render(s, cam, pose)
    rep, ok = assert_images_close(g, o)
    assert o["opacity"].max() > 0.9 and (o["count"] > 3).mean() > 0.3


@pytest.mark.parametrize("tile", [(8, 32), (32, 8)])
def test_render_fwd_tile_shapes_agree(torch_cuda, tile):
    s, cam, pose = scenes.slab_scene(1), scenes.slab_camera(), scenes.identity_pose()
    _, _, _, a = gpu_render(s, cam, pose, tile=(16, 16))
    _, _, _, b = gpu_render(s, cam, pose, tile=tile)
    # the tile only changes where the intersection is re-based: FP32 rounding
    ref = {k: a[k].astype(np.float64) for k in ("rgb", "depth", "normal", "opacity")}
    assert_images_close(b, ref)


def test_render_fwd_room_sampled_pixels(torch_cuda, orc):
    """Full-size tracking workload (200k surfels, 640x480): random pixels and
    a 64x64 crop against the oracle evaluated pixel by pixel."""
    s, cam, pose = scenes.room_scene(0, 200_000), scenes.tracking_camera(), scenes.room_pose(1)
    _, _, _, g = gpu_render(s, cam, pose)
    pix = scenes.pixel_sample(3, cam.height, cam.width, 2048)
    ys, xs = np.mgrid[200:264, 300:364]
    pix = np.concatenate([pix, np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)])
    o = orc.render(s, cam, pose, pixels=pix)
    gs = {k: g[k][pix[:, 1], pix[:, 0]] for k in ("rgb", "depth", "normal", "opacity")}
    assert_images_close(gs, o)
    assert np.median(o["opacity"]) > 0.95


@pytest.mark.parametrize("tile,px", [((16, 16), 1), ((16, 32), 2), ((16, 48), 3), ((32, 32), 4)])
def test_render_edge_cases(torch_cuda, orc, tile, px):
    cam = scenes.Camera(50.0, 50.0, 20.5, 10.0, 37, 21)   # ragged tiles both ways
    # everything behind the camera: empty image
    s = scenes.slab_scene(2, 300)
    s.mu[:, 2] *= -1
    _, _, _, g = gpu_render(s, cam, scenes.identity_pose(), tile=tile, px=px)
    assert np.all(g["opacity"] == 0) and np.all(g["t_final"] == 1) and np.all(g["n_last"] == 0)
    # a single surfel, and a surfel straddling the camera plane (full-image footprint)
    s1 = scenes.Surfels(np.array([[0.0, 0.0, 1.0], [0.05, 0.0, 0.06]]),
                        np.array([[1.0, 0, 0, 0], [0.7, 0.7, 0.0, 0.0]]),
                        np.array([[0.05, 0.05], [0.3, 0.3]]), np.array([0.8, 0.6]),
                        np.array([[1.0, 0.5, 0.2], [0.1, 0.9, 0.3]]))
    _, _, _, g = gpu_render(s1, cam, scenes.identity_pose(), tile=tile, px=px)
    o = orc.render(s1, cam, scenes.identity_pose())
    assert_images_close(g, o)


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------
def _slab_loss_setup(orc):
    s, cam, gt = scenes.slab_scene(0), scenes.slab_camera(), scenes.identity_pose()
    target_pose = scenes.perturb_pose(gt, 0.02, 1.0, seed=11)
    tgt = orc.render(s, cam, target_pose)
    return s, cam, gt, tgt


@pytest.mark.parametrize("tile,px", [((16, 16), 1), ((32, 16), 2), ((32, 24), 3), ((32, 32), 4)])
def test_render_bwd_slab_all_params_and_pose(torch_cuda, orc, tile, px):
    """Workload 1: L1 colour + L1 depth against a target rendered at a pose
    offset by 2 cm / 1 degree; gradients to all surfel params and the pose
    (1, 2 and 4 pixels per thread)."""
    torch = torch_cuda
    s, cam, pose, tgt = _slab_loss_setup(orc)
    r, ds, pose_t, g = gpu_render(s, cam, pose, tile=tile, px=px)
    # upstream gradient of sum|rgb - rgb_t| + sum|D - D_t| from the oracle image
    o = orc.render(s, cam, pose)
    d_rgb = np.sign(o["rgb"] - tgt["rgb"])
    d_depth = np.sign(o["depth"] - tgt["depth"])
    zeros3 = np.zeros_like(d_rgb)
    zeros1 = np.zeros_like(d_depth)
    og = orc.render_bwd(s, cam, pose, d_rgb, d_depth, zeros3, zeros1)
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    gg = r.backward(ds, pose_t, T(d_rgb), T(d_depth), None, None, full=True)
    torch.cuda.synchronize()
    ok = grad_rows_ok(og)
    for k in ("mu", "quat", "scale", "opacity", "rgb"):
        assert_grads_close(to_np(gg[k]), og[k], k, rows_ok=ok)
    assert_grads_close(to_np(gg["pose6"]), og["pose6"], "pose6", tol=1e-3)
    # tracking mode returns the same pose gradient
    gp = r.backward(ds, pose_t, T(d_rgb), T(d_depth), None, None, full=False)
    assert_grads_close(to_np(gp["pose6"]), og["pose6"], "pose6 (tracking mode)")


@pytest.mark.parametrize("tile,px", [((16, 16), 1), ((16, 64), 4)])
def test_render_bwd_with_normal_and_opacity_grads(torch_cuda, orc, tile, px):
    torch = torch_cuda
    s, cam, pose = scenes.slab_scene(4), scenes.slab_camera(), scenes.identity_pose()
    r, ds, pose_t, _ = gpu_render(s, cam, pose, tile=tile, px=px)
    up = scenes.random_upstream(5, cam.height, cam.width)
    og = orc.render_bwd(s, cam, pose, *up)
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    gg = r.backward(ds, pose_t, T(up[0]), T(up[1]), T(up[2]), T(up[3]), full=True)
    ok = grad_rows_ok(og)
    # random-sign upstream gradients make many surfel sums cancel: the
    # floor of the per-element bound covers their FP32 rounding
    for k in ("mu", "quat", "scale", "opacity", "rgb"):
        assert_grads_close(to_np(gg[k]), og[k], k, rows_ok=ok)
    assert_grads_close(to_np(gg["pose6"]), og["pose6"], "pose6")
    gp = r.backward(ds, pose_t, T(up[0]), T(up[1]), T(up[2]), T(up[3]), full=False)
    assert_grads_close(to_np(gp["pose6"]), og["pose6"], "pose6 (tracking mode)")


def test_render_bwd_deterministic(torch_cuda):
    torch = torch_cuda
    s, cam, pose = scenes.slab_scene(3), scenes.slab_camera(), scenes.identity_pose()
    r, ds, pose_t, _ = gpu_render(s, cam, pose)
    up = scenes.random_upstream(6, cam.height, cam.width)
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    a = r.backward(ds, pose_t, *(T(u) for u in up), full=True)
    a = {k: v.clone() for k, v in a.items()}
    b = r.backward(ds, pose_t, *(T(u) for u in up), full=True)
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_render_bwd_room_pixel_subset(torch_cuda, orc):
    """Full-size backward (200k surfels, 640x480) with the upstream gradient
    non-zero on a 48x48 crop only, so the oracle can evaluate it exactly."""
    torch = torch_cuda
    s, cam, pose = scenes.room_scene(0, 200_000), scenes.tracking_camera(), scenes.room_pose(1)
    r, ds, pose_t, _ = gpu_render(s, cam, pose)
    up = [np.zeros((cam.height, cam.width, 3)), np.zeros((cam.height, cam.width)),
          np.zeros((cam.height, cam.width, 3)), np.zeros((cam.height, cam.width))]
    rnd = scenes.random_upstream(8, 48, 48)
    ys, xs = np.mgrid[300:348, 210:258]
    for a, b in zip(up, rnd):
        a[ys, xs] = b
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    og = orc.render_bwd(s, cam, pose, *(u[ys, xs].reshape(-1, *u.shape[2:]) for u in up), pixels=pix)
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    gg = r.backward(ds, pose_t, *(T(u) for u in up), full=True)
    touched = np.abs(og["rgb"]).sum(1) > 0
    assert touched.sum() > 100
    ok = grad_rows_ok(og)
    for k in ("mu", "quat", "scale", "opacity", "rgb"):
        assert_grads_close(to_np(gg[k]), og[k], k, rows_ok=ok, min_rows=0.5)
    assert_grads_close(to_np(gg["pose6"]), og["pose6"], "pose6")


def test_autograd_render_matches_oracle_gradient(torch_cuda, orc):
    """A loss written with torch ops on the images of the autograd binding
    (L1 colour + L1 depth against a target 2 cm / 1 deg away) back-propagates
    through gs2d_render_bwd to the oracle's gradients of every surfel
    parameter and of the pose tangent."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import autograd, gs2d
    s, cam, pose, tgt = _slab_loss_setup(orc)
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    params = [T(s.mu).requires_grad_(), T(s.quat).requires_grad_(), T(s.scale).requires_grad_(),
              T(s.opacity).requires_grad_(), T(s.rgb).requires_grad_()]
    tau = torch.zeros(6, device="cuda", requires_grad=True)
    rast = gs2d.Rasterizer(cam, s.n)
    rgb, depth, normal, opac = autograd.render(*params, tau, gs2d.pose_tensor(pose), rast)
    loss = (rgb - T(tgt["rgb"])).abs().sum() + (depth - T(tgt["depth"])).abs().sum()
    loss.backward()
    o = orc.render(s, cam, pose)
    og = orc.render_bwd(s, cam, pose, np.sign(o["rgb"] - tgt["rgb"]), np.sign(o["depth"] - tgt["depth"]),
                        np.zeros_like(o["rgb"]), np.zeros_like(o["depth"]))
    ok = grad_rows_ok(og)
    for k, p in zip(("mu", "quat", "scale", "opacity", "rgb"), params):
        assert_grads_close(to_np(p.grad), og[k], k, rows_ok=ok)
    assert_grads_close(to_np(tau.grad), og["pose6"], "pose6")
    # a non-zero tangent renders at Exp(tau) T
    tau2 = torch.tensor([0.01, 0.0, 0.0, 0.0, 0.0, 0.0], device="cuda")
    with torch.no_grad():
        rgb2, *_ = autograd.render(*params, tau2, gs2d.pose_tensor(pose), rast)
    moved = scenes.Pose(pose.R.copy(), pose.t + np.array([0.01, 0.0, 0.0]))
    _, _, _, ref = gpu_render(s, cam, moved)
    assert np.abs(rgb2.cpu().numpy() - ref["rgb"]).max() < 1e-4


def test_forward_only_binning_matches(torch_cuda):
    """Bins without emission arrays (gs2d_bin_sort skips the emission scan)
    hold the same surfel order and tile ranges, and the forward renders the
    same bits."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cam, pose = scenes.room_scene(2, 50_000), scenes.tracking_camera(), scenes.room_pose(3)
    r, ds, pose_t, g = gpu_render(s, cam, pose)
    K = int(r.n_isect.item())
    vals = r.vals[:K].clone()
    ranges = r.ranges.clone()
    rgb = r.rgb.clone()
    r.vals.fill_(-1)
    r.status.zero_()
    fb = gs2d.Bins(r.bins.keys, r.bins.vals, None, None, r.bins.tile_ranges, r.bins.n_isect,
                   r.bins.status, r.bins.capacity)
    gs2d.gs2d_bin_sort(r.proj, r.tiles, r.n, r.cam, r.cfg, r.sort_ws, fb)
    r.render_fwd()
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0 and int(r.n_isect.item()) == K
    assert torch.equal(r.vals[:K], vals) and torch.equal(r.ranges, ranges)
    assert torch.equal(r.rgb, rgb)

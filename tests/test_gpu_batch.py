"""Batched views (one persistent launch per render pass over all views):
per-view images equal the single-view entry points bit for bit; surfel
gradients summed over views, with active subsets, uneven resolutions and
per-view tile shapes, equal the sum of the oracle's per-view gradients."""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes
from gpu_helpers import (EDGE_ON_COS, GRAD_FLOOR, TOL_GRAD, assert_grads_close, gpu_render,
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


def _setup(n_views=4, seed=0):
    s = scenes.slab_scene(seed, 3000)
    rng = np.random.default_rng(seed)
    cams = [scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120),
            scenes.Camera(100.0, 100.0, 48.0, 32.0, 96, 64),
            scenes.Camera(170.0, 170.0, 100.5, 75.0, 200, 150),
            scenes.Camera(120.0, 120.0, 60.0, 44.0, 120, 88)][:n_views]
    poses = [scenes.perturb_pose(scenes.identity_pose(), 0.05, 3.0, seed=10 + v) for v in range(n_views)]
    actives = [None, np.sort(rng.choice(s.n, 1800, replace=False)).astype(np.int32), None,
               np.sort(rng.choice(s.n, 900, replace=False)).astype(np.int32)][:n_views]
    tiles = [(16, 16), (8, 32), (32, 8), (16, 16)][:n_views]
    return s, cams, poses, actives, tiles


@pytest.mark.parametrize("px", [1, 2, 3, 4])
def test_batch_forward_equals_single_views(torch_cuda, px):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cams, poses, actives, tiles = _setup()
    if px != 1:
        shapes = gs2d.TILE_SHAPES[px]
        tiles = [shapes[v % len(shapes)] for v in range(len(cams))]
    ds = gs2d.DeviceSurfels(s)
    br = gs2d.BatchRasterizer(cams, s.n, actives=actives, tiles=tiles, px=px)
    br.set_poses(poses)
    br.forward(ds)
    torch.cuda.synchronize()
    for v in range(len(cams)):
        sub = s if actives[v] is None else s.subset(actives[v])
        _, _, _, g = gpu_render(sub, cams[v], poses[v], tile=tiles[v], px=px)
        b = br.keep[v]
        for k in ("rgb", "depth", "normal", "opacity", "t_final", "n_last"):
            np.testing.assert_array_equal(b[k].cpu().numpy(), g[k], err_msg=f"view {v} {k}")


def _well_conditioned(orc, s, cams, poses, actives, min_cos=0.02):
    """The scene without surfels that some view sees within ~1.1 degrees of
    edge-on (oracle min_cos), where the FP32 ray-surfel intersection is
    ill-conditioned; active subsets are re-indexed."""
    mc = np.ones(s.n)
    for v in range(len(cams)):
        ids = np.arange(s.n) if actives[v] is None else actives[v]
        z3 = np.zeros((cams[v].height, cams[v].width, 3))
        z1 = np.zeros((cams[v].height, cams[v].width))
        og = orc.render_bwd(s.subset(ids), cams[v], poses[v], z3, z1, z3, z1)
        mc[ids] = np.minimum(mc[ids], og["min_cos"])
    keep = np.nonzero(mc > min_cos)[0]
    new_id = np.full(s.n, -1, np.int64)
    new_id[keep] = np.arange(len(keep))
    acts = [None if a is None else new_id[a][new_id[a] >= 0].astype(np.int32) for a in actives]
    return s.subset(keep), acts


def test_batch_backward_matches_oracle_sum(torch_cuda, orc):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cams, poses, actives, tiles = _setup()
    s, actives = _well_conditioned(orc, s, cams, poses, actives)
    ds = gs2d.DeviceSurfels(s)
    br = gs2d.BatchRasterizer(cams, s.n, actives=actives, tiles=tiles)
    br.set_poses(poses)
    br.forward(ds)
    total = {k: np.zeros(getattr(s, k).shape) for k in ("mu", "quat", "scale", "opacity", "rgb")}
    mincos = np.ones(s.n)
    flagged = np.zeros(s.n, bool)
    pose6 = []
    for v in range(len(cams)):
        up = scenes.random_upstream(20 + v, cams[v].height, cams[v].width)
        # L1-like signs on colour and depth
        d_rgb, d_d = np.sign(up[0]), np.sign(up[1])
        b = br.keep[v]
        b["d_rgb"].copy_(torch.tensor(d_rgb, dtype=torch.float32))
        b["d_depth"].copy_(torch.tensor(d_d, dtype=torch.float32))
        ids = np.arange(s.n) if actives[v] is None else actives[v]
        og = orc.render_bwd(s.subset(ids), cams[v], poses[v], d_rgb, d_d, np.zeros_like(d_rgb),
                            np.zeros_like(d_d))
        for k in total:
            total[k][ids] += og[k]
        mincos[ids] = np.minimum(mincos[ids], og["min_cos"])
        flagged[ids] |= og["ambiguous"]
        pose6.append(og["pose6"])
    g = br.backward(ds)
    torch.cuda.synchronize()
    # per element, no exceptions, on the surfels that no view's oracle pass
    # flags (a candidate at a pixel with a threshold decision within
    # rounding) and that no view sees within ~3 degrees of edge-on
    ok = ~flagged & (mincos > EDGE_ON_COS)
    for k in total:
        assert_grads_close(to_np(g[k]), total[k], k, rows_ok=ok, floor=GRAD_FLOOR * len(cams))
    # the batch equals the single-view entry points summed over views (same
    # per-pair arithmetic; only the FP32 order of the sum over views differs)
    single = {k: np.zeros(getattr(s, k).shape) for k in total}
    for v in range(len(cams)):
        ids = np.arange(s.n) if actives[v] is None else actives[v]
        sub = s.subset(ids)
        r, dsub, pt, _ = gpu_render(sub, cams[v], poses[v], tile=tiles[v])
        b = br.keep[v]
        gv = r.backward(dsub, pt, b["d_rgb"], b["d_depth"], None, None, full=True)
        for k in single:
            single[k][ids] += to_np(gv[k])
    torch.cuda.synchronize()
    for k in single:
        a = to_np(g[k])
        assert np.abs(a - single[k]).max() <= 1e-6 * np.abs(single[k]).max() * len(cams), k
    for v in range(len(cams)):
        p = br.keep[v]["d_pose6"].cpu().numpy().astype(np.float64)
        assert np.abs(p - pose6[v]).max() <= TOL_GRAD * np.abs(pose6[v]).max(), (v, p, pose6[v])
    # surfels outside every subset and every view get exactly zero
    seen = np.zeros(s.n, bool)
    for v in range(len(cams)):
        seen[np.arange(s.n) if actives[v] is None else actives[v]] = True
    assert seen.all() or np.all(to_np(g["mu"])[~seen] == 0)


@pytest.mark.parametrize("extra", [0, 5])
def test_batch_binning_equals_per_view_binning(torch_cuda, extra):
    """gs2d_bin_sort_batch gives every view the bins gs2d_bin_sort gives it
    alone, bit for bit, on synthetic tile records -- with 8 views (one side
    stream each) and 13 (one launch per stage over all views): views of
    several tile grids, one with more tiles than the per-block shared-memory
    histograms hold (81 x 76), one whose histograms need more than 48 KB of
    shared memory (80 x 68), two whose four tiles hold segments longer than
    a shared-memory sort (~6k and ~40k keys), several with more surfels than
    a scan chunk (several look-back chunks), one without emission arrays, and
    an empty one."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    specs = [(4097, 10, 8, 3, True), (20000, 81, 76, 4, True), (9000, 2, 2, 6, True),
             (60000, 2, 2, 7, True), (1, 5, 4, 1, True), (7000, 12, 9, 8, False),
             (0, 5, 4, 0, True), (30000, 80, 68, 9, True)]
    specs += [(5000 + 3000 * k, 20 - k, 14, 20 + k, k % 2 == 0) for k in range(extra)]
    i32 = dict(dtype=torch.int32, device="cuda")
    views, keep = [], []
    for n, tx, ty, seed, emit in specs:
        if n:
            rect, depth, count = scenes.random_tile_records(seed, n, tx, ty)
        else:
            rect, depth, count = np.zeros((0, 4), np.int32), np.zeros(0, np.float32), np.zeros(0, np.int32)
        proj, tiles = records_to_proj(torch, rect, depth, count)
        cam = gs2d.camera(scenes.Camera(100.0, 100.0, 8.0, 8.0, tx * 16 - 5, ty * 16 - 3))
        cfg = gs2d.default_config((16, 16))
        cap = int(count.sum()) + 17
        act = torch.arange(max(n, 1), **i32)

        def bufs():
            return dict(vals=torch.full((cap,), -7, **i32), emit=torch.full((cap,), -7, **i32),
                        off=torch.full((max(n, 1),), -7, **i32),
                        ranges=torch.full((2 * tx * ty,), -7, **i32),
                        n_isect=torch.zeros(1, **i32), status=torch.zeros(1, **i32))

        def mk_bins(o):
            return gs2d.Bins(None, o["vals"].data_ptr(), o["emit"].data_ptr() if emit else None,
                             o["off"].data_ptr() if emit else None, o["ranges"].data_ptr(),
                             o["n_isect"].data_ptr(), o["status"].data_ptr(), cap)

        batch, single = bufs(), bufs()
        views.append(gs2d.View(cam, cfg, None, act.data_ptr(), n, proj.data_ptr(),
                               tiles.data_ptr(), mk_bins(batch)))
        keep.append((n, emit, cam, cfg, cap, proj, tiles, act, batch, single, mk_bins(single)))
    arr = (gs2d.View * len(views))(*views)
    ws = torch.empty(gs2d.lib().gs2d_bin_sort_batch_workspace(arr, len(views), 0),
                     dtype=torch.uint8, device="cuda")
    gs2d.gs2d_bin_sort_batch(views, 0, ws)
    torch.cuda.synchronize()
    for v, (n, emit, cam, cfg, cap, proj, tiles, act, batch, single, sb) in enumerate(keep):
        w1 = torch.empty(gs2d.gs2d_bin_sort_workspace(n, cap), dtype=torch.uint8, device="cuda")
        gs2d.gs2d_bin_sort(proj, tiles, n, cam, cfg, w1, sb)
        torch.cuda.synchronize()
        assert int(batch["status"].item()) == 0 and int(single["status"].item()) == 0, v
        K = int(single["n_isect"].item())
        assert int(batch["n_isect"].item()) == K and (K > 0 or n < 10), v
        assert torch.equal(batch["ranges"], single["ranges"]), v
        assert torch.equal(batch["vals"][:K], single["vals"][:K]), v
        if emit:
            assert torch.equal(batch["emit"][:K], single["emit"][:K]), v
            assert torch.equal(batch["off"][:n], single["off"][:n]), v
    r = keep[3][8]["ranges"].view(-1, 2)
    assert int((r[:, 1] - r[:, 0]).max()) > 16384


def test_batch_capacity_error_is_per_view(torch_cuda):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cams, poses, actives, tiles = _setup(n_views=2)
    ds = gs2d.DeviceSurfels(s)
    br = gs2d.BatchRasterizer(cams, s.n, actives=actives, tiles=tiles, capacities=[50, 100000])
    br.set_poses(poses)
    with pytest.raises(gs2d.Gs2dError):
        br.forward(ds)
    assert int(br.keep[0]["status"].item()) == 3 and int(br.keep[1]["status"].item()) == 0


def test_batch_fit_grows_capacity_and_graph_replay_is_bit_identical(torch_cuda):
    """fit() regrows views whose intersections overflow; a whole batched
    step (forward + backward) captured in a CUDA graph and replayed
    reproduces the direct calls bit for bit."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cams, poses, actives, tiles = _setup(n_views=3)
    ds = gs2d.DeviceSurfels(s)
    br = gs2d.BatchRasterizer(cams, s.n, actives=actives, tiles=tiles, capacities=[64, 64, 64])
    br.set_poses(poses)
    k = br.fit(ds)
    assert all(kv > 64 for kv in k)
    assert all(b["cap"] >= kv for b, kv in zip(br.keep, k))
    for v, b in enumerate(br.keep):
        up = scenes.random_upstream(40 + v, cams[v].height, cams[v].width)
        b["d_rgb"].copy_(torch.tensor(up[0], dtype=torch.float32))
        b["d_depth"].copy_(torch.tensor(up[1], dtype=torch.float32))

    def step():
        br.forward(ds, check_status=False)
        br.backward(ds)

    br.forward(ds)
    g = br.backward(ds)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in g.items()}
    ref_img = [b["rgb"].clone() for b in br.keep]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        for t in g.values():
            t.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        assert all(int(b["status"].item()) == 0 for b in br.keep)
        for k in ref:
            assert torch.equal(g[k], ref[k]), k
        for b, im in zip(br.keep, ref_img):
            assert torch.equal(b["rgb"], im)


def test_autotune_picks_a_candidate_and_caches(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2506_00970_gb300 import autotune, gs2d
    s, cams, poses, actives, _ = _setup(n_views=2)
    ds = gs2d.DeviceSurfels(s)
    path = str(tmp_path / "tune.json")
    autotune._cache.clear()
    tiles, table = autotune.tune_tiles(ds, cams, poses, actives, reps=1, cache_path=path)
    assert all(t in autotune.TILE_SHAPES[1] for t in tiles)
    assert set(table) == {f"{c.width}x{c.height}" for c in cams}
    for c, t in zip(cams, tiles):
        row = table[f"{c.width}x{c.height}"]
        assert row[f"{t[0]}x{t[1]}"] == min(row.values())
    autotune._cache.clear()
    tiles2, table2 = autotune.tune_tiles(ds, cams, poses, actives, cache_path=path)
    assert tiles2 == tiles and table2 == {}


@pytest.mark.parametrize("px,tiles", [(2, [(16, 32), (32, 16), (16, 32)]),
                                      (3, [(32, 24), (64, 12), (16, 48)])])
def test_batch_backward_several_pixels_per_thread_equals_single_views(torch_cuda, px, tiles):
    """The persistent backward with 2 or 3 pixels per thread equals the
    single-view backward (same per-pair arithmetic) summed over views."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cams, poses, actives, _ = _setup(n_views=3)
    ds = gs2d.DeviceSurfels(s)
    br = gs2d.BatchRasterizer(cams, s.n, actives=actives, tiles=tiles, px=px)
    br.set_poses(poses)
    br.forward(ds)
    for v, b in enumerate(br.keep):
        up = scenes.random_upstream(70 + v, cams[v].height, cams[v].width)
        b["d_rgb"].copy_(torch.tensor(up[0], dtype=torch.float32))
        b["d_depth"].copy_(torch.tensor(up[1], dtype=torch.float32))
    g = br.backward(ds)
    single = {k: np.zeros(getattr(s, k).shape) for k in g}
    for v in range(len(cams)):
        ids = np.arange(s.n) if actives[v] is None else actives[v]
        r, dsub, pt, _ = gpu_render(s.subset(ids), cams[v], poses[v], tile=tiles[v], px=px)
        b = br.keep[v]
        gv = r.backward(dsub, pt, b["d_rgb"], b["d_depth"], None, None, full=True)
        for k in single:
            single[k][ids] += to_np(gv[k])
    torch.cuda.synchronize()
    for k in single:
        assert np.abs(to_np(g[k]) - single[k]).max() <= 1e-6 * np.abs(single[k]).max() * 3, k


def test_autotune_sweeps_pixels_per_thread(torch_cuda):
    from paper_2506_00970_gb300 import autotune, gs2d
    s, cams, poses, actives, _ = _setup(n_views=2)
    ds = gs2d.DeviceSurfels(s)
    autotune._cache.clear()
    px, tiles, table = autotune.tune(ds, cams, poses, actives, reps=1)
    assert px in (1, 2, 3, 4) and all(t in gs2d.TILE_SHAPES[px] for t in tiles)
    assert set(table) == {"px1", "px2", "px3", "px4"}

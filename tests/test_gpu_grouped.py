"""The grouped one-pixel compositing loops (four (pixel, surfel) evaluations
in flight per thread, chosen for tile grids too small to fill the GPU)
against the plain loops: the same evaluations blended in the same order, so
forward images, compositing state and whole tracking frames are
bit-identical whichever form runs."""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    yield torch
    gs2d.gs2d_set_grouped_tiles(-1)


def _forward(gs2d, ds, cam, pose, grouped):
    gs2d.gs2d_set_grouped_tiles(1 << 30 if grouped else 0)
    r = gs2d.Rasterizer(cam, ds.n)
    out = r.forward(ds, gs2d.pose_tensor(pose))
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


CASES = [
    # (scene, camera, pose): the c1-style slab, a small room view, a dense
    # low-resolution view of a large room (long tile lists), a ragged image
    ("slab", scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120), None),
    ("room30k", scenes.Camera(262.5, 262.5, 160.0, 120.0, 320, 240), 3),
    ("room200k", scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120), 100),
    ("room30k", scenes.Camera(200.0, 210.0, 97.0, 53.5, 197, 109), 5),
]


def _scene(name, seed):
    if name == "slab":
        return scenes.slab_scene(0, 4096), scenes.identity_pose()
    n = 30_000 if name == "room30k" else 200_000
    return scenes.room_scene(0, n), scenes.room_pose(seed)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_grouped_forward_is_bit_identical(torch_cuda, case):
    from paper_2506_00970_gb300 import gs2d
    name, cam, seed = CASES[case]
    s, pose = _scene(name, seed)
    ds = gs2d.DeviceSurfels(s)
    a = _forward(gs2d, ds, cam, pose, grouped=False)
    b = _forward(gs2d, ds, cam, pose, grouped=True)
    gs2d.gs2d_set_grouped_tiles(-1)
    assert a["opacity"].max() > 0.5
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("case", [1, 2, 3])
def test_grouped_tracking_frame_is_bit_identical(torch_cuda, case):
    """20 fused tracking iterations (forward, loss, pose backward, AdamW,
    retraction) give the same loss and pose histories in both forms."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    name, cam, seed = CASES[case]
    s, gt = _scene(name, seed)
    ds = gs2d.DeviceSurfels(s)
    img = _forward(gs2d, ds, cam, gt, grouped=False)
    obs_rgb = torch.tensor(img["rgb"], device="cuda")
    obs_d = torch.tensor(img["depth"] / np.maximum(img["opacity"], 1e-6), device="cuda")
    start = gs2d.pose_tensor(scenes.perturb_pose(gt, 0.02, 1.0, seed=7))
    ccam, cfg = gs2d.camera(cam), gs2d.default_config()
    prm = gs2d.default_track_params(stop_tol=0.0)
    cap = 8 * s.n
    hist = []
    for grouped in (False, True):
        gs2d.gs2d_set_grouped_tiles(1 << 30 if grouped else 0)
        ws = torch.empty(gs2d.gs2d_track_workspace(s.n, cap, ccam, cfg), dtype=torch.uint8,
                         device="cuda")
        pose = start.clone()
        lh = torch.zeros(20, device="cuda")
        ph = torch.zeros(20, 12, device="cuda")
        gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, 20, cap, lh, ph, ws)
        torch.cuda.synchronize()
        assert int(gs2d.gs2d_track_status(ws).item()) == 0
        hist.append((lh.cpu().numpy(), ph.cpu().numpy(), pose.cpu().numpy()))
    gs2d.gs2d_set_grouped_tiles(-1)
    assert hist[0][0][0] > 0
    for x, y in zip(hist[0], hist[1]):
        np.testing.assert_array_equal(x, y)

"""End-to-end keyframe bookkeeping on the GPU through ``SurfelMap``
(Sec. III-D, III-E, III-F, IV-C), with the steps' own parity covered by
test_gpu_contrib / test_gpu_map / test_gpu_expand.  Checked here: a map
grown from an RGB-D keyframe renders that keyframe's depth back; a second,
overlapping keyframe adds surfels only in free voxels; the covisibility
keyframe rule; the state update and the voxel table's rebuild after
deactivation; occlusion removal removes exactly the surfels the rule names;
the map correction moves exactly the surfels of the corrected keyframe.
"""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes
from gpu_helpers import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


def test_surfel_map_keyframe_flow(torch_cuda):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    from paper_2506_00970_gb300.surfel_map import SurfelMap
    cam = scenes.Camera(300.0, 300.0, 160.0, 120.0, 320, 240)
    p0 = scenes.identity_pose()
    p1 = scenes.perturb_pose(p0, 0.05, 3.0, seed=1)
    p2 = scenes.perturb_pose(p0, 0.30, 10.0, seed=2)
    T = lambda a: torch.tensor(a, device="cuda")
    P = gs2d.pose_tensor
    gen = torch.Generator(device="cuda").manual_seed(0)
    M = SurfelMap(400_000, voxel=0.02, inactive_after=0)
    rgb0, d0 = scenes.rgbd_frame(0, cam, pose=p0)
    k0 = M.expand(T(rgb0), T(d0), cam, P(p0), 0, 0.25, gen)
    assert k0 > 5000 and M.n == k0
    st = M.map_state()
    assert bool((st.delta == 1).all()) and bool((st.t_c == 0).all()) and bool((st.t_l == 0).all())
    # the new map renders the keyframe's depth back
    r = gs2d.Rasterizer(cam, M.n)
    out = r.forward(M.surfels(), P(p0))
    O = to_np(out["opacity"])
    Dh = to_np(out["depth"]) / np.maximum(O, 1e-6)
    mask = (O > 0.5) & (d0 > 0)
    assert mask.mean() > 0.6
    assert np.median(np.abs(Dh[mask] - d0[mask])) < 0.01
    # contributions and the state update from the same keyframe
    c0 = M.contributions(cam, P(p0))
    vis, closer, deact, react = M.observe(c0, P(p0), 0)
    assert vis > 0.3 * M.n and deact == 0 and react == 0
    # an overlapping keyframe adds surfels only where the voxels were free
    rgb1, d1 = scenes.rgbd_frame(1, cam, pose=p1)
    occ_before = M.table.query(M.params.mu[:M.n]).clone()
    n_before = M.n
    k1 = M.expand(T(rgb1), T(d1), cam, P(p1), 1, 0.25, gen)
    assert 0 < k1 < k0
    assert bool(occ_before.all())
    # covisibility: the nearby view is covisible, the far one triggers a keyframe
    c1 = M.contributions(cam, P(p1))
    s01, kf01 = M.keyframe_test(c1, c0, P(p1), P(p0), c_k=0.0)
    assert 0.0 < s01 <= 1.0 and not kf01
    c2 = M.contributions(cam, P(p2))
    _, kf02 = M.keyframe_test(c2, c0, P(p2), P(p0), c_k=0.0)
    assert kf02                                  # 30 cm apart
    # occlusion removal for keyframe 0: exactly the rule's surfels go
    cr = M.contributions(cam, P(p0), active_only=False)
    t_c = M.state.t_c[:M.n].cpu().numpy()
    expect = int(((t_c == 0) & (cr.cpu().numpy() < 0.5)).sum())
    n_pre = M.n
    removed = M.prune(cr, 0)
    assert removed == expect and M.n == n_pre - removed
    # map correction: keyframe 1 moves by 5 cm along x, keyframe 0 stays
    old = torch.stack([P(p0), P(p1)]).reshape(-1)
    new = old.clone()
    new[12 + 9:12 + 12] = new[12 + 9:12 + 12] - torch.tensor(
        np.asarray(p1.R, np.float32) @ np.array([0.05, 0.0, 0.0], np.float32), device="cuda")
    mu0 = M.params.mu[:M.n].clone()
    tc = M.state.t_c[:M.n].clone()
    assert M.correct(old, new) == 0
    d = (M.params.mu[:M.n] - mu0).cpu().numpy()
    sel1 = (tc == 1).cpu().numpy()
    np.testing.assert_allclose(d[sel1], np.tile([0.05, 0.0, 0.0], (sel1.sum(), 1)), atol=2e-5)
    np.testing.assert_allclose(d[~sel1], 0.0, atol=2e-6)
    # deactivation: a keyframe that sees nothing of the map (all surfels
    # unobserved, 0 keyframes allowed) empties the active map and the table
    vis, _, deact, _ = M.observe(torch.zeros(M.n, device="cuda"), P(p0), 5)
    assert vis == 0 and deact == M.n
    assert not bool(M.table.query(M.params.mu[:M.n]).any())
    # the freed voxels take new surfels again
    k3 = M.expand(T(rgb0), T(d0), cam, P(p0), 6, 0.25, gen)
    assert k3 > 0.5 * k0


def test_surfel_map_checkpoint(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    from paper_2506_00970_gb300.surfel_map import SurfelMap
    cam = scenes.Camera(300.0, 300.0, 160.0, 120.0, 320, 240)
    p0 = scenes.identity_pose()
    M = SurfelMap(200_000, voxel=0.03)
    rgb, d = scenes.rgbd_frame(4, cam, pose=p0)
    T = lambda a: torch.tensor(a, device="cuda")
    M.expand(T(rgb), T(d), cam, gs2d.pose_tensor(p0), 2, 0.2,
             torch.Generator(device="cuda").manual_seed(1))
    M.state.delta[: M.n : 3] = 0                     # some inactive surfels
    M.rebuild_table()
    path = str(tmp_path / "map.npz")
    M.save(path)
    L = SurfelMap.load(path)
    assert L.n == M.n and L.capacity == M.capacity and L.table.voxel == M.table.voxel
    for name in ("mu", "quat", "scale", "opacity", "rgb"):
        assert torch.equal(getattr(L.params, name)[:L.n], getattr(M.params, name)[:M.n]), name
    for name in ("delta", "t_c", "d_c", "t_l"):
        assert torch.equal(getattr(L.state, name)[:L.n], getattr(M.state, name)[:M.n]), name
    q = M.params.mu[: M.n]
    assert torch.equal(L.table.query(q), M.table.query(q))

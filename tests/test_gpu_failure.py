"""Failure paths of the binning on the GPU, made without a fault.

The emission scan of gs2d_bin_sort waits (boundedly) for each predecessor
block's published sum.  gs2d_set_lookback_wait withholds one block's sum --
a flag that nothing sets -- and shortens the wait, so the next block's wait
runs out: the call must record GS2D_ERR_TIMEOUT in its status word, keep
every write in bounds, make every later kernel skip (outputs keep their
sentinel values, the forward render gated on the same word writes nothing),
and leave the context usable: the same binning afterwards equals the
oracle's library sort.
"""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes

pytestmark = pytest.mark.gpu

SENTINEL = -7


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


def test_lookback_timeout_is_reported_and_gates_later_kernels(torch_cuda, orc):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cam, pose = scenes.room_scene(3, 50_000), scenes.tracking_camera(), scenes.room_pose(4)
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, s.n, capacity=40 * s.n, keys=True)
    pose_t = gs2d.pose_tensor(pose)
    r.project(ds, pose_t)
    torch.cuda.synchronize()
    n_chunks = (s.n + 4095) // 4096
    assert n_chunks >= 8
    for t in (r.vals, r.emit, r.ranges):
        t.fill_(SENTINEL)
    r.surfel_off.fill_(SENTINEL)
    r.rgb.fill_(float(SENTINEL))
    r.status.zero_()
    gs2d.gs2d_set_lookback_wait(256, 3)
    try:
        gs2d.gs2d_bin_sort(r.proj, r.tiles, r.n, r.cam, r.cfg, r.sort_ws, r.bins)
        r.render_fwd()
        torch.cuda.synchronize()
    finally:
        gs2d.gs2d_set_lookback_wait(0, -1)
    assert int(r.status.item()) == 5   # GS2D_ERR_TIMEOUT
    # the scan wrote every surfel's offset, each within the total
    off = r.surfel_off.cpu().numpy().astype(np.int64)
    total = int(r.tiles[: s.n].sum().item())
    assert np.all((off >= 0) & (off <= total))
    # the kernels after the scan skipped: outputs untouched
    for t in (r.vals, r.emit, r.ranges):
        assert torch.all(t == SENTINEL)
    assert torch.all(r.rgb == float(SENTINEL))
    # the context is still usable: the same binning, without the withheld
    # block, equals the library stable sort of the oracle
    r.bin_sort(grow=False)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0
    proj = r.proj.cpu().numpy().reshape(-1, 32)[: s.n]
    r01, r23 = proj[:, 28].view(np.uint32), proj[:, 29].view(np.uint32)
    rect = np.stack([r01 & 0xFFFF, r01 >> 16, r23 & 0xFFFF, r23 >> 16], 1).astype(np.int32)
    _, ov, _ = orc.bin_sort(rect, proj[:, 26], r.tiles_x, r.tiles_y)
    K = int(r.n_isect.item())
    assert K == len(ov)
    np.testing.assert_array_equal(r.vals[:K].cpu().numpy().astype(np.uint32), ov)


def test_lookback_default_wait_is_restored(torch_cuda):
    """With the default wait (and no withheld block) many back-to-back
    binnings of a large map all finish with GS2D_OK."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cam, pose = scenes.room_scene(4, 200_000), scenes.tracking_camera(), scenes.room_pose(5)
    ds = gs2d.DeviceSurfels(s)
    r = gs2d.Rasterizer(cam, s.n, capacity=16 * s.n)
    r.project(ds, gs2d.pose_tensor(pose))
    for _ in range(20):
        r.status.zero_()
        gs2d.gs2d_bin_sort(r.proj, r.tiles, r.n, r.cam, r.cfg, r.sort_ws, r.bins)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 0

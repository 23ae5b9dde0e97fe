"""GPU parity of gs2d_render_contrib and gs2d_covisibility (through the C
ABI) against the FP64 oracle (Sec. III-D, Eq. weight and Eq. contribution).

Tolerance: a surfel's contribution is a sum of its per-pixel weights, each
within the forward's FP32 rounding (about 1e-7 relative, far inside the
1e-4 opacity tolerance), so |C_gpu - C_orc| <= 1e-4 (1 + C_orc).  Surfels
the oracle flags as candidates at a pixel whose evaluation sits on a
threshold (FP32 may decide that pixel otherwise, moving at most a few
hundredths of weight) or that blend into a ray within ~3 degrees of edge-on
are held to 0.05 + 1e-3 C_orc (each test also requires a minimum number of
tightly checked surfels).  Visibility (C > 0.5) must agree wherever
the oracle's contribution is outside that band.
"""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes
from gpu_helpers import gpu_render, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


def _check(g, o, rows=None):
    c_o, c_g = o["contrib"], np.asarray(g, np.float64)
    loose = o["ambiguous"] | (o["min_cos"] < 0.05)
    sel = np.ones(len(c_o), bool) if rows is None else rows
    err = np.abs(c_g - c_o)
    tight = sel & ~loose
    assert np.all(err[tight] <= 1e-4 * (1 + c_o[tight])), err[tight].max()
    assert np.all(err[sel & loose] <= 0.05 + 1e-3 * c_o[sel & loose])
    band = np.abs(c_o - 0.5) <= 0.05 + 1e-3
    vis_bad = (c_g > 0.5) != (c_o > 0.5)
    assert not np.any(vis_bad & sel & ~band)
    return int(tight.sum())


@pytest.mark.parametrize("tile,px", [((16, 16), 1), ((8, 32), 1), ((32, 16), 2), ((32, 24), 3),
                                     ((32, 32), 4)])
def test_contrib_slab_full_image(torch_cuda, orc, tile, px):
    torch = torch_cuda
    s, cam, pose = scenes.slab_scene(0), scenes.slab_camera(), scenes.identity_pose()
    r, _, _, g = gpu_render(s, cam, pose, tile=tile, px=px)
    c = r.contribution()
    torch.cuda.synchronize()
    o = orc.contrib(s, cam, pose)
    n_tight = _check(to_np(c), o)
    assert n_tight > 0.8 * s.n
    # the weights of every pixel sum to its opacity (both from the GPU)
    np.testing.assert_allclose(to_np(c).sum(), g["opacity"].astype(np.float64).sum(), rtol=2e-5)
    # deterministic
    c2 = r.contribution().clone()
    assert torch.equal(c, c2)


def test_contrib_room_full_size_crop(torch_cuda, orc):
    """The 200k-surfel room at 640x480: the contributions of the surfels whose
    whole footprint lies inside a 128x128 crop, against the oracle over the crop;
    and sum C = sum O over the full image."""
    torch = torch_cuda
    s, cam, pose = scenes.room_scene(0, 200_000), scenes.tracking_camera(), scenes.room_pose(1)
    r, _, _, g = gpu_render(s, cam, pose)
    c = to_np(r.contribution())
    torch.cuda.synchronize()
    x0, y0, side = 256, 176, 128
    ys, xs = np.mgrid[y0:y0 + side, x0:x0 + side]
    pix = np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    o = orc.contrib(s, cam, pose, pixels=pix)
    b = o["bbox"]
    inside = (b[:, 0] > x0) & (b[:, 1] > y0) & (b[:, 2] < x0 + side - 1) & (b[:, 3] < y0 + side - 1)
    assert inside.sum() > 150
    # a dense room puts a cutoff decision within FP32 reach of ~1/3 of them
    assert _check(c, o, rows=inside) > 100
    np.testing.assert_allclose(c.sum(), g["opacity"].astype(np.float64).sum(), rtol=2e-5)


def test_contrib_edge_cases(torch_cuda, orc):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    cam = scenes.Camera(50.0, 50.0, 20.5, 10.0, 37, 21)      # ragged tiles both ways
    s = scenes.slab_scene(2, 300)
    s.mu[:, 2] *= -1                                       # everything behind the camera
    r, _, _, _ = gpu_render(s, cam, scenes.identity_pose())
    assert float(r.contribution().abs().max()) == 0.0
    s1 = scenes.Surfels(np.array([[0.0, 0.0, 1.0], [0.05, 0.0, 0.06]]),
                        np.array([[1.0, 0, 0, 0], [0.7, 0.7, 0.0, 0.0]]),
                        np.array([[0.05, 0.05], [0.3, 0.3]]), np.array([0.8, 0.6]),
                        np.array([[1.0, 0.5, 0.2], [0.1, 0.9, 0.3]]))
    r, _, _, _ = gpu_render(s1, cam, scenes.identity_pose())
    _check(to_np(r.contribution()), orc.contrib(s1, cam, scenes.identity_pose()))
    # a binning that overflowed its capacity gates the kernels: contrib untouched
    s2 = scenes.slab_scene(3, 2000)
    r2 = gs2d.Rasterizer(scenes.slab_camera(), s2.n, capacity=64)
    ds = gs2d.DeviceSurfels(s2)
    r2.project(ds, gs2d.pose_tensor(scenes.identity_pose()))
    r2.bin_sort(grow=False)
    out = torch.full((s2.n,), -7.0, device="cuda")
    r2.contribution(out=out)
    torch.cuda.synchronize()
    assert int(r2.status.item()) == 3 and bool((out == -7.0).all())


def test_covisibility_counts_and_keyframe_rule(torch_cuda, orc):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(7)
    for n in (0, 1, 1000, 300_001):
        ca = rng.uniform(0, 1, n).astype(np.float32)
        cb = rng.uniform(0, 1, n).astype(np.float32)
        if n > 10:
            ca[:5] = 0.5                                   # exactly on the threshold
            cb[5:10] = np.nextafter(np.float32(0.5), np.float32(1))
        inter, union, score = orc.covisibility(ca, cb)
        T = lambda a, dt=torch.float32: torch.tensor(np.asarray(a), dtype=dt, device="cuda")
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        sc = torch.zeros(1, device="cuda")
        kf = torch.zeros(1, dtype=torch.int32, device="cuda")
        pa = np.concatenate([np.eye(3).reshape(-1), [0.0, 0.0, 0.0]]).astype(np.float32)
        for tb, c_k in (((0.05, 0.0, 0.0), 0.0), ((0.3, 0.0, 0.0), 0.0), ((0.0, 0.0, 0.0), 1.1)):
            pb = pa.copy()
            pb[9:] = tb
            gs2d.gs2d_covisibility(T(ca) if n else T(np.zeros(1)), T(cb) if n else T(np.zeros(1)),
                                   n, 0.5, T(pa), T(pb), c_k, 0.15, counts, sc, kf)
            torch.cuda.synchronize()
            assert tuple(counts.cpu().numpy().tolist()) == (inter, union)
            assert float(sc.item()) == float(np.float32(score))
            assert bool(kf.item()) == orc.keyframe_rule(float(np.float32(score)), pa[9:], pb[9:],
                                                        c_k, 0.15)

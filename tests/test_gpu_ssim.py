"""GPU parity of the SSIM term (gs2d_ssim_loss) and of the full mapping loss
with it (gs2d_mapping_loss_ssim, Sec. III-E with the Table I weight) against
the FP64 oracle.

The loss is a mean of per-pixel SSIM values computed from FP32 window sums
of values in [0, 1]: within 1e-5 relative.  Gradients within the contract's
1e-3 relative (max over the image against its scale, and per element above
1% of the scale).  Sizes: ragged tiles (37 x 29), several tiles (128 x 96),
and the mapping view (1200 x 680).
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


def _grad_close(a, b, tol=1e-3):
    scale = np.abs(b).max()
    err = np.abs(a - b)
    assert err.max() <= tol * scale, err.max() / scale
    big = np.abs(b) > 1e-2 * scale
    assert np.mean(err[big] / np.abs(b[big]) > tol) < 2e-3


def _images(seed, h, w):
    rng = np.random.default_rng(seed)
    # smooth structure plus noise, like a rendering against its observation
    yy, xx = np.mgrid[0:h, 0:w]
    base = 0.5 + 0.4 * np.sin(xx[..., None] / 7.0 + np.arange(3)) * np.cos(yy[..., None] / 11.0)
    y = np.clip(base + rng.normal(scale=0.05, size=(h, w, 3)), 0, 1)
    x = np.clip(y + rng.normal(scale=0.1, size=(h, w, 3)), 0, 1)
    return x.astype(np.float32), y.astype(np.float32)


@pytest.mark.parametrize("h,w", [(29, 37), (96, 128), (680, 1200), (1, 1)])
def test_ssim_loss_and_gradient(torch_cuda, orc, h, w):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    x, y = _images(h * w, h, w)
    L, g = orc.ssim_loss(x, y, weight=0.125)
    T = lambda a: torch.tensor(a, device="cuda")
    g_x = torch.zeros(h, w, 3, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ws = torch.empty(gs2d.gs2d_ssim_workspace(h, w), dtype=torch.uint8, device="cuda")
    gs2d.gs2d_ssim_loss(T(x), T(y), h, w, 0.125, g_x, loss, ws)
    torch.cuda.synchronize()
    assert float(loss.item()) == pytest.approx(L, rel=1e-5, abs=1e-9)
    _grad_close(to_np(g_x), g)
    # the call adds to its outputs (FP32 sums of the same values); deterministic
    base = torch.tensor(np.random.default_rng(5).normal(size=x.shape).astype(np.float32),
                        device="cuda")
    g2 = base.clone()
    loss2 = torch.full((1,), 0.25, device="cuda")
    gs2d.gs2d_ssim_loss(T(x), T(y), h, w, 0.125, g2, loss2, ws)
    torch.cuda.synchronize()
    assert torch.equal(g2, base + g_x)
    assert float(loss2.item()) == pytest.approx(0.25 + float(loss.item()), abs=1e-7)


def test_mapping_loss_with_ssim(torch_cuda, orc):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    s, cam, pose = scenes.slab_scene(2), scenes.slab_camera(), scenes.identity_pose()
    o = orc.render(s, cam, pose)
    img = {k: o[k] for k in ("rgb", "depth", "normal", "opacity")}
    obs_rgb, obs_d = scenes.random_images(3, cam.height, cam.width, (1.0, 3.0))
    L, g = orc.mapping_loss(img, obs_rgb, obs_d, cam, w_d=0.5, w_n=0.02, w_ssim=0.125)
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    f = dict(dtype=torch.float32, device="cuda")
    out = [torch.empty(cam.height, cam.width, 3, **f), torch.empty(cam.height, cam.width, **f),
           torch.empty(cam.height, cam.width, 3, **f), torch.empty(cam.height, cam.width, **f)]
    loss = torch.empty(1, **f)
    ccam = gs2d.camera(cam)
    ws = torch.empty(gs2d.gs2d_mapping_loss_ssim_workspace(ccam), dtype=torch.uint8, device="cuda")
    gs2d.gs2d_mapping_loss_ssim(T(img["rgb"]), T(img["depth"]), T(img["normal"]),
                                T(img["opacity"]), T(obs_rgb), T(obs_d), ccam, 0.125, 0.5, 0.02,
                                *out, loss, ws)
    torch.cuda.synchronize()
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    _grad_close(to_np(out[0]), g["rgb"])

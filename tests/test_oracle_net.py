"""Pins of the proposal-network oracle (oracle/net.py) against things other
than itself: torch's bfloat16 conversion and conv2d (library routines),
central finite differences, torch autograd, and closed forms."""
import numpy as np
import pytest
import torch

from oracle import net
from paper_2506_00970_gb300 import scenes


def test_to_bf16_matches_torch_rounding():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, 65504.0]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(net.to_bf16(x), ref)
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert net.to_bf16(1.0 + 2.0 ** -8) == 1.0
    assert net.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_spatial_sizes_and_layout():
    hw = net.spatial_sizes()
    assert hw == [(120, 160), (60, 80), (30, 40), (15, 20), (8, 10), (4, 5), (2, 3)]
    items, total = net.param_layout()
    d = dict((n, (s, o)) for n, s, o in items)
    assert d["fc1.W"][0] == (256, 2 * 3 * 256)
    conv = sum(co * 9 * ci + co for ci, co in net.CONV)
    assert total == conv + 256 * 1536 + 256 + 6 * 256 + 6


def _torch_conv(x, W, b):
    xt = torch.tensor(x).permute(0, 3, 1, 2)
    wt = torch.tensor(W).permute(0, 3, 1, 2)
    y = torch.nn.functional.conv2d(xt, wt, torch.tensor(b), stride=2, padding=1)
    return y.permute(0, 2, 3, 1).numpy()


@pytest.mark.parametrize("shape", [(2, 9, 11, 5, 7), (1, 8, 10, 8, 4), (3, 1, 1, 2, 3)])
def test_conv_fwd_matches_torch_conv2d(shape):
    B, H, W, Ci, Co = shape
    rng = np.random.default_rng(1)
    x = rng.normal(size=(B, H, W, Ci))
    Wt = rng.normal(size=(Co, 3, 3, Ci))
    b = rng.normal(size=Co)
    np.testing.assert_allclose(net.conv_fwd(x, Wt, b), _torch_conv(x, Wt, b), rtol=1e-12, atol=1e-12)


def test_conv_bwd_matches_autograd_and_finite_differences():
    rng = np.random.default_rng(2)
    B, H, W, Ci, Co = 2, 7, 6, 3, 4
    x = rng.normal(size=(B, H, W, Ci))
    Wt = rng.normal(size=(Co, 3, 3, Ci))
    b = rng.normal(size=Co)
    g = rng.normal(size=(B, 4, 3, Co))
    dx, dW, db = net.conv_bwd(x, Wt, g)
    xt = torch.tensor(x, requires_grad=True)
    wt = torch.tensor(Wt, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    y = torch.nn.functional.conv2d(xt.permute(0, 3, 1, 2), wt.permute(0, 3, 1, 2), bt, stride=2,
                                   padding=1).permute(0, 2, 3, 1)
    (y * torch.tensor(g)).sum().backward()
    np.testing.assert_allclose(dx, xt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dW, wt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(db, bt.grad.numpy(), rtol=1e-12, atol=1e-12)
    # central differences on a few entries of each
    L = lambda x_, W_, b_: float(np.sum(g * net.conv_fwd(x_, W_, b_)))
    h = 1e-6
    for arr, grad in ((x, dx), (Wt, dW), (b, db)):
        for idx in list(np.ndindex(arr.shape))[::7][:12]:
            p, m = [a.copy() for a in (x, Wt, b)], [a.copy() for a in (x, Wt, b)]
            k = [x is arr, Wt is arr, b is arr].index(True)
            p[k][idx] += h
            m[k][idx] -= h
            fd = (L(*p) - L(*m)) / (2 * h)
            assert fd == pytest.approx(grad[idx], rel=1e-6, abs=1e-8)


def _tiny():
    conv = ((8, 4), (4, 6))
    h, w = 7, 9
    items, total = net.param_layout(conv, h, w)
    rng = np.random.default_rng(3)
    params = rng.normal(0, 0.5, total)
    x = rng.normal(size=(3, h, w, 8))
    t = rng.normal(size=(3, 6))
    return conv, params, x, t


def test_network_gradient_matches_finite_differences():
    conv, params, x, t = _tiny()
    y, acts = net.forward(params, x, conv)
    L0, dy = net.loss_and_grad(y, t)
    g = net.backward(params, acts, dy, conv)

    def L(p):
        return net.loss_and_grad(net.forward(p, x, conv)[0], t)[0]

    h = 1e-6
    rng = np.random.default_rng(4)
    for i in rng.choice(params.size, 60, replace=False):
        p, m = params.copy(), params.copy()
        p[i] += h
        m[i] -= h
        assert (L(p) - L(m)) / (2 * h) == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_network_gradient_matches_autograd():
    """The whole network written with torch ops (conv2d, relu, linear) and
    differentiated by autograd gives the same flat gradient."""
    conv, params, x, t = _tiny()
    y, acts = net.forward(params, x, conv)
    _, dy = net.loss_and_grad(y, t)
    g = net.backward(params, acts, dy, conv)
    pt = torch.tensor(params, requires_grad=True)
    items, _ = net.param_layout(conv, x.shape[1], x.shape[2])
    P = {n: pt[o:o + int(np.prod(s))].reshape(s) for n, s, o in items}
    a = torch.tensor(x).permute(0, 3, 1, 2)
    for i in range(len(conv)):
        a = torch.relu(torch.nn.functional.conv2d(a, P[f"conv{i}.W"].permute(0, 3, 1, 2),
                                                  P[f"conv{i}.b"], stride=2, padding=1))
    f = a.permute(0, 2, 3, 1).reshape(x.shape[0], -1)
    hdn = torch.relu(f @ P["fc1.W"].T + P["fc1.b"])
    yt = hdn @ P["fc2.W"].T + P["fc2.b"]
    np.testing.assert_allclose(yt.detach().numpy(), y, rtol=1e-12, atol=1e-12)
    (0.5 * ((yt - torch.tensor(t)) ** 2).sum() / x.shape[0]).backward()
    np.testing.assert_allclose(g, pt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_bf16_mode_rounds_only_at_storage_points():
    """With every stored value already a bfloat16 the bf16 mode differs from
    the exact mode only through the rounding of the activations."""
    conv, params, x, t = _tiny()
    xb = net.to_bf16(x)
    y0, _ = net.forward(params, xb, conv)
    y1, acts = net.forward(params, xb, conv, bf16=True)
    assert np.all([np.array_equal(a, net.to_bf16(a)) for a in acts])
    assert np.abs(y1 - y0).max() < 3e-2 * np.abs(y0).max()


def test_target_delta_recovers_the_ground_truth_pose():
    for seed in range(5):
        gt = scenes.room_pose(seed)
        init = scenes.perturb_pose(gt, 0.05, 3.0, seed=100 + seed)
        d = net.target_delta(init, gt)
        back = net.apply_delta(init, d)
        np.testing.assert_allclose(back.R, gt.R, atol=1e-12)
        np.testing.assert_allclose(back.t, gt.t, atol=1e-12)
        # magnitudes: |rho| ~ translation of the camera frame, |theta| = 3 degrees
        assert np.linalg.norm(d[3:] * net.TAU_SCALE[3:]) == pytest.approx(np.radians(3.0), rel=1e-9)


def test_pack_input_closed_form():
    r_rgb = np.full((1, 2, 2, 3), 0.25)
    r_d = np.array([[[2.0, 1.5], [0.0, 3.0]]])
    r_o = np.array([[[1.0, 0.5], [0.0, 0.75]]])
    o_rgb = np.full((1, 2, 2, 3), 0.5)
    o_d = np.array([[[2.5, 0.0], [4.0, 1.0]]])
    x = net.pack_input(r_rgb, r_d, r_o, o_rgb, o_d)
    assert x.shape == (1, 2, 2, 8)
    np.testing.assert_array_equal(x[0, :, :, 3], [[-0.5, 0.0], [0.0, 1.5]])
    np.testing.assert_array_equal(x[0, :, :, 7], [[0.0, 0.0], [1.5, -1.5]])
    np.testing.assert_array_equal(x[..., :3], 0.25)
    np.testing.assert_array_equal(x[..., 4:7], 0.5)


def test_net_init_draws_he_normal_weights_and_zero_biases():
    items, total = net.param_layout()
    blocks = [(int(np.prod(s)), int(np.prod(s[1:])) if len(s) > 1 else 0) for _, s, _ in items]
    p = scenes.net_init(7, blocks)
    assert p.dtype == np.float32 and p.size == total
    P = net.unflatten(p.astype(np.float64))
    for name, shape, _ in items:
        v = P[name]
        if name.endswith(".b"):
            assert np.all(v == 0)
        elif v.size > 5000:
            assert np.std(v) == pytest.approx(net.he_scale(int(np.prod(shape[1:]))), rel=0.05)


def test_downsample_rgbd_hand_case():
    from oracle import net
    rgb = np.zeros((4, 4, 3))
    rgb[:2, :2] = 1.0
    rgb[2:, 2:, 0] = 0.5
    depth = np.array([[1.0, 3.0, 0.0, 0.0],
                      [0.0, 2.0, 0.0, 0.0],
                      [5.0, 5.0, 4.0, np.inf],
                      [5.0, 5.0, 0.0, 2.0]])
    c, d = net.downsample_rgbd(rgb, depth, 2)
    np.testing.assert_allclose(c[0, 0], 1.0)
    np.testing.assert_allclose(c[1, 1], [0.5, 0.0, 0.0])
    np.testing.assert_allclose(c[0, 1], 0.0)
    # means of the valid depths; a block without any is 0
    np.testing.assert_allclose(d, [[2.0, 0.0], [5.0, 3.0]])

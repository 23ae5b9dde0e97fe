"""GPU parity of the learned-proposal network kernels (include/gs2d_net.h)
against the FP64 oracle (oracle/net.py) in its bfloat16-storage mode: the
same values are rounded to bfloat16 at the same points, so the remaining
differences come from FP32 accumulation order on the tensor cores and the
bfloat16 roundings it flips (one unit in the last place, 2^-8 relative,
propagating through later layers)."""
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


def _setup(torch, B, seed=0):
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    params = scenes.net_init(seed, gs2d.net_init_blocks())
    rng = np.random.default_rng(seed + 1)
    # small random biases so the bias paths are exercised
    items, _ = net.param_layout()
    for name, shape, off in items:
        if name.endswith(".b"):
            params[off:off + shape[0]] = rng.normal(0, 0.05, shape[0])
    x = net.to_bf16(rng.uniform(-1.0, 1.0, (B, 120, 160, 8)))
    t = rng.normal(0, 1, (B, 6))
    P = torch.tensor(params, device="cuda")
    X = torch.tensor(x, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    ws = torch.empty(gs2d.gs2d_net_workspace(B), dtype=torch.uint8, device="cuda")
    return params.astype(np.float64), x, t, P, X, T, ws


def test_net_forward_matches_oracle(torch_cuda):
    torch = torch_cuda
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    params, x, t, P, X, T, ws = _setup(torch, 3)
    y = torch.empty(3, 6, device="cuda")
    gs2d.gs2d_net_forward(P, X, y, ws)
    torch.cuda.synchronize()
    yo, _ = net.forward(params, x, bf16=True)
    err = np.abs(to_np(y) - yo)
    assert err.max() <= 1e-2 * np.abs(yo).max(), (err.max(), np.abs(yo).max())


def test_net_rows_are_independent_of_batch_tiling(torch_cuda):
    """Each output row's accumulation order does not depend on the batch
    size (M tiling), so a ragged batch equals per-sample calls bit for bit."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    params, x, t, P, X, T, ws = _setup(torch, 37, seed=3)
    y = torch.empty(37, 6, device="cuda")
    gs2d.gs2d_net_forward(P, X, y, ws)
    ws1 = torch.empty(gs2d.gs2d_net_workspace(1), dtype=torch.uint8, device="cuda")
    for b in (0, 17, 36):
        y1 = torch.empty(1, 6, device="cuda")
        gs2d.gs2d_net_forward(P, X[b:b + 1].contiguous(), y1, ws1)
        torch.cuda.synchronize()
        assert torch.equal(y1[0], y[b]), b


def test_net_rows_of_a_full_batch_equal_single_samples(torch_cuda):
    """At a batch that fills the GPU (160 samples) the layers 2-4
    convolutions run with fewer pipeline stages per CTA than for a single
    sample; a tile sums its K steps in the same order either way, so rows
    of the full batch equal single-sample calls bit for bit."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    params, x, t, P, X, T, ws = _setup(torch, 160, seed=5)
    y = torch.empty(160, 6, device="cuda")
    gs2d.gs2d_net_forward(P, X, y, ws)
    ws1 = torch.empty(gs2d.gs2d_net_workspace(1), dtype=torch.uint8, device="cuda")
    for b in (0, 77, 159):
        y1 = torch.empty(1, 6, device="cuda")
        gs2d.gs2d_net_forward(P, X[b:b + 1].contiguous(), y1, ws1)
        torch.cuda.synchronize()
        assert torch.equal(y1[0], y[b]), b


def _exact_setup(torch, B, seed):
    """Inputs on which every FP32 accumulation is exact: x and the biases
    integer multiples of 1/4, weights sparse in {-1, 0, 1} (about 3.5
    non-zero taps per output), targets multiples of 1/4, B a power of two.
    Every stored value is then a multiple of 1/16 well inside FP32's 24-bit
    range, both sides round the same exact values to bfloat16 at the same
    points, and the results must agree bit for bit."""
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(seed)
    items, total = net.param_layout()
    params = np.zeros(total)
    for name, shape, off in items:
        n = int(np.prod(shape))
        if name.endswith(".b"):
            params[off:off + n] = rng.integers(-1, 2, n) * 0.25
        else:
            fan = int(np.prod(shape[1:]))
            nz = rng.uniform(size=n) < 3.5 / fan
            params[off:off + n] = np.where(nz, rng.choice([-1.0, 1.0], n), 0.0)
    x = rng.integers(-4, 5, (B, 120, 160, 8)) * 0.25
    t = rng.integers(-8, 9, (B, 6)) * 0.25
    P = torch.tensor(params, dtype=torch.float32, device="cuda")
    X = torch.tensor(x, dtype=torch.float32, device="cuda").to(torch.bfloat16)
    T = torch.tensor(t, dtype=torch.float32, device="cuda")
    ws = torch.empty(gs2d.gs2d_net_workspace(B), dtype=torch.uint8, device="cuda")
    return params, x, t, P, X, T, ws


@pytest.mark.parametrize("B", [4, 32])
def test_net_is_bit_exact_on_exactly_representable_inputs(torch_cuda, B):
    """Every GEMM form (conv forward, data and weight gradients, both fully
    connected layers' three products), every epilogue, the bias gradients,
    the loss and the split-K reductions, pinned bit for bit.  At batch 32
    the first two layers' direct backward kernels walk more tiles than
    their grids hold blocks, so their next-tile staging runs too."""
    torch = torch_cuda
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    params, x, t, P, X, T, ws = _exact_setup(torch, B, seed=21)
    loss = torch.empty(1, device="cuda")
    grad = torch.empty(gs2d.gs2d_net_param_count(), device="cuda")
    y = torch.empty(B, 6, device="cuda")
    gs2d.gs2d_net_grad(P, X, T, loss, grad, ws, y=y)
    torch.cuda.synchronize()
    yo, acts = net.forward(params, x, bf16=True)
    Lo, dy = net.loss_and_grad(yo, t)
    go = net.backward(params, acts, dy, bf16=True)
    assert np.abs(yo).max() > 0 and np.count_nonzero(go) > 1000
    np.testing.assert_array_equal(to_np(y), yo)
    assert float(loss.item()) == pytest.approx(Lo, rel=1e-6)
    g = to_np(grad)
    items, _ = net.param_layout()
    for name, shape, off in items:
        n = int(np.prod(shape))
        np.testing.assert_array_equal(g[off:off + n], go[off:off + n], err_msg=name)


def test_net_grad_matches_oracle(torch_cuda):
    """Random inputs: bfloat16 rounding flips ReLU masks (a unit active in
    one evaluation and not the other moves a whole row of its weight
    gradient), so the GPU is compared with the oracle's bfloat16 mode per
    layer in the L2 norm, against the oracle's own bfloat16-vs-FP64
    difference: both are rounding noise of the same size."""
    torch = torch_cuda
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    B = 4
    params, x, t, P, X, T, ws = _setup(torch, B, seed=5)
    loss = torch.empty(1, device="cuda")
    grad = torch.empty(gs2d.gs2d_net_param_count(), device="cuda")
    y = torch.empty(B, 6, device="cuda")
    gs2d.gs2d_net_grad(P, X, T, loss, grad, ws, y=y)
    torch.cuda.synchronize()
    yo, acts = net.forward(params, x, bf16=True)
    Lo, dy = net.loss_and_grad(yo, t)
    go = net.backward(params, acts, dy, bf16=True)
    ye, ae = net.forward(params, x)
    _, dye = net.loss_and_grad(ye, t)
    ge = net.backward(params, ae, dye)
    assert float(loss.item()) == pytest.approx(Lo, rel=1e-2)
    g = to_np(grad)
    items, _ = net.param_layout()
    for name, shape, off in items:
        sl = slice(off, off + int(np.prod(shape)))
        a, r, e = g[sl], go[sl], ge[sl]
        noise = np.linalg.norm(r - e)
        assert np.linalg.norm(a - r) <= 2.0 * noise + 1e-3 * np.linalg.norm(r), \
            (name, np.linalg.norm(a - r), noise, np.linalg.norm(r))


def test_pack_input_matches_oracle(torch_cuda):
    torch = torch_cuda
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(9)
    B, H, W = 2, 12, 20
    r_rgb = rng.uniform(0, 1, (B, H, W, 3)).astype(np.float32)
    r_o = np.where(rng.uniform(size=(B, H, W)) < 0.3, rng.uniform(0, 0.6, (B, H, W)),
                   rng.uniform(0.6, 1.0, (B, H, W))).astype(np.float32)
    r_d = (r_o * rng.uniform(0.5, 5.0, (B, H, W))).astype(np.float32)
    o_rgb = rng.uniform(0, 1, (B, H, W, 3)).astype(np.float32)
    o_d = np.where(rng.uniform(size=(B, H, W)) < 0.1, 0.0,
                   rng.uniform(0.5, 5.0, (B, H, W))).astype(np.float32)
    T = lambda a: torch.tensor(a, device="cuda")
    x = torch.empty(B, H, W, 8, dtype=torch.bfloat16, device="cuda")
    gs2d.gs2d_net_pack_input(T(r_rgb), T(r_d), T(r_o), T(o_rgb), T(o_d), x)
    torch.cuda.synchronize()
    got = x.float().cpu().numpy().astype(np.float64)
    ref = net.pack_input(r_rgb.astype(np.float64), r_d.astype(np.float64), r_o.astype(np.float64),
                         o_rgb.astype(np.float64), o_d.astype(np.float64))
    np.testing.assert_array_equal(got[..., [0, 1, 2, 4, 5, 6, 7]], ref[..., [0, 1, 2, 4, 5, 6, 7]])
    # the rendered depth D/O is an FP32 division before the bf16 rounding:
    # at most one bfloat16 step apart
    d = np.abs(got[..., 3] - ref[..., 3])
    assert np.all(d <= 2.0 ** -7 * np.maximum(np.abs(ref[..., 3]), 1e-30) + 1e-30)


def test_adamw_and_apply_match_oracle(torch_cuda):
    torch = torch_cuda
    import oracle
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(11)
    n = 1000
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    p, g = f32(rng.normal(size=n)), f32(rng.normal(size=n))
    m, v = f32(rng.normal(size=n) * 0.1), f32(rng.uniform(0, 0.1, n))
    st = oracle.AdamState(m.copy(), v.copy(), step=4)
    # the kernel takes its hyper-parameters as FP32 values: so does the oracle
    hp = [float(np.float32(z)) for z in (1e-3, 0.9, 0.999, 1e-8, 0.01)]
    ref = oracle.adamw_step(p, g, st, lr=hp[0], betas=(hp[1], hp[2]), eps=hp[3], wd=hp[4])
    T = lambda a: torch.tensor(np.asarray(a, np.float32), device="cuda")
    P, G, M, V = T(p), T(g), T(m), T(v)
    gs2d.gs2d_net_adamw(P, G, M, V, 5, lr=1e-3, wd=0.01)
    torch.cuda.synchronize()
    np.testing.assert_allclose(to_np(P), ref, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(to_np(M), st.m, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(to_np(V), st.v, rtol=1e-5, atol=1e-8)
    # proposals applied on the left
    poses = [scenes.room_pose(s) for s in range(5)]
    y = rng.normal(0, 1, (5, 6))
    pt = torch.stack([gs2d.pose_tensor(q) for q in poses])
    gs2d.gs2d_net_apply(T(y), pt)
    torch.cuda.synchronize()
    for b in range(5):
        ref = net.apply_delta(poses[b], y[b])
        got = pt[b].cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got[:9].reshape(3, 3), ref.R, atol=2e-6)
        np.testing.assert_allclose(got[9:], ref.t, atol=2e-5)


def test_net_training_reduces_the_loss(torch_cuda):
    """A few hundred AdamW steps on one fixed batch fit it (the kernels'
    gradient is a descent direction of the kernels' loss)."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    B = 16
    params, x, t, P, X, T, ws = _setup(torch, B, seed=13)
    T.mul_(0.5)
    n = gs2d.gs2d_net_param_count()
    grad = torch.empty(n, device="cuda")
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    loss = torch.empty(1, device="cuda")
    hist = []
    for step in range(1, 201):
        gs2d.gs2d_net_grad(P, X, T, loss, grad, ws)
        gs2d.gs2d_net_adamw(P, grad, m, v, step, lr=1e-3)
        if step == 1 or step % 50 == 0:
            hist.append(float(loss.item()))
    assert hist[-1] < 0.05 * hist[0], hist


def test_target_and_accept_kernels(torch_cuda):
    torch = torch_cuda
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    gts = [scenes.room_pose(40 + i) for i in range(6)]
    inits = [scenes.perturb_uniform(g, 0.05, 3.0, seed=60 + i) for i, g in enumerate(gts)]
    inits[0] = gts[0]                      # zero delta
    inits[1] = scenes.perturb_pose(gts[1], 0.0, 0.004, seed=3)   # tiny angle, series branch
    I = torch.stack([gs2d.pose_tensor(p) for p in inits])
    G = torch.stack([gs2d.pose_tensor(p) for p in gts])
    tgt = torch.empty(6, 6, device="cuda")
    gs2d.gs2d_net_target(I, G, tgt)
    torch.cuda.synchronize()
    for b in range(6):
        # the oracle on the same FP32 poses
        Pi = I[b].cpu().numpy().astype(np.float64)
        Pg = G[b].cpu().numpy().astype(np.float64)
        ref = net.target_delta(scenes.Pose(Pi[:9].reshape(3, 3), Pi[9:]),
                               scenes.Pose(Pg[:9].reshape(3, 3), Pg[9:]))
        np.testing.assert_allclose(tgt[b].cpu().numpy(), ref, atol=2e-4, err_msg=str(b))
    lp = torch.tensor([1.0, 2.0, 3.0, 3.0, 0.5, 9.0], device="cuda")
    li = torch.tensor([2.0, 1.0, 3.0, 2.0, 0.6, 8.0], device="cuda")
    prop = torch.arange(72, dtype=torch.float32, device="cuda").reshape(6, 12)
    poses = -torch.ones(6, 12, device="cuda")
    acc = torch.empty(6, dtype=torch.int32, device="cuda")
    gs2d.gs2d_net_accept(lp, li, prop, poses, acc)
    torch.cuda.synchronize()
    want = [1, 0, 1, 0, 1, 0]
    assert acc.cpu().tolist() == want
    for b in range(6):
        assert torch.equal(poses[b], prop[b] if want[b] else -torch.ones(12, device="cuda"))


def test_accept_keep_copies_the_taken_images_and_losses(torch_cuda):
    """gs2d_net_accept_keep: the same decisions as gs2d_net_accept; where a
    proposal is taken its images and loss replace the kept ones, elsewhere
    the kept ones are untouched (bit for bit)."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    B, H, W = 6, 7, 9
    g = torch.Generator(device="cuda")
    g.manual_seed(4)
    lp = torch.tensor([1.0, 2.0, 3.0, 3.0, 0.5, 9.0], device="cuda")
    li = torch.tensor([2.0, 1.0, 3.0, 2.0, 0.6, 8.0], device="cuda")
    prop = torch.arange(72, dtype=torch.float32, device="cuda").reshape(6, 12)
    poses = -torch.ones(6, 12, device="cuda")
    acc = torch.empty(6, dtype=torch.int32, device="cuda")
    P = [torch.rand(B, H, W, 3, generator=g, device="cuda"), torch.rand(B, H, W, generator=g, device="cuda"),
         torch.rand(B, H, W, generator=g, device="cuda")]
    K = [torch.rand(B, H, W, 3, generator=g, device="cuda"), torch.rand(B, H, W, generator=g, device="cuda"),
         torch.rand(B, H, W, generator=g, device="cuda")]
    K0 = [k.clone() for k in K]
    li0 = li.clone()
    gs2d.gs2d_net_accept_keep(lp, li, prop, poses, P, K, acc)
    torch.cuda.synchronize()
    want = [1, 0, 1, 0, 1, 0]
    assert acc.cpu().tolist() == want
    for b in range(B):
        take = bool(want[b])
        assert torch.equal(poses[b], prop[b] if take else -torch.ones(12, device="cuda"))
        assert float(li[b]) == float(lp[b] if take else li0[b])
        for k, p0, k0 in zip(K, P, K0):
            assert torch.equal(k[b], p0[b] if take else k0[b])


def test_downsample_rgbd_matches_oracle(torch_cuda):
    """640x480 -> 160x120 box downsampling of an observation with holes:
    block sums of 16 values in FP32 against FP64 (1e-6 relative); blocks
    without a valid depth are 0 on both sides."""
    torch = torch_cuda
    from oracle import net
    from paper_2506_00970_gb300 import gs2d
    cam = scenes.tracking_camera()
    rgb, depth = scenes.rgbd_frame(3, cam, hole_frac=0.3)
    depth[:8, :8] = 0.0                      # a block of holes
    c_o, d_o = net.downsample_rgbd(rgb, depth, 4)
    T = lambda a: torch.tensor(a, device="cuda")
    c = torch.empty(120, 160, 3, device="cuda")
    d = torch.empty(120, 160, device="cuda")
    gs2d.gs2d_net_downsample_rgbd(T(rgb), T(depth), 4, c, d)
    torch.cuda.synchronize()
    np.testing.assert_allclose(c.cpu().numpy(), c_o, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(d.cpu().numpy(), d_o, rtol=1e-6, atol=0)
    assert float(d[0, 0]) == 0.0 and float(d[0, 1]) == 0.0


def test_prepared_forward_is_the_forward(torch_cuda):
    """gs2d_net_forward_prepared after gs2d_net_prepare gives the bits of
    gs2d_net_forward (the same bfloat16 weights, cast once)."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    params = torch.tensor(scenes.net_init(4, gs2d.net_init_blocks()), device="cuda")
    x = (torch.rand(3, 120, 160, 8, device="cuda") * 2 - 1).to(torch.bfloat16)
    ws = torch.empty(gs2d.gs2d_net_workspace(3), dtype=torch.uint8, device="cuda")
    y0 = torch.empty(3, 6, device="cuda")
    y1 = torch.empty(3, 6, device="cuda")
    gs2d.gs2d_net_forward(params, x, y0, ws)
    ws.zero_()
    gs2d.gs2d_net_prepare(params, 3, ws)
    gs2d.gs2d_net_forward_prepared(params, x, y1, ws)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)

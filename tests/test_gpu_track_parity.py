"""Element-wise parity of the fused tracking call gs2d_track_step with the
oracle, iteration by iteration (the tracking loop of Sec. III-D: the masked
L1 loss of Eq. tracking_loss, its pose gradient through Sec. III-B's
Eq. derivatives, AdamW on tau and the left retraction T <- Exp(tau) T).

Each iteration k is checked at the pose the GPU actually held before it
(pose_hist[k-1], the start pose for k = 0), so FP32 rounding never
compounds across iterations:
  * loss_hist[k] against the oracle's loss at that pose: 1e-4 relative;
  * grad_hist[k] (the 6-vector the fused kernel hands to AdamW) against the
    oracle's pose gradient there: 1e-3 of its largest component;
  * pose_hist[k] against the oracle's AdamW step (moments fed with the GPU's
    gradients) and retraction applied to that pose: 2e-6.
Exemptions come from the oracle only, each with the amount it may move:
pixels whose opacity or normal-mask value lies within 1e-5 of the mask
threshold (an FP32 transmittance differs from the FP64 one by about 1e-6
there): the pixel's whole term; pixels whose L1 residual lies within 1e-5 of
zero (the sub-gradient of |x| is not unique there): twice its term; pixels
with a compositing decision on a threshold (oracle ``ambiguous``): the
largest change of the pixel's term when the oracle re-evaluates it with one
threshold moved by the diagnostic's margin.  The oracle evaluates these
terms pixel by pixel, and the test also checks that they stay a small
fraction of the bound they widen.

The observation is the ground-truth render shifted by +0.3 in colour and by
5% in depth, so every active residual is bounded away from zero and the loss
is differentiable at every pixel; the tracking itself (convergence from a
2 cm / 1 degree start) is tested on unshifted observations elsewhere.
Configurations: the grouped one-pixel loops (160x120, 80 tiles), the plain
one-pixel loops (the grouped form switched off), three pixels per thread,
and the 640x480 default path.
"""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes

pytestmark = pytest.mark.gpu

MASK_MARGIN = 1e-5
RESID_MARGIN = 1e-5
TOL_LOSS = 1e-4
TOL_G = 1e-3
TOL_POSE = 2e-6


def F32(x):
    """The FP64 value of an FP32 number."""
    return float(np.float32(x))


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


def _scene(orc, n, scale_cm, cam, seed=0):
    """Room scene with the surfels seen within ~3 degrees of edge-on at the
    ground-truth or the start pose removed (an oracle pre-pass): their FP32
    intersection is ill-conditioned, and the pose gradient sums every
    surfel."""
    s = scenes.room_scene(seed, n, scale_cm=scale_cm)
    gt = scenes.room_pose(seed + 1)
    start = scenes.perturb_pose(gt, 0.02, 1.0, seed=seed + 4)
    keep = np.ones(s.n, bool)
    H, W = cam.height, cam.width
    ones = (np.ones((H, W, 3)), np.ones((H, W)), np.zeros((H, W, 3)), np.zeros((H, W)))
    for p in (gt, start):
        keep &= orc.render_bwd(s, cam, p, *ones)["min_cos"] > 0.05
    s = scenes.Surfels(s.mu[keep], s.quat[keep], s.scale[keep], s.opacity[keep], s.rgb[keep])
    return s, gt, start


def _observation(orc, s, cam, gt):
    o = orc.render(s, cam, gt)
    rgb = (o["rgb"] + 0.3).astype(np.float32)
    depth = (1.05 * o["depth"] / np.maximum(o["opacity"], 1e-6)).astype(np.float32)
    return rgb, depth


def _rays(cam):
    x = (np.arange(cam.width) + 0.5 - cam.cx) / cam.fx
    y = (np.arange(cam.height) + 0.5 - cam.cy) / cam.fy
    return np.meshgrid(x, y)


def _pixel_term(orc, s, cam, pose, x, y, obs_rgb, obs_d, rule=None, force_active=False,
                lam=1.0):
    """Loss term and pose gradient of pixel (x, y) alone under the oracle's
    compositing rules `rule` and the camera `cam` (force_active: both masks
    taken as on)."""
    pix = np.array([[x, y]], np.int32)
    rule = rule or orc.Rule()
    o = orc.render(s, cam, pose, rule, pixels=pix)
    P = cam.width * cam.height
    rx, ry = (x + 0.5 - cam.cx) / cam.fx, (y + 0.5 - cam.cy) / cam.fy
    O = o["opacity"][0]
    nr = o["normal"][0] @ np.array([rx, ry, 1.0])
    if not (force_active or (nr > 0 and O > 0.95)):
        return 0.0, np.zeros(6)
    Oc = max(O, 1e-6)
    D = o["depth"][0]
    res_d = D / Oc - obs_d[y, x]
    loss = (np.abs(o["rgb"][0] - obs_rgb[y, x]).sum() + lam * abs(res_d)) / P
    sd = lam * np.sign(res_d) / P
    up = ((np.sign(o["rgb"][0] - obs_rgb[y, x]) / P)[None], np.array([sd / Oc]), np.zeros((1, 3)),
          np.array([-sd * D / (O * O) if O > 1e-6 else 0.0]))
    return loss, orc.render_bwd(s, cam, pose, *up, rule=rule, pixels=pix)["pose6"]


def _nudged(orc, cam):
    """The oracle's rules and cameras with one threshold moved by the margin
    of its threshold diagnostic, each way."""
    t, ts = orc.AMBIGUITY_TIGHT, orc.AMBIGUITY_STOP
    base = orc.Rule()
    out = []
    for sgn in (-1.0, 1.0):
        out.append((orc.Rule(cutoff_r2=base.cutoff_r2 * (1 + sgn * t)), cam))
        out.append((orc.Rule(alpha_min=base.alpha_min * (1 + sgn * t)), cam))
        out.append((orc.Rule(t_min=base.t_min * (1 + sgn * ts)), cam))
        out.append((base, scenes.Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                                        cam.near * (1 + sgn * t))))
    return out


def _allowances(orc, s, cam, pose, img, obs_rgb, obs_d, lam=1.0):
    """Pixels whose mask, residual sign or compositing decision FP32 may take
    otherwise (all decided by the oracle), and the loss and gradient they can
    move.  A mask within MASK_MARGIN of its threshold: the pixel's whole term
    (a flip adds or drops it).  A residual within RESID_MARGIN of zero:
    twice its term (a sign flip).  A compositing decision on a threshold
    (oracle ``ambiguous``): the largest change of the pixel's term when one
    threshold moves by the oracle's margin either way."""
    X, Y = _rays(cam)
    O = img["opacity"]
    N = img["normal"]
    nr = N[..., 0] * X + N[..., 1] * Y + N[..., 2]
    Dh = img["depth"] / np.maximum(O, 1e-6)
    on = (nr > 0) & (O > 0.95)
    near_o = np.abs(O - 0.95) <= MASK_MARGIN
    near_n = (np.abs(nr) <= MASK_MARGIN * O * (np.abs(X) + np.abs(Y) + 1)) & (O > 0.95 - MASK_MARGIN)
    near_0 = on & ((np.abs(img["rgb"] - obs_rgb) <= RESID_MARGIN).any(-1)
                   | (np.abs(Dh - obs_d) <= RESID_MARGIN * np.abs(Dh)))
    thr = img["ambiguous"] & ~(near_o | near_n | near_0)
    amb = near_o | near_n | near_0 | thr
    loss_allow, g_allow = 0.0, np.zeros(6)
    for y, x in zip(*np.nonzero(near_o | near_n | near_0)):
        lp, gp = _pixel_term(orc, s, cam, pose, x, y, obs_rgb, obs_d, force_active=True, lam=lam)
        k = 2.0 if near_0[y, x] else 1.0
        loss_allow += lp
        g_allow += k * np.abs(gp)
    nudged = _nudged(orc, cam)
    for y, x in zip(*np.nonzero(thr)):
        l0, g0 = _pixel_term(orc, s, cam, pose, x, y, obs_rgb, obs_d, lam=lam)
        dl, dg = 0.0, np.zeros(6)
        for rule, c in nudged:
            l1, g1 = _pixel_term(orc, s, c, pose, x, y, obs_rgb, obs_d, rule=rule, lam=lam)
            dl = max(dl, abs(l1 - l0))
            dg = np.maximum(dg, np.abs(g1 - g0))
        loss_allow += dl
        g_allow += dg
    return int(amb.sum()), loss_allow, g_allow


CASES = {
    "160x120_grouped_p1": (scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120), 8000, (6.0, 10.0),
                           (16, 16), 1, -1, 8),
    "160x120_plain_p1": (scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120), 8000, (6.0, 10.0),
                         (16, 16), 1, 0, 8),
    "160x120_p3": (scenes.Camera(150.0, 150.0, 80.0, 60.0, 160, 120), 8000, (6.0, 10.0),
                   (32, 24), 3, -1, 8),
    "640x480_plain_p1": (scenes.Camera(525.0, 525.0, 320.0, 240.0, 640, 480), 5000, (8.0, 12.0),
                         (16, 16), 1, -1, 3),
}


@pytest.mark.parametrize("case", list(CASES))
def test_track_step_iterations_match_oracle(torch_cuda, orc, case):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    cam, n, scale_cm, tile, px, grouped, n_iter = CASES[case]
    s, gt, start = _scene(orc, n, scale_cm, cam)
    obs_rgb, obs_d = _observation(orc, s, cam, gt)
    ds = gs2d.DeviceSurfels(s)
    ccam, cfg = gs2d.camera(cam), gs2d.default_config(tile, px)
    prm = gs2d.default_track_params(stop_tol=0.0)
    cap = 256 * s.n
    ws = torch.empty(gs2d.gs2d_track_workspace(s.n, cap, ccam, cfg), dtype=torch.uint8, device="cuda")
    f = dict(dtype=torch.float32, device="cuda")
    pose = gs2d.pose_tensor(start)
    adam = torch.zeros(16, **f)
    lh, ph, gh = torch.zeros(n_iter, **f), torch.zeros(n_iter, 12, **f), torch.zeros(n_iter, 6, **f)
    gs2d.gs2d_set_grouped_tiles(grouped)
    try:
        gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, torch.tensor(obs_rgb, device="cuda"),
                             torch.tensor(obs_d, device="cuda"), n_iter, cap, lh, ph, ws,
                             adam_state=adam, grad_hist=gh)
        torch.cuda.synchronize()
    finally:
        gs2d.gs2d_set_grouped_tiles(-1)
    assert int(gs2d.gs2d_track_status(ws).item()) == 0
    lh = lh.cpu().numpy().astype(np.float64)
    ph = ph.cpu().numpy().astype(np.float64)
    gh = gh.cpu().numpy().astype(np.float64)
    o_rgb, o_d = obs_rgb.astype(np.float64), obs_d.astype(np.float64)
    st = orc.AdamState(np.zeros(6), np.zeros(6))
    pose_k = start
    n_amb_total = 0
    for k in range(n_iter):
        if k:
            pose_k = scenes.Pose(ph[k - 1, :9].reshape(3, 3), ph[k - 1, 9:])
        img = orc.render(s, cam, pose_k)
        L, g = orc.tracking_loss(img, o_rgb, o_d, cam)
        og = orc.render_bwd(s, cam, pose_k, g["rgb"], g["depth"], g["normal"], g["opacity"])["pose6"]
        n_amb, loss_allow, g_allow = _allowances(orc, s, cam, pose_k, img, o_rgb, o_d)
        n_amb_total += n_amb
        scale = np.abs(og).max()
        assert L > 0.1 and scale > 0
        # the exemptions stay small next to what they exempt
        assert n_amb <= 5e-3 * cam.width * cam.height, (k, n_amb)
        assert np.all(g_allow <= 3.0 * TOL_G * scale), (k, g_allow / scale)
        assert loss_allow <= 10.0 * TOL_LOSS * L, (k, loss_allow / L)
        assert abs(lh[k] - L) <= TOL_LOSS * L + loss_allow, (k, lh[k], L, loss_allow)
        err = np.abs(gh[k] - og)
        assert np.all(err <= TOL_G * scale + g_allow), (k, err / scale, g_allow / scale)
        # AdamW on the GPU's gradient and the left retraction, in FP64 with
        # the hyper-parameters the ABI takes (FP32: 1 - beta2 of the FP32
        # 0.999 differs from the FP64 one by 1.3e-5 relative)
        tau = orc.adamw_step(np.zeros(6), gh[k], st, lr=F32(prm.lr),
                             betas=(F32(prm.beta1), F32(prm.beta2)), eps=F32(prm.eps))
        ref = orc.retract(pose_k, tau)
        np.testing.assert_allclose(ph[k, :9], ref.R.reshape(-1), rtol=0, atol=TOL_POSE)
        np.testing.assert_allclose(ph[k, 9:], ref.t, rtol=0,
                                   atol=TOL_POSE * (1.0 + np.abs(ref.t).max()))
    # the caller's AdamW state holds the moments and the step count
    a = adam.cpu().numpy().astype(np.float64)
    assert a[12] == n_iter
    np.testing.assert_allclose(a[:6], st.m, rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(a[6:12], st.v, rtol=1e-5, atol=1e-18)
    np.testing.assert_array_equal(pose.cpu().numpy(), ph[-1].astype(np.float32))


def test_track_step_split_calls_are_bit_identical(torch_cuda, orc):
    """A frame run as 2 + 4 iterations in two calls that share the caller's
    AdamW state gives the same bits as one call of 6."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    cam, n, scale_cm, tile, px, _, _ = CASES["160x120_grouped_p1"]
    s = scenes.room_scene(5, n, scale_cm=scale_cm)
    gt = scenes.room_pose(6)
    o = orc.render(s, cam, gt)
    obs_rgb = torch.tensor(o["rgb"].astype(np.float32), device="cuda")
    obs_d = torch.tensor((o["depth"] / np.maximum(o["opacity"], 1e-6)).astype(np.float32), device="cuda")
    start = gs2d.pose_tensor(scenes.perturb_pose(gt, 0.02, 1.0, seed=9))
    ds = gs2d.DeviceSurfels(s)
    ccam, cfg = gs2d.camera(cam), gs2d.default_config(tile, px)
    prm = gs2d.default_track_params(stop_tol=0.0)
    cap = 256 * s.n
    ws = torch.empty(gs2d.gs2d_track_workspace(s.n, cap, ccam, cfg), dtype=torch.uint8, device="cuda")
    f = dict(dtype=torch.float32, device="cuda")

    def run(splits):
        pose = start.clone()
        adam = torch.zeros(16, **f)
        lh, ph, gh = [], [], []
        for m in splits:
            l, p, g = torch.zeros(m, **f), torch.zeros(m, 12, **f), torch.zeros(m, 6, **f)
            gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, m, cap, l, p, ws,
                                 adam_state=adam, grad_hist=g)
            torch.cuda.synchronize()
            assert int(gs2d.gs2d_track_status(ws).item()) == 0
            lh.append(l), ph.append(p), gh.append(g)
        return pose, adam, torch.cat(lh), torch.cat(ph), torch.cat(gh)

    one, two = run([6]), run([2, 4])
    for a, b in zip(one, two):
        assert torch.equal(a, b)
    assert float(one[1][12].item()) == 6.0
    # without a caller state every call starts from zero moments
    pose = start.clone()
    l = torch.zeros(4, **f)
    gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, 2, cap, l[:2], None, ws)
    gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, 2, cap, l[2:], None, ws)
    torch.cuda.synchronize()
    assert torch.equal(l[:2], one[2][:2])
    assert not torch.equal(pose, one[3][3])


def test_track_step_nonfinite_observation_keeps_the_pose(torch_cuda, orc):
    """A NaN in the observed depth at an active pixel makes the loss
    non-finite: the call records GS2D_ERR_NONFINITE, leaves the pose and the
    AdamW state as they were, and every later iteration skips its work."""
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    cam, n, scale_cm, tile, px, _, _ = CASES["160x120_grouped_p1"]
    s = scenes.room_scene(7, n, scale_cm=scale_cm)
    gt = scenes.room_pose(8)
    o = orc.render(s, cam, gt)
    d = (o["depth"] / np.maximum(o["opacity"], 1e-6)).astype(np.float32)
    ys, xs = np.nonzero(o["opacity"] > 0.99)
    assert len(ys) > 100
    d[ys[::50], xs[::50]] = np.nan
    obs_rgb = torch.tensor(o["rgb"].astype(np.float32), device="cuda")
    obs_d = torch.tensor(d, device="cuda")
    start = gs2d.pose_tensor(scenes.perturb_pose(gt, 0.002, 0.1, seed=3))
    ds = gs2d.DeviceSurfels(s)
    ccam, cfg = gs2d.camera(cam), gs2d.default_config()
    prm = gs2d.default_track_params()
    cap = 256 * s.n
    ws = torch.empty(gs2d.gs2d_track_workspace(s.n, cap, ccam, cfg), dtype=torch.uint8, device="cuda")
    f = dict(dtype=torch.float32, device="cuda")
    pose = start.clone()
    adam = torch.zeros(16, **f)
    lh = torch.full((5,), -1.0, **f)
    ph = torch.full((5, 12), -1.0, **f)
    gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d, 5, cap, lh, ph, ws,
                         adam_state=adam)
    torch.cuda.synchronize()
    assert int(gs2d.gs2d_track_status(ws).item()) == 6   # GS2D_ERR_NONFINITE
    assert torch.equal(pose, start)
    assert torch.equal(adam, torch.zeros(16, **f))
    assert torch.isnan(lh[0])
    assert torch.all(lh[1:] == -1.0) and torch.all(ph == -1.0)
    # the same call on the finite observation runs normally afterwards
    obs_d2 = torch.tensor(np.nan_to_num(d, nan=2.0), device="cuda")
    gs2d.gs2d_track_step(ds, ccam, cfg, prm, pose, obs_rgb, obs_d2, 5, cap, lh, ph, ws,
                         adam_state=adam)
    torch.cuda.synchronize()
    assert int(gs2d.gs2d_track_status(ws).item()) in (0, gs2d.CONVERGED)
    assert torch.isfinite(lh).all() and float(adam[12].item()) >= 1.0

"""FP64 CPU oracle for the 2D Gaussian surfel rasterizer of 2DGS-SLAM.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product path.  It
shares no code with the CUDA implementation; the only common module is the
seeded input generator ``paper_2506_00970_gb300.scenes`` (no method
arithmetic in it).

Contents (each cites the passage it follows):
  * ``render`` / ``render_bwd``  -- brute-force per-pixel renderer and its
    hand-written reverse mode (C++, ``gs2d_oracle.cpp``): Sec. III-A
    (Eq. Puv, hc, homo, wth, alpha_blending) and Sec. III-B
    (Eq. derivatives, the manifold derivative and its Jacobians).
  * ``contrib``                  -- per-surfel contribution, the sum of its
    blending weights over the image (Sec. III-D, Eq. weight, contribution);
    ``visible`` / ``covisibility`` / ``keyframe_rule`` -- the visibility
    threshold, the covisibility score and the keyframe rule of Sec. III-D.
  * ``tile_rects`` / ``bin_sort`` -- FP64 tile footprint and a stable library
    sort of (tile, depth) keys (the depth ordering of Sec. III-A).
  * ``se3_exp`` / ``se3_log``     -- SE(3) exponential / logarithm used by the
    left perturbation Exp(tau) o T (Sec. III-B), tau = (rho, theta).
  * ``adamw_step``               -- AdamW (Loshchilov & Hutter), the pose
    optimiser of Sec. III-D.
  * ``tracking_loss``            -- masked L1 colour + depth loss, Eq.
    normal_mask, opacity_mask, tracking_loss (Sec. III-D).
  * ``normal_from_depth`` / ``mapping_loss`` -- Eq. normal_fromD and the
    mapping loss of Sec. III-E, with or without the SSIM term;
    ``ssim`` / ``ssim_loss`` -- SSIM of Wang et al. 2004 (11 x 11 Gaussian
    window, sigma 1.5) and its loss term with gradient.
  * ``track``                    -- the frame-to-map tracking loop of
    Sec. III-D: render, loss, pose gradient, AdamW, retraction.
  * ``net`` (oracle/net.py)      -- the learned tracking-pose proposal
    network (not in the paper; it replaces the starting pose of the loop of
    Sec. III-D): convolutions, MLP, loss, their reverse mode, input packing
    and the se(3) target.
Parity pins live in ``tests/test_oracle_*.py``.  The convergence *rate* of
``track`` is "parity unpinned": the paper prints no per-iteration numbers.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_render.restype = ctypes.c_int
        lib.orc_render_bwd.restype = ctypes.c_int
        lib.orc_tile_rects.restype = ctypes.c_int
        lib.orc_bin_sort.restype = ctypes.c_longlong
        lib.orc_contrib.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# Relative margins of the oracle's threshold diagnostic (``ambiguous`` of
# render / render_bwd; the constants kTight and kLooseT of gs2d_oracle.cpp):
# cutoff radius, alpha_min and near plane; the stop test against t_min.
AMBIGUITY_TIGHT = 2e-5
AMBIGUITY_STOP = 1e-4


@dataclasses.dataclass
class Rule:
    """Compositing constants (readings of points the paper leaves open)."""
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    cutoff_r2: float = 9.0
    exact: bool = False

    def vec(self):
        return np.array([self.alpha_min, self.alpha_max, self.t_min, self.cutoff_r2], np.float64)


def _cam5(cam):
    return np.array([cam.fx, cam.fy, cam.cx, cam.cy, cam.near], np.float64)


def _surfel_arrays(s):
    return _d(s.mu), _d(s.quat), _d(s.scale), _d(s.opacity), _d(s.rgb)


def default_threads() -> int:
    return int(os.environ.get("GS2D_ORACLE_THREADS", os.cpu_count() or 1))


def render(surfels, cam, pose, rule: Rule = Rule(), pixels=None, n_threads: int = 0):
    """Render colour, depth (literal sum of w z), normal, opacity, the final
    transmittance, the number of blended surfels, the smallest |cos|
    between the ray and a blended surfel's normal (``min_cos``) and
    ``ambiguous``: pixels holding a compositing decision (cutoff, alpha_min,
    near plane, stop test) within rounding of its threshold, which an FP32
    evaluation may legitimately take otherwise (a diagnostic of the parity
    tests).

    ``pixels``: optional (P,2) int array of (x, y); then every output has a
    leading P axis instead of (H, W)."""
    mu, q, sc, op, rgb = _surfel_arrays(surfels)
    W, H = cam.width, cam.height
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    npx = W * H if pix is None else pix.shape[0]
    out_rgb = np.zeros((npx, 3))
    out_d = np.zeros(npx)
    out_n = np.zeros((npx, 3))
    out_o = np.zeros(npx)
    out_t = np.zeros(npx)
    out_c = np.zeros(npx, np.int32)
    out_m = np.zeros(npx)
    out_a = np.zeros(npx, np.int32)
    _lib().orc_render(surfels.n, _p(mu), _p(q), _p(sc), _p(op), _p(rgb), _p(_cam5(cam)), W, H,
                      _p(_d(pose.R)), _p(_d(pose.t)), _p(rule.vec()), int(rule.exact), npx,
                      _p(pix, ctypes.c_int), _p(out_rgb), _p(out_d), _p(out_n), _p(out_o), _p(out_t),
                      _p(out_c, ctypes.c_int), _p(out_m), _p(out_a, ctypes.c_int),
                      int(n_threads or default_threads()))
    amb = out_a.astype(bool)
    if pix is None:
        return dict(rgb=out_rgb.reshape(H, W, 3), depth=out_d.reshape(H, W),
                    normal=out_n.reshape(H, W, 3), opacity=out_o.reshape(H, W),
                    t_final=out_t.reshape(H, W), count=out_c.reshape(H, W),
                    min_cos=out_m.reshape(H, W), ambiguous=amb.reshape(H, W))
    return dict(rgb=out_rgb, depth=out_d, normal=out_n, opacity=out_o, t_final=out_t, count=out_c,
                min_cos=out_m, ambiguous=amb)


def render_bwd(surfels, cam, pose, g_rgb, g_depth, g_normal, g_opacity, rule: Rule = Rule(),
               pixels=None, n_threads: int = 0):
    """Gradients of L w.r.t. the surfel parameters and the pose tangent,
    given dL/d(rgb, depth, normal, opacity) of the rendered images (or of the
    listed pixels).  Returns dict(mu, quat, scale, opacity, rgb, pose6),
    min_cos, per surfel the smallest |cos| between a ray it blends into and
    its normal (an ill-conditioning measure for the parity tests), and
    ``ambiguous``, per surfel whether it is a candidate at a pixel that holds
    a compositing decision within rounding of its threshold (see render):
    there an FP32 evaluation may legitimately give it other gradient
    terms."""
    mu, q, sc, op, rgb = _surfel_arrays(surfels)
    W, H = cam.width, cam.height
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    npx = W * H if pix is None else pix.shape[0]
    n = surfels.n
    d_mu = np.zeros((n, 3))
    d_q = np.zeros((n, 4))
    d_s = np.zeros((n, 2))
    d_o = np.zeros(n)
    d_c = np.zeros((n, 3))
    d_pose = np.zeros(6)
    d_mc = np.ones(n)
    d_amb = np.zeros(n, np.int32)
    _lib().orc_render_bwd(n, _p(mu), _p(q), _p(sc), _p(op), _p(rgb), _p(_cam5(cam)), W, H,
                          _p(_d(pose.R)), _p(_d(pose.t)), _p(rule.vec()), int(rule.exact), npx,
                          _p(pix, ctypes.c_int), _p(_d(g_rgb).reshape(-1)),
                          _p(_d(g_depth).reshape(-1)), _p(_d(g_normal).reshape(-1)),
                          _p(_d(g_opacity).reshape(-1)), _p(d_mu), _p(d_q), _p(d_s), _p(d_o),
                          _p(d_c), _p(d_pose), _p(d_mc), _p(d_amb, ctypes.c_int),
                          int(n_threads or default_threads()))
    return dict(mu=d_mu, quat=d_q, scale=d_s, opacity=d_o, rgb=d_c, pose6=d_pose, min_cos=d_mc,
                ambiguous=d_amb.astype(bool))


def contrib(surfels, cam, pose, rule: Rule = Rule(), pixels=None, n_threads: int = 0):
    """Per-surfel contribution C_k = sum_p w_k(p) over the image (or the
    listed pixels), Eq. contribution of Sec. III-D with w_k(p) of Eq. weight
    (the renderer's items and stop rule).  Also, per surfel: ``ambiguous``
    (a candidate at a pixel whose evaluation lies within a small relative
    margin of a threshold), ``bbox`` (x0, y0, x1, y1 of the listed pixels
    where it is a candidate; x0 = -1 if none) and ``min_cos``."""
    mu, q, sc, op, rgb = _surfel_arrays(surfels)
    W, H = cam.width, cam.height
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    npx = W * H if pix is None else pix.shape[0]
    n = surfels.n
    out = np.zeros(n)
    flag = np.zeros(n, np.int32)
    bbox = np.zeros((n, 4), np.int32)
    mc = np.ones(n)
    _lib().orc_contrib(n, _p(mu), _p(q), _p(sc), _p(op), _p(rgb), _p(_cam5(cam)), W, H,
                       _p(_d(pose.R)), _p(_d(pose.t)), _p(rule.vec()), int(rule.exact), npx,
                       _p(pix, ctypes.c_int), _p(out), _p(flag, ctypes.c_int),
                       _p(bbox, ctypes.c_int), _p(mc), int(n_threads or default_threads()))
    return dict(contrib=out, ambiguous=flag.astype(bool), bbox=bbox, min_cos=mc)


def visible(c, threshold: float = 0.5):
    """Visibility of Sec. III-D: a surfel is visible from a view when its
    contribution exceeds 0.5."""
    return np.asarray(c) > threshold


def covisibility(c_a, c_b, threshold: float = 0.5):
    """(|G_A n G_B|, |G_A u G_B|, S_cov) with G_X the surfels visible from
    view X (Sec. III-D); S_cov = 0 when both sets are empty."""
    ga = set(np.flatnonzero(visible(c_a, threshold)).tolist())
    gb = set(np.flatnonzero(visible(c_b, threshold)).tolist())
    inter, union = len(ga & gb), len(ga | gb)
    return inter, union, (inter / union if union else 0.0)


def keyframe_rule(score, t_a, t_b, c_k: float = 0.9, d_k: float = 0.15):
    """Keyframe selection of Sec. III-D: a new keyframe when the
    covisibility with the last keyframe falls below c_k or the distance
    between the translation vectors of the two world-to-camera poses exceeds
    d_k (Table I: 0.9 and 15 cm)."""
    d = math.sqrt(sum((float(a) - float(b)) ** 2 for a, b in zip(t_a, t_b)))
    return bool(score < c_k or d > d_k)


def tile_rects(surfels, cam, pose, rule: Rule = Rule(), tile=(16, 16)):
    """FP64 tile rectangle (tx0, ty0, tx1, ty1) of every surfel's footprint
    ((1,1,0,0) if culled) and its centre depth mu_c.z."""
    mu, q, sc, op, _ = _surfel_arrays(surfels)
    rect = np.zeros((surfels.n, 4), np.int32)
    depth = np.zeros(surfels.n)
    _lib().orc_tile_rects(surfels.n, _p(mu), _p(q), _p(sc), _p(op), _p(_cam5(cam)), cam.width,
                          cam.height, _p(_d(pose.R)), _p(_d(pose.t)), _p(rule.vec()),
                          int(tile[0]), int(tile[1]), _p(rect, ctypes.c_int), _p(depth))
    return rect, depth


def bin_sort(rect, depth_f32, tiles_x: int, tiles_y: int):
    """Stable sort of (tile << 32 | depth bits, surfel id) pairs.  ``depth_f32``
    is the FP32 centre depth whose bit pattern is the key (positive floats
    order like their bit patterns).  Returns (keys u64, vals u32, ranges
    (n_tiles, 2) int32)."""
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    bits = np.ascontiguousarray(np.asarray(depth_f32, np.float32)).view(np.uint32)
    n = rect.shape[0]
    area = np.where(rect[:, 2] >= rect[:, 0], rect[:, 2] - rect[:, 0] + 1, 0) * \
        np.where(rect[:, 3] >= rect[:, 1], rect[:, 3] - rect[:, 1] + 1, 0)
    cap = int(area.sum())
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    ranges = np.zeros((tiles_x * tiles_y, 2), np.int32)
    k = _lib().orc_bin_sort(n, _p(rect, ctypes.c_int), _p(bits, ctypes.c_uint32), tiles_x,
                            tiles_y, _p(keys, ctypes.c_uint64), _p(vals, ctypes.c_uint32), cap,
                            _p(ranges, ctypes.c_int))
    assert k == cap
    return keys[:k], vals[:k], ranges


# --------------------------------------------------------------------------
# SE(3) (Sec. III-B: left perturbation Exp(tau) o T, tau = (rho, theta))
# --------------------------------------------------------------------------
def hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def _so3_coeffs(th):
    """sin(t)/t, (1-cos t)/t^2, (t - sin t)/t^3 with series near zero."""
    if th < 1e-4:
        t2 = th * th
        return 1 - t2 / 6 + t2 * t2 / 120, 0.5 - t2 / 24 + t2 * t2 / 720, 1 / 6 - t2 / 120
    return math.sin(th) / th, (1 - math.cos(th)) / th ** 2, (th - math.sin(th)) / th ** 3


def se3_exp(tau):
    """Exp of tau = (rho, theta): R = Rodrigues(theta), t = V(theta) rho."""
    tau = np.asarray(tau, np.float64)
    rho, w = tau[:3], tau[3:]
    th = float(np.linalg.norm(w))
    A, B, C = _so3_coeffs(th)
    K = hat(w)
    R = np.eye(3) + A * K + B * K @ K
    V = np.eye(3) + B * K + C * K @ K
    return R, V @ rho


def se3_log(R, t):
    """Inverse of se3_exp for rotation angles below pi."""
    c = np.clip((np.trace(R) - 1) / 2, -1.0, 1.0)
    th = math.acos(c)
    if th < 1e-6:
        w = 0.5 * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    else:
        w = th / (2 * math.sin(th)) * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    A, B, C = _so3_coeffs(float(np.linalg.norm(w)))
    K = hat(w)
    V = np.eye(3) + B * K + C * K @ K
    return np.concatenate([np.linalg.solve(V, t), w])


def retract(pose, tau):
    """Left update T <- Exp(tau) T."""
    from paper_2506_00970_gb300.scenes import Pose
    dR, dt = se3_exp(tau)
    return Pose(dR @ pose.R, dR @ pose.t + dt)


def pose_error(pose, gt):
    """Translation error of the camera centres (m) and geodesic rotation
    error (degrees)."""
    c = -pose.R.T @ pose.t
    cg = -gt.R.T @ gt.t
    cosang = np.clip((np.trace(pose.R @ gt.R.T) - 1) / 2, -1.0, 1.0)
    return float(np.linalg.norm(c - cg)), math.degrees(math.acos(cosang))


# --------------------------------------------------------------------------
# AdamW (Loshchilov & Hutter), the tracking optimiser of Sec. III-D
# --------------------------------------------------------------------------
@dataclasses.dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    step: int = 0


def adamw_step(param, grad, st: AdamState, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, wd=0.0):
    st.step += 1
    b1, b2 = betas
    param = param * (1 - lr * wd)
    st.m = b1 * st.m + (1 - b1) * grad
    st.v = b2 * st.v + (1 - b2) * grad * grad
    mhat = st.m / (1 - b1 ** st.step)
    vhat = st.v / (1 - b2 ** st.step)
    return param - lr * mhat / (np.sqrt(vhat) + eps)


# --------------------------------------------------------------------------
# losses (Sec. III-D, III-E), FP64 torch on the CPU; gradients by autograd
# --------------------------------------------------------------------------
def _ray_grid(cam):
    x = np.arange(cam.width) + 0.5
    y = np.arange(cam.height) + 0.5
    X, Y = np.meshgrid(x, y)
    return np.stack([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, np.ones_like(X)], axis=-1)


def _expected_depth(D, O, depth_mode):
    import torch
    return D / torch.clamp(O, min=1e-6) if depth_mode == 1 else D


def tracking_loss(img, obs_rgb, obs_depth, cam, lambda_d=1.0, depth_mode=1, mask_thresh=0.95):
    """L_t = 1/|Omega| sum_p M_n M_o (|I_r - I|_1 + lambda_d |D_r - D|)
    (Eq. tracking_loss) with M_n = [N_r . r > 0] (Eq. normal_mask) and
    M_o = [O > 0.95] (Eq. opacity_mask).  The masks carry no gradient.
    ``img``: dict of rendered rgb (H,W,3), depth, normal, opacity.
    Returns (L, grads dict for rgb, depth, normal, opacity)."""
    import torch
    t = {k: torch.tensor(np.asarray(img[k], np.float64), requires_grad=True)
         for k in ("rgb", "depth", "normal", "opacity")}
    I = torch.tensor(np.asarray(obs_rgb, np.float64))
    D = torch.tensor(np.asarray(obs_depth, np.float64))
    r = torch.tensor(_ray_grid(cam))
    with torch.no_grad():
        Mn = ((t["normal"] * r).sum(-1) > 0).double()
        Mo = (t["opacity"] > mask_thresh).double()
    Dr = _expected_depth(t["depth"], t["opacity"], depth_mode)
    per = (t["rgb"] - I).abs().sum(-1) + lambda_d * (Dr - D).abs()
    L = (Mn * Mo * per).sum() / (cam.width * cam.height)
    L.backward()
    return float(L.detach()), {k: (v.grad.numpy().copy() if v.grad is not None else np.zeros(v.shape))
                               for k, v in t.items()}


def normal_from_depth(depth, cam):
    """Eq. normal_fromD on the back-projected point map X = D r with central
    differences; returns (N_D (H,W,3), valid (H,W)) where border pixels and
    degenerate cross products are invalid.  Accepts numpy or torch."""
    import torch
    D = depth if isinstance(depth, torch.Tensor) else torch.tensor(np.asarray(depth, np.float64))
    r = torch.tensor(_ray_grid(cam), dtype=D.dtype)
    X = D[..., None] * r
    gx = torch.zeros_like(X)
    gy = torch.zeros_like(X)
    gx[1:-1, 1:-1] = (X[1:-1, 2:] - X[1:-1, :-2]) / 2
    gy[1:-1, 1:-1] = (X[2:, 1:-1] - X[:-2, 1:-1]) / 2
    n = torch.cross(gx, gy, dim=-1)
    nn = torch.linalg.norm(n, dim=-1)
    valid = nn > 0
    ND = torch.where(valid[..., None], n / torch.where(valid, nn, torch.ones_like(nn))[..., None],
                     torch.zeros_like(n))
    return ND, valid


def ssim_window(radius: int = 5, sigma: float = 1.5):
    """The SSIM window of Wang et al. 2004: an 11 x 11 Gaussian, sigma 1.5,
    normalised to sum 1 (the outer product of the normalised 1D Gaussian)."""
    d = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-d * d / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def _ssim_torch(x, y, C1=1e-4, C2=9e-4):
    """Per-pixel, per-channel SSIM (Wang et al. 2004) of H x W x C tensors:
    local means, variances and covariance under the window with zero padding
    (a library 2D convolution), then the SSIM formula."""
    import torch
    import torch.nn.functional as F
    C = x.shape[-1]
    w = torch.tensor(ssim_window(), dtype=torch.float64)[None, None].repeat(C, 1, 1, 1)
    X = x.permute(2, 0, 1)[None]
    Y = y.permute(2, 0, 1)[None]
    f = lambda a: F.conv2d(a, w, padding=5, groups=C)
    mx, my = f(X), f(Y)
    sxx = f(X * X) - mx * mx
    syy = f(Y * Y) - my * my
    sxy = f(X * Y) - mx * my
    S = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return S[0].permute(1, 2, 0)


def ssim(x, y):
    """SSIM map (H x W x C, FP64) of x against y."""
    import torch
    return _ssim_torch(torch.tensor(np.asarray(x, np.float64)),
                       torch.tensor(np.asarray(y, np.float64))).numpy()


def ssim_loss(x, y, weight=1.0):
    """weight / |Omega| sum_p (1 - mean_c SSIM_c(p)) and its gradient w.r.t. x."""
    import torch
    t = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    S = _ssim_torch(t, torch.tensor(np.asarray(y, np.float64)))
    H, W = S.shape[0], S.shape[1]
    L = weight * (1.0 - S.mean(-1)).sum() / (H * W)
    L.backward()
    return float(L.detach()), t.grad.numpy().copy()


def mapping_loss(img, obs_rgb, obs_depth, cam, w_d=0.5, w_n=0.02, depth_mode=1, valid_opacity=0.5,
                 w_ssim=0.0):
    """L_m = 1/|Omega| sum_p (L_c + w_d |D_r - D| + w_n (1 - N_{D_r} . N_r))
    (Sec. III-E) with L_c = (1 - w_ssim) |I_r - I|_1 + w_ssim (1 - SSIM(p)),
    SSIM(p) the channel mean (w_ssim = 0: the colour term without SSIM;
    Table I gives the SSIM term 0.125).  The normal term counts at interior
    pixels whose own and 4-neighbour opacities exceed 0.5."""
    import torch
    t = {k: torch.tensor(np.asarray(img[k], np.float64), requires_grad=True)
         for k in ("rgb", "depth", "normal", "opacity")}
    I = torch.tensor(np.asarray(obs_rgb, np.float64))
    D = torch.tensor(np.asarray(obs_depth, np.float64))
    Dr = _expected_depth(t["depth"], t["opacity"], depth_mode)
    ND, valid = normal_from_depth(Dr, cam)
    with torch.no_grad():
        O = t["opacity"]
        ok = torch.zeros_like(O, dtype=torch.bool)
        ok[1:-1, 1:-1] = ((O[1:-1, 1:-1] > valid_opacity) & (O[1:-1, 2:] > valid_opacity)
                          & (O[1:-1, :-2] > valid_opacity) & (O[2:, 1:-1] > valid_opacity)
                          & (O[:-2, 1:-1] > valid_opacity))
        ok &= valid
    Ln = torch.where(ok, 1.0 - (ND * t["normal"]).sum(-1), torch.zeros_like(O))
    Lc = (1.0 - w_ssim) * (t["rgb"] - I).abs().sum(-1)
    if w_ssim > 0.0:
        Lc = Lc + w_ssim * (1.0 - _ssim_torch(t["rgb"], I).mean(-1))
    per = Lc + w_d * (Dr - D).abs() + w_n * Ln
    L = per.sum() / (cam.width * cam.height)
    L.backward()
    return float(L.detach()), {k: (v.grad.numpy().copy() if v.grad is not None else np.zeros(v.shape))
                               for k, v in t.items()}


# --------------------------------------------------------------------------
# frame-to-map tracking (Sec. III-D)
# --------------------------------------------------------------------------
def track(surfels, cam, pose0, obs_rgb, obs_depth, n_iter=100, lr=1e-3, betas=(0.9, 0.999),
          eps=1e-8, wd=0.0, lambda_d=1.0, stop_tol=1e-5, rule: Rule = Rule(), n_threads=0,
          callback=None):
    """Optimise T_cw by AdamW on the left-perturbation tangent tau, which is
    reset to zero after every retraction T <- Exp(tau) T (moments kept);
    stops when |tau| < stop_tol or after n_iter iterations.
    Returns (pose, list of per-iteration losses)."""
    pose = pose0.copy()
    st = AdamState(np.zeros(6), np.zeros(6))
    losses = []
    for it in range(n_iter):
        img = render(surfels, cam, pose, rule, n_threads=n_threads)
        L, g = tracking_loss(img, obs_rgb, obs_depth, cam, lambda_d)
        losses.append(L)
        gr = render_bwd(surfels, cam, pose, g["rgb"], g["depth"], g["normal"], g["opacity"], rule,
                        n_threads=n_threads)
        tau = adamw_step(np.zeros(6), gr["pose6"], st, lr, betas, eps, wd)
        pose = retract(pose, tau)
        if callback:
            callback(it, pose, L)
        if np.linalg.norm(tau) < stop_tol:
            break
    return pose, losses

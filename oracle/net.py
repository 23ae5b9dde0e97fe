"""FP64 CPU oracle of the learned tracking-pose proposal network.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by
``tests/`` and ``bench.py``'s CPU-baseline leg, never by the product path.

The paper has no learned component: each frame's tracking starts from the
previous frame's pose and refines it with the gradient loop of Sec. III-D.
The proposal network is an addition whose output only replaces that starting
pose (the plain loop still refines it and judges it by the tracking loss of
Eq. tracking_loss).  Its definition, written out here plainly:

  * input x: [B, 120, 160, 8] channels-last (NHWC): the rendered colour and
    depth at the current pose estimate T_init and the observed colour and
    depth (``pack_input``);
  * six convolutions, 3x3 kernel, stride 2, zero padding 1, each followed by
    ReLU; channels 8 -> 32 -> 64 -> 128 -> 256 -> 256 -> 256; spatial
    120x160 -> 60x80 -> 30x40 -> 15x20 -> 8x10 -> 4x5 -> 2x3; weights
    W[c_out, ky, kx, c_in], output pixel (oy, ox) reads input pixel
    (2 oy - 1 + ky, 2 ox - 1 + kx);
  * flatten (h, w, c order) to 1536, FC 1536 -> 256 with ReLU, FC 256 -> 6;
  * the 6 outputs times ``TAU_SCALE`` are a twist delta = (rho, theta) of
    se(3), applied on the left: T <- Exp(delta) T_init (the left
    perturbation of Sec. III-B);
  * training target: delta* = Log(T_gt T_init^-1) / TAU_SCALE, loss
    L = 1/(2B) sum_b |y_b - delta*_b|^2.

Flat parameter vector (float32 on the device, float64 here): for every conv
layer W (c_out*9*c_in) then b (c_out); then FC1 W [256, 1536], b [256]; then
FC2 W [6, 256], b [6].

Precision points of the device path, mirrored when ``bf16=True``: the input,
the weights and every stored activation and activation gradient are rounded
to bfloat16 (round to nearest even); products accumulate in FP32 (here FP64);
biases, the network output, the loss and the weight gradients stay FP32.
"""
from __future__ import annotations

import math

import numpy as np

from . import se3_exp, se3_log

IN_H, IN_W, IN_C = 120, 160, 8
CONV = ((8, 32), (32, 64), (64, 128), (128, 256), (256, 256), (256, 256))
FC_HIDDEN = 256
N_OUT = 6
TAU_SCALE = np.array([0.03, 0.03, 0.03, 0.03, 0.03, 0.03])
DEPTH_OFFSET = 2.5      # metres subtracted from valid depths in the input
VALID_OPACITY = 0.5     # rendered pixels with O <= this get depth channel 0


def to_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Works on the float32 bit pattern: add 0x7FFF plus the lowest kept bit,
    then clear the 16 dropped bits."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv_out_hw(h: int, w: int):
    return (h + 1) // 2, (w + 1) // 2


def spatial_sizes(h=IN_H, w=IN_W, n_layers=len(CONV)):
    out = [(h, w)]
    for _ in range(n_layers):
        h, w = conv_out_hw(h, w)
        out.append((h, w))
    return out


def param_layout(conv=CONV, h=IN_H, w=IN_W, hidden=FC_HIDDEN, n_out=N_OUT):
    """[(name, shape, offset)] of the flat parameter vector."""
    hs = spatial_sizes(h, w, len(conv))[-1]
    flat = hs[0] * hs[1] * conv[-1][1]
    items = []
    off = 0
    for i, (ci, co) in enumerate(conv):
        for name, shape in ((f"conv{i}.W", (co, 3, 3, ci)), (f"conv{i}.b", (co,))):
            items.append((name, shape, off))
            off += int(np.prod(shape))
    for name, shape in (("fc1.W", (hidden, flat)), ("fc1.b", (hidden,)),
                        ("fc2.W", (n_out, hidden)), ("fc2.b", (n_out,))):
        items.append((name, shape, off))
        off += int(np.prod(shape))
    return items, off


def unflatten(params, conv=CONV, h=IN_H, w=IN_W):
    items, total = param_layout(conv, h, w)
    assert params.size == total
    return {name: params[off:off + int(np.prod(shape))].reshape(shape)
            for name, shape, off in items}


def flatten(d, conv=CONV, h=IN_H, w=IN_W):
    items, total = param_layout(conv, h, w)
    out = np.zeros(total)
    for name, shape, off in items:
        out[off:off + int(np.prod(shape))] = np.asarray(d[name], np.float64).ravel()
    return out


# --------------------------------------------------------------------------
# convolution 3x3, stride 2, padding 1 (NHWC) and its reverse mode
# --------------------------------------------------------------------------
def conv_fwd(x, W, b):
    """y[b, oy, ox, o] = b[o] + sum_{ky, kx, i} W[o, ky, kx, i] x[b, 2oy-1+ky, 2ox-1+kx, i]
    (out-of-range input pixels are zero)."""
    B, H, Wd, Ci = x.shape
    Co = W.shape[0]
    Ho, Wo = conv_out_hw(H, Wd)
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:H + 1, 1:Wd + 1] = x
    y = np.zeros((B, Ho, Wo, Co)) + b
    for ky in range(3):
        for kx in range(3):
            # padded row of input row 2 oy - 1 + ky is 2 oy + ky
            patch = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]
            y += patch @ W[:, ky, kx, :].T
    return y


def conv_bwd(x, W, dy):
    """Gradients of conv_fwd w.r.t. x, W and b given dL/dy."""
    B, H, Wd, Ci = x.shape
    Ho, Wo = dy.shape[1:3]
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:H + 1, 1:Wd + 1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwi->oi", dy, patch)
            dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :] += dy @ W[:, ky, kx, :]
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, 1:H + 1, 1:Wd + 1], dW, db


# --------------------------------------------------------------------------
# the network
# --------------------------------------------------------------------------
def forward(params, x, conv=CONV, bf16=False):
    """Returns the 6 outputs per sample and the stored activations."""
    rnd = to_bf16 if bf16 else (lambda a: a)
    B, H, Wd, _ = x.shape
    P = unflatten(params, conv, H, Wd)
    acts = [rnd(x)]
    a = acts[0]
    for i in range(len(conv)):
        a = rnd(np.maximum(conv_fwd(a, rnd(P[f"conv{i}.W"]), P[f"conv{i}.b"]), 0.0))
        acts.append(a)
    f = a.reshape(B, -1)
    h = rnd(np.maximum(f @ rnd(P["fc1.W"]).T + P["fc1.b"], 0.0))
    acts.append(h)
    y = h @ rnd(P["fc2.W"]).T + P["fc2.b"]
    return y, acts


def loss_and_grad(y, target):
    """L = 1/(2B) sum |y - t|^2 and dL/dy."""
    B = y.shape[0]
    d = y - target
    return 0.5 * float(np.sum(d * d)) / B, d / B


def backward(params, acts, dy, conv=CONV, bf16=False):
    """Flat gradient of the loss w.r.t. the parameters given dL/dy, through
    the stored activations of ``forward``."""
    rnd = to_bf16 if bf16 else (lambda a: a)
    x = acts[0]
    B, H, Wd, _ = x.shape
    P = unflatten(params, conv, H, Wd)
    G = {}
    h = acts[-1]
    dz2 = rnd(dy)
    G["fc2.W"] = dz2.T @ h
    G["fc2.b"] = dz2.sum(0)
    dz1 = rnd((dz2 @ rnd(P["fc2.W"])) * (h > 0))
    a6 = acts[-2]
    f = a6.reshape(B, -1)
    G["fc1.W"] = dz1.T @ f
    G["fc1.b"] = dz1.sum(0)
    dz = rnd(((dz1 @ rnd(P["fc1.W"])) * (f > 0)).reshape(a6.shape))
    for i in range(len(conv) - 1, -1, -1):
        a_in = acts[i]
        dx, dW, db = conv_bwd(a_in, rnd(P[f"conv{i}.W"]), dz)
        G[f"conv{i}.W"] = dW
        G[f"conv{i}.b"] = db
        if i > 0:
            dz = rnd(dx * (a_in > 0))
    return flatten(G, conv, H, Wd)


# --------------------------------------------------------------------------
# data: input packing, targets, applying a proposal
# --------------------------------------------------------------------------
def pack_input(r_rgb, r_depth, r_opacity, o_rgb, o_depth):
    """[B,H,W,8]: rendered colour, rendered expected depth D/O - offset (0
    where O <= 0.5), observed colour, observed depth - offset (0 where the
    observation is not positive), rounded to bfloat16."""
    r_rgb = np.asarray(r_rgb, np.float64)
    valid = r_opacity > VALID_OPACITY
    dr = np.where(valid, r_depth / np.where(valid, r_opacity, 1.0) - DEPTH_OFFSET, 0.0)
    do = np.where(o_depth > 0, o_depth - DEPTH_OFFSET, 0.0)
    return to_bf16(np.concatenate([r_rgb, dr[..., None], o_rgb, do[..., None]], axis=-1))


def downsample_rgbd(rgb, depth, factor):
    """The network's view of a full-resolution observation: colour averaged
    over factor x factor blocks, depth the mean of each block's valid
    (finite, positive) values, 0 where a block has none."""
    rgb = np.asarray(rgb, np.float64)
    d = np.asarray(depth, np.float64)
    H, W = d.shape
    f = int(factor)
    c = rgb.reshape(H // f, f, W // f, f, 3).mean(axis=(1, 3))
    ok = np.isfinite(d) & (d > 0)
    s = np.where(ok, d, 0.0).reshape(H // f, f, W // f, f).sum(axis=(1, 3))
    k = ok.reshape(H // f, f, W // f, f).sum(axis=(1, 3))
    return c, np.where(k > 0, s / np.maximum(k, 1), 0.0)


def target_delta(T_init, T_gt):
    """delta* with Exp(delta* * TAU_SCALE) T_init = T_gt."""
    R = T_gt.R @ T_init.R.T
    t = T_gt.t - R @ T_init.t
    return se3_log(R, t) / TAU_SCALE


def apply_delta(T, y):
    """T <- Exp(y * TAU_SCALE) T."""
    from paper_2506_00970_gb300.scenes import Pose
    dR, dt = se3_exp(np.asarray(y, np.float64) * TAU_SCALE)
    return Pose(dR @ T.R, dR @ T.t + dt)


def he_scale(fan_in: int) -> float:
    return math.sqrt(2.0 / fan_in)

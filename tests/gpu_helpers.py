"""Shared helpers of the GPU parity tests: run the CUDA path through the
C ABI binding and compare with the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np


# tolerances of the parity contract: colour / opacity max-abs, depth and
# normal relative, gradients relative
TOL_ABS = 1e-4
TOL_REL = 1e-4
TOL_GRAD = 1e-3


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def gpu_render(surfels, cam, pose, tile=(16, 16), capacity=None, keys=False, px=1):
    from paper_2506_00970_gb300 import gs2d
    import torch
    ds = gs2d.DeviceSurfels(surfels)
    r = gs2d.Rasterizer(cam, ds.n, capacity=capacity, tile=tile, keys=keys, px=px)
    pose_t = gs2d.pose_tensor(pose)
    out = r.forward(ds, pose_t)
    torch.cuda.synchronize()
    return r, ds, pose_t, {k: v.detach().cpu().numpy() for k, v in out.items()}


def image_mismatch(a, b, rel, atol):
    """Elementwise |a-b| <= rel*|b| + atol over pixels (any channel)."""
    bad = np.abs(a - b) > rel * np.abs(b) + atol
    if bad.ndim == 3:
        bad = bad.any(-1)
    return bad


GRAZING_COS = 0.02   # a blended surfel within ~1.1 degrees of edge-on
EDGE_ON_COS = 0.05   # a surfel seen within ~3 degrees of edge-on (gradients)
GRAD_FLOOR = 2.0 ** -17


def grad_rows_ok(og):
    """Surfels held to the per-element gradient bound: not flagged by the
    oracle (a candidate at a pixel whose compositing decision sits within
    rounding of its threshold, where FP32 may legitimately blend otherwise)
    and not seen within ~3 degrees of edge-on (ill-conditioned FP32
    intersection)."""
    return ~np.asarray(og["ambiguous"], bool) & (np.asarray(og["min_cos"]) > EDGE_ON_COS)


FLAGGED_TOL = 1e-2


def assert_grads_close(a, b, name, rows_ok=None, tol=TOL_GRAD, min_rows=0.9, floor=GRAD_FLOOR):
    """Gradient parity at the contract's 1e-3 relative.
    Per element on rows_ok (all rows if None): |a - b| <= tol |b| +
    GRAD_FLOOR max|b|, no exceptions.  The floor, 2^-17 of the array's
    largest element (128 units of FP32 rounding at that scale), covers the
    FP32 rounding of a surfel's sum over up to a few hundred per-pixel terms
    where they cancel.  The other rows (flagged by the oracle, or seen
    nearly edge-on): |a - b| <= FLAGGED_TOL max|b| -- a threshold decision
    taken otherwise moves a surfel's gradient by about one pixel's term.
    min_rows: the share of surfels with a non-zero gradient row that must be
    held to the per-element bound (the exemptions stay few).  floor: the
    floor's share of the scale (a sum over V views takes V times it: every
    view's sum rounds at its own scale)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b)
    if rows_ok is None or b.ndim == 0 or b.shape[0] != rows_ok.shape[0]:
        bad = err > tol * np.abs(b) + floor * scale
        assert not bad.any(), (name, int(bad.sum()), (err[bad] / scale)[:4], (np.abs(b[bad]) / scale)[:4])
        return
    live = np.abs(b.reshape(len(b), -1)).max(1) > 0
    assert (rows_ok & live).sum() >= min_rows * live.sum(), (name, int((rows_ok & live).sum()), int(live.sum()))
    e, r = err[rows_ok], b[rows_ok]
    bad = e > tol * np.abs(r) + floor * scale
    assert not bad.any(), (name, int(bad.sum()), (e[bad] / scale)[:4], (np.abs(r[bad]) / scale)[:4])
    if (~rows_ok).any():
        assert err[~rows_ok].max() <= FLAGGED_TOL * scale, (name, err[~rows_ok].max() / scale)


def assert_images_close(gpu, orc, max_bad_frac=1e-4, min_bad=2, grazing_frac=1e-2):
    """Colour/opacity within TOL_ABS absolute; depth within TOL_REL of the
    depth; the normal image N = sum w t_nc within TOL_REL of the pixel's
    opacity O = sum w (which bounds |N|; per-component relative error is
    meaningless where normals of different surfels cancel).  Pixels whose
    evaluation sits on a threshold may differ: at most max_bad_frac of them
    (at least min_bad).  Pixels that blend a surfel seen within ~1 degree of
    edge-on (oracle min_cos < GRAZING_COS) have an ill-conditioned FP32
    intersection; they are held to 10x the tolerance and may make up at most
    grazing_frac of the image."""
    P = orc["opacity"].size
    allow = max(min_bad, int(max_bad_frac * P))
    g = {k: np.asarray(gpu[k], np.float64) for k in ("rgb", "opacity", "depth", "normal")}
    bad = {
        "rgb": (np.abs(g["rgb"] - orc["rgb"]) > TOL_ABS).any(-1),
        "opacity": np.abs(g["opacity"] - orc["opacity"]) > TOL_ABS,
        "depth": np.abs(g["depth"] - orc["depth"]) > TOL_REL * np.abs(orc["depth"]) + 1e-6,
        "normal": np.abs(g["normal"] - orc["normal"]).max(-1) > TOL_REL * orc["opacity"] + 1e-6,
    }
    bad_any = np.zeros(orc["opacity"].shape, bool)
    for v in bad.values():
        bad_any |= v
    grazing = orc["min_cos"] < GRAZING_COS if "min_cos" in orc else np.zeros_like(bad_any)
    report = {k: int((v & ~grazing).sum()) for k, v in bad.items()}
    report["grazing_px"] = int(grazing.sum())
    assert (bad_any & ~grazing).sum() <= allow, (report, allow)
    assert grazing.sum() <= max(min_bad, grazing_frac * P), report
    loose = {
        "rgb": (np.abs(g["rgb"] - orc["rgb"]) > 10 * TOL_ABS).any(-1),
        "opacity": np.abs(g["opacity"] - orc["opacity"]) > 10 * TOL_ABS,
        "depth": np.abs(g["depth"] - orc["depth"]) > 10 * TOL_REL * np.abs(orc["depth"]) + 1e-5,
        "normal": np.abs(g["normal"] - orc["normal"]).max(-1) > 10 * TOL_REL * orc["opacity"] + 1e-5,
    }
    loose_bad = np.zeros_like(bad_any)
    for v in loose.values():
        loose_bad |= v
    assert (loose_bad & grazing).sum() <= allow, report
    return report, ~bad_any


def records_to_proj(torch, rect, depth, count):
    """Projection records (device, PROJ_FLOATS per record) carrying only what
    the binning reads: the tile rectangle and the centre depth; and the
    per-record tile counts."""
    from paper_2506_00970_gb300 import gs2d
    n = len(depth)
    proj = np.zeros((max(n, 1), gs2d.PROJ_FLOATS), np.float32)
    if n:
        proj[:n, 26] = depth
        r01 = (rect[:, 0].astype(np.uint32) | (rect[:, 1].astype(np.uint32) << 16))
        r23 = (rect[:, 2].astype(np.uint32) | (rect[:, 3].astype(np.uint32) << 16))
        proj[:n, 28] = r01.view(np.float32)
        proj[:n, 29] = r23.view(np.float32)
    return (torch.tensor(proj.reshape(-1), device="cuda"),
            torch.tensor(np.asarray(count, np.int32).reshape(-1) if n else np.zeros(1, np.int32),
                         device="cuda"))

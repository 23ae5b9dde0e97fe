"""FP64 oracle of the map-state bookkeeping of 2DGS-SLAM (test infrastructure
only: imported by ``tests/`` and never by the product path).

* ``observe``     -- the state update after keyframe n (Sec. III-F) of the
  per-surfel state of Eq. map (Sec. III-C): last observation t^l, closest
  observing keyframe t^c and distance d^c, active flag delta, deactivation
  after a time threshold and reactivation after a loop closure;
* ``increment`` / ``correct`` -- the map correction of Sec. IV-C:
  dT_j = T^o_j T_j^-1 (camera-to-world poses), mu' = dT mu, R' = dR R;
* ``prune_keep``  -- the occlusion removal of Sec. III-F for a sampled
  keyframe r: surfels with t^c = r and contribution below 0.5 go;
* ``compact``     -- the map without the removed surfels, order kept
  (numpy boolean indexing).
Poses are world-to-camera T_cw (R, t); a camera-to-world pose is its
inverse.  Visibility is the contribution threshold of Sec. III-D.
"""
from __future__ import annotations

import numpy as np


def camera_centre(R_cw, t_cw):
    """Viewpoint of a world-to-camera pose: c = -R^T t."""
    return -np.asarray(R_cw, np.float64).T @ np.asarray(t_cw, np.float64)


def observe(contrib, mu, R_cw, t_cw, kf_id, state, vis_threshold=0.5, inactive_after=10,
            reactivate=False, loop_h=-1):
    """Sec. III-F for keyframe ``kf_id``; ``state`` = dict(delta, t_c, d_c,
    t_l) (arrays, not modified).  Returns (new state, counts) with counts =
    (visible active, closest updates, deactivations, reactivations).

    Active surfels (delta = 1 on entry) visible from the keyframe get
    t^l = n; their distance to the keyframe's viewpoint replaces d^c (and n
    replaces t^c) when it is smaller; an active surfel unobserved for more
    than ``inactive_after`` keyframes (n - t^l > threshold) becomes inactive.
    Within the keyframes that follow a loop closure with K_h
    (``reactivate``), an inactive surfel that is observed and whose t^c is
    after h becomes active again with t^l = n."""
    delta = np.asarray(state["delta"]).astype(np.int64).copy()
    t_c = np.asarray(state["t_c"]).astype(np.int64).copy()
    d_c = np.asarray(state["d_c"], np.float64).copy()
    t_l = np.asarray(state["t_l"]).astype(np.int64).copy()
    vis = np.asarray(contrib, np.float64) > vis_threshold
    active = delta == 1
    c = camera_centre(R_cw, t_cw)
    dist = np.linalg.norm(np.asarray(mu, np.float64) - c[None, :], axis=1)
    seen = active & vis
    t_l[seen] = kf_id
    closer = seen & (dist < d_c)
    d_c[closer] = dist[closer]
    t_c[closer] = kf_id
    deact = active & (kf_id - t_l > inactive_after)
    delta[deact] = 0
    react = np.zeros_like(active)
    if reactivate:
        react = ~active & vis & (t_c > loop_h)
        delta[react] = 1
        t_l[react] = kf_id
    new = dict(delta=delta, t_c=t_c, d_c=d_c, t_l=t_l)
    return new, (int(seen.sum()), int(closer.sum()), int(deact.sum()), int(react.sum()))


def increment(R_old, t_old, R_new, t_new):
    """dT = T^o T^-1 with T, T^o the camera-to-world poses, from the
    world-to-camera poses (R, t) before and (R_new, t_new) after pose graph
    optimisation: the camera-to-world pose is (R^T, -R^T t)."""
    def c2w(R, t):
        M = np.eye(4)
        M[:3, :3] = np.asarray(R, np.float64).T
        M[:3, 3] = -np.asarray(R, np.float64).T @ np.asarray(t, np.float64)
        return M
    D = c2w(R_new, t_new) @ np.linalg.inv(c2w(R_old, t_old))
    return D[:3, :3], D[:3, 3]


def quat_matrix(q):
    """Rotation matrices of (w, x, y, z) quaternions (normalised first)."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def correct(mu, quat, t_c, poses_old, poses_new):
    """Sec. IV-C: every surfel follows its closest keyframe t^c's increment:
    mu' = dR mu + dt, R' = dR R.  poses_*: lists of (R, t) world-to-camera.
    Surfels whose t^c is not a keyframe index are left unchanged.  Returns
    (mu', R' as matrices [n, 3, 3], skipped count)."""
    mu = np.asarray(mu, np.float64)
    R = quat_matrix(quat)
    t_c = np.asarray(t_c)
    mu_o, R_o = mu.copy(), R.copy()
    n_kf = len(poses_old)
    ok = (t_c >= 0) & (t_c < n_kf)
    for j in range(n_kf):
        sel = ok & (t_c == j)
        if not sel.any():
            continue
        dR, dt = increment(*poses_old[j], *poses_new[j])
        mu_o[sel] = mu[sel] @ dR.T + dt
        R_o[sel] = dR[None] @ R[sel]
    return mu_o, R_o, int((~ok).sum())


def prune_keep(contrib, t_c, r, vis_threshold=0.5):
    """Sec. III-F: for a sampled keyframe r, a surfel with t^c = r whose
    contribution is below 0.5 is removed (False), every other kept (True)."""
    return ~((np.asarray(t_c) == r) & (np.asarray(contrib, np.float64) < vis_threshold))


def compact(keep, *arrays):
    """The arrays restricted to the kept surfels, order kept, and each
    surfel's new index (-1 if removed)."""
    keep = np.asarray(keep, bool)
    new_index = np.where(keep, np.cumsum(keep) - 1, -1)
    return [np.asarray(a)[keep] for a in arrays], new_index

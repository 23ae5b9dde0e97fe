"""Pins of the oracle's hand-written reverse mode (Sec. III-B) against
central finite differences in FP64 and against an invariance of the
pose gradient (no GPU).

* surfel-parameter gradients: central differences, h = 1e-6, on tiny scenes
  in exact mode (no clamp / skip / stop / cutoff, so the images are smooth);
* pose gradient: central differences along the left perturbation
  Exp(h e_k) o T_cw (the manifold derivative of Sec. III-B);
* translation invariance: moving the camera by rho equals moving every
  surfel by R_cw^T rho, so dL/drho = R_cw sum_k dL/dmu_k.
"""
import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes


def _scene(seed, n=6):
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-0.15, 0.15, n), rng.uniform(-0.15, 0.15, n),
                   rng.uniform(0.8, 1.2, n)], 1)
    q = rng.normal(size=(n, 4))
    q[:, 0] += 2.0            # mostly facing the camera
    sc = rng.uniform(0.04, 0.09, (n, 2))
    op = rng.uniform(0.3, 0.8, n)
    rgb = rng.uniform(0, 1, (n, 3))
    return scenes.Surfels(mu, q, sc, op, rgb)


CAM = scenes.Camera(40.0, 44.0, 8.3, 7.9, 16, 16)


def _loss(orc, s, pose, g, rule):
    out = orc.render(s, CAM, pose, rule)
    return (np.sum(out["rgb"] * g[0]) + np.sum(out["depth"] * g[1]) +
            np.sum(out["normal"] * g[2]) + np.sum(out["opacity"] * g[3]))


def _check_fd(orc, s, pose, rule, tol):
    g = scenes.random_upstream(1, CAM.height, CAM.width)
    an = orc.render_bwd(s, CAM, pose, *g, rule=rule)
    h = 1e-6
    worst = 0.0
    for name in ("mu", "quat", "scale", "opacity", "rgb"):
        arr = getattr(s, name)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            lp = _loss(orc, s, pose, g, rule)
            arr[idx] = old - h
            lm = _loss(orc, s, pose, g, rule)
            arr[idx] = old
            fd[idx] = (lp - lm) / (2 * h)
        scale = max(np.max(np.abs(fd)), 1e-3)
        err = np.max(np.abs(an[name] - fd)) / scale
        worst = max(worst, err)
        assert err < tol, (name, err)
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        lp = _loss(orc, s, orc.retract(pose, e), g, rule)
        lm = _loss(orc, s, orc.retract(pose, -e), g, rule)
        fd[k] = (lp - lm) / (2 * h)
    err = np.max(np.abs(an["pose6"] - fd)) / max(np.max(np.abs(fd)), 1e-3)
    assert err < tol, ("pose", err, an["pose6"], fd)
    return an


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fd_exact_mode(orc, seed):
    s = _scene(seed)
    pose = orc.retract(scenes.identity_pose(), np.array([0.01, -0.02, 0.03, 0.02, -0.01, 0.015]))
    _check_fd(orc, s, pose, orc.Rule(exact=True), 1e-6)


def test_fd_thresholded_mode(orc):
    """With the skip / clamp / stop rules active: away from the thresholds the
    rendered images are still smooth, and clamped surfels get no alpha gradient."""
    s = _scene(5, n=8)
    s.opacity[:3] = 0.999      # clamped at alpha_max near their centres
    s.scale *= 1.5
    pose = scenes.identity_pose()
    _check_fd(orc, s, pose, orc.Rule(), 1e-5)


def test_translation_invariance_of_pose_gradient(orc):
    s = _scene(3, n=10)
    pose = orc.retract(scenes.identity_pose(), np.array([0.02, 0.0, -0.01, 0.03, 0.01, -0.02]))
    g = scenes.random_upstream(2, CAM.height, CAM.width)
    an = orc.render_bwd(s, CAM, pose, *g, rule=orc.Rule())
    np.testing.assert_allclose(an["pose6"][:3], pose.R @ an["mu"].sum(0), rtol=1e-10, atol=1e-12)


def test_rotation_invariance_of_pose_gradient(orc):
    """Rotating the camera by theta about its centre equals rotating every
    surfel about the camera centre by R_cw^T theta; the surfel rotation acts on
    the centre and on the frame (q -> dq * q).  Checked by finite differences
    of the world-space rigid motion, independent of the pose formula."""
    from scipy.spatial.transform import Rotation
    s = _scene(4, n=7)
    pose = orc.retract(scenes.identity_pose(), np.array([0.01, 0.02, 0.0, -0.02, 0.01, 0.03]))
    g = scenes.random_upstream(3, CAM.height, CAM.width)
    rule = orc.Rule(exact=True)
    an = orc.render_bwd(s, CAM, pose, *g, rule=rule)
    cw = -pose.R.T @ pose.t        # camera centre in world space
    h = 1e-6
    for k in range(3):
        vals = []
        for sgn in (1, -1):
            w = np.zeros(3)
            w[k] = sgn * h
            # camera rotation Exp(w) o T_cw == world rotation exp(R^T w) about cw
            Rw = Rotation.from_rotvec(pose.R.T @ w).as_matrix()
            mu = (s.mu - cw) @ Rw.T + cw
            q = s.quat / np.linalg.norm(s.quat, axis=1, keepdims=True)
            Rq = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
            q2 = Rotation.from_matrix(Rw[None] @ Rq).as_quat()
            q2 = np.concatenate([q2[:, 3:], q2[:, :3]], 1)
            s2 = scenes.Surfels(mu, q2, s.scale, s.opacity, s.rgb)
            vals.append(_loss(orc, s2, pose, g, rule))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert fd == pytest.approx(an["pose6"][3 + k], rel=1e-6, abs=1e-9)

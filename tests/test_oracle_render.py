"""Pins of the FP64 oracle's forward renderer against closed forms and
identities fixed by the paper and by geometry (no GPU).

Each test names the passage it pins:
  * camera-facing surfel: Eq. Puv/homo give u = dx d/(f s_u), z = d;
  * single surfel: Eq. alpha_blending with N = 1 gives O = alpha G, C = O c,
    D / O = z;
  * depth consistency of 2DGS (Sec. III-A; the multi-view depth property the
    method relies on): the blended depth of a planar surfel lies on its plane
    from every viewpoint;
  * transmittance identities of Eq. alpha_blending;
  * the paper's skip/stop rules are our readings (alpha_min, alpha_max,
    t_min, cutoff): their closed-form consequences.
"""
import math

import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes

def _rule(orc, exact=True):
    return orc.Rule(exact=exact)


def _facing(mu, s_u, s_v, alpha, rgb):
    return scenes.Surfels(np.array([mu], float), np.array([[1.0, 0, 0, 0]]),
                          np.array([[s_u, s_v]]), np.array([alpha]), np.array([rgb], float))


def test_camera_facing_closed_form(orc):
    cam = scenes.Camera(100.0, 120.0, 16.0, 12.0, 32, 24)
    X, Y, d, su, sv, al = 0.03, -0.02, 1.7, 0.05, 0.08, 0.8
    s = _facing((X, Y, d), su, sv, al, (0.2, 0.5, 0.9))
    out = orc.render(s, cam, scenes.identity_pose(), _rule(orc))
    x = np.arange(cam.width) + 0.5
    y = np.arange(cam.height) + 0.5
    x0 = cam.fx * X / d + cam.cx
    y0 = cam.fy * Y / d + cam.cy
    u = (x[None, :] - x0) * d / (cam.fx * su)
    v = (y[:, None] - y0) * d / (cam.fy * sv)
    G = np.exp(-(u * u + v * v) / 2)
    np.testing.assert_allclose(out["opacity"], al * G, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["rgb"], (al * G)[..., None] * np.array([0.2, 0.5, 0.9]),
                               rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["depth"], d * al * G, rtol=1e-12, atol=1e-15)
    m = out["opacity"] > 1e-3
    np.testing.assert_allclose(out["depth"][m] / out["opacity"][m], d, rtol=1e-12)
    np.testing.assert_allclose(out["normal"][..., 2], al * G, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out["t_final"], 1 - al * G, rtol=1e-12)


def test_centre_pixel_has_unit_gaussian(orc):
    cam = scenes.Camera(100.0, 100.0, 8.0, 8.0, 16, 16)
    d = 2.0
    # centre projects exactly onto the centre of pixel (5, 9)
    X = (5.5 - cam.cx) * d / cam.fx
    Y = (9.5 - cam.cy) * d / cam.fy
    s = _facing((X, Y, d), 0.03, 0.03, 0.7, (1, 1, 1))
    out = orc.render(s, cam, scenes.identity_pose(), _rule(orc))
    assert out["opacity"][9, 5] == pytest.approx(0.7, abs=1e-14)


def test_single_surfel_any_orientation(orc):
    rng = np.random.default_rng(3)
    cam = scenes.Camera(80.0, 80.0, 10.0, 10.0, 20, 20)
    for trial in range(5):
        q = rng.normal(size=4)
        s = scenes.Surfels(np.array([[0.02, -0.01, 1.5]]), q[None], np.array([[0.1, 0.06]]),
                           np.array([0.6]), np.array([[0.3, 0.6, 0.1]]))
        out = orc.render(s, cam, scenes.identity_pose(), _rule(orc))
        O = out["opacity"]
        # O = 1 - T loses relative precision for tiny O, so compare where O > 1e-4
        m = O > 1e-4
        assert m.sum() > 10
        np.testing.assert_allclose(out["rgb"][m], O[m][:, None] * np.array([0.3, 0.6, 0.1]), rtol=1e-10)
        assert np.all(O <= 0.6 + 1e-15)


def _plane_pose_views(rng, mu, k):
    poses = []
    for _ in range(k):
        eye = mu + rng.normal(size=3) * 0.4 + np.array([0, 0, -1.5])
        poses.append(scenes.look_at(eye, mu + rng.normal(size=3) * 0.05, down=(0, 1, 0)))
    return poses


def test_depth_consistency_planar_surfel(orc):
    """Blended depth D/O of one planar surfel back-projects onto its plane from
    any viewpoint, and equals the ray-plane depth (n.mu_c)/(n.r)."""
    rng = np.random.default_rng(7)
    cam = scenes.Camera(60.0, 60.0, 16.0, 16.0, 32, 32)
    mu = np.array([0.1, -0.05, 0.3])
    q = np.array([0.9, 0.2, -0.3, 0.1])
    s = scenes.Surfels(mu[None], q[None], np.array([[0.15, 0.1]]), np.array([0.9]),
                       np.array([[1.0, 1.0, 1.0]]))
    # plane normal in world space = third column of R(q), written via scipy
    from scipy.spatial.transform import Rotation
    qn = q / np.linalg.norm(q)
    n_w = Rotation.from_quat([qn[1], qn[2], qn[3], qn[0]]).as_matrix()[:, 2]
    x = np.arange(cam.width) + 0.5
    y = np.arange(cam.height) + 0.5
    X, Y = np.meshgrid(x, y)
    r = np.stack([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, np.ones_like(X)], -1)
    covered = 0
    for pose in _plane_pose_views(rng, mu, 6):
        out = orc.render(s, cam, pose, _rule(orc))
        m = out["opacity"] > 1e-4
        covered += m.sum()
        z = out["depth"][m] / out["opacity"][m]
        Xc = z[:, None] * r[m]
        Xw = (Xc - pose.t) @ pose.R
        assert np.max(np.abs((Xw - mu) @ n_w)) < 1e-9
        n_c = pose.R @ n_w
        mu_c = pose.R @ mu + pose.t
        np.testing.assert_allclose(z, (n_c @ mu_c) / (r[m] @ n_c), rtol=1e-12)
    assert covered > 200


def test_blending_weights_sum_with_transmittance(orc):
    """Eq. alpha_blending with v = 1 for every surfel: sum_i w_i + T_final = 1."""
    s = scenes.slab_scene(11, 200)
    s.rgb[:] = 1.0
    s.scale *= 4
    cam = scenes.Camera(40.0, 40.0, 12.0, 10.0, 24, 20)
    for exact in (True, False):
        out = orc.render(s, cam, scenes.identity_pose(), _rule(orc, exact))
        np.testing.assert_allclose(out["rgb"][..., 0] + out["t_final"], 1.0, atol=1e-13)
        assert out["count"].max() >= 3


def _ray_plane_alpha(s, cam, px, py):
    """Independent per-surfel alpha at one pixel via the plane normal and an
    orthonormal tangent frame (scipy rotation), exact mode."""
    from scipy.spatial.transform import Rotation
    r = np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0])
    out = []
    for i in range(s.n):
        q = s.quat[i] / np.linalg.norm(s.quat[i])
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        n = R[:, 2]
        z = (n @ s.mu[i]) / (n @ r)
        P = z * r - s.mu[i]
        u = (P @ R[:, 0]) / s.scale[i, 0]
        v = (P @ R[:, 1]) / s.scale[i, 1]
        ok = z > cam.near and s.mu[i, 2] > cam.near
        out.append((s.mu[i, 2], i, s.opacity[i] * math.exp(-(u * u + v * v) / 2) if ok else 0.0))
    return out


def test_opacity_is_one_minus_product_and_order_invariant(orc):
    s = scenes.slab_scene(5, 60)
    s.scale *= 5
    cam = scenes.Camera(40.0, 40.0, 8.0, 8.0, 16, 16)
    rule = _rule(orc)
    out = orc.render(s, cam, scenes.identity_pose(), rule)
    for (px, py) in [(3, 4), (8, 8), (12, 2), (0, 15)]:
        items = _ray_plane_alpha(s, cam, px, py)
        O = 1 - np.prod([1 - a for (_, _, a) in items])
        assert out["opacity"][py, px] == pytest.approx(O, abs=1e-12)
        items.sort()
        T, C = 1.0, np.zeros(3)
        for (_, i, a) in items:
            C += a * T * s.rgb[i]
            T *= 1 - a
        np.testing.assert_allclose(out["rgb"][py, px], C, atol=1e-12)
    perm = np.random.default_rng(0).permutation(s.n)
    out2 = orc.render(s.subset(perm), cam, scenes.identity_pose(), rule)
    np.testing.assert_allclose(out2["opacity"], out["opacity"], atol=1e-13)
    np.testing.assert_allclose(out2["rgb"], out["rgb"], atol=1e-13)


def test_stacked_identical_surfels(orc):
    """M identical camera-facing surfels at one depth: O = 1 - (1 - alpha G)^M;
    equal centre depths blend in surfel-id order."""
    cam = scenes.Camera(50.0, 50.0, 8.0, 8.0, 16, 16)
    M = 5
    mu = np.tile([[0.0, 0.0, 2.0]], (M, 1))
    cols = np.random.default_rng(1).uniform(size=(M, 3))
    s = scenes.Surfels(mu, np.tile([[1.0, 0, 0, 0]], (M, 1)), np.full((M, 2), 0.1),
                       np.full(M, 0.3), cols)
    out = orc.render(s, cam, scenes.identity_pose(), _rule(orc))
    single = orc.render(s.subset(np.arange(1)), cam, scenes.identity_pose(), _rule(orc))
    a = single["opacity"]
    np.testing.assert_allclose(out["opacity"], 1 - (1 - a) ** M, atol=1e-14)
    expect = sum((a * (1 - a) ** k)[..., None] * cols[k] for k in range(M))
    np.testing.assert_allclose(out["rgb"], expect, atol=1e-14)


def test_skip_clamp_and_stop_rules(orc):
    cam = scenes.Camera(50.0, 50.0, 8.0, 8.0, 16, 16)
    rule = orc.Rule()
    # cutoff: only pixels with u^2 + v^2 <= 9 are touched
    s = _facing((0.0, 0.0, 1.0), 0.02, 0.02, 0.95, (1, 1, 1))
    out = orc.render(s, cam, scenes.identity_pose(), rule)
    x = np.arange(16) + 0.5
    u = (x - 8.0) * 1.0 / (50.0 * 0.02)
    r2 = u[None, :] ** 2 + u[:, None] ** 2
    assert np.all(out["opacity"][r2 > 9] == 0)
    assert np.all(out["opacity"][r2 <= 9] > 0)
    # alpha_min: a < 1/255 is skipped
    s2 = _facing((0.0, 0.0, 1.0), 0.05, 0.05, 0.5 / 255 * 2.2, (1, 1, 1))
    out2 = orc.render(s2, cam, scenes.identity_pose(), rule)
    a = s2.opacity[0] * np.exp(-r2 * (0.02 / 0.05) ** 2 / 2)
    np.testing.assert_allclose(out2["opacity"], np.where(a >= 1 / 255, a, 0.0), atol=1e-15)
    # alpha_max clamp at 0.99 and stop before T drops below t_min:
    # M stacked a = 0.99 surfels blend floor(log(1e-4)/log(0.01)) = 2 of them
    M = 6
    s3 = scenes.Surfels(np.tile([[0.0, 0.0, 1.0]], (M, 1)), np.tile([[1.0, 0, 0, 0]], (M, 1)),
                        np.full((M, 2), 10.0), np.full(M, 0.999), np.ones((M, 3)))
    out3 = orc.render(s3, cam, scenes.identity_pose(), rule)
    assert np.all(out3["count"] == 2)
    np.testing.assert_allclose(out3["t_final"], (1 - 0.99) ** 2, rtol=1e-12)
    # with a = 0.9, stop after floor(4 / 1) = 4 surfels (0.1^4 = 1e-4 is kept)
    s4 = scenes.Surfels(s3.mu, s3.quat, s3.scale, np.full(M, 0.9), s3.rgb)
    out4 = orc.render(s4, cam, scenes.identity_pose(), rule)
    G = np.exp(-r2 * (0.02 / 10.0) ** 2 / 2)
    a4 = 0.9 * G
    kmax = np.floor(np.log(1e-4) / np.log(1 - a4) + 1e-9)
    np.testing.assert_array_equal(out4["count"], np.minimum(kmax, M).astype(int))


def test_near_plane_and_behind_camera(orc):
    cam = scenes.Camera(50.0, 50.0, 8.0, 8.0, 16, 16)
    s = _facing((0.0, 0.0, -1.0), 0.1, 0.1, 0.9, (1, 1, 1))
    assert orc.render(s, cam, scenes.identity_pose(), _rule(orc))["opacity"].max() == 0
    s = _facing((0.0, 0.0, 0.04), 0.1, 0.1, 0.9, (1, 1, 1))
    assert orc.render(s, cam, scenes.identity_pose(), _rule(orc))["opacity"].max() == 0


def test_pixel_subset_matches_full(orc):
    s = scenes.slab_scene(2, 300)
    cam = scenes.Camera(60.0, 60.0, 12.0, 9.0, 24, 18)
    full = orc.render(s, cam, scenes.identity_pose())
    pix = scenes.pixel_sample(4, cam.height, cam.width, 50)
    sub = orc.render(s, cam, scenes.identity_pose(), pixels=pix)
    np.testing.assert_array_equal(sub["rgb"], full["rgb"][pix[:, 1], pix[:, 0]])
    np.testing.assert_array_equal(sub["depth"], full["depth"][pix[:, 1], pix[:, 0]])

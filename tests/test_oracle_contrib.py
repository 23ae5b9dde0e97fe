"""Pins of the oracle's per-surfel contribution, visibility, covisibility and
keyframe rule (Sec. III-D, Eq. weight and Eq. contribution; Table I) against
closed forms, identities and hand-worked cases (no GPU).

  * sum over surfels of C_k = sum over pixels of the rendered opacity: the
    weights of a pixel telescope to 1 - T (Eq. alpha_blending), computed by
    the renderer as a product;
  * a camera-facing surfel in exact mode: sum over pixel centres of
    alpha G = alpha 2 pi sigma_x sigma_y (sigma in pixels; the Gaussian's
    sum over a unit lattice equals its integral to far below FP64 rounding
    for sigma >= 2);
  * two camera-facing surfels with the same pixel footprint at different
    depths: the front one gets alpha_1 2 pi sigma^2, the back one
    alpha_2 pi sigma^2 (2 - alpha_1) (its weight carries T = 1 - alpha_1 G
    and the sum of G^2 over the lattice is pi sigma^2);
  * covisibility and the keyframe rule on hand-worked sets and poses.
"""
import math

import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes


def _facing(mus, scales, alphas):
    n = len(mus)
    return scenes.Surfels(np.array(mus, float), np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)),
                          np.array(scales, float), np.array(alphas, float),
                          np.full((n, 3), 0.5))


def test_contributions_sum_to_opacity(orc):
    s, cam, pose = scenes.slab_scene(3, 600), scenes.slab_camera(), scenes.identity_pose()
    c = orc.contrib(s, cam, pose)
    o = orc.render(s, cam, pose)
    assert c["contrib"].min() >= 0.0
    np.testing.assert_allclose(c["contrib"].sum(), o["opacity"].sum(), rtol=1e-12)
    # and per surfel it is bounded by its footprint's pixel count times alpha
    assert np.all(c["contrib"] <= s.opacity * cam.width * cam.height + 1e-12)


def test_single_facing_surfel_gaussian_sum(orc):
    cam = scenes.Camera(400.0, 300.0, 100.3, 80.7, 200, 160)
    d, su, sv, al = 2.0, 0.05, 0.06, 0.7
    s = _facing([(0.0, 0.0, d)], [(su, sv)], [al])
    c = orc.contrib(s, cam, scenes.identity_pose(), orc.Rule(exact=True))["contrib"][0]
    sx, sy = cam.fx * su / d, cam.fy * sv / d        # 10 px and 9 px
    np.testing.assert_allclose(c, al * 2 * math.pi * sx * sy, rtol=1e-9)


def test_single_facing_surfel_with_cutoff(orc):
    """With the cutoff u^2 + v^2 <= 9 (and alpha G >= 1/255 implied by it at
    alpha = 0.9) the sum approaches alpha 2 pi sigma_x sigma_y (1 - e^-4.5);
    the lattice error is O(perimeter / area) = O(1 / sigma)."""
    cam = scenes.Camera(800.0, 800.0, 100.0, 100.0, 200, 200)
    d, s_w, al = 2.0, 0.05, 0.9
    s = _facing([(0.0, 0.0, d)], [(s_w, s_w)], [al])
    c = orc.contrib(s, cam, scenes.identity_pose())["contrib"][0]
    sig = cam.fx * s_w / d                           # 20 px
    np.testing.assert_allclose(c, al * 2 * math.pi * sig * sig * (1 - math.exp(-4.5)), rtol=5e-3)


def test_stacked_facing_surfels(orc):
    cam = scenes.Camera(400.0, 400.0, 60.0, 60.0, 120, 120)
    d1, d2, s1, a1, a2 = 1.0, 1.5, 0.02, 0.6, 0.8
    s2 = s1 * d2 / d1                                # the same footprint in pixels
    s = _facing([(0.0, 0.0, d2), (0.0, 0.0, d1)], [(s2, s2), (s1, s1)], [a2, a1])
    c = orc.contrib(s, cam, scenes.identity_pose(), orc.Rule(exact=True))["contrib"]
    sig = cam.fx * s1 / d1                           # 8 px
    np.testing.assert_allclose(c[1], a1 * 2 * math.pi * sig * sig, rtol=1e-9)
    np.testing.assert_allclose(c[0], a2 * math.pi * sig * sig * (2 - a1), rtol=1e-9)


def test_visibility_and_covisibility_hand_cases(orc):
    ca = np.array([0.6, 0.4, 0.9, 0.0, 0.51, 0.5])
    cb = np.array([0.7, 0.6, 0.2, 0.0, 0.5, 0.50001])
    assert list(np.flatnonzero(orc.visible(ca))) == [0, 2, 4]     # 0.5 itself is not visible
    assert list(np.flatnonzero(orc.visible(cb))) == [0, 1, 5]
    inter, union, score = orc.covisibility(ca, cb)
    assert (inter, union) == (1, 5) and score == pytest.approx(0.2)
    assert orc.covisibility(np.zeros(4), np.zeros(4)) == (0, 0, 0.0)
    assert orc.covisibility(ca, ca)[2] == 1.0


@pytest.mark.parametrize("score,ta,tb,expect", [
    (0.95, (0.0, 0.0, 0.0), (0.10, 0.0, 0.0), False),    # covisible, 10 cm apart
    (0.95, (0.0, 0.0, 0.0), (0.10, 0.10, 0.06), True),   # 15.4 cm > d_k
    (0.95, (1.0, 2.0, 3.0), (1.0, 2.0, 3.149), False),   # 14.9 cm
    (0.85, (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), True),      # covisibility below c_k
    (0.90, (1.0, 2.0, 3.0), (1.0, 2.1, 3.0), False),     # score == c_k is not below it
])
def test_keyframe_rule_hand_cases(orc, score, ta, tb, expect):
    assert orc.keyframe_rule(score, ta, tb) is expect

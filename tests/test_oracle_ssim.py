"""Pins of the oracle's SSIM term of the mapping loss (Sec. III-E, L_c with
L_SSIM of Wang et al. 2004; Table I weight) against closed forms and the
plain definition (no GPU):

  * the window: normalised, symmetric, Gaussian ratios of sigma 1.5;
  * SSIM(x, x) = 1 at every pixel (borders included): zero loss, zero
    gradient;
  * constant images a, b: interior SSIM = (2ab + C1) / (a^2 + b^2 + C1);
  * the library-convolution map against the definition written out as a
    sum over the 121 window offsets with zero padding, at border, corner
    and interior pixels;
  * the gradient against central finite differences;
  * the mapping loss with the SSIM weight: linear in the weight between the
    L1 term and the SSIM term.
"""
import math

import numpy as np

from paper_2506_00970_gb300 import scenes


def test_window(orc):
    w = orc.ssim_window()
    assert w.shape == (11, 11)
    np.testing.assert_allclose(w.sum(), 1.0, rtol=1e-14)
    np.testing.assert_allclose(w, w.T, rtol=0, atol=0)
    np.testing.assert_allclose(w, w[::-1, ::-1], rtol=0, atol=0)
    np.testing.assert_allclose(w[5, 5] / w[5, 6], math.exp(1.0 / (2 * 1.5 ** 2)), rtol=1e-13)
    np.testing.assert_allclose(w[5, 5] / w[6, 6], math.exp(2.0 / (2 * 1.5 ** 2)), rtol=1e-13)


def test_identical_images(orc):
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(23, 31, 3))
    np.testing.assert_allclose(orc.ssim(x, x), 1.0, rtol=0, atol=1e-12)
    L, g = orc.ssim_loss(x, x, weight=0.7)
    assert abs(L) < 1e-12 and np.abs(g).max() < 1e-12


def test_constant_images_closed_form(orc):
    a, b = 0.3, 0.8
    S = orc.ssim(np.full((30, 30, 3), a), np.full((30, 30, 3), b))
    C1 = 1e-4
    np.testing.assert_allclose(S[5:-5, 5:-5], (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)


def test_map_matches_definition(orc):
    rng = np.random.default_rng(1)
    H, W = 17, 14
    x = rng.uniform(size=(H, W, 3))
    y = np.clip(x + rng.normal(scale=0.2, size=x.shape), 0, 1)
    S = orc.ssim(x, y)
    w = orc.ssim_window()
    C1, C2 = 1e-4, 9e-4

    def at(img, r, c, ch):
        return img[r, c, ch] if 0 <= r < H and 0 <= c < W else 0.0

    for (r, c) in [(0, 0), (0, 7), (8, 0), (8, 7), (16, 13), (3, 12)]:
        for ch in range(3):
            m = np.zeros(5)
            for dr in range(-5, 6):
                for dc in range(-5, 6):
                    a, b = at(x, r + dr, c + dc, ch), at(y, r + dr, c + dc, ch)
                    m += w[dr + 5, dc + 5] * np.array([a, b, a * a, b * b, a * b])
            mx, my, exx, eyy, exy = m
            s = ((2 * mx * my + C1) * (2 * (exy - mx * my) + C2)) / (
                (mx * mx + my * my + C1) * (exx - mx * mx + eyy - my * my + C2))
            np.testing.assert_allclose(S[r, c, ch], s, rtol=1e-12)


def test_gradient_finite_differences(orc):
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(9, 8, 3))
    y = rng.uniform(size=(9, 8, 3))
    L, g = orc.ssim_loss(x, y, weight=0.5)
    h = 1e-6
    for idx in [(0, 0, 0), (4, 3, 1), (8, 7, 2), (2, 6, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (orc.ssim_loss(xp, y, 0.5)[0] - orc.ssim_loss(xm, y, 0.5)[0]) / (2 * h)
        np.testing.assert_allclose(g[idx], fd, rtol=1e-6, atol=1e-10)


def test_mapping_loss_ssim_weight_is_linear(orc):
    rng = np.random.default_rng(3)
    cam = scenes.Camera(40.0, 40.0, 12.0, 10.0, 24, 20)
    img = dict(rgb=rng.uniform(size=(20, 24, 3)), depth=rng.uniform(1, 2, (20, 24)),
               normal=rng.normal(size=(20, 24, 3)), opacity=rng.uniform(0.6, 1, (20, 24)))
    obs_rgb = rng.uniform(size=(20, 24, 3))
    obs_d = rng.uniform(1, 2, (20, 24))
    L0, g0 = orc.mapping_loss(img, obs_rgb, obs_d, cam, w_ssim=0.0)
    L1, g1 = orc.mapping_loss(img, obs_rgb, obs_d, cam, w_ssim=1.0)
    Lh, gh = orc.mapping_loss(img, obs_rgb, obs_d, cam, w_ssim=0.125)
    np.testing.assert_allclose(Lh, 0.875 * L0 + 0.125 * L1, rtol=1e-12)
    np.testing.assert_allclose(gh["rgb"], 0.875 * g0["rgb"] + 0.125 * g1["rgb"], atol=1e-15)
    Ls, gs = orc.ssim_loss(img["rgb"], obs_rgb)
    l1 = np.abs(img["rgb"] - obs_rgb).sum() / (20 * 24)
    np.testing.assert_allclose(L1 - L0, Ls - l1, rtol=1e-12)

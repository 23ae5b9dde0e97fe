"""Pins of the oracle's threshold diagnostic (no GPU).

``render(...)["ambiguous"]`` marks pixels that hold a compositing decision
within rounding of its threshold -- the cutoff radius u^2 + v^2 = 9, the skip
a = alpha_min, the near plane, or the stop test T = t_min (our readings of
the blending rules of Eq. alpha_blending) -- at or before the position where
the pixel stops blending.  ``render_bwd(...)["ambiguous"]`` marks the surfels
that are candidates at such pixels.  The parity tests exempt exactly these
from their tight bounds, so the diagnostic is pinned here on constructed
scenes whose decisions sit on a threshold by closed form (camera-facing
surfels: u = dx d / (f s_u), Eq. Puv / homo), and shown to be rare on a
generic scene.
"""
import math

import numpy as np

from paper_2506_00970_gb300 import scenes

F, D = 100.0, 2.0
CAM = scenes.Camera(F, F, 16.0, 8.5, 32, 17)   # pixel (15, 8) has its centre on the axis


def _facing(rows):
    """Camera-facing surfels: rows of (x, y, z, s_u, s_v, alpha)."""
    a = np.asarray(rows, float)
    n = len(a)
    return scenes.Surfels(a[:, :3], np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), a[:, 3:5], a[:, 5],
                          np.tile([0.4, 0.5, 0.6], (n, 1)))


def _x(col, z=D):
    """Camera-space x of a surfel centre at depth z that projects onto
    column col's pixel centre."""
    return (col + 0.5 - CAM.cx) * z / F


def test_cutoff_radius_is_flagged(orc):
    # centre on pixel (12, 8); s_u so that the pixel 3 columns right has u = 3
    s_u = 3.0 * D / (3.0 * F)
    s = _facing([(_x(12), 0.0, D, s_u, 1.0, 0.9)])
    o = orc.render(s, CAM, scenes.identity_pose(), orc.Rule())
    amb = o["ambiguous"]
    assert amb[8, 15] and amb[8, 9]          # u = +-3: on the cutoff
    assert not amb[8, 14] and not amb[8, 10]  # u = +-2
    assert not amb[8, 12] and not amb[8, 16]  # centre; u = 4 (outside, not near)
    assert amb.sum() == 2


def test_alpha_min_is_flagged(orc):
    # alpha G at u = 2 equals alpha_min exactly
    s_u = 1.0 * D / (1.0 * F)                 # u = column offset
    alpha = (1.0 / 255.0) / math.exp(-2.0)
    s = _facing([(_x(12), 0.0, D, s_u, s_u, alpha)])     # v = row offset
    o = orc.render(s, CAM, scenes.identity_pose(), orc.Rule())
    amb = o["ambiguous"]
    # u^2 + v^2 = 4 at two columns and two rows from the centre pixel (12, 8)
    assert amb[8, 14] and amb[8, 10] and amb[6, 12] and amb[10, 12]
    assert not amb[8, 13] and not amb[8, 11] and not amb[8, 12] and not amb[7, 13]
    assert amb.sum() == 4


def test_stop_test_is_flagged(orc):
    # three stacked surfels of alpha a: (1 - a)^3 = t_min at the axis pixel
    a = 1.0 - 1e-4 ** (1.0 / 3.0)
    rows = [(_x(15), 0.0, D + 0.01 * k, 0.2, 0.2, a) for k in range(3)]
    o = orc.render(_facing(rows), CAM, scenes.identity_pose(), orc.Rule())
    amb = o["ambiguous"]
    assert amb[8, 15]
    # off the axis pixel G < 1 moves (1 - a G)^3 far from t_min
    assert amb.sum() == 1


def test_decision_after_the_stop_is_not_flagged(orc):
    # an opaque stack stops blending well away from t_min; a surfel on its
    # cutoff behind the stack is never reached, in front of it it is
    stack = [(_x(15, D + 0.01 * k), 0.0, D + 0.01 * k, 1.0, 1.0, 0.98) for k in range(3)]
    for z, flagged in ((D + 0.5, False), (D - 0.5, True)):
        # centre on column 12 at depth z; u = 3 three columns right
        edge = (_x(12, z), 0.0, z, 3.0 * z / (3.0 * F), 1.0, 0.9)
        o = orc.render(_facing(stack + [edge]), CAM, scenes.identity_pose(), orc.Rule())
        assert o["ambiguous"][8, 15] == flagged, z


def test_exact_mode_has_no_thresholds(orc):
    s_u = 3.0 * D / (3.0 * F)
    s = _facing([(_x(12), 0.0, D, s_u, 1.0, 0.9)])
    o = orc.render(s, CAM, scenes.identity_pose(), orc.Rule(exact=True))
    assert not o["ambiguous"].any()


def test_backward_flags_the_candidates_of_ambiguous_pixels(orc):
    s_u = 3.0 * D / (3.0 * F)
    s = _facing([
        (_x(12), 0.0, D, s_u, 1.0, 0.9),           # on the cutoff at (15, 8) and (9, 8)
        (_x(15), 0.0, D + 0.2, 0.05, 0.05, 0.5),   # covers (15, 8), behind
        (_x(27), 0.0, D, 0.013, 0.013, 0.5),       # far from both; no pixel on a threshold
    ])
    up = scenes.random_upstream(0, CAM.height, CAM.width)
    g = orc.render_bwd(s, CAM, scenes.identity_pose(), *up, rule=orc.Rule())
    assert list(g["ambiguous"]) == [True, True, False]
    # only the listed pixels count
    pix = np.array([[27, 8], [26, 8]], np.int32)
    sub = [u[pix[:, 1], pix[:, 0]] for u in up]
    g = orc.render_bwd(s, CAM, scenes.identity_pose(), *sub, rule=orc.Rule(), pixels=pix)
    assert not g["ambiguous"].any()


def test_rare_on_a_generic_scene(orc):
    s, cam, pose = scenes.slab_scene(0), scenes.slab_camera(), scenes.identity_pose()
    o = orc.render(s, cam, pose)
    assert o["ambiguous"].mean() < 5e-3
    up = scenes.random_upstream(1, cam.height, cam.width)
    g = orc.render_bwd(s, cam, pose, *up)
    # every flagged surfel is a candidate at a flagged pixel: few of them
    assert g["ambiguous"].mean() < 0.05

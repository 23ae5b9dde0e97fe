"""Pins of the map-state oracle (Eq. map, Sec. III-F state update, Sec. IV-C
map correction, Sec. III-F occlusion removal) against hand-worked cases and
geometric identities (no GPU).

  * the state update on a hand-worked table (each row's expected values are
    derived in its comment from the rules of Sec. III-F);
  * map correction: the corrected map seen from a keyframe's optimised pose
    equals the original map seen from its original pose (both the surfel
    centres and orientations in camera space, and the rendered images) --
    the property that makes the map follow the optimised keyframes; an
    unchanged pose graph leaves the map unchanged;
  * quaternion-to-matrix on known rotations;
  * pruning and compaction on a hand-worked case.
"""
import math

import numpy as np

import oracle.map_state as ms
from paper_2506_00970_gb300 import scenes


def _state(delta, t_c, d_c, t_l):
    return dict(delta=np.array(delta), t_c=np.array(t_c), d_c=np.array(d_c, float),
                t_l=np.array(t_l))


def test_observe_hand_table():
    # keyframe 7 at R = I, t = (-1, 0, 0): viewpoint c = (1, 0, 0)
    R, t = np.eye(3), np.array([-1.0, 0.0, 0.0])
    mu = np.array([[1.0, 0, 2], [1.0, 0, 4], [0.0, 0, 0], [5.0, 0, 0], [1.0, 1, 0], [1.0, 2, 0],
                   [1.0, 3, 0]])
    contrib = np.array([0.8, 0.9, 0.2, 0.5, 0.9, 0.1, 0.7])
    st = _state(delta=[1, 1, 1, 1, 0, 0, 0], t_c=[2, 3, 1, 1, 6, 6, 3],
                d_c=[3.0, 1.5, 0.5, 9.0, 1.0, 1.0, 1.0], t_l=[5, 6, 4, 3, 2, 2, 2])
    new, counts = ms.observe(contrib, mu, R, t, 7, st, inactive_after=3)
    # 0: visible, distance 2 < 3: t_l = 7, d_c = 2, t_c = 7
    # 1: visible, distance 4 > 1.5: t_l = 7, closest kept
    # 2: not visible, 7 - 4 = 3 is not above 3: stays active
    # 3: contribution 0.5 is not above 0.5; 7 - 3 = 4 > 3: deactivated
    # 4, 5, 6: inactive, no reactivation outside a loop window
    assert new["delta"].tolist() == [1, 1, 1, 0, 0, 0, 0]
    assert new["t_l"].tolist() == [7, 7, 4, 3, 2, 2, 2]
    assert new["t_c"].tolist() == [7, 3, 1, 1, 6, 6, 3]
    np.testing.assert_allclose(new["d_c"], [2.0, 1.5, 0.5, 9.0, 1.0, 1.0, 1.0])
    assert counts == (2, 1, 1, 0)
    # within a loop window with K_h = 4: surfel 4 (visible, t_c = 6 > 4) comes
    # back with t_l = 7; 5 is not visible; 6 has t_c = 3, not after h
    new2, counts2 = ms.observe(contrib, mu, R, t, 7, st, inactive_after=3, reactivate=True,
                               loop_h=4)
    assert new2["delta"].tolist() == [1, 1, 1, 0, 1, 0, 0]
    assert new2["t_l"].tolist() == [7, 7, 4, 3, 7, 2, 2]
    assert counts2 == (2, 1, 1, 1)


def test_quat_matrix_known_rotations():
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    Rz = ms.quat_matrix([c, 0.0, 0.0, s])             # 90 degrees about z
    np.testing.assert_allclose(Rz, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)
    Rx = ms.quat_matrix([0.0, 2.0, 0.0, 0.0])          # 180 degrees about x, unnormalised
    np.testing.assert_allclose(Rx, np.diag([1.0, -1.0, -1.0]), atol=1e-15)


def _random_pose(rng):
    q = rng.normal(size=4)
    R = ms.quat_matrix(q)
    return R, rng.normal(size=3)


def test_correct_follows_keyframes():
    rng = np.random.default_rng(3)
    n, n_kf = 400, 5
    mu = rng.normal(size=(n, 3)) * 2
    quat = rng.normal(size=(n, 4))
    t_c = rng.integers(-1, n_kf + 1, n)                # includes invalid ids -1 and n_kf
    old = [_random_pose(rng) for _ in range(n_kf)]
    new = [_random_pose(rng) for _ in range(n_kf)]
    mu2, R2, skipped = ms.correct(mu, quat, t_c, old, new)
    R = ms.quat_matrix(quat)
    assert skipped == int(((t_c < 0) | (t_c >= n_kf)).sum())
    for j in range(n_kf):
        sel = t_c == j
        (Ro, to), (Rn, tn) = old[j], new[j]
        # camera-space centre and orientation from the optimised pose are the
        # original ones from the original pose
        np.testing.assert_allclose(mu2[sel] @ Rn.T + tn, mu[sel] @ Ro.T + to, atol=1e-12)
        np.testing.assert_allclose(Rn[None] @ R2[sel], Ro[None] @ R[sel], atol=1e-12)
    bad = (t_c < 0) | (t_c >= n_kf)
    np.testing.assert_array_equal(mu2[bad], mu[bad])
    # an unchanged pose graph changes nothing
    mu3, R3, _ = ms.correct(mu, quat, t_c, old, old)
    np.testing.assert_allclose(mu3, mu, atol=1e-12)
    np.testing.assert_allclose(R3, R, atol=1e-12)


def test_correct_render_invariance(orc):
    """A keyframe's surfels render the same image from its optimised pose
    after the correction as from its original pose before it."""
    s, cam = scenes.slab_scene(5, 300), scenes.slab_camera()
    old = scenes.identity_pose()
    new = scenes.perturb_pose(old, 0.05, 3.0, seed=9)
    t_c = np.zeros(s.n, int)
    mu2, R2, _ = ms.correct(s.mu, s.quat, t_c, [(old.R, old.t)], [(new.R, new.t)])
    q2 = np.array([scenes._quat_wxyz_from_matrix(Rk) for Rk in R2])
    s2 = scenes.Surfels(mu2, q2, s.scale, s.opacity, s.rgb)
    a = orc.render(s, cam, old)
    b = orc.render(s2, cam, new)
    for k in ("rgb", "depth", "normal", "opacity"):
        np.testing.assert_allclose(b[k], a[k], atol=1e-9)
    assert a["opacity"].max() > 0.5


def test_prune_and_compact_hand_case():
    contrib = np.array([0.3, 0.7, 0.49, 0.5, 0.1, 0.0])
    t_c = np.array([4, 4, 4, 4, 3, 4])
    keep = ms.prune_keep(contrib, t_c, 4)
    # t_c = 4 and contribution < 0.5 go: 0, 2, 5; 3 (exactly 0.5) and 4 (t_c = 3) stay
    assert keep.tolist() == [False, True, False, True, True, False]
    (a, b), new_index = ms.compact(keep, np.arange(6) * 10, np.arange(12).reshape(6, 2))
    assert a.tolist() == [10, 30, 40]
    assert b.tolist() == [[2, 3], [6, 7], [8, 9]]
    assert new_index.tolist() == [-1, 0, -1, 1, 2, -1]

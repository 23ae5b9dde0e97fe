"""Pins of the map-expansion oracle (Sec. III-E: RGB-D to points, random
downsampling, nearest-neighbour scales, normals from Eq. normal_fromD,
random tangents, the voxel occupancy gate) against closed forms and
hand-checked cases (no GPU):

  * the tangent basis of Duff et al. 2017: orthonormal, right-handed, also
    at the poles;
  * a fronto-parallel plane: every point at depth d, normal (0, 0, 1) (away
    from the camera, as Eq. normal_fromD gives it), nearest-neighbour
    distance = one pixel's footprint d / f, viewpoint distance |X_c|;
  * a tilted plane seen from a moved camera: world points on the plane,
    world normals equal to the plane normal (central differences of a plane
    are exact), rotation matrices proper with t_n as third column;
  * downsampling keeps exactly the pixels with u < ratio; holes and their
    neighbours get no surfel; occupied voxels block creation.
"""

import numpy as np

import oracle.expand as ex
import oracle.map_state as ms
from paper_2506_00970_gb300 import scenes


def test_duff_basis():
    rng = np.random.default_rng(0)
    n = rng.normal(size=(500, 3))
    n = np.concatenate([n, [[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, -1.0, 1e-9]]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    b1, b2 = ex.duff_basis(n)
    for a, b in ((b1, b1), (b2, b2)):
        np.testing.assert_allclose((a * b).sum(-1), 1.0, atol=1e-12)
    np.testing.assert_allclose((b1 * b2).sum(-1), 0.0, atol=1e-12)
    np.testing.assert_allclose((b1 * n).sum(-1), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(b1, b2), n, atol=1e-12)


def test_fronto_parallel_plane():
    cam = scenes.Camera(100.0, 100.0, 16.0, 12.0, 32, 24)
    d = 2.0
    depth = np.full((24, 32), d)
    rgb = np.random.default_rng(1).uniform(size=(24, 32, 3))
    out = ex.expand(rgb, depth, cam, np.eye(3), np.zeros(3), np.zeros((24, 32)),
                    np.zeros((24, 32)), 1.0, kf_id=4)
    # interior pixels only (the normal needs four neighbours)
    assert len(out["mu"]) == 22 * 30
    np.testing.assert_allclose(out["mu"][:, 2], d, atol=1e-15)
    np.testing.assert_allclose(out["R"][:, :, 2], np.tile([0, 0, 1.0], (22 * 30, 1)), atol=1e-12)
    np.testing.assert_allclose(out["scale"], d / 100.0, rtol=1e-12)
    np.testing.assert_allclose(out["d_c"], np.linalg.norm(out["mu"], axis=1), rtol=1e-12)
    # u_angle = 0: t_u is b1 of the basis, here (1, 0, 0)
    np.testing.assert_allclose(out["R"][:, :, 0], np.tile([1.0, 0, 0], (22 * 30, 1)), atol=1e-12)
    assert np.all(out["t_c"] == 4) and np.all(out["t_l"] == 4) and np.all(out["delta"] == 1)
    np.testing.assert_allclose(out["opacity"], 0.99)
    np.testing.assert_array_equal(out["rgb"], rgb.reshape(-1, 3)[out["pixel"]])


def test_tilted_plane_from_moved_camera():
    cam = scenes.Camera(120.0, 110.0, 20.0, 15.0, 40, 30)
    # plane n . X_c = c in the camera frame
    n_c = np.array([0.3, -0.2, 1.0])
    n_c /= np.linalg.norm(n_c)
    c = 1.8
    x = (np.arange(40) + 0.5 - cam.cx) / cam.fx
    y = (np.arange(30) + 0.5 - cam.cy) / cam.fy
    rx, ry = np.meshgrid(x, y)
    depth = c / (n_c[0] * rx + n_c[1] * ry + n_c[2])
    rng = np.random.default_rng(2)
    R = ms.quat_matrix(rng.normal(size=4))
    t = rng.normal(size=3)
    out = ex.expand(np.zeros((30, 40, 3)), depth, cam, R, t, rng.uniform(size=(30, 40)),
                    rng.uniform(size=(30, 40)), 0.5, kf_id=1)
    assert len(out["mu"]) > 100
    n_w = R.T @ n_c
    # world points on the plane n_w . X = c + n_c . t  (X_c = R X + t)
    np.testing.assert_allclose(out["mu"] @ n_w, c - n_c @ t, atol=1e-12)
    # the normal of Eq. normal_fromD is the plane normal, away from the camera
    np.testing.assert_allclose(out["R"][:, :, 2], np.tile(n_w, (len(out["mu"]), 1)), atol=1e-9)
    Rs = out["R"]
    np.testing.assert_allclose(np.einsum("kij,kil->kjl", Rs, Rs), np.tile(np.eye(3), (len(Rs), 1, 1)),
                               atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(Rs), 1.0, atol=1e-12)


def test_downsampling_holes_and_voxel_gate():
    cam = scenes.Camera(100.0, 100.0, 10.0, 10.0, 20, 20)
    depth = np.full((20, 20), 1.5)
    depth[7, 9] = 0.0                                   # a hole
    u = np.random.default_rng(3).uniform(size=(20, 20))
    out = ex.expand(np.zeros((20, 20, 3)), depth, cam, np.eye(3), np.zeros(3), u,
                    np.zeros((20, 20)), 0.3, kf_id=0)
    keep = (u < 0.3) & (depth > 0)
    np.testing.assert_array_equal(out["ps_pixel"], np.flatnonzero(keep.ravel()))
    made = set(out["pixel"].tolist())
    for p in (7 * 20 + 9, 7 * 20 + 8, 7 * 20 + 10, 6 * 20 + 9, 8 * 20 + 9):
        assert p not in made                             # the hole and its neighbours
    # block the voxels of the first three candidates
    occ = {tuple(v) for v in ex.voxel_index(out["mu"][:3], 0.05)}
    out2 = ex.expand(np.zeros((20, 20, 3)), depth, cam, np.eye(3), np.zeros(3), u,
                     np.zeros((20, 20)), 0.3, kf_id=0, occupied=occ, voxel=0.05)
    vox2 = {tuple(v) for v in ex.voxel_index(out2["mu"], 0.05)}
    assert not (vox2 & occ)
    assert len(out2["mu"]) < len(out["mu"])

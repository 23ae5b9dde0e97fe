"""FP64 oracle of the map expansion of 2DGS-SLAM (Sec. III-E) -- test
infrastructure only (imported by ``tests/``, never by the product path).

The steps, in the paper's order: the keyframe's RGB-D image as a coloured
point cloud P (pixels with a valid depth, back-projected at the pixel
centre), random downsampling to P_s (the random numbers are inputs: pixel p
is kept when u_keep[p] < ratio), P_s in world coordinates, and a new surfel
for every point of P_s with a normal in N_D (Eq. normal_fromD of the
observed depth) whose voxel of edge r_h holds no surfel of the active map:
scales s_u = s_v = the distance to the nearest other point of P_s (a library
k-d tree query), opacity 0.99, the pixel's colour, t_n = R^T N_D and random
tangents t_u, t_v perpendicular to it (angle 2 pi u_angle[p] in the basis of
Duff et al. 2017), t^c = t^l = the keyframe id, delta = 1, and d^c the
distance to the keyframe's viewpoint.
"""
from __future__ import annotations

import math

import numpy as np


def voxel_index(X, voxel):
    """Integer voxel coordinates floor(X / r_h) per axis."""
    return np.floor(np.asarray(X, np.float64) / voxel).astype(np.int64)


def duff_basis(n):
    """Orthonormal b1, b2 with b1 x b2 = n for unit n (Duff et al., "Building
    an Orthonormal Basis, Revisited", JCGT 2017)."""
    n = np.asarray(n, np.float64)
    sg = np.where(n[..., 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sg + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    b1 = np.stack([1 + sg * n[..., 0] ** 2 * a, sg * b, -sg * n[..., 0]], -1)
    b2 = np.stack([b, sg + n[..., 1] ** 2 * a, -n[..., 1]], -1)
    return b1, b2


def _rays(cam):
    x = (np.arange(cam.width) + 0.5 - cam.cx) / cam.fx
    y = (np.arange(cam.height) + 0.5 - cam.cy) / cam.fy
    return np.stack([np.broadcast_to(x[None, :], (cam.height, cam.width)),
                     np.broadcast_to(y[:, None], (cam.height, cam.width)),
                     np.ones((cam.height, cam.width))], -1)


def observed_normals(depth, cam):
    """N_D of Eq. normal_fromD from an observed depth image (camera frame):
    central differences of the back-projected points; defined at interior
    pixels whose own and four neighbours' depths are valid and whose cross
    product is not zero.  Returns (N (H, W, 3), valid (H, W))."""
    D = np.asarray(depth, np.float64)
    ok_d = np.isfinite(D) & (D > 0)
    X = np.where(ok_d, D, 0.0)[..., None] * _rays(cam)
    H, W = D.shape
    N = np.zeros((H, W, 3))
    valid = np.zeros((H, W), bool)
    gx = (X[1:-1, 2:] - X[1:-1, :-2]) / 2
    gy = (X[2:, 1:-1] - X[:-2, 1:-1]) / 2
    c = np.cross(gx, gy)
    ln = np.linalg.norm(c, axis=-1)
    inner = (ok_d[1:-1, 1:-1] & ok_d[1:-1, 2:] & ok_d[1:-1, :-2] & ok_d[2:, 1:-1] & ok_d[:-2, 1:-1]
             & (ln > 0))
    N[1:-1, 1:-1] = np.where(inner[..., None], c / np.where(ln > 0, ln, 1.0)[..., None], 0.0)
    valid[1:-1, 1:-1] = inner
    return N, valid


def nearest_distance(P):
    """Distance from each point to its nearest other point (inf if alone)."""
    P = np.asarray(P, np.float64)
    if len(P) < 2:
        return np.full(len(P), np.inf)
    from scipy.spatial import cKDTree
    d, _ = cKDTree(P).query(P, k=2)
    return d[:, 1]


def expand(rgb, depth, cam, R_cw, t_cw, u_keep, u_angle, ratio, kf_id, occupied=(), voxel=0.05,
           opacity=0.99, max_scale=0.05):
    """New surfels (in pixel order) as a dict of arrays: mu, R (rotation
    matrices [t_u, t_v, t_n]), scale, opacity, rgb, delta, t_c, t_l, d_c, and
    the pixel index of each; plus P_s itself (pixel indices and world
    points).  ``occupied``: a set of voxel index triples of the active map."""
    R = np.asarray(R_cw, np.float64)
    t = np.asarray(t_cw, np.float64)
    D = np.asarray(depth, np.float64)
    H, W = D.shape
    ok = np.isfinite(D) & (D > 0)
    keep = ok & (np.asarray(u_keep) < ratio)
    pix = np.flatnonzero(keep.ravel())                       # P_s in pixel order
    Xc = (np.where(ok, D, 0.0)[..., None] * _rays(cam)).reshape(-1, 3)[pix]
    Xw = (Xc - t) @ R                                        # R^T (X_c - t)
    nnd = nearest_distance(Xw)
    N, nvalid = observed_normals(D, cam)
    N = N.reshape(-1, 3)[pix]
    nvalid = nvalid.ravel()[pix]
    vox = voxel_index(Xw, voxel)
    occ = set(map(tuple, occupied))
    free = np.array([tuple(v) not in occ for v in vox], bool) if len(pix) else np.zeros(0, bool)
    make = nvalid & free
    tn = N[make] @ R                                         # R^T N
    b1, b2 = duff_basis(tn)
    phi = 2 * math.pi * np.asarray(u_angle, np.float64).ravel()[pix[make]]
    tu = np.cos(phi)[:, None] * b1 + np.sin(phi)[:, None] * b2
    tv = np.cross(tn, tu)
    rot = np.stack([tu, tv, tn], -1)                          # columns
    k = int(make.sum())
    s = np.where(np.isfinite(nnd[make]), nnd[make], max_scale)
    return dict(mu=Xw[make], R=rot, scale=np.stack([s, s], -1), opacity=np.full(k, opacity),
                rgb=np.asarray(rgb, np.float64).reshape(-1, 3)[pix[make]],
                delta=np.ones(k, np.int64), t_c=np.full(k, kf_id), t_l=np.full(k, kf_id),
                d_c=np.linalg.norm(Xc[make], axis=1), pixel=pix[make],
                ps_pixel=pix, ps_world=Xw, ps_nn=nnd, ps_voxel=vox)

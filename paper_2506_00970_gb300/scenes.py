"""Seeded synthetic inputs for the 2D Gaussian surfel rasterizer.

This module only *draws inputs*: surfel parameters, pinhole cameras, camera
poses, pose perturbations, random images and random per-pixel gradients.  It
holds none of the rasterizer's arithmetic (no projection, intersection,
blending, loss or pose update), so that the CPU oracle and the CUDA path can
both consume its output without sharing any of the method's code.

Surfel parameters follow the paper's parameterisation (Sec. III-A, Eq. Puv):
centre ``mu`` (N,3), rotation as a unit quaternion ``quat`` (N,4, order
w,x,y,z) whose matrix columns are ``t_u, t_v, t_n``, tangent scales ``scale``
(N,2) = (s_u, s_v), opacity ``opacity`` (N,) in (0,1) and colour ``rgb`` (N,3).
Poses are world-to-camera ``T_cw`` as a row-major 3x3 ``R`` and a 3-vector
``t`` (x_c = R x_w + t); camera axes are x right, y down, z forward.

Workload shapes stand in for the paper's RGB-D datasets (Sec. IV-A: Replica at
1200x680, TUM/ScanNet-like 640x480); none of their content is reproduced.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation


# --------------------------------------------------------------------------
# containers
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Surfels:
    mu: np.ndarray        # (N,3) float
    quat: np.ndarray      # (N,4) float, (w,x,y,z)
    scale: np.ndarray     # (N,2) float, (s_u, s_v) > 0
    opacity: np.ndarray   # (N,)  float in (0,1)
    rgb: np.ndarray       # (N,3) float

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    def astype(self, dtype) -> "Surfels":
        return Surfels(*(np.ascontiguousarray(a, dtype=dtype) for a in
                         (self.mu, self.quat, self.scale, self.opacity, self.rgb)))

    def subset(self, idx: np.ndarray) -> "Surfels":
        return Surfels(self.mu[idx], self.quat[idx], self.scale[idx],
                       self.opacity[idx], self.rgb[idx])


@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.05


@dataclasses.dataclass
class Pose:
    R: np.ndarray   # (3,3) world->camera rotation
    t: np.ndarray   # (3,)  world->camera translation

    def copy(self) -> "Pose":
        return Pose(self.R.copy(), self.t.copy())


def identity_pose() -> Pose:
    return Pose(np.eye(3), np.zeros(3))


# --------------------------------------------------------------------------
# small helpers (input drawing only)
# --------------------------------------------------------------------------
def _quat_wxyz_from_matrix(R: np.ndarray) -> np.ndarray:
    q = Rotation.from_matrix(R).as_quat()          # scipy order (x,y,z,w)
    return np.concatenate([q[..., 3:4], q[..., 0:3]], axis=-1)


def _random_unit(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _unit(a):
    n = math.sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2])
    return (a[0] / n, a[1] / n, a[2] / n)


def look_at(eye, target, down=(0.0, 0.0, -1.0)) -> Pose:
    """World->camera pose of a camera at ``eye`` looking at ``target``.

    Camera x points right, y down, z forward; the world z axis is up.
    """
    e = [float(v) for v in eye]
    f = _unit([float(target[k]) - e[k] for k in range(3)])
    x = _unit(_cross([float(v) for v in down], f))
    y = _cross(f, x)
    R = np.array([x, y, f])                      # rows: the camera axes in world coordinates
    return Pose(R, -(R @ np.array(e)))


def _rodrigues(axis, angle: float) -> np.ndarray:
    """Rotation by ``angle`` (radians) about the unit ``axis``."""
    kx, ky, kz = (float(v) for v in axis)
    c, s = math.cos(angle), math.sin(angle)
    v = 1.0 - c
    return np.array([[c + kx * kx * v, kx * ky * v - kz * s, kx * kz * v + ky * s],
                     [ky * kx * v + kz * s, c + ky * ky * v, ky * kz * v - kx * s],
                     [kz * kx * v - ky * s, kz * ky * v + kx * s, c + kz * kz * v]])


def perturb_pose(pose: Pose, trans_m: float, rot_deg: float, seed: int) -> Pose:
    """Pose offset by a rotation of ``rot_deg`` about a random axis and a
    translation of ``trans_m`` in a random direction, both applied on the
    camera side (left): R' = dR R, t' = dR t + dt."""
    rng = np.random.default_rng(seed)
    axis = _random_unit(rng, 1)[0]
    dR = _rodrigues(axis, math.radians(rot_deg))
    dt = _random_unit(rng, 1)[0] * trans_m
    return Pose(dR @ pose.R, dR @ pose.t + dt)


# --------------------------------------------------------------------------
# workload 1: random slab in front of the camera
# --------------------------------------------------------------------------
def perturb_uniform(pose: Pose, max_trans_m: float, max_rot_deg: float, seed: int) -> Pose:
    """perturb_pose with magnitudes drawn uniformly in [0, max]."""
    rng = np.random.default_rng(seed)
    return perturb_pose(pose, rng.uniform(0.0, max_trans_m), rng.uniform(0.0, max_rot_deg),
                        seed=seed + 7_000_000)


def slab_scene(seed: int = 0, n: int = 4096) -> Surfels:
    """Centres uniform in [-1,1]^2 x [1,3] m (camera frame = world frame),
    log-uniform scales in [1,5] cm, uniform random rotations,
    sigmoid(N(0,1)) opacity and uniform [0,1] colour."""
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                   rng.uniform(1, 3, n)], axis=1)
    scale = np.exp(rng.uniform(math.log(0.01), math.log(0.05), size=(n, 2)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(size=n)))
    rgb = rng.uniform(0, 1, size=(n, 3))
    return Surfels(mu, q, scale, opacity, rgb)


def slab_camera() -> Camera:
    return Camera(150.0, 150.0, 80.0, 60.0, 160, 120)


# --------------------------------------------------------------------------
# room scenes (workloads 2-5)
# --------------------------------------------------------------------------
ROOM = (5.0, 4.0, 3.0)
CAM_ZONE = (np.array([1.6, 1.3, 1.1]), np.array([3.4, 2.7, 1.9]))


@dataclasses.dataclass
class _Patch:
    kind: str            # 'rect' or 'sphere'
    area: float
    origin: np.ndarray = None
    e1: np.ndarray = None   # rect edge vectors
    e2: np.ndarray = None
    normal: np.ndarray = None  # into the material
    centre: np.ndarray = None
    radius: float = 0.0
    albedo: np.ndarray = None


def _box_faces(lo, hi, inward: bool, skip_bottom: bool):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    d = hi - lo
    faces = []
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for side in (0, 1):
            if skip_bottom and ax == 2 and side == 0:
                continue
            origin = lo.copy()
            origin[ax] = hi[ax] if side else lo[ax]
            e1 = np.zeros(3)
            e1[o1] = d[o1]
            e2 = np.zeros(3)
            e2[o2] = d[o2]
            outward = np.zeros(3)
            outward[ax] = 1.0 if side else -1.0
            faces.append((origin, e1, e2, outward if not inward else -outward))
    return faces


def _room_patches(rng: np.random.Generator, n_objects: int = 20):
    patches = []
    # walls: the material lies outside the room, so the normal points outward
    for origin, e1, e2, nrm in _box_faces((0, 0, 0), ROOM, inward=False, skip_bottom=False):
        patches.append(_Patch('rect', float(np.linalg.norm(np.cross(e1, e2))), origin, e1, e2, nrm,
                              albedo=rng.uniform(0, 1, 3)))
    lo_c, hi_c = CAM_ZONE
    placed = 0
    while placed < n_objects:
        if rng.uniform() < 0.5:
            size = rng.uniform(0.2, 1.0, 3)
            pos = np.array([rng.uniform(0, ROOM[0] - size[0]), rng.uniform(0, ROOM[1] - size[1]), 0.0])
            if rng.uniform() < 0.3:
                pos[2] = rng.uniform(0.0, ROOM[2] - size[2])
            lo, hi = pos, pos + size
            if np.all(hi > lo_c - 0.3) and np.all(lo < hi_c + 0.3):
                continue
            # the material is inside the box: normal points into the box
            for origin, e1, e2, nrm in _box_faces(lo, hi, inward=True, skip_bottom=pos[2] == 0.0):
                patches.append(_Patch('rect', float(np.linalg.norm(np.cross(e1, e2))), origin, e1, e2,
                                      nrm, albedo=rng.uniform(0, 1, 3)))
        else:
            r = rng.uniform(0.1, 0.5)
            c = np.array([rng.uniform(r, ROOM[0] - r), rng.uniform(r, ROOM[1] - r),
                          r if rng.uniform() < 0.6 else rng.uniform(r, ROOM[2] - r)])
            if np.all(c + r > lo_c - 0.3) and np.all(c - r < hi_c + 0.3):
                continue
            patches.append(_Patch('sphere', 4 * math.pi * r * r, centre=c, radius=r,
                                  albedo=rng.uniform(0, 1, 3)))
        placed += 1
    return patches


def room_scene(seed: int = 0, n: int = 200_000, scale_cm=(1.0, 3.0), opacity: float = 0.9,
               albedo_noise: float = 0.03) -> Surfels:
    """Surfels on a 5x4x3 m room (six walls) plus 20 random boxes and
    spheres, sampled uniformly by area, tangent to the surfaces with t_n
    pointing into the material (away from a viewer in free space)."""
    rng = np.random.default_rng(seed)
    patches = _room_patches(rng)
    areas = np.array([p.area for p in patches])
    counts = rng.multinomial(n, areas / areas.sum())
    mus, nrms, cols = [], [], []
    for p, k in zip(patches, counts):
        if k == 0:
            continue
        if p.kind == 'rect':
            a = rng.uniform(0, 1, (k, 1))
            b = rng.uniform(0, 1, (k, 1))
            mus.append(p.origin + a * p.e1 + b * p.e2)
            nrms.append(np.broadcast_to(p.normal, (k, 3)))
        else:
            d = _random_unit(rng, k)
            mus.append(p.centre + p.radius * d)
            nrms.append(-d)
        cols.append(np.clip(p.albedo + rng.normal(0, albedo_noise, (k, 3)), 0.0, 1.0))
    mu = np.concatenate(mus)
    t_n = np.concatenate(nrms).astype(float)
    rgb = np.concatenate(cols)
    # random tangent t_u orthogonal to t_n, t_v completes a right-handed frame
    r = rng.normal(size=(n, 3))
    t_u = r - np.sum(r * t_n, axis=1, keepdims=True) * t_n
    t_u /= np.linalg.norm(t_u, axis=1, keepdims=True)
    t_v = np.cross(t_n, t_u)
    Rm = np.stack([t_u, t_v, t_n], axis=2)
    quat = _quat_wxyz_from_matrix(Rm)
    scale = rng.uniform(scale_cm[0] / 100.0, scale_cm[1] / 100.0, size=(n, 2))
    op = np.full(n, opacity)
    perm = rng.permutation(n)          # surfel ids carry no spatial order
    return Surfels(mu[perm], quat[perm], scale[perm], op[perm], rgb[perm])


def room_pose(seed: int) -> Pose:
    """A camera inside the free central zone looking at a random point on a wall."""
    rng = np.random.default_rng(seed)
    lo, hi = CAM_ZONE
    eye = rng.uniform(lo, hi)
    wall = rng.integers(0, 4)
    tgt = np.array([rng.uniform(0.5, ROOM[0] - 0.5), rng.uniform(0.5, ROOM[1] - 0.5),
                    rng.uniform(0.6, ROOM[2] - 0.6)])
    tgt[wall // 2] = 0.0 if wall % 2 == 0 else ROOM[wall // 2]
    return look_at(eye, tgt)


def room_trajectory(seed: int, n_views: int):
    """Keyframe poses on a smooth path: each coordinate is a sum of three
    sinusoids inside the free zone; the look-at point sweeps along the walls."""
    rng = np.random.default_rng(seed)
    lo, hi = CAM_ZONE
    s = np.linspace(0.0, 1.0, n_views)
    centre = (lo + hi) / 2
    half = (hi - lo) / 2
    eyes = np.zeros((n_views, 3))
    for ax in range(3):
        amp = rng.uniform(0.1, 0.33, 3)
        freq = rng.uniform(0.5, 2.0, 3)
        ph = rng.uniform(0, 2 * math.pi, 3)
        eyes[:, ax] = centre[ax] + half[ax] * np.sum(
            amp[None] * np.sin(2 * math.pi * freq[None] * s[:, None] + ph[None]), axis=1)
    ang0 = rng.uniform(0, 2 * math.pi)
    poses = []
    for i in range(n_views):
        ang = ang0 + 1.2 * math.pi * s[i]
        d = np.array([math.cos(ang), math.sin(ang), rng.uniform(-0.15, 0.15)])
        poses.append(look_at(eyes[i], eyes[i] + d))
    return poses


def tracking_camera() -> Camera:
    return Camera(525.0, 525.0, 320.0, 240.0, 640, 480)


def mapping_camera() -> Camera:
    return Camera(600.0, 600.0, 600.0, 340.0, 1200, 680)


def uneven_cameras(seed: int, n_views: int):
    """Resolutions drawn from {320x240, 640x480, 1200x680}; the focal length
    keeps a ~62 degree horizontal field of view."""
    rng = np.random.default_rng(seed)
    opts = [(320, 240, 262.5), (640, 480, 525.0), (1200, 680, 600.0)]
    cams = []
    for k in rng.integers(0, 3, n_views):
        w, h, f = opts[int(k)]
        cams.append(Camera(f, f, w / 2, h / 2, w, h))
    return cams


def active_subset(s: Surfels, pose: Pose, size: int, reach: float = 1.5) -> np.ndarray:
    """An active-map subset for one view: the ``size`` surfels nearest to a
    point ``reach`` metres ahead of the camera along its optical axis (a ball
    around the viewed region, grown until it holds ``size`` surfels), as
    sorted int32 ids."""
    eye = -pose.R.T @ pose.t
    ahead = eye + reach * pose.R[2]
    d2 = np.sum((s.mu - ahead) ** 2, axis=1)
    size = min(int(size), s.n)
    ids = np.argpartition(d2, size - 1)[:size] if size < s.n else np.arange(s.n)
    return np.sort(ids).astype(np.int32)


def uneven_batch(seed: int, s: Surfels, n_views: int = 32, sizes=(50_000, 1_000_000)):
    """Views of one room for the uneven batch: resolution drawn from
    {320x240, 640x480, 1200x680}, a pose from the room's camera zone, and an
    active subset whose size is log-uniform in ``sizes``."""
    rng = np.random.default_rng(seed)
    cams = uneven_cameras(seed, n_views)
    poses = [room_pose(10_000 + 97 * seed + v) for v in range(n_views)]
    lo, hi = np.log(sizes[0]), np.log(sizes[1])
    actives = [active_subset(s, p, int(np.exp(rng.uniform(lo, hi)))) for p in poses]
    return cams, poses, actives


def net_init(seed: int, blocks) -> np.ndarray:
    """Seeded initial parameters of a network as one flat float32 vector:
    ``blocks`` is a list of (count, fan_in); a block with fan_in > 0 is drawn
    from N(0, 2 / fan_in) (He initialisation), one with fan_in == 0 is zero."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, math.sqrt(2.0 / f), int(c)) if f > 0 else np.zeros(int(c))
             for c, f in blocks]
    return np.concatenate(parts).astype(np.float32)


# --------------------------------------------------------------------------
# generic random tensors for kernel-level tests
# --------------------------------------------------------------------------
def random_images(seed: int, h: int, w: int, depth_range=(0.5, 4.0)):
    rng = np.random.default_rng(seed)
    rgb = rng.uniform(0, 1, (h, w, 3))
    depth = rng.uniform(*depth_range, (h, w))
    return rgb, depth


def random_upstream(seed: int, h: int, w: int, scale: float = 1.0):
    """Random per-pixel gradients of a scalar loss w.r.t. the rendered
    colour (h,w,3), depth (h,w), normal (h,w,3) and opacity (h,w)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(0, scale, (h, w, 3)), rng.normal(0, scale, (h, w)),
            rng.normal(0, scale, (h, w, 3)), rng.normal(0, scale, (h, w)))


def random_tile_records(seed: int, n: int, tiles_x: int, tiles_y: int, cull_frac: float = 0.2,
                        max_extent: int = 4, tie_frac: float = 0.1):
    """Synthetic per-surfel tile rectangles (tx0,ty0,tx1,ty1) and positive
    FP32 centre depths for exercising binning and sorting on its own.
    A fraction is culled (empty rectangle, encoded tx0 > tx1) and a fraction
    share an exact depth with another surfel so that ties occur."""
    rng = np.random.default_rng(seed)
    tx0 = rng.integers(0, tiles_x, n)
    ty0 = rng.integers(0, tiles_y, n)
    tx1 = np.minimum(tx0 + rng.integers(0, max_extent, n), tiles_x - 1)
    ty1 = np.minimum(ty0 + rng.integers(0, max_extent, n), tiles_y - 1)
    culled = rng.uniform(size=n) < cull_frac
    rect = np.stack([tx0, ty0, tx1, ty1], axis=1).astype(np.int32)
    rect[culled] = np.array([1, 1, 0, 0], np.int32)
    depth = rng.uniform(0.1, 10.0, n).astype(np.float32)
    ties = rng.uniform(size=n) < tie_frac
    depth[ties] = depth[rng.integers(0, n, int(ties.sum()))]
    count = np.where(culled, 0, (rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1))
    return rect, depth, count.astype(np.int32)


def pixel_sample(seed: int, h: int, w: int, n: int):
    """``n`` distinct pixel coordinates (x, y) drawn uniformly."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(h * w, size=min(n, h * w), replace=False)
    return np.stack([idx % w, idx // w], axis=1).astype(np.int32)


def rgbd_frame(seed: int, cam: Camera, noise_m: float = 0.001, hole_frac: float = 0.03,
               pose: Pose | None = None):
    """A synthetic observed RGB-D frame of a box room seen from inside --
    back wall z = 3.2, side walls x = +-2.1, floor y = 1.3, ceiling y = -1.4
    (y down), front wall z = -2.0 -- with a sphere of radius 0.45 m at
    (0.3, 0.25, 2.0), all in world coordinates, seen from the world-to-camera
    ``pose`` (identity: the camera at the origin looking along +z).  Depth is
    the camera-frame z of the first hit, with Gaussian noise and holes (depth
    0) at a random fraction of the pixels; colour a smooth random pattern
    over the image plus noise, in [0, 1].  Returns (rgb (H, W, 3), depth
    (H, W)) float32."""
    rng = np.random.default_rng(seed)
    R = np.eye(3) if pose is None else np.asarray(pose.R, np.float64)
    tt = np.zeros(3) if pose is None else np.asarray(pose.t, np.float64)
    c0 = -R.T @ tt
    x = (np.arange(cam.width) + 0.5 - cam.cx) / cam.fx
    y = (np.arange(cam.height) + 0.5 - cam.cy) / cam.fy
    rx, ry = np.meshgrid(x, y)
    r = np.stack([rx, ry, np.ones_like(rx)], -1) @ R      # world direction, camera z = 1
    d = np.full(rx.shape, np.inf)
    for n, c in (((0, 0, 1), 3.2), ((0, 0, -1), 2.0), ((1, 0, 0), 2.1), ((-1, 0, 0), 2.1),
                 ((0, 1, 0), 1.3), ((0, -1, 0), 1.4)):
        n = np.array(n, float)
        nr = r @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(nr > 1e-9, (c - n @ c0) / nr, np.inf)
        d = np.minimum(d, np.where(t > 0, t, np.inf))
    C, rho = np.array([0.3, 0.25, 2.0]) - c0, 0.45
    a = (r * r).sum(-1)
    b = -2 * (r @ C)
    q = C @ C - rho * rho
    disc = b * b - 4 * a * q
    with np.errstate(invalid="ignore"):
        t = np.where(disc >= 0, (-b - np.sqrt(np.maximum(disc, 0))) / (2 * a), np.inf)
    d = np.minimum(d, np.where(t > 0, t, np.inf))
    d = np.where(np.isfinite(d), d, 0.0)
    d = d + rng.normal(0, noise_m, d.shape) * (d > 0)
    d[rng.uniform(size=d.shape) < hole_frac] = 0.0
    f = rng.uniform(0.05, 0.3, 3)
    ph = rng.uniform(0, 2 * np.pi, 3)
    u, v = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    rgb = 0.5 + 0.35 * np.sin(f[None, None, :] * u[..., None] + ph) * np.cos(
        0.7 * f[None, None, :] * v[..., None])
    rgb = np.clip(rgb + rng.normal(0, 0.03, rgb.shape), 0, 1)
    return rgb.astype(np.float32), d.astype(np.float32)

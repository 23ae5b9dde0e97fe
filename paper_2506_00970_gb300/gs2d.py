"""Thin Python binding of the gs2d C ABI (include/gs2d.h).

Functions named like the C entry points marshal torch CUDA tensors into
device pointers and call the library; every step of the rasterizer runs in
the library's CUDA kernels.  PyTorch only provides device memory and streams.
There is no CPU fallback: importing the binding without the built library
(``python -c "import __graft_entry__ as g; g.build()"``) raises.

``Rasterizer`` bundles the buffers of one camera for convenience (tests,
benchmark); it sizes the intersection capacity from the device count, which
costs a host synchronisation only when the capacity has to grow.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

_LIB = None

PROJ_FLOATS = 32
CONVERGED = 256
STATUS = {0: "ok", 1: "invalid argument", 2: "workspace", 3: "capacity", 4: "cuda",
          5: "timeout", 6: "non-finite", 256: "converged"}


class Gs2dError(RuntimeError):
    pass


class Camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("near_z", ctypes.c_float)]


class Surfels(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("scale", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("rgb", ctypes.c_void_p), ("n", ctypes.c_int)]


class Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("px_per_thread", ctypes.c_int),
                ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("cutoff_r2", ctypes.c_float)]


class Bins(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("isect_emit", ctypes.c_void_p), ("surfel_off", ctypes.c_void_p),
                ("tile_ranges", ctypes.c_void_p), ("n_isect", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("capacity", ctypes.c_size_t)]


class TrackParams(ctypes.Structure):
    _fields_ = [("lambda_d", ctypes.c_float), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("weight_decay", ctypes.c_float), ("stop_tol", ctypes.c_float),
                ("opacity_thresh", ctypes.c_float), ("depth_mode", ctypes.c_int)]


class View(ctypes.Structure):
    _fields_ = [("cam", Camera), ("cfg", Config), ("pose", ctypes.c_void_p),
                ("active", ctypes.c_void_p), ("n_active", ctypes.c_int),
                ("proj", ctypes.c_void_p), ("tiles_per_surfel", ctypes.c_void_p), ("bins", Bins),
                ("rgb", ctypes.c_void_p), ("depth", ctypes.c_void_p), ("normal", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("t_final", ctypes.c_void_p),
                ("n_last", ctypes.c_void_p), ("d_rgb", ctypes.c_void_p),
                ("d_depth", ctypes.c_void_p), ("d_normal", ctypes.c_void_p),
                ("d_opacity", ctypes.c_void_p), ("d_pose6", ctypes.c_void_p)]


class LossView(ctypes.Structure):
    _fields_ = [("cam", Camera), ("rgb", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("normal", ctypes.c_void_p), ("opacity", ctypes.c_void_p),
                ("obs_rgb", ctypes.c_void_p), ("obs_depth", ctypes.c_void_p),
                ("g_rgb", ctypes.c_void_p), ("g_depth", ctypes.c_void_p),
                ("g_normal", ctypes.c_void_p), ("g_opacity", ctypes.c_void_p)]


class MapState(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_void_p), ("t_c", ctypes.c_void_p), ("d_c", ctypes.c_void_p),
                ("t_l", ctypes.c_void_p)]


class StateParams(ctypes.Structure):
    _fields_ = [("vis_threshold", ctypes.c_float), ("inactive_after", ctypes.c_int),
                ("reactivate", ctypes.c_int), ("loop_h", ctypes.c_int)]


class VoxelTable(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("capacity", ctypes.c_uint32), ("voxel", ctypes.c_float),
                ("status", ctypes.c_void_p)]


class ExpandParams(ctypes.Structure):
    _fields_ = [("ratio", ctypes.c_float), ("opacity", ctypes.c_float),
                ("max_scale", ctypes.c_float), ("kf_id", ctypes.c_int),
                ("insert_new", ctypes.c_int)]


MAX_VIEWS = 32

EXPORTS = ["gs2d_default_config", "gs2d_default_track_params", "gs2d_status_string",
           "gs2d_tiles_x", "gs2d_tiles_y", "gs2d_project", "gs2d_bin_sort_workspace",
           "gs2d_bin_sort", "gs2d_render_fwd", "gs2d_render_bwd_workspace", "gs2d_render_bwd",
           "gs2d_tracking_loss", "gs2d_mapping_loss", "gs2d_track_workspace", "gs2d_track_step",
           "gs2d_track_status", "gs2d_track_tile_order", "gs2d_render_count", "gs2d_bin_sort_static",
           "gs2d_set_grouped_tiles", "gs2d_set_lookback_wait",
           "gs2d_profile_track_kernel", "gs2d_profile_track_kernel_count",
           "gs2d_profile_track_kernel_every",
           "gs2d_project_batch", "gs2d_bin_sort_batch_workspace", "gs2d_bin_sort_batch",
           "gs2d_render_batch_workspace", "gs2d_render_fwd_batch", "gs2d_render_bwd_batch",
           "gs2d_net_param_count", "gs2d_net_layout", "gs2d_net_workspace",
           "gs2d_net_pack_input", "gs2d_net_forward", "gs2d_net_grad", "gs2d_net_adamw",
           "gs2d_net_apply", "gs2d_net_target", "gs2d_net_accept", "gs2d_net_accept_keep",
           "gs2d_render_contrib_workspace", "gs2d_render_contrib", "gs2d_covisibility",
           "gs2d_map_observe", "gs2d_map_correct_workspace", "gs2d_map_correct",
           "gs2d_map_prune", "gs2d_map_compact_workspace", "gs2d_map_compact",
           "gs2d_mapping_loss_ssim_workspace", "gs2d_mapping_loss_ssim", "gs2d_ssim_workspace",
           "gs2d_ssim_loss", "gs2d_voxel_clear", "gs2d_voxel_insert", "gs2d_voxel_query",
           "gs2d_expand_workspace", "gs2d_expand", "gs2d_map_expand_values",
           "gs2d_net_downsample_rgbd", "gs2d_net_prepare", "gs2d_net_forward_prepared",
           "gs2d_mapping_loss_batch_workspace", "gs2d_mapping_loss_batch"]

NET_LAYERS = 8
NET_IN = (120, 160, 8)
NET_OUT = 6
NET_TAU_SCALE = 0.03


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise Gs2dError(f"gs2d CUDA library not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, sz, ip = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        L.gs2d_default_config.restype = Config
        L.gs2d_default_track_params.restype = TrackParams
        L.gs2d_status_string.restype = ctypes.c_char_p
        L.gs2d_status_string.argtypes = [ip]
        L.gs2d_tiles_x.argtypes = [vp, vp]
        L.gs2d_tiles_y.argtypes = [vp, vp]
        L.gs2d_project.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.gs2d_bin_sort_workspace.restype = sz
        L.gs2d_bin_sort_workspace.argtypes = [ip, sz]
        L.gs2d_bin_sort.argtypes = [vp, vp, ip, vp, vp, vp, sz, vp, vp, vp]
        L.gs2d_bin_sort_static.argtypes = [vp, vp, ip, vp, vp, vp, vp]
        L.gs2d_render_fwd.argtypes = [vp] * 11
        L.gs2d_render_count.argtypes = [vp] * 6
        L.gs2d_set_grouped_tiles.argtypes = [ip]
        L.gs2d_set_grouped_tiles.restype = None
        L.gs2d_set_lookback_wait.argtypes = [ip, ip]
        L.gs2d_set_lookback_wait.restype = None
        L.gs2d_render_bwd_workspace.restype = sz
        L.gs2d_render_bwd_workspace.argtypes = [ip, sz, ip]
        L.gs2d_render_bwd.argtypes = [vp] * 20 + [sz, vp, vp]
        L.gs2d_tracking_loss.argtypes = [vp] * 13 + [sz, vp, vp]
        L.gs2d_mapping_loss.argtypes = [vp] * 7 + [ctypes.c_float, ctypes.c_float] + [vp] * 6 + [sz, vp, vp]
        L.gs2d_track_workspace.restype = sz
        L.gs2d_track_workspace.argtypes = [ip, sz, vp, vp]
        L.gs2d_track_step.argtypes = [vp] * 8 + [ip, sz, vp, vp, vp, vp, sz, vp, vp]
        L.gs2d_profile_track_kernel.argtypes = [vp, vp, ip]
        L.gs2d_profile_track_kernel_count.restype = ip
        L.gs2d_profile_track_kernel_every.argtypes = [ip]
        L.gs2d_project_batch.argtypes = [vp, vp, ip, vp]
        L.gs2d_bin_sort_batch_workspace.restype = sz
        L.gs2d_bin_sort_batch_workspace.argtypes = [vp, ip, ip]
        L.gs2d_bin_sort_batch.argtypes = [vp, ip, ip, vp, sz, vp, vp]
        L.gs2d_render_batch_workspace.restype = sz
        L.gs2d_render_batch_workspace.argtypes = [vp, ip, ip]
        L.gs2d_render_fwd_batch.argtypes = [vp, ip, vp, sz, vp, vp]
        L.gs2d_render_bwd_batch.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp, vp, sz, vp, vp]
        L.gs2d_track_status.restype = vp
        L.gs2d_track_status.argtypes = [vp]
        L.gs2d_track_tile_order.restype = vp
        L.gs2d_track_tile_order.argtypes = [vp, ip, sz, vp, vp]
        fl = ctypes.c_float
        L.gs2d_net_param_count.restype = sz
        L.gs2d_net_layout.argtypes = [vp, vp, vp]
        L.gs2d_net_workspace.restype = sz
        L.gs2d_net_workspace.argtypes = [ip]
        L.gs2d_net_pack_input.argtypes = [vp] * 5 + [ip, ip, ip, vp, vp]
        L.gs2d_net_forward.argtypes = [vp, vp, ip, vp, vp, sz, vp, vp]
        L.gs2d_net_grad.argtypes = [vp, vp, vp, ip, vp, vp, vp, vp, sz, vp, vp]
        L.gs2d_net_adamw.argtypes = [vp, vp, vp, vp, sz, ip, fl, fl, fl, fl, fl, vp]
        L.gs2d_net_apply.argtypes = [vp, ip, vp, vp]
        L.gs2d_net_target.argtypes = [vp, vp, ip, vp, vp]
        L.gs2d_net_accept.argtypes = [vp, vp, vp, ip, vp, vp, vp]
        L.gs2d_net_accept_keep.argtypes = [vp, vp, vp, ip, vp, vp, sz] + [vp] * 7
        L.gs2d_net_downsample_rgbd.argtypes = [vp, vp, ip, ip, ip, vp, vp, vp]
        L.gs2d_net_prepare.argtypes = [vp, ip, vp, sz, vp, vp]
        L.gs2d_net_forward_prepared.argtypes = [vp, vp, ip, vp, vp, sz, vp, vp]
        L.gs2d_render_contrib_workspace.restype = sz
        L.gs2d_render_contrib_workspace.argtypes = [sz]
        L.gs2d_render_contrib.argtypes = [vp, vp, vp, ip, vp, vp, vp, vp, sz, vp, vp]
        L.gs2d_covisibility.argtypes = [vp, vp, ip, fl, vp, vp, fl, fl, vp, vp, vp, vp]
        L.gs2d_map_observe.argtypes = [vp, vp, ip, vp, ip, vp, vp, vp, vp]
        L.gs2d_map_correct_workspace.restype = sz
        L.gs2d_map_correct_workspace.argtypes = [ip]
        L.gs2d_map_correct.argtypes = [vp, vp, vp, ip, vp, vp, ip, vp, sz, vp, vp, vp]
        L.gs2d_map_prune.argtypes = [vp, vp, ip, ip, fl, vp, vp]
        L.gs2d_mapping_loss_batch_workspace.restype = sz
        L.gs2d_mapping_loss_batch_workspace.argtypes = [vp, ip]
        L.gs2d_mapping_loss_batch.argtypes = [vp, ip, fl, fl, vp, vp, sz, vp, vp]
        L.gs2d_mapping_loss_ssim_workspace.restype = sz
        L.gs2d_mapping_loss_ssim_workspace.argtypes = [vp]
        L.gs2d_mapping_loss_ssim.argtypes = [vp] * 7 + [fl, fl, fl] + [vp] * 6 + [sz, vp, vp]
        L.gs2d_ssim_workspace.restype = sz
        L.gs2d_ssim_workspace.argtypes = [ip, ip]
        L.gs2d_ssim_loss.argtypes = [vp, vp, ip, ip, fl, vp, vp, vp, sz, vp, vp]
        L.gs2d_voxel_clear.argtypes = [vp, vp]
        L.gs2d_map_expand_values.argtypes = [vp, vp, ip, fl, vp, vp]
        L.gs2d_voxel_insert.argtypes = [vp, vp, vp, ip, vp]
        L.gs2d_voxel_query.argtypes = [vp, vp, ip, vp, vp]
        L.gs2d_expand_workspace.restype = sz
        L.gs2d_expand_workspace.argtypes = [vp]
        L.gs2d_expand.argtypes = [vp] * 8 + [ip, ip] + [vp] * 7 + [vp, sz, vp, vp]
        L.gs2d_map_compact_workspace.restype = sz
        L.gs2d_map_compact_workspace.argtypes = [ip]
        L.gs2d_map_compact.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp,
                                       vp]
        _LIB = L
    return _LIB


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ref(s):
    return ctypes.byref(s)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def check(rc: int, what: str):
    if rc != 0:
        raise Gs2dError(f"{what}: {lib().gs2d_status_string(rc).decode()} ({rc})")


def camera(cam) -> Camera:
    return Camera(cam.fx, cam.fy, cam.cx, cam.cy, int(cam.width), int(cam.height), cam.near)


def default_config(tile=(16, 16), px: int = 1) -> Config:
    """The library's default compositing constants with a tile shape and a
    pixels-per-thread count (tile_w * tile_h = 256 px)."""
    c = lib().gs2d_default_config()
    c.tile_w, c.tile_h = int(tile[0]), int(tile[1])
    c.px_per_thread = int(px)
    return c


# tile shapes of each pixels-per-thread count (256 P pixels, widths a
# multiple of 8, heights of 4P)
TILE_SHAPES = {1: ((16, 16), (8, 32), (32, 8)), 2: ((16, 32), (32, 16)),
               3: ((32, 24), (64, 12), (16, 48)), 4: ((32, 32), (16, 64))}


def default_track_params(**kw) -> TrackParams:
    p = lib().gs2d_default_track_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# device-side containers
# ---------------------------------------------------------------------------
class DeviceSurfels:
    """Surfel parameters as contiguous float32 CUDA tensors (SoA)."""

    def __init__(self, surfels, device="cuda"):
        def t(a, cols):
            x = torch.as_tensor(np.asarray(a, np.float32), device=device)
            return x.reshape(-1, cols).contiguous() if cols > 1 else x.reshape(-1).contiguous()
        self.mu = t(surfels.mu, 3)
        self.quat = t(surfels.quat, 4)
        self.scale = t(surfels.scale, 2)
        self.opacity = t(surfels.opacity, 1)
        self.rgb = t(surfels.rgb, 3)

    @classmethod
    def from_tensors(cls, mu, quat, scale, opacity, rgb):
        o = cls.__new__(cls)
        o.mu, o.quat, o.scale, o.opacity, o.rgb = (x.contiguous() for x in (mu, quat, scale, opacity, rgb))
        return o

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    def struct(self) -> Surfels:
        return Surfels(self.mu.data_ptr(), self.quat.data_ptr(), self.scale.data_ptr(),
                       self.opacity.data_ptr(), self.rgb.data_ptr(), self.n)


def pose_tensor(pose, device="cuda") -> torch.Tensor:
    v = np.concatenate([np.asarray(pose.R, np.float64).reshape(-1), np.asarray(pose.t, np.float64)])
    return torch.tensor(v, dtype=torch.float32, device=device)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def gs2d_project(surf: DeviceSurfels, cam: Camera, pose: torch.Tensor, cfg: Config,
                 proj: torch.Tensor, tiles: torch.Tensor, stream=None):
    s = surf.struct()
    check(lib().gs2d_project(_ref(s), _ref(cam), _ptr(pose), _ref(cfg), _ptr(proj), _ptr(tiles),
                             _stream(stream)), "gs2d_project")


def gs2d_bin_sort_workspace(n: int, capacity: int) -> int:
    return int(lib().gs2d_bin_sort_workspace(int(n), int(capacity)))


def gs2d_bin_sort(proj, tiles, n, cam: Camera, cfg: Config, workspace: torch.Tensor, bins: Bins,
                  stream=None):
    check(lib().gs2d_bin_sort(_ptr(proj), _ptr(tiles), int(n), _ref(cam), _ref(cfg),
                              _ptr(workspace), workspace.numel() * workspace.element_size(), None,
                              _ref(bins), _stream(stream)), "gs2d_bin_sort")


def gs2d_bin_sort_static(proj, tiles, n, cam: Camera, cfg: Config, bins: Bins, stream=None):
    """gs2d_bin_sort with the library's own fixed device scratch (no
    workspace argument, no allocation)."""
    check(lib().gs2d_bin_sort_static(_ptr(proj), _ptr(tiles), int(n), _ref(cam), _ref(cfg),
                                     _ref(bins), _stream(stream)), "gs2d_bin_sort_static")


def gs2d_render_fwd(proj, bins: Bins, cam: Camera, cfg: Config, rgb, depth, normal, opacity,
                    t_final, n_last, stream=None):
    check(lib().gs2d_render_fwd(_ptr(proj), _ref(bins), _ref(cam), _ref(cfg), _ptr(rgb),
                                _ptr(depth), _ptr(normal), _ptr(opacity), _ptr(t_final),
                                _ptr(n_last), _stream(stream)), "gs2d_render_fwd")


def gs2d_render_count(proj, bins: Bins, cam: Camera, cfg: Config, counts, stream=None):
    """counts: device int64 [5] (see gs2d.h)."""
    if counts.numel() < 5 or counts.element_size() != 8:
        raise Gs2dError("gs2d_render_count needs a 5-element 64-bit counts buffer")
    check(lib().gs2d_render_count(_ptr(proj), _ref(bins), _ref(cam), _ref(cfg), _ptr(counts),
                                  _stream(stream)), "gs2d_render_count")


def gs2d_set_grouped_tiles(max_tiles: int):
    """Tile grids of at most max_tiles tiles run the grouped one-pixel
    compositing loops (-1: twice the SM count, the default; 0: never)."""
    lib().gs2d_set_grouped_tiles(int(max_tiles))


def gs2d_set_lookback_wait(spin_limit: int = 0, withheld_chunk: int = -1):
    """Polls of a binning scan block's look-back wait before it records
    GS2D_ERR_TIMEOUT (0: the default), and the scan block (4096 surfels) that
    never publishes its sum (-1: none) -- for tests of the timeout path."""
    lib().gs2d_set_lookback_wait(int(spin_limit), int(withheld_chunk))


def gs2d_render_contrib_workspace(capacity) -> int:
    return int(lib().gs2d_render_contrib_workspace(int(capacity)))


def gs2d_render_contrib(proj, bins: Bins, tiles, n, cam: Camera, cfg: Config, contrib, workspace,
                        stream=None):
    check(lib().gs2d_render_contrib(_ptr(proj), _ref(bins), _ptr(tiles), int(n), _ref(cam),
                                    _ref(cfg), _ptr(contrib), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), None,
                                    _stream(stream)), "gs2d_render_contrib")


def gs2d_covisibility(contrib_a, contrib_b, n, vis_threshold, pose_a, pose_b, c_k, d_k, counts,
                      score=None, is_keyframe=None, stream=None):
    check(lib().gs2d_covisibility(_ptr(contrib_a), _ptr(contrib_b), int(n), float(vis_threshold),
                                  _ptr(pose_a), _ptr(pose_b), float(c_k), float(d_k),
                                  _ptr(counts), _ptr(score), _ptr(is_keyframe), _stream(stream)),
          "gs2d_covisibility")


class DeviceMapState:
    """Per-surfel state of Eq. map (Sec. III-C) as CUDA tensors: delta
    (uint8, 1 = active), t_c (int32), d_c (float32), t_l (int32)."""

    def __init__(self, n, kf_id=0, d_c=float("inf"), device="cuda", active=True):
        self.delta = torch.full((n,), 1 if active else 0, dtype=torch.uint8, device=device)
        self.t_c = torch.full((n,), int(kf_id), dtype=torch.int32, device=device)
        self.d_c = torch.full((n,), float(d_c), dtype=torch.float32, device=device)
        self.t_l = torch.full((n,), int(kf_id), dtype=torch.int32, device=device)

    @classmethod
    def from_tensors(cls, delta, t_c, d_c, t_l):
        o = cls.__new__(cls)
        o.delta, o.t_c, o.d_c, o.t_l = (x.contiguous() for x in (delta, t_c, d_c, t_l))
        return o

    def struct(self) -> MapState:
        return MapState(self.delta.data_ptr(), self.t_c.data_ptr(), self.d_c.data_ptr(),
                        self.t_l.data_ptr())


def gs2d_map_observe(contrib, mu, n, pose_cw, kf_id, prm: StateParams, st: DeviceMapState,
                     counts=None, stream=None):
    ms = st.struct()
    check(lib().gs2d_map_observe(_ptr(contrib), _ptr(mu), int(n), _ptr(pose_cw), int(kf_id),
                                 _ref(prm), _ref(ms), _ptr(counts), _stream(stream)),
          "gs2d_map_observe")


def gs2d_map_correct_workspace(n_kf) -> int:
    return int(lib().gs2d_map_correct_workspace(int(n_kf)))


def gs2d_map_correct(mu, quat, t_c, n, poses_old, poses_new, n_kf, workspace, n_skipped=None,
                     stream=None):
    check(lib().gs2d_map_correct(_ptr(mu), _ptr(quat), _ptr(t_c), int(n), _ptr(poses_old),
                                 _ptr(poses_new), int(n_kf), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), None,
                                 _ptr(n_skipped), _stream(stream)), "gs2d_map_correct")


def gs2d_map_prune(contrib, t_c, n, r, vis_threshold, keep, stream=None):
    check(lib().gs2d_map_prune(_ptr(contrib), _ptr(t_c), int(n), int(r), float(vis_threshold),
                               _ptr(keep), _stream(stream)), "gs2d_map_prune")


def gs2d_map_expand_values(vals, new_index, n, fill, out, stream=None):
    check(lib().gs2d_map_expand_values(_ptr(vals), _ptr(new_index), int(n), float(fill), _ptr(out),
                                       _stream(stream)), "gs2d_map_expand_values")


def gs2d_map_compact_workspace(n) -> int:
    return int(lib().gs2d_map_compact_workspace(int(n)))


def gs2d_map_compact(keep, n, surf: "DeviceSurfels", st, out: "DeviceSurfels", st_out, new_index,
                     n_out, workspace, stream=None):
    sv = surf.struct()
    si = st.struct() if st is not None else None
    so = st_out.struct() if st_out is not None else None
    check(lib().gs2d_map_compact(_ptr(keep), int(n), _ref(sv), _ref(si) if si else None,
                                 _ptr(out.mu), _ptr(out.quat), _ptr(out.scale), _ptr(out.opacity),
                                 _ptr(out.rgb), _ref(so) if so else None, _ptr(new_index),
                                 _ptr(n_out), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), None,
                                 _stream(stream)), "gs2d_map_compact")


def gs2d_render_bwd_workspace(n, capacity, n_tiles) -> int:
    return int(lib().gs2d_render_bwd_workspace(int(n), int(capacity), int(n_tiles)))


def gs2d_render_bwd(proj, bins: Bins, tiles, surf: DeviceSurfels, pose, cam: Camera, cfg: Config,
                    t_final, n_last, d_rgb, d_depth, d_normal, d_opacity, d_mu, d_quat, d_scale,
                    d_opac, d_rgb_out, d_pose6, workspace, stream=None):
    s = surf.struct()
    check(lib().gs2d_render_bwd(_ptr(proj), _ref(bins), _ptr(tiles), _ref(s), _ptr(pose),
                                _ref(cam), _ref(cfg), _ptr(t_final), _ptr(n_last), _ptr(d_rgb),
                                _ptr(d_depth), _ptr(d_normal), _ptr(d_opacity), _ptr(d_mu),
                                _ptr(d_quat), _ptr(d_scale), _ptr(d_opac), _ptr(d_rgb_out),
                                _ptr(d_pose6), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), None,
                                _stream(stream)), "gs2d_render_bwd")


def gs2d_tracking_loss(rgb, depth, normal, opacity, obs_rgb, obs_depth, cam: Camera,
                       prm: TrackParams, g_rgb, g_depth, g_opacity, loss_out, workspace,
                       stream=None):
    check(lib().gs2d_tracking_loss(_ptr(rgb), _ptr(depth), _ptr(normal), _ptr(opacity),
                                   _ptr(obs_rgb), _ptr(obs_depth), _ref(cam), _ref(prm),
                                   _ptr(g_rgb), _ptr(g_depth), _ptr(g_opacity), _ptr(loss_out),
                                   _ptr(workspace), workspace.numel() * workspace.element_size(),
                                   None, _stream(stream)), "gs2d_tracking_loss")


def gs2d_mapping_loss(rgb, depth, normal, opacity, obs_rgb, obs_depth, cam: Camera, w_d, w_n,
                      g_rgb, g_depth, g_normal, g_opacity, loss_out, workspace, stream=None):
    check(lib().gs2d_mapping_loss(_ptr(rgb), _ptr(depth), _ptr(normal), _ptr(opacity),
                                  _ptr(obs_rgb), _ptr(obs_depth), _ref(cam), float(w_d), float(w_n),
                                  _ptr(g_rgb), _ptr(g_depth), _ptr(g_normal), _ptr(g_opacity),
                                  _ptr(loss_out), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), None,
                                  _stream(stream)), "gs2d_mapping_loss")


def loss_views(views):
    """ctypes array of LossView from (cam, rgb, depth, normal, opacity,
    obs_rgb, obs_depth, g_rgb, g_depth, g_normal, g_opacity) tuples."""
    arr = (LossView * len(views))()
    for k, v in enumerate(views):
        arr[k] = LossView(v[0], *[t.data_ptr() for t in v[1:]])
    return arr


def gs2d_mapping_loss_batch_workspace(views) -> int:
    arr = views if isinstance(views, ctypes.Array) else loss_views(views)
    return int(lib().gs2d_mapping_loss_batch_workspace(arr, len(arr)))


def gs2d_mapping_loss_batch(views, w_d, w_n, loss_out, workspace, stream=None):
    """gs2d_mapping_loss over every view in one launch; views as for
    loss_views (or its result), loss_out device [n_views]."""
    arr = views if isinstance(views, ctypes.Array) else loss_views(views)
    check(lib().gs2d_mapping_loss_batch(arr, len(arr), float(w_d), float(w_n), _ptr(loss_out),
                                        _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), None,
                                        _stream(stream)), "gs2d_mapping_loss_batch")


def gs2d_mapping_loss_ssim_workspace(cam: Camera) -> int:
    return int(lib().gs2d_mapping_loss_ssim_workspace(_ref(cam)))


def gs2d_mapping_loss_ssim(rgb, depth, normal, opacity, obs_rgb, obs_depth, cam: Camera, w_ssim,
                           w_d, w_n, g_rgb, g_depth, g_normal, g_opacity, loss_out, workspace,
                           stream=None):
    check(lib().gs2d_mapping_loss_ssim(_ptr(rgb), _ptr(depth), _ptr(normal), _ptr(opacity),
                                       _ptr(obs_rgb), _ptr(obs_depth), _ref(cam), float(w_ssim),
                                       float(w_d), float(w_n), _ptr(g_rgb), _ptr(g_depth),
                                       _ptr(g_normal), _ptr(g_opacity), _ptr(loss_out),
                                       _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), None,
                                       _stream(stream)), "gs2d_mapping_loss_ssim")


def gs2d_ssim_workspace(height, width) -> int:
    return int(lib().gs2d_ssim_workspace(int(height), int(width)))


def gs2d_ssim_loss(x, y, height, width, weight, g_x, loss, workspace, stream=None):
    check(lib().gs2d_ssim_loss(_ptr(x), _ptr(y), int(height), int(width), float(weight), _ptr(g_x),
                               _ptr(loss), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), None,
                               _stream(stream)), "gs2d_ssim_loss")


class DeviceVoxelTable:
    """Voxel hash table of occupied space (Sec. III-E) on the device."""

    def __init__(self, capacity: int, voxel: float, device="cuda"):
        cap = 1 << max(0, int(capacity - 1).bit_length())
        self.keys = torch.empty(cap, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.capacity = cap
        self.voxel = float(voxel)
        self.clear()

    def struct(self) -> VoxelTable:
        return VoxelTable(self.keys.data_ptr(), self.capacity, self.voxel, self.status.data_ptr())

    def clear(self, stream=None):
        t = self.struct()
        check(lib().gs2d_voxel_clear(_ref(t), _stream(stream)), "gs2d_voxel_clear")

    def insert(self, points, mask=None, stream=None):
        t = self.struct()
        check(lib().gs2d_voxel_insert(_ref(t), _ptr(points), _ptr(mask), int(points.shape[0]),
                                      _stream(stream)), "gs2d_voxel_insert")

    def query(self, points, out=None, stream=None):
        t = self.struct()
        m = int(points.shape[0])
        occ = out if out is not None else torch.empty(max(m, 1), dtype=torch.uint8,
                                                      device=points.device)
        check(lib().gs2d_voxel_query(_ref(t), _ptr(points), m, _ptr(occ), _stream(stream)),
              "gs2d_voxel_query")
        return occ[:m]


def gs2d_expand_workspace(cam: Camera) -> int:
    return int(lib().gs2d_expand_workspace(_ref(cam)))


def gs2d_expand(rgb, depth, cam: Camera, pose_cw, u_keep, u_angle, table, prm: ExpandParams,
                n_map, capacity, out: "DeviceSurfels", st, n_new, workspace, stream=None):
    tb = table.struct() if table is not None else None
    ms = st.struct() if st is not None else None
    check(lib().gs2d_expand(_ptr(rgb), _ptr(depth), _ref(cam), _ptr(pose_cw), _ptr(u_keep),
                            _ptr(u_angle), _ref(tb) if tb else None, _ref(prm), int(n_map),
                            int(capacity), _ptr(out.mu), _ptr(out.quat), _ptr(out.scale),
                            _ptr(out.opacity), _ptr(out.rgb), _ref(ms) if ms else None,
                            _ptr(n_new), _ptr(workspace),
                            workspace.numel() * workspace.element_size(), None, _stream(stream)),
          "gs2d_expand")


def gs2d_track_workspace(n, capacity, cam: Camera, cfg: Config) -> int:
    return int(lib().gs2d_track_workspace(int(n), int(capacity), _ref(cam), _ref(cfg)))


def gs2d_track_step(surf: DeviceSurfels, cam: Camera, cfg: Config, prm: TrackParams, pose,
                    obs_rgb, obs_depth, n_iter, capacity, loss_hist, pose_hist, workspace,
                    stream=None, adam_state=None, grad_hist=None):
    """n_iter tracking iterations (see gs2d.h).  adam_state: optional
    caller-owned device [16] AdamW state (zero it to start a frame; NULL =
    reset at every call); grad_hist: optional device [n_iter, 6] pose
    gradients."""
    s = surf.struct()
    check(lib().gs2d_track_step(_ref(s), _ref(cam), _ref(cfg), _ref(prm), _ptr(pose),
                                _ptr(adam_state), _ptr(obs_rgb), _ptr(obs_depth), int(n_iter),
                                int(capacity), _ptr(loss_hist), _ptr(pose_hist), _ptr(grad_hist),
                                _ptr(workspace), workspace.numel() * workspace.element_size(),
                                None, _stream(stream)), "gs2d_track_step")


def gs2d_profile_track_kernel(events_start, events_stop):
    """Record the given torch.cuda.Event pairs around the next launches of
    the fused tracking kernel (empty lists switch it off)."""
    n = len(events_start)
    if n == 0:
        check(lib().gs2d_profile_track_kernel(None, None, 0), "gs2d_profile_track_kernel")
        _PROFILE_KEEP.clear()
        return
    for e in list(events_start) + list(events_stop):
        e.record()   # make sure the underlying cudaEvent_t exists
    a = (ctypes.c_void_p * n)(*[e.cuda_event for e in events_start])
    b = (ctypes.c_void_p * n)(*[e.cuda_event for e in events_stop])
    _PROFILE_KEEP[:] = [a, b, list(events_start), list(events_stop)]
    check(lib().gs2d_profile_track_kernel(a, b, n), "gs2d_profile_track_kernel")


def gs2d_profile_track_kernel_count() -> int:
    return int(lib().gs2d_profile_track_kernel_count())


def gs2d_profile_track_kernel_every(every: int):
    """Bracket only the launches of iterations it % every == 0."""
    check(lib().gs2d_profile_track_kernel_every(int(every)), "gs2d_profile_track_kernel_every")


_PROFILE_KEEP = []


def gs2d_track_status(workspace) -> torch.Tensor:
    """The int32 status word of a track workspace, as a 1-element view."""
    return workspace.view(torch.int32)[:1]


def gs2d_track_tile_order(workspace, n: int, capacity: int, cam, cfg) -> torch.Tensor:
    """The tile launch order of the last tracking iteration (int32 view of
    the workspace, one entry per tile)."""
    p = lib().gs2d_track_tile_order(ctypes.c_void_p(workspace.data_ptr()), int(n), int(capacity),
                                    _ref(cam), _ref(cfg))
    if not p:
        raise Gs2dError("gs2d_track_tile_order: invalid arguments")
    off = p - workspace.data_ptr()
    nt = int(lib().gs2d_tiles_x(_ref(cam), _ref(cfg))) * int(lib().gs2d_tiles_y(_ref(cam), _ref(cfg)))
    return workspace[off:off + 4 * nt].view(torch.int32)


def gs2d_project_batch(surf: DeviceSurfels, views, stream=None):
    arr = (View * len(views))(*views)
    sv = surf.struct()
    check(lib().gs2d_project_batch(_ref(sv), arr, len(views), _stream(stream)), "gs2d_project_batch")


def gs2d_bin_sort_batch(views, n, workspace, stream=None):
    arr = (View * len(views))(*views)
    check(lib().gs2d_bin_sort_batch(arr, len(views), int(n), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), None,
                                    _stream(stream)), "gs2d_bin_sort_batch")


def gs2d_render_fwd_batch(views, workspace, stream=None):
    arr = (View * len(views))(*views)
    check(lib().gs2d_render_fwd_batch(arr, len(views), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), None,
                                      _stream(stream)), "gs2d_render_fwd_batch")


def gs2d_render_bwd_batch(views, surf: DeviceSurfels, d_mu, d_quat, d_scale, d_opac, d_rgb,
                          workspace, stream=None):
    arr = (View * len(views))(*views)
    sv = surf.struct()
    check(lib().gs2d_render_bwd_batch(arr, len(views), _ref(sv), _ptr(d_mu), _ptr(d_quat),
                                      _ptr(d_scale), _ptr(d_opac), _ptr(d_rgb), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), None,
                                      _stream(stream)), "gs2d_render_bwd_batch")


# ---------------------------------------------------------------------------
# learned pose proposal (include/gs2d_net.h)
# ---------------------------------------------------------------------------
def gs2d_net_param_count() -> int:
    return int(lib().gs2d_net_param_count())


def gs2d_net_layout():
    w = (ctypes.c_size_t * NET_LAYERS)()
    b = (ctypes.c_size_t * NET_LAYERS)()
    f = (ctypes.c_int * NET_LAYERS)()
    check(lib().gs2d_net_layout(w, b, f), "gs2d_net_layout")
    return list(w), list(b), list(f)


def gs2d_net_workspace(batch: int) -> int:
    return int(lib().gs2d_net_workspace(int(batch)))


def gs2d_net_pack_input(r_rgb, r_depth, r_opacity, o_rgb, o_depth, x, stream=None):
    B, H, W = r_depth.shape
    check(lib().gs2d_net_pack_input(_ptr(r_rgb), _ptr(r_depth), _ptr(r_opacity), _ptr(o_rgb),
                                    _ptr(o_depth), B, H, W, _ptr(x), _stream(stream)),
          "gs2d_net_pack_input")


def gs2d_net_downsample_rgbd(rgb, depth, factor, rgb_out, depth_out, stream=None):
    H, W = int(depth.shape[-2]), int(depth.shape[-1])
    check(lib().gs2d_net_downsample_rgbd(_ptr(rgb), _ptr(depth), H, W, int(factor), _ptr(rgb_out),
                                         _ptr(depth_out), _stream(stream)),
          "gs2d_net_downsample_rgbd")


def gs2d_net_prepare(params, batch, workspace, stream=None):
    check(lib().gs2d_net_prepare(_ptr(params), int(batch), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), None,
                                 _stream(stream)), "gs2d_net_prepare")


def gs2d_net_forward_prepared(params, x, y, workspace, stream=None):
    check(lib().gs2d_net_forward_prepared(_ptr(params), _ptr(x), int(x.shape[0]), _ptr(y),
                                          _ptr(workspace),
                                          workspace.numel() * workspace.element_size(), None,
                                          _stream(stream)), "gs2d_net_forward_prepared")


def gs2d_net_forward(params, x, y, workspace, stream=None):
    check(lib().gs2d_net_forward(_ptr(params), _ptr(x), int(x.shape[0]), _ptr(y), _ptr(workspace),
                                 workspace.numel() * workspace.element_size(), None,
                                 _stream(stream)), "gs2d_net_forward")


def gs2d_net_grad(params, x, target, loss, grad, workspace, y=None, stream=None):
    check(lib().gs2d_net_grad(_ptr(params), _ptr(x), _ptr(target), int(x.shape[0]), _ptr(loss),
                              _ptr(grad), _ptr(y), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), None,
                              _stream(stream)), "gs2d_net_grad")


def gs2d_net_adamw(params, grad, m, v, step, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, wd=0.0,
                   stream=None):
    check(lib().gs2d_net_adamw(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(),
                               int(step), float(lr), float(betas[0]), float(betas[1]), float(eps),
                               float(wd), _stream(stream)), "gs2d_net_adamw")


def gs2d_net_apply(y, poses, stream=None):
    check(lib().gs2d_net_apply(_ptr(y), int(y.shape[0]), _ptr(poses), _stream(stream)),
          "gs2d_net_apply")


def gs2d_net_target(poses_init, poses_gt, target, stream=None):
    check(lib().gs2d_net_target(_ptr(poses_init), _ptr(poses_gt), int(poses_init.shape[0]),
                                _ptr(target), _stream(stream)), "gs2d_net_target")


def gs2d_net_accept(loss_prop, loss_init, proposal, poses, accepted=None, stream=None):
    check(lib().gs2d_net_accept(_ptr(loss_prop), _ptr(loss_init), _ptr(proposal),
                                int(poses.shape[0]), _ptr(poses), _ptr(accepted),
                                _stream(stream)), "gs2d_net_accept")


def gs2d_net_accept_keep(loss_prop, loss_init, proposal, poses, prop_images, kept_images,
                         accepted=None, stream=None):
    """gs2d_net_accept that also copies the taken proposals' images (rgb,
    depth, opacity of prop_images) over kept_images and their loss over
    loss_init."""
    n_px = int(prop_images[1].numel()) // int(poses.shape[0])
    check(lib().gs2d_net_accept_keep(_ptr(loss_prop), _ptr(loss_init), _ptr(proposal),
                                     int(poses.shape[0]), _ptr(poses), _ptr(accepted), n_px,
                                     *[_ptr(t) for t in prop_images],
                                     *[_ptr(t) for t in kept_images], _stream(stream)),
          "gs2d_net_accept_keep")


def net_init_blocks():
    """(count, fan_in) blocks of the flat parameter vector, in layout order,
    for the seeded initialiser (weights He-normal, biases zero)."""
    w_off, b_off, fan = gs2d_net_layout()
    total = gs2d_net_param_count()
    blocks = []
    for l in range(NET_LAYERS):
        blocks.append((b_off[l] - w_off[l], fan[l]))
        end = w_off[l + 1] if l + 1 < NET_LAYERS else total
        blocks.append((end - b_off[l], 0))
    return blocks


class BatchRasterizer:
    """Buffers of a batch of views (up to 32): per view its records, bins,
    images and upstream gradients; projection, binning and the two render
    passes each run as one batched call."""

    def __init__(self, cams, n: int, actives=None, tiles=None, capacities=None, device="cuda",
                 px: int = 1):
        self.n = int(n)
        self.px = int(px)
        self.device = device
        self.nv = len(cams)
        assert 0 < self.nv <= MAX_VIEWS
        self.keep = []
        f = dict(dtype=torch.float32, device=device)
        # views of one size share stacked [V, H, W, ...] image tensors
        sizes = {(int(c.height), int(c.width)) for c in cams}
        self.stacked = None
        if len(sizes) == 1:
            H, W = sizes.pop()
            V = self.nv
            self.stacked = dict(rgb=torch.empty(V, H, W, 3, **f), depth=torch.empty(V, H, W, **f),
                                normal=torch.empty(V, H, W, 3, **f),
                                opacity=torch.empty(V, H, W, **f))
        for v, cam in enumerate(cams):
            act = None if actives is None or actives[v] is None else \
                torch.as_tensor(np.asarray(actives[v], np.int32), device=device)
            m = self.n if act is None else int(act.numel())
            cfg = default_config(tiles[v] if tiles else TILE_SHAPES[self.px][0], self.px)
            ccam = camera(cam)
            tx = int(lib().gs2d_tiles_x(_ref(ccam), _ref(cfg)))
            ty = int(lib().gs2d_tiles_y(_ref(ccam), _ref(cfg)))
            H, W = int(cam.height), int(cam.width)
            b = dict(pose=torch.empty(12, **f), active=act,
                     proj=torch.empty(max(m, 1) * PROJ_FLOATS, **f),
                     tiles=torch.empty(max(m, 1), dtype=torch.int32, device=device),
                     off=torch.empty(max(m, 1), dtype=torch.int32, device=device),
                     ranges=torch.empty(2 * tx * ty, dtype=torch.int32, device=device),
                     n_isect=torch.zeros(1, dtype=torch.int32, device=device),
                     status=torch.zeros(1, dtype=torch.int32, device=device),
                     rgb=self.stacked["rgb"][v] if self.stacked else torch.empty(H, W, 3, **f),
                     depth=self.stacked["depth"][v] if self.stacked else torch.empty(H, W, **f),
                     normal=self.stacked["normal"][v] if self.stacked else torch.empty(H, W, 3, **f),
                     opacity=self.stacked["opacity"][v] if self.stacked else torch.empty(H, W, **f),
                     t_final=torch.empty(H, W, **f),
                     n_last=torch.empty(H, W, dtype=torch.int32, device=device),
                     d_rgb=torch.zeros(H, W, 3, **f), d_depth=torch.zeros(H, W, **f),
                     d_normal=torch.zeros(H, W, 3, **f), d_opacity=torch.zeros(H, W, **f),
                     d_pose6=torch.zeros(6, **f), m=m, cam=cam, ccam=ccam, cfg=cfg,
                     n_tiles=tx * ty)
            self._alloc_bins(b, int(capacities[v]) if capacities else max(8 * m, 1024))
            self.keep.append(b)
        self._rebuild()
        self.grads = dict(mu=torch.empty(self.n, 3, **f), quat=torch.empty(self.n, 4, **f),
                          scale=torch.empty(self.n, 2, **f), opacity=torch.empty(self.n, **f),
                          rgb=torch.empty(self.n, 3, **f))

    def _alloc_bins(self, b, cap):
        b["cap"] = int(cap)
        b["vals"] = torch.empty(b["cap"], dtype=torch.int32, device=self.device)
        b["emit"] = torch.empty(b["cap"], dtype=torch.int32, device=self.device)

    def _rebuild(self):
        """The C view table and the batch workspaces from the buffers."""
        self.views = []
        for b in self.keep:
            act = b["active"]
            bins = Bins(None, b["vals"].data_ptr(), b["emit"].data_ptr(), b["off"].data_ptr(),
                        b["ranges"].data_ptr(), b["n_isect"].data_ptr(), b["status"].data_ptr(),
                        b["cap"])
            b["bins"] = bins
            self.views.append(View(
                b["ccam"], b["cfg"], b["pose"].data_ptr(),
                _ptr(act).value if act is not None else None, b["m"], b["proj"].data_ptr(),
                b["tiles"].data_ptr(), bins, b["rgb"].data_ptr(), b["depth"].data_ptr(),
                b["normal"].data_ptr(), b["opacity"].data_ptr(), b["t_final"].data_ptr(),
                b["n_last"].data_ptr(), b["d_rgb"].data_ptr(), b["d_depth"].data_ptr(),
                b["d_normal"].data_ptr(), b["d_opacity"].data_ptr(), b["d_pose6"].data_ptr()))
        arr = (View * self.nv)(*self.views)
        self.sort_ws = None
        self.render_ws = None
        self.sort_ws = _bytes(lib().gs2d_bin_sort_batch_workspace(arr, self.nv, self.n),
                              self.device)
        self.render_ws = _bytes(lib().gs2d_render_batch_workspace(arr, self.nv, self.n),
                                self.device)

    def set_poses(self, poses):
        for b, p in zip(self.keep, poses):
            b["pose"].copy_(p if isinstance(p, torch.Tensor) else pose_tensor(p, self.device))

    def fit(self, surf: DeviceSurfels, margin: float = 1.25, stream=None):
        """Project and bin at the current poses and regrow every view whose
        intersection count exceeded its capacity (to margin x the count).
        Returns the counts K per view."""
        for b in self.keep:
            b["status"].zero_()
        gs2d_project_batch(surf, self.views, stream)
        gs2d_bin_sort_batch(self.views, self.n, self.sort_ws, stream)
        k = [int(b["n_isect"].item()) for b in self.keep]
        grow = False
        for b, kv in zip(self.keep, k):
            if kv > b["cap"]:
                self._alloc_bins(b, int(kv * margin) + 1024)
                grow = True
        if grow:
            self._rebuild()
        for b in self.keep:
            b["status"].zero_()
        return k

    def forward(self, surf: DeviceSurfels, stream=None, check_status=True):
        for b in self.keep:
            b["status"].zero_()
        gs2d_project_batch(surf, self.views, stream)
        gs2d_bin_sort_batch(self.views, self.n, self.sort_ws, stream)
        gs2d_render_fwd_batch(self.views, self.render_ws, stream)
        if check_status:
            st = [int(b["status"].item()) for b in self.keep]
            if any(st):
                raise Gs2dError(f"batch status {st} (n_isect {[int(b['n_isect'].item()) for b in self.keep]})")

    def backward(self, surf: DeviceSurfels, stream=None):
        g = self.grads
        gs2d_render_bwd_batch(self.views, surf, g["mu"], g["quat"], g["scale"], g["opacity"],
                              g["rgb"], self.render_ws, stream)
        return g


# ---------------------------------------------------------------------------
# convenience: buffers of one camera
# ---------------------------------------------------------------------------
def _bytes(n, device):
    return torch.empty(max(int(n), 1), dtype=torch.uint8, device=device)


class Rasterizer:
    """Owns the intermediate buffers for rendering one camera:
    project -> bin_sort -> render_fwd, and render_bwd."""

    def __init__(self, cam, n: int, capacity: int | None = None, tile=(16, 16), device="cuda",
                 keys: bool = False, px: int = 1):
        self.cam = camera(cam)
        self.cfg = default_config(tile, px)
        self.n = int(n)
        self.device = device
        self.tiles_x = int(lib().gs2d_tiles_x(_ref(self.cam), _ref(self.cfg)))
        self.tiles_y = int(lib().gs2d_tiles_y(_ref(self.cam), _ref(self.cfg)))
        self.n_tiles = self.tiles_x * self.tiles_y
        self.want_keys = keys
        self.proj = torch.empty(max(self.n, 1) * PROJ_FLOATS, dtype=torch.float32, device=device)
        self.tiles = torch.empty(max(self.n, 1), dtype=torch.int32, device=device)
        self.surfel_off = torch.empty(max(self.n, 1), dtype=torch.int32, device=device)
        self.ranges = torch.empty(2 * self.n_tiles, dtype=torch.int32, device=device)
        self.n_isect = torch.zeros(1, dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        H, W = int(cam.height), int(cam.width)
        self.H, self.W = H, W
        f = dict(dtype=torch.float32, device=device)
        self.rgb = torch.empty(H, W, 3, **f)
        self.depth = torch.empty(H, W, **f)
        self.normal = torch.empty(H, W, 3, **f)
        self.opacity = torch.empty(H, W, **f)
        self.t_final = torch.empty(H, W, **f)
        self.n_last = torch.empty(H, W, dtype=torch.int32, device=device)
        self._alloc(capacity if capacity is not None else max(4 * self.n, 1024))

    def _alloc(self, capacity):
        self.capacity = int(capacity)
        d = self.device
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=d)
        self.emit = torch.empty(self.capacity, dtype=torch.int32, device=d)
        self.keys = torch.empty(self.capacity, dtype=torch.int64, device=d) if self.want_keys else None
        self.sort_ws = _bytes(gs2d_bin_sort_workspace(self.n, self.capacity), d)
        self.bwd_ws = _bytes(gs2d_render_bwd_workspace(self.n, self.capacity, self.n_tiles), d)
        self.bins = Bins(_ptr(self.keys).value if self.keys is not None else None,
                         self.vals.data_ptr(), self.emit.data_ptr(), self.surfel_off.data_ptr(),
                         self.ranges.data_ptr(), self.n_isect.data_ptr(), self.status.data_ptr(),
                         self.capacity)

    def project(self, surf: DeviceSurfels, pose: torch.Tensor, stream=None):
        gs2d_project(surf, self.cam, pose, self.cfg, self.proj, self.tiles, stream)

    def bin_sort(self, stream=None, grow: bool = True):
        self.status.zero_()
        gs2d_bin_sort(self.proj, self.tiles, self.n, self.cam, self.cfg, self.sort_ws, self.bins,
                      stream)
        if grow:
            st = int(self.status.item())
            if st == 3:
                need = int(self.n_isect.item())
                self._alloc(int(need * 1.25) + 1024)
                self.status.zero_()
                gs2d_bin_sort(self.proj, self.tiles, self.n, self.cam, self.cfg, self.sort_ws,
                              self.bins, stream)
                st = int(self.status.item())
            if st != 0:
                raise Gs2dError(f"gs2d_bin_sort device status {STATUS.get(st, st)}")

    def render_fwd(self, stream=None):
        gs2d_render_fwd(self.proj, self.bins, self.cam, self.cfg, self.rgb, self.depth, self.normal,
                        self.opacity, self.t_final, self.n_last, stream)

    def forward(self, surf: DeviceSurfels, pose: torch.Tensor, stream=None):
        self.project(surf, pose, stream)
        self.bin_sort(stream)
        self.render_fwd(stream)
        return dict(rgb=self.rgb, depth=self.depth, normal=self.normal, opacity=self.opacity,
                    t_final=self.t_final, n_last=self.n_last)

    def contribution(self, out=None, stream=None):
        """Per-surfel contribution (sum of blending weights over the image)
        of the last projected and binned view; device [n] FP32."""
        contrib = out if out is not None else torch.empty(max(self.n, 1), dtype=torch.float32,
                                                          device=self.device)
        need = gs2d_render_contrib_workspace(self.capacity)
        ws = getattr(self, "contrib_ws", None)
        if ws is None or ws.numel() < need:
            ws = self.contrib_ws = _bytes(need, self.device)
        gs2d_render_contrib(self.proj, self.bins, self.tiles, self.n, self.cam, self.cfg, contrib,
                            ws, stream)
        return contrib[: self.n]

    def backward(self, surf: DeviceSurfels, pose, d_rgb, d_depth, d_normal=None, d_opacity=None,
                 full: bool = True, stream=None):
        n = self.n
        f = dict(dtype=torch.float32, device=self.device)
        d_pose6 = torch.empty(6, **f)
        out = dict(pose6=d_pose6)
        if full:
            out.update(mu=torch.empty(n, 3, **f), quat=torch.empty(n, 4, **f),
                       scale=torch.empty(n, 2, **f), opacity=torch.empty(n, **f),
                       rgb=torch.empty(n, 3, **f))
        gs2d_render_bwd(self.proj, self.bins, self.tiles, surf, pose, self.cam, self.cfg,
                        self.t_final, self.n_last, d_rgb.contiguous(), d_depth.contiguous(),
                        None if d_normal is None else d_normal.contiguous(),
                        None if d_opacity is None else d_opacity.contiguous(),
                        out.get("mu"), out.get("quat"), out.get("scale"), out.get("opacity"),
                        out.get("rgb"), d_pose6, self.bwd_ws, stream)
        return out

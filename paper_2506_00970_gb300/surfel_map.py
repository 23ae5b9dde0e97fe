"""A growable surfel map on the GPU with the per-surfel state of Eq. map and
its voxel occupancy table, and the keyframe bookkeeping of 2DGS-SLAM as calls
into the library: map expansion (Sec. III-E), per-surfel contributions and the
covisibility keyframe rule (Sec. III-D), the state update after a keyframe and
occlusion removal (Sec. III-F), and the map correction after pose graph
optimisation (Sec. IV-C).

This module owns buffers and orders calls; every step on the data runs in the
library's kernels.  Host round trips happen only where the host must learn a
size (the number of new or kept surfels).
"""
from __future__ import annotations

import numpy as np
import torch

from . import gs2d


class SurfelMap:
    def __init__(self, capacity: int, voxel: float = 0.02, table_capacity: int | None = None,
                 inactive_after: int = 20, device="cuda"):
        self.capacity = int(capacity)
        self.device = device
        self.n = 0
        self.inactive_after = int(inactive_after)
        self._alloc_arrays()
        self.table = gs2d.DeviceVoxelTable(table_capacity or 2 * self.capacity, voxel, device)
        self._counts = torch.zeros(4, dtype=torch.int32, device=device)
        self._n_dev = torch.zeros(1, dtype=torch.int32, device=device)

    def _alloc_arrays(self):
        f = dict(dtype=torch.float32, device=self.device)
        c = self.capacity
        self.params = gs2d.DeviceSurfels.from_tensors(torch.zeros(c, 3, **f), torch.zeros(c, 4, **f),
                                                      torch.zeros(c, 2, **f), torch.zeros(c, **f),
                                                      torch.zeros(c, 3, **f))
        self.state = gs2d.DeviceMapState(c, device=self.device)

    # checkpoint ----------------------------------------------------------------
    def save(self, path: str):
        """The map's parameters and state (the first n surfels) and settings
        as a NumPy .npz; the voxel table is rebuilt on load."""
        n = self.n
        p, st = self.params, self.state
        np.savez(path, mu=p.mu[:n].cpu().numpy(), quat=p.quat[:n].cpu().numpy(),
                 scale=p.scale[:n].cpu().numpy(), opacity=p.opacity[:n].cpu().numpy(),
                 rgb=p.rgb[:n].cpu().numpy(), delta=st.delta[:n].cpu().numpy(),
                 t_c=st.t_c[:n].cpu().numpy(), d_c=st.d_c[:n].cpu().numpy(),
                 t_l=st.t_l[:n].cpu().numpy(),
                 settings=np.array([self.capacity, self.table.voxel, self.table.capacity,
                                    self.inactive_after], np.float64))

    @classmethod
    def load(cls, path: str, device="cuda") -> "SurfelMap":
        z = np.load(path)
        cap, voxel, tcap, after = z["settings"]
        m = cls(int(cap), float(voxel), int(tcap), int(after), device)
        n = int(z["mu"].shape[0])
        for name in ("mu", "quat", "scale", "opacity", "rgb"):
            getattr(m.params, name)[:n].copy_(torch.from_numpy(z[name]))
        for name in ("delta", "t_c", "d_c", "t_l"):
            getattr(m.state, name)[:n].copy_(torch.from_numpy(z[name]))
        m.n = n
        m.rebuild_table()
        return m

    # views of the first n surfels ------------------------------------------
    def surfels(self) -> gs2d.DeviceSurfels:
        p = self.params
        n = self.n
        return gs2d.DeviceSurfels.from_tensors(p.mu[:n], p.quat[:n], p.scale[:n], p.opacity[:n],
                                               p.rgb[:n])

    def map_state(self) -> gs2d.DeviceMapState:
        s = self.state
        n = self.n
        return gs2d.DeviceMapState.from_tensors(s.delta[:n], s.t_c[:n], s.d_c[:n], s.t_l[:n])

    # Sec. III-E ----------------------------------------------------------------
    def expand(self, rgb, depth, cam, pose_t, kf_id: int, ratio: float, generator=None,
               opacity: float = 0.99, max_scale: float = 0.05) -> int:
        """New surfels from an RGB-D keyframe in the free voxels of the active
        map; returns how many were added (their voxels join the table)."""
        H, W = depth.shape[0], depth.shape[1]
        g = generator
        u_keep = torch.rand(H, W, generator=g, device=self.device)
        u_ang = torch.rand(H, W, generator=g, device=self.device)
        ccam = gs2d.camera(cam)
        ws = torch.empty(gs2d.gs2d_expand_workspace(ccam), dtype=torch.uint8, device=self.device)
        prm = gs2d.ExpandParams(ratio, opacity, max_scale, int(kf_id), 1)
        gs2d.gs2d_expand(rgb.contiguous(), depth.contiguous(), ccam, pose_t, u_keep, u_ang,
                         self.table, prm, self.n, self.capacity, self.params, self.state,
                         self._n_dev, ws)
        k = int(self._n_dev.item())
        if int(self.table.status.item()) != 0:
            raise gs2d.Gs2dError(f"map expansion: capacity {self.capacity} or voxel table full "
                                 f"(needs {self.n + k} surfels)")
        self.n += k
        return k

    def rebuild_table(self):
        """The voxel table of the active surfels (after state changes)."""
        self.table.clear()
        if self.n:
            self.table.insert(self.params.mu[:self.n], self.state.delta[:self.n])

    # Sec. III-D ----------------------------------------------------------------
    def contributions(self, cam, pose_t, active_only: bool = True, tile=(16, 16)):
        """Per-surfel contribution (device [n]) of the view, rendering the
        active map (or the whole map); surfels not rendered get 0."""
        n = self.n
        if n == 0:
            return torch.zeros(0, device=self.device)
        if not active_only:
            r = gs2d.Rasterizer(cam, n, tile=tile, device=self.device)
            r.forward(self.surfels(), pose_t)
            return r.contribution().clone()
        sub = gs2d.DeviceSurfels.from_tensors(*(torch.empty_like(t) for t in (
            self.params.mu[:n], self.params.quat[:n], self.params.scale[:n],
            self.params.opacity[:n], self.params.rgb[:n])))
        new_index = torch.empty(n, dtype=torch.int32, device=self.device)
        n_out = torch.zeros(1, dtype=torch.int32, device=self.device)
        ws = torch.empty(gs2d.gs2d_map_compact_workspace(n), dtype=torch.uint8, device=self.device)
        gs2d.gs2d_map_compact(self.state.delta[:n], n, self.surfels(), None, sub, None, new_index,
                              n_out, ws)
        m = int(n_out.item())
        out = torch.zeros(n, device=self.device)
        if m == 0:
            return out
        act = gs2d.DeviceSurfels.from_tensors(sub.mu[:m], sub.quat[:m], sub.scale[:m],
                                              sub.opacity[:m], sub.rgb[:m])
        r = gs2d.Rasterizer(cam, m, tile=tile, device=self.device)
        r.forward(act, pose_t)
        c = r.contribution()
        gs2d.gs2d_map_expand_values(c, new_index, n, 0.0, out)
        return out

    def keyframe_test(self, c_cur, c_kf, pose_cur, pose_kf, c_k: float = 0.9, d_k: float = 0.15):
        """(covisibility score, is_keyframe) of the current view against the
        last keyframe's contributions (Table I thresholds)."""
        counts = torch.zeros(2, dtype=torch.int32, device=self.device)
        score = torch.zeros(1, device=self.device)
        kf = torch.zeros(1, dtype=torch.int32, device=self.device)
        gs2d.gs2d_covisibility(c_cur, c_kf, self.n, 0.5, pose_cur, pose_kf, c_k, d_k, counts,
                               score, kf)
        return float(score.item()), bool(kf.item())

    # Sec. III-F ----------------------------------------------------------------
    def observe(self, contrib, pose_t, kf_id: int, reactivate: bool = False, loop_h: int = -1):
        """State update for keyframe kf_id; returns (visible, closer,
        deactivated, reactivated) and rebuilds the voxel table when states
        changed."""
        prm = gs2d.StateParams(0.5, self.inactive_after, int(reactivate), int(loop_h))
        gs2d.gs2d_map_observe(contrib, self.params.mu[:self.n], self.n, pose_t, int(kf_id), prm,
                              self.map_state(), self._counts)
        counts = tuple(int(x) for x in self._counts.cpu().numpy())
        if counts[2] or counts[3]:
            self.rebuild_table()
        return counts

    def prune(self, contrib, r: int) -> int:
        """Removes the surfels of keyframe r (t^c = r) whose contribution to
        its view is below 0.5; returns how many were removed."""
        n = self.n
        if n == 0:
            return 0
        keep = torch.empty(n, dtype=torch.uint8, device=self.device)
        gs2d.gs2d_map_prune(contrib, self.state.t_c[:n], n, int(r), 0.5, keep)
        old_p, old_s = self.params, self.state
        self._alloc_arrays()
        n_out = torch.zeros(1, dtype=torch.int32, device=self.device)
        ws = torch.empty(gs2d.gs2d_map_compact_workspace(n), dtype=torch.uint8, device=self.device)
        src = gs2d.DeviceSurfels.from_tensors(old_p.mu[:n], old_p.quat[:n], old_p.scale[:n],
                                              old_p.opacity[:n], old_p.rgb[:n])
        src_st = gs2d.DeviceMapState.from_tensors(old_s.delta[:n], old_s.t_c[:n], old_s.d_c[:n],
                                                  old_s.t_l[:n])
        gs2d.gs2d_map_compact(keep, n, src, src_st, self.params, self.state, None, n_out, ws)
        self.n = int(n_out.item())
        self.rebuild_table()
        return n - self.n

    # Sec. IV-C -----------------------------------------------------------------
    def correct(self, poses_old, poses_new) -> int:
        """Map correction by the keyframes' pose increments (device
        [n_kf * 12] world-to-camera poses before and after pose graph
        optimisation); returns the number of surfels left unchanged."""
        n_kf = int(poses_old.numel() // 12)
        ws = torch.empty(gs2d.gs2d_map_correct_workspace(n_kf), dtype=torch.uint8,
                         device=self.device)
        skipped = torch.zeros(1, dtype=torch.int32, device=self.device)
        gs2d.gs2d_map_correct(self.params.mu[:self.n], self.params.quat[:self.n],
                              self.state.t_c[:self.n], self.n, poses_old, poses_new, n_kf, ws,
                              skipped)
        self.rebuild_table()
        return int(skipped.item())

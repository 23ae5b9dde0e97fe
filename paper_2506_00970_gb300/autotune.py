"""Tile-shape and pixels-per-thread autotuner for batched rendering.

For every pixels-per-thread count P (1, 2, 3, 4) and every resolution class
(width x height) of a batch, each tile shape of P is timed on a forward +
backward pass of up to ``max_views`` of that class's views (CUDA events on
the launching stream, the median of ``reps`` repetitions after one warm-up);
the fastest shape per class is kept.  One batched launch runs one P, so P is
chosen for the whole batch: the one whose per-class best times, weighted by
the number of views in each class, sum lowest.  Results are cached per device
name and resolution class (and the P decision per set of classes), in memory
and optionally in a JSON file, so a later batch with the same classes skips
the sweep.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import gs2d

TILE_SHAPES = gs2d.TILE_SHAPES
PX_COUNTS = (1, 2, 3, 4)

_cache: dict[str, list] = {}


def _key(device_name: str, w: int, h: int, px: int) -> str:
    return f"{device_name}|{w}x{h}|px{px}"


def _load(path):
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                _cache.update(json.load(f))
        except (OSError, ValueError):
            pass


def _store(path):
    if path:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        with open(path, "w") as f:
            json.dump(_cache, f, indent=1, sort_keys=True)


def time_batch(surf, cams, poses, actives, tile, px=1, reps=3, stream=None):
    """Median ms of project + bin_sort + forward + backward of one batch with
    one tile shape and pixels-per-thread count for all views (unit upstream
    gradients on colour and depth)."""
    br = gs2d.BatchRasterizer(cams, surf.n, actives=actives, tiles=[tile] * len(cams), px=px)
    br.set_poses(poses)
    br.fit(surf)
    for b in br.keep:
        b["d_rgb"].fill_(1.0)
        b["d_depth"].fill_(1.0)
    st = stream if stream is not None else torch.cuda.current_stream()
    ms = []
    for r in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        br.forward(surf, stream, check_status=False)
        br.backward(surf, stream)
        e1.record(st)
        e1.synchronize()
        if r:
            ms.append(e0.elapsed_time(e1))
    bad = [int(b["status"].item()) for b in br.keep]
    if any(bad):
        raise gs2d.Gs2dError(f"autotune batch status {bad}")
    del br
    return float(np.median(ms))


def tune(surf, cams, poses, actives=None, max_views=3, reps=3, cache_path=None, stream=None,
         px_counts=PX_COUNTS):
    """(P, tile shape per view, sweep table {"pxP": {class: {tile: ms}}})."""
    _load(cache_path)
    dev = torch.cuda.get_device_name()
    classes: dict[tuple[int, int], list[int]] = {}
    for v, c in enumerate(cams):
        classes.setdefault((int(c.width), int(c.height)), []).append(v)
    table = {}
    best = {}      # (px, class) -> (tile, ms)
    for px in px_counts:
        for (w, h), idx in classes.items():
            key = _key(dev, w, h, px)
            if key in _cache:
                tw, th, ms = _cache[key]
                best[(px, (w, h))] = ((int(tw), int(th)), float(ms))
                continue
            pick = idx[:max_views]
            sub_c = [cams[v] for v in pick]
            sub_p = [poses[v] for v in pick]
            sub_a = None if actives is None else [actives[v] for v in pick]
            t = {}
            for tile in TILE_SHAPES[px]:
                t[f"{tile[0]}x{tile[1]}"] = time_batch(surf, sub_c, sub_p, sub_a, tile, px, reps,
                                                       stream) / len(pick)
            table.setdefault(f"px{px}", {})[f"{w}x{h}"] = t
            win = min(t, key=t.get)
            tile = tuple(int(x) for x in win.split("x"))
            best[(px, (w, h))] = (tile, t[win])
            _cache[key] = [tile[0], tile[1], t[win]]
            torch.cuda.empty_cache()
    _store(cache_path)
    total = {px: sum(best[(px, cl)][1] * len(idx) for cl, idx in classes.items())
             for px in px_counts}
    px = min(total, key=total.get)
    tiles = [best[(px, (int(c.width), int(c.height)))][0] for c in cams]
    return px, tiles, table


def tune_tiles(surf, cams, poses, actives=None, **kw):
    """Tile shape per view at one pixel per thread (see ``tune``)."""
    px, tiles, table = tune(surf, cams, poses, actives, px_counts=(1,), **kw)
    return tiles, table.get("px1", {})

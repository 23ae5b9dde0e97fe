"""Tile-shape autotuner for batched rendering.

For every resolution class (width x height) of a batch, each candidate tile
shape is timed on a forward + backward pass of up to ``max_views`` of that
class's views (CUDA events on the launching stream, the median of ``reps``
repetitions after one warm-up) and the fastest is kept.  Results are cached
per device name and resolution class, in memory and optionally in a JSON file,
so a later batch with the same classes skips the sweep.

The compositing kernels map one thread to one pixel (a 256-thread block per
tile), so the candidates are the three 256-pixel shapes; the pixels-per-thread
field of the config stays 1.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import gs2d

TILE_SHAPES = ((16, 16), (8, 32), (32, 8))

_cache: dict[str, list[int]] = {}


def _key(device_name: str, w: int, h: int) -> str:
    return f"{device_name}|{w}x{h}"


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


def time_batch(surf, cams, poses, actives, tile, reps=3, stream=None):
    """Median ms of project + bin_sort + forward + backward of one batch with
    one tile shape for all views (unit upstream gradients on colour and
    depth)."""
    br = gs2d.BatchRasterizer(cams, surf.n, actives=actives, tiles=[tile] * len(cams))
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


def tune_tiles(surf, cams, poses, actives=None, max_views=3, reps=3, cache_path=None,
               stream=None):
    """Tile shape per view: the fastest candidate of the view's resolution
    class.  Returns (tiles per view, sweep table {class: {tile: ms}})."""
    _load(cache_path)
    dev = torch.cuda.get_device_name()
    classes: dict[tuple[int, int], list[int]] = {}
    for v, c in enumerate(cams):
        classes.setdefault((int(c.width), int(c.height)), []).append(v)
    table = {}
    best = {}
    for (w, h), idx in classes.items():
        key = _key(dev, w, h)
        if key in _cache:
            best[(w, h)] = tuple(_cache[key])
            continue
        pick = idx[:max_views]
        sub_c = [cams[v] for v in pick]
        sub_p = [poses[v] for v in pick]
        sub_a = None if actives is None else [actives[v] for v in pick]
        t = {}
        for tile in TILE_SHAPES:
            t[f"{tile[0]}x{tile[1]}"] = time_batch(surf, sub_c, sub_p, sub_a, tile, reps, stream)
        table[f"{w}x{h}"] = t
        win = min(t, key=t.get)
        best[(w, h)] = tuple(int(x) for x in win.split("x"))
        _cache[key] = list(best[(w, h)])
        torch.cuda.empty_cache()
    _store(cache_path)
    return [best[(int(c.width), int(c.height))] for c in cams], table

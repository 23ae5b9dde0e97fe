"""GPU parity of the map-state calls (include/gs2d_map.h) against the FP64
oracle ``oracle.map_state``:

* gs2d_map_observe: active flags, t^l and t^c bit-exact and d^c within FP32
  rounding, except where the FP64 distance lies within 1e-5 of the stored
  d^c (the FP32 kernel may take that decision either way: both results are
  checked to be valid); counts exact when no such tie exists;
* gs2d_map_correct: centres within 1e-5 (1 + |mu|), rotation matrices within
  1e-5, quaternion norms kept, invalid keyframe ids left as they are and
  counted;
* gs2d_map_prune and gs2d_map_compact: bit-exact (integer and copy work),
  at sizes from 0 to several scan blocks of blocks.
"""
import numpy as np
import pytest

import oracle.map_state as ms
from gpu_helpers import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


def _pose12(R, t):
    return np.concatenate([np.asarray(R).reshape(-1), np.asarray(t)]).astype(np.float32)


def _rand_rot(rng):
    return ms.quat_matrix(rng.normal(size=4))


@pytest.mark.parametrize("n,react", [(1, False), (5000, False), (5000, True), (1_000_003, True)])
def test_map_observe(torch_cuda, n, react):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(n + react)
    f32 = lambda a: np.asarray(a, np.float32)
    mu = f32(rng.uniform(-4, 4, (n, 3)))
    contrib = f32(rng.choice([0.0, 0.2, 0.5, 0.7, 3.0], n))
    st = dict(delta=rng.integers(0, 2, n).astype(np.uint8), t_c=rng.integers(0, 20, n).astype(np.int32),
              d_c=f32(rng.uniform(0.5, 8.0, n)), t_l=rng.integers(0, 20, n).astype(np.int32))
    R, t = _rand_rot(rng), rng.normal(size=3)
    pose = _pose12(R, t)
    kf, after, loop_h = 20, 5, 10
    o, ocounts = ms.observe(contrib, mu, pose[:9].reshape(3, 3).astype(np.float64),
                            pose[9:].astype(np.float64), kf, st, 0.5, after, react, loop_h)
    T = lambda a: torch.tensor(a, device="cuda")
    dst = gs2d.DeviceMapState.from_tensors(T(st["delta"]), T(st["t_c"]), T(st["d_c"]),
                                           T(st["t_l"]))
    prm = gs2d.StateParams(0.5, after, int(react), loop_h)
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    gs2d.gs2d_map_observe(T(contrib), T(mu), n, T(pose), kf, prm, dst, counts)
    torch.cuda.synchronize()
    g = {k: getattr(dst, k).cpu().numpy() for k in ("delta", "t_c", "d_c", "t_l")}
    # ties: the FP32 distance may fall on either side of d_c
    c = ms.camera_centre(pose[:9].reshape(3, 3).astype(np.float64), pose[9:].astype(np.float64))
    dist = np.linalg.norm(mu.astype(np.float64) - c, axis=1)
    tie = np.abs(dist - st["d_c"]) <= 1e-5 * st["d_c"]
    assert np.array_equal(g["delta"], o["delta"]) and np.array_equal(g["t_l"], o["t_l"])
    ok = ~tie
    assert np.array_equal(g["t_c"][ok], o["t_c"][ok])
    np.testing.assert_allclose(g["d_c"][ok], o["d_c"][ok], rtol=1e-6)
    # at a tie either outcome is valid: unchanged, or (distance, kf)
    kept = (g["t_c"][tie] == st["t_c"][tie]) & (g["d_c"][tie] == st["d_c"][tie])
    took = (g["t_c"][tie] == kf) & (np.abs(g["d_c"][tie] - dist[tie]) <= 1e-6 * dist[tie])
    assert np.all(kept | took)
    gc = tuple(counts.cpu().numpy().tolist())
    assert gc[0] == ocounts[0] and gc[2:] == ocounts[2:]
    if not tie.any():
        assert gc[1] == ocounts[1]


@pytest.mark.parametrize("n,n_kf", [(0, 3), (1, 1), (4097, 7), (500_000, 64)])
def test_map_correct(torch_cuda, n, n_kf):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(n + n_kf)
    mu = rng.uniform(-5, 5, (n, 3)).astype(np.float32)
    quat = rng.normal(size=(n, 4)).astype(np.float32)
    t_c = rng.integers(-1, n_kf + 1, n).astype(np.int32)
    old = [(_rand_rot(rng), rng.normal(size=3)) for _ in range(n_kf)]
    new = [(R @ ms.quat_matrix(np.r_[1.0, rng.normal(scale=0.05, size=3)]),
            t + rng.normal(scale=0.1, size=3)) for R, t in old]
    # the FP32 copies of the poses are the inputs of both sides
    old32 = [(R.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64))
             for R, t in old]
    new32 = [(R.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64))
             for R, t in new]
    mu_o, R_o, skipped = ms.correct(mu, quat, t_c, old32, new32)
    T = lambda a: torch.tensor(a, device="cuda")
    pm = lambda ps: T(np.concatenate([_pose12(R, t) for R, t in ps]) if ps else np.zeros(12, np.float32))
    g_mu = T(mu.reshape(-1, 3) if n else np.zeros((1, 3), np.float32))
    g_q = T(quat.reshape(-1, 4) if n else np.zeros((1, 4), np.float32))
    ws = torch.empty(gs2d.gs2d_map_correct_workspace(n_kf), dtype=torch.uint8, device="cuda")
    nsk = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    gs2d.gs2d_map_correct(g_mu, g_q, T(t_c) if n else T(np.zeros(1, np.int32)), n, pm(old32),
                          pm(new32), n_kf, ws, nsk)
    torch.cuda.synchronize()
    assert int(nsk.item()) == skipped
    if n == 0:
        return
    gm, gq = to_np(g_mu), to_np(g_q)
    np.testing.assert_allclose(gm, mu_o, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(ms.quat_matrix(gq), R_o, atol=1e-5)
    np.testing.assert_allclose(np.linalg.norm(gq, axis=1),
                               np.linalg.norm(quat.astype(np.float64), axis=1), rtol=1e-5)
    bad = (t_c < 0) | (t_c >= n_kf)
    assert np.array_equal(gm[bad], mu[bad].astype(np.float64))


@pytest.mark.parametrize("n", [0, 1, 1023, 1024, 1025, 70_000, 3_000_001])
def test_map_prune_and_compact(torch_cuda, n):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    rng = np.random.default_rng(n)
    contrib = rng.choice(np.float32([0.0, 0.3, 0.5, 0.9]), n)
    t_c = rng.integers(0, 4, n).astype(np.int32)
    keep_o = ms.prune_keep(contrib, t_c, 2)
    T = lambda a: torch.tensor(a, device="cuda")
    m = max(n, 1)
    keep = torch.empty(m, dtype=torch.uint8, device="cuda")
    gs2d.gs2d_map_prune(T(contrib) if n else T(np.zeros(1, np.float32)),
                        T(t_c) if n else T(np.zeros(1, np.int32)), n, 2, 0.5, keep)
    torch.cuda.synchronize()
    assert np.array_equal(keep.cpu().numpy()[:n].astype(bool), keep_o)
    arrays = dict(mu=rng.normal(size=(m, 3)).astype(np.float32),
                  quat=rng.normal(size=(m, 4)).astype(np.float32),
                  scale=rng.uniform(size=(m, 2)).astype(np.float32),
                  opacity=rng.uniform(size=m).astype(np.float32),
                  rgb=rng.uniform(size=(m, 3)).astype(np.float32))
    state = dict(delta=rng.integers(0, 2, m).astype(np.uint8), t_c=t_c if n else np.zeros(1, np.int32),
                 d_c=rng.uniform(size=m).astype(np.float32), t_l=rng.integers(0, 9, m).astype(np.int32))
    surf = gs2d.DeviceSurfels.from_tensors(*(T(arrays[k]) for k in ("mu", "quat", "scale", "opacity", "rgb")))
    out = gs2d.DeviceSurfels.from_tensors(*(torch.full_like(T(arrays[k]), -9)
                                            for k in ("mu", "quat", "scale", "opacity", "rgb")))
    st = gs2d.DeviceMapState.from_tensors(*(T(state[k]) for k in ("delta", "t_c", "d_c", "t_l")))
    st_o = gs2d.DeviceMapState.from_tensors(*(torch.zeros_like(T(state[k]))
                                              for k in ("delta", "t_c", "d_c", "t_l")))
    new_index = torch.empty(m, dtype=torch.int32, device="cuda")
    n_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ws = torch.empty(gs2d.gs2d_map_compact_workspace(n), dtype=torch.uint8, device="cuda")
    gs2d.gs2d_map_compact(keep, n, surf, st, out, st_o, new_index, n_out, ws)
    torch.cuda.synchronize()
    k = int(n_out.item())
    assert k == int(keep_o.sum())
    names = ("mu", "quat", "scale", "opacity", "rgb")
    expect, idx = ms.compact(keep_o, *(arrays[nm][:n] for nm in names),
                             *(state[nm][:n] for nm in ("delta", "t_c", "d_c", "t_l")))
    for nm, e in zip(names, expect[:5]):
        assert np.array_equal(getattr(out, nm).cpu().numpy()[:k], e), nm
    for nm, e in zip(("delta", "t_c", "d_c", "t_l"), expect[5:]):
        assert np.array_equal(getattr(st_o, nm).cpu().numpy()[:k], e), nm
    if n:
        assert np.array_equal(new_index.cpu().numpy()[:n], idx)

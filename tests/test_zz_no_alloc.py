"""gs2d_bin_sort_static, the binning entry point that allocates nothing: for
callers that cannot allocate device memory when they bin (inside a CUDA stream
capture, under a no-allocation rule, or in a framework that owns all device
memory), it uses a fixed scratch array inside the library instead of a caller
workspace.  It must return exactly what gs2d_bin_sort returns, call after
call (the scratch keeps the previous call's contents), and refuse sizes its
scratch cannot hold.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2506_00970_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_00970_gb300 import gs2d
    gs2d.lib()
    return torch


def _inputs(torch, seed, n, tx, ty):
    from paper_2506_00970_gb300 import gs2d
    rect, depth, count = scenes.random_tile_records(seed, n, tx, ty)
    proj = np.zeros((n, gs2d.PROJ_FLOATS), np.float32)
    proj[:, 26] = depth
    proj[:, 28] = (rect[:, 0].astype(np.uint32) | (rect[:, 1].astype(np.uint32) << 16)).view(np.float32)
    proj[:, 29] = (rect[:, 2].astype(np.uint32) | (rect[:, 3].astype(np.uint32) << 16)).view(np.float32)
    return (torch.tensor(proj.reshape(-1), device="cuda"),
            torch.tensor(count.astype(np.int32), device="cuda"), int(count.sum()))


def _outputs(torch, n, n_tiles, cap):
    from paper_2506_00970_gb300 import gs2d
    o = dict(keys=torch.empty(cap, dtype=torch.int64, device="cuda"),
             vals=torch.empty(cap, dtype=torch.int32, device="cuda"),
             emit=torch.empty(cap, dtype=torch.int32, device="cuda"),
             off=torch.empty(n, dtype=torch.int32, device="cuda"),
             ranges=torch.empty(2 * n_tiles, dtype=torch.int32, device="cuda"),
             n_isect=torch.zeros(1, dtype=torch.int32, device="cuda"),
             status=torch.zeros(1, dtype=torch.int32, device="cuda"))
    o["bins"] = gs2d.Bins(o["keys"].data_ptr(), o["vals"].data_ptr(), o["emit"].data_ptr(),
                          o["off"].data_ptr(), o["ranges"].data_ptr(), o["n_isect"].data_ptr(),
                          o["status"].data_ptr(), cap)
    return o


@pytest.mark.parametrize("case", [(1, 20000, 40, 30), (2, 150_000, 75, 43)])
def test_static_bin_sort_matches_workspace_bin_sort_twice(torch_cuda, case):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    seed, n, tx, ty = case
    cam = gs2d.Camera(100.0, 100.0, 8.0, 8.0, tx * 16, ty * 16, 0.05)
    cfg = gs2d.default_config()
    L = gs2d.lib()
    for call in range(2):          # two calls in a row, different inputs
        proj, tiles, K = _inputs(torch, seed + 10 * call, n, tx, ty)
        cap = K + 101
        ref = _outputs(torch, n, tx * ty, cap)
        ws = torch.empty(gs2d.gs2d_bin_sort_workspace(n, cap), dtype=torch.uint8, device="cuda")
        gs2d.gs2d_bin_sort(proj, tiles, n, cam, cfg, ws, ref["bins"])
        got = _outputs(torch, n, tx * ty, cap)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = L.gs2d_bin_sort_static(ctypes.c_void_p(proj.data_ptr()), ctypes.c_void_p(tiles.data_ptr()),
                                    n, ctypes.byref(cam), ctypes.byref(cfg), ctypes.byref(got["bins"]),
                                    stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert int(got["status"].item()) == 0 and int(ref["status"].item()) == 0
        assert int(got["n_isect"].item()) == int(ref["n_isect"].item()) == K
        for k in ("keys", "vals", "emit"):
            assert torch.equal(got[k][:K], ref[k][:K]), (call, k)
        assert torch.equal(got["off"], ref["off"]) and torch.equal(got["ranges"], ref["ranges"])


def test_static_bin_sort_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_2506_00970_gb300 import gs2d
    L = gs2d.lib()
    cam = gs2d.Camera(100.0, 100.0, 8.0, 8.0, 640, 480, 0.05)
    cfg = gs2d.default_config()
    n, cap = 1_000_000, 8_000_000
    assert gs2d.gs2d_bin_sort_workspace(n, cap) > (32 << 20)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    bins = gs2d.Bins(None, 16, 16, 16, 16, 16, status.data_ptr(), cap)
    rc = L.gs2d_bin_sort_static(None, None, n, ctypes.byref(cam), ctypes.byref(cfg),
                                ctypes.byref(bins), None)
    assert rc == 2            # GS2D_ERR_WORKSPACE, nothing launched
    torch.cuda.synchronize()
    assert int(status.item()) == 0

"""The multi-GPU path runs replicas (no collective on the data path); its
plumbing -- process group, barrier, max-over-ranks timing, per-rank seeds,
the whole-job weak-scaling value -- runs here as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_2506_00970_gb300 import replicas
    ws, r, local = replicas.init("gloo")
    replicas.barrier()
    slowest = replicas.max_over_ranks(10.0 + 5.0 * r)     # rank r "took" 10 + 5 r ms
    value = replicas.weak_scaling_value(ws, 1000.0, slowest)
    q.put((r, ws, local, slowest, value, replicas.seed_base(r)))
    replicas.finish()


def test_two_gloo_ranks_aggregate_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    # every rank sees the slowest rank's time; the job value counts both ranks' units
    assert all(r[3] == pytest.approx(15.0) for r in res)
    assert all(r[4] == pytest.approx(2 * 1000.0 / 0.015) for r in res)
    assert res[0][5] != res[1][5]


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2506_00970_gb300 import replicas
    assert replicas.init("gloo") == (1, 0, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.weak_scaling_value(1, 10.0, 2.0) == pytest.approx(5000.0)

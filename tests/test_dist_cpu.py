"""The multi-process replica path of the benchmark on CPU: two gloo ranks, barrier and
max/sum reductions of per-rank values (the only collectives a replica run uses)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2507_08820_gb300 import dist
    info = dist.rank_info()
    assert (info.rank, info.world) == (rank, world)
    dist.init(info, "gloo")
    dist.barrier(info)
    mx = dist.max_over_ranks(info, 1.5 + rank)
    sm = dist.sum_over_ranks(info, 10.0 * (rank + 1))
    out[rank] = (mx, sm)
    dist.finalize(info)


def test_two_gloo_ranks_reduce_times():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.5, 30.0)


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2507_08820_gb300 import dist
    info = dist.rank_info()
    assert (info.rank, info.world, info.local_rank) == (0, 1, 0)
    assert dist.init(info, "gloo") is None
    assert dist.max_over_ranks(info, 3.0) == 3.0

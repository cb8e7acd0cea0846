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


# ---------------------------------------------------------------- z-slab decomposition
SLAB_SHAPE = (6, 5, 10)   # nx, ny, nz_global
SLAB_STEPS = 3


def _global_state():
    import numpy as np
    from oracle import rflbm_oracle as o
    from paper_2507_08820_gb300 import workloads as W
    nx, ny, nz = SLAB_SHAPE
    rho, u = W.random_fields(nx, ny, nz, seed=21, drho=0.02, du=0.03)
    n = nx * ny * nz
    return np.ascontiguousarray(o.equilibrium_state(rho, u) + W.population_perturbation(n, 22, 2e-4))


def _slab_worker(rank, world, port, out):
    """One z-slab of the box on a gloo rank: the oracle's collision on the slab's sites
    (noise keyed by their global index), the faces exchanged by dist.exchange_faces on the
    ring, then streaming with the received rows as the rows beyond the slab's faces."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    from oracle import rflbm_oracle as o
    from paper_2507_08820_gb300 import dist
    info = dist.rank_info()
    dist.init(info, "gloo")
    nx, ny, nzg = SLAB_SHAPE
    nxy = nx * ny
    z0, nz = dist.slab_bounds(nzg, info.world, info.rank)
    c = o.velocities()
    up = [i for i in range(27) if c[i, 2] == 1]      # populations leaving through the top face
    down = [i for i in range(27) if c[i, 2] == -1]   # ... through the bottom face
    f = _global_state()[:, z0 * nxy:(z0 + nz) * nxy].copy()
    sites = np.arange(z0 * nxy, (z0 + nz) * nxy, dtype=np.uint64)
    for t in range(SLAB_STEPS):
        fs = o.collide(f, 0.8, 1e-4, 7, t, sites).reshape(27, nz, ny, nx)
        send_up = [torch.from_numpy(np.ascontiguousarray(fs[i, nz - 1])) for i in up]
        send_down = [torch.from_numpy(np.ascontiguousarray(fs[i, 0])) for i in down]
        recv_below = [torch.empty((ny, nx), dtype=torch.float64) for _ in up]
        recv_above = [torch.empty((ny, nx), dtype=torch.float64) for _ in down]
        dist.exchange_faces(info, send_up, send_down, recv_below, recv_above)
        ext = np.zeros((27, nz + 2, ny, nx))   # rows: ghost below, own rows, ghost above
        ext[:, 1:nz + 1] = fs
        for k, i in enumerate(up):
            ext[i, 0] = recv_below[k].numpy()
        for k, i in enumerate(down):
            ext[i, nz + 1] = recv_above[k].numpy()
        new = np.empty((27, nz, ny, nx))
        for i in range(27):  # f_i(x) = f*_i(x - c_i): periodic in x and y, ghost rows in z
            rolled = np.roll(ext[i], shift=(c[i, 1], c[i, 0]), axis=(1, 2))
            new[i] = rolled[1 - c[i, 2]:1 - c[i, 2] + nz]
        f = new.reshape(27, nz * nxy)
    out[rank] = (z0, nz, f)
    dist.finalize(info)


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_reproduce_the_undecomposed_oracle_run(world):
    """world gloo ranks, each a z-slab of a 6 x 5 x 10 box, reproduce the oracle's run of
    the whole periodic box (3 steps with noise) within FP64 round-off."""
    import numpy as np
    from oracle import rflbm_oracle as o
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    want = o.run(_global_state(), SLAB_SHAPE, 0.8, 1e-4, 7, SLAB_STEPS)
    nxy = SLAB_SHAPE[0] * SLAB_SHAPE[1]
    rows = 0
    for r in range(world):
        z0, nz, f = out[r]
        assert z0 == rows
        rows += nz
        assert np.allclose(f, want[:, z0 * nxy:(z0 + nz) * nxy], rtol=1e-13, atol=1e-15)
    assert rows == SLAB_SHAPE[2]


def test_slab_bounds_split_the_rows():
    from paper_2507_08820_gb300 import dist
    for nzg, world in ((10, 3), (7, 7), (1024, 8), (5, 2)):
        parts = [dist.slab_bounds(nzg, world, r) for r in range(world)]
        assert sum(nz for _, nz in parts) == nzg
        assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        assert max(nz for _, nz in parts) - min(nz for _, nz in parts) <= 1
    with pytest.raises(ValueError):
        dist.slab_bounds(3, 4, 0)

"""Process-group plumbing, one process per GPU: independent replicas, and the z-slab
decomposition of one box.

Replicas: the Reg-FLBM step has no exchange between independent boxes, so N replicas run
with no data-path collective (weak scaling): rank r advances its own box with Philox
replica word r, and the only collectives are a barrier around the timed region and a
max-reduction of the per-rank times.

z-slabs (the paper's linear decomposition along z, Sec. IV): rank r holds rows
z0 .. z0 + nz - 1 of one periodic box (`slab_bounds`); after every step each rank sends the
face of its top row to the rank above and the face of its bottom row to the rank below, and
receives the matching faces into its ghost rows (`exchange_faces`: grouped point-to-point
sends and receives on a periodic ring). torch.distributed carries the bytes (NCCL on GPUs,
gloo on CPU); which rows and populations form a face is the library's business
(rflbm_slab_faces).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class RankInfo:
    rank: int
    world: int
    local_rank: int


def rank_info() -> RankInfo:
    """RANK / WORLD_SIZE / LOCAL_RANK from the environment (torchrun), else 0 / 1 / 0."""
    return RankInfo(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                    int(os.environ.get("LOCAL_RANK", "0")))


def init(info: RankInfo, backend: str):
    """Initialises the default process group when world > 1 (env:// rendezvous)."""
    if info.world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=info.rank, world_size=info.world)
    return dist


def barrier(info: RankInfo, device=None):
    if info.world <= 1:
        return
    import torch.distributed as dist
    if device is not None and dist.get_backend() == "nccl":
        dist.barrier(device_ids=[device])
    else:
        dist.barrier()


def max_over_ranks(info: RankInfo, value: float, device=None) -> float:
    """Maximum of a float over all ranks (the slowest rank's time)."""
    if info.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(info: RankInfo, value: float, device=None) -> float:
    if info.world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def finalize(info: RankInfo):
    if info.world <= 1:
        return
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def slab_bounds(nz_global: int, world: int, rank: int):
    """(z0, nz) of rank's z-slab when nz_global rows are split as evenly as possible over
    world ranks (the first nz_global % world ranks take one row more)."""
    if not 1 <= world <= nz_global:
        raise ValueError(f"cannot split {nz_global} rows over {world} ranks")
    base, extra = divmod(nz_global, world)
    nz = base + (1 if rank < extra else 0)
    z0 = rank * base + min(rank, extra)
    return z0, nz


def ring_neighbours(info: RankInfo):
    """(rank above, rank below) on the periodic ring of z-slabs."""
    return (info.rank + 1) % info.world, (info.rank - 1) % info.world


def exchange_faces(info: RankInfo, send_up, send_down, recv_below, recv_above):
    """One face exchange on the ring of z-slabs. Each argument is a list of equally long
    lists of tensors (the plane rows of a face, in the library's run and plane order);
    send_up goes to the rank above into its recv_below, send_down to the rank below into
    its recv_above. With one rank the slab is its own neighbour (local copies). The
    operations are posted as one group: the two sends to a peer are matched in order by
    the peer's two receives (up before down), which also pairs them correctly when the
    rank above and the rank below are the same peer (two ranks)."""
    if info.world <= 1:
        for d, s in zip(recv_below, send_up):
            d.copy_(s)
        for d, s in zip(recv_above, send_down):
            d.copy_(s)
        return
    import torch.distributed as dist
    up, down = ring_neighbours(info)
    ops = [dist.P2POp(dist.isend, t, up) for t in send_up]
    ops += [dist.P2POp(dist.isend, t, down) for t in send_down]
    ops += [dist.P2POp(dist.irecv, t, down) for t in recv_below]
    ops += [dist.P2POp(dist.irecv, t, up) for t in recv_above]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def face_rows(buffers, face):
    """The 9 plane rows of a face (an rflbm_face_t: three runs of three plane rows) as uint8
    views of the torch tensors that hold the slab's population buffers."""
    rows = []
    for r in range(3):
        for p in range(3):
            addr = face.run[r] + p * face.plane_pitch
            for t in buffers:
                off = addr - t.data_ptr()
                if 0 <= off and off + face.row_bytes <= t.numel():
                    rows.append(t[off:off + face.row_bytes])
                    break
            else:
                raise ValueError("face row outside the slab's buffers")
    return rows


def exchange_slab(R, box, info: RankInfo, stream):
    """The face exchange after a step of this rank's z-slab (a Box created with
    torch_buffers=True): the copy stream waits for the slab's boundary rows, the faces
    travel on it (exchange_faces), and the slab's next step waits for the stream."""
    import torch
    send_up, send_down, recv_below, recv_above = R.rflbm_slab_faces(box.h)
    R.rflbm_slab_faces_ready(box.h, stream.cuda_stream)
    with torch.cuda.stream(stream):
        exchange_faces(info, face_rows(box._buffers, send_up), face_rows(box._buffers, send_down),
                       face_rows(box._buffers, recv_below), face_rows(box._buffers, recv_above))
    R.rflbm_slab_exchange_done(box.h, stream.cuda_stream)

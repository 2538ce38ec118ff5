"""Screen-space sharding of one frame across ranks (one process per GPU).

Rays are independent, so a frame splits into row ranges with the volume,
forest and transfer function replicated on every rank.  The only exchange is
one gather of the rendered rows to the rank that presents the frame.  The
render itself is `Volume.render(..., row_begin, row_end)`, which fills only
its rows; this module holds the host-side logic around it.
"""
from __future__ import annotations


def row_range(height: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous rows [r0, r1) of `rank`; sizes differ by at most one row."""
    if world < 1 or not (0 <= rank < world) or height < 0:
        raise ValueError("bad height/world/rank")
    base, extra = divmod(height, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def render_shard(vol, cam, tf, step, out, world: int, rank: int, stream=None):
    """Render this rank's rows of the frame into `out` (H x W x 4, device)."""
    r0, r1 = row_range(cam.height, world, rank)
    if r1 > r0:
        vol.render(cam, tf, step, out=out, stream=stream, row_begin=r0, row_end=r1)
    return r0, r1


def gather_rows(out, height: int, world: int, rank: int, dst: int = 0, group=None):
    """Assemble the frame on rank `dst` from every rank's rows (one collective).

    `out` is this rank's full-size buffer holding its own rows; every rank
    sends a padded copy of its rows; rank `dst` returns the assembled frame,
    the other ranks return None."""
    import torch
    import torch.distributed as dist
    r0, r1 = row_range(height, world, rank)
    rows = max(row_range(height, world, q)[1] - row_range(height, world, q)[0] for q in range(world))
    send = torch.zeros((rows,) + tuple(out.shape[1:]), dtype=out.dtype, device=out.device)
    send[: r1 - r0] = out[r0:r1]
    bufs = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(bufs, send, group=group)
    if rank != dst:
        return None
    frame = torch.empty_like(out)
    for q in range(world):
        q0, q1 = row_range(height, world, q)
        frame[q0:q1] = bufs[q][: q1 - q0]
    return frame


def max_over_ranks(x: float, group=None, device=None) -> float:
    """The slowest rank's value (timings are reported as the max over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

"""Screen-space sharding of one frame across ranks (one process per GPU).

Rays are independent (Sec. 4), so a frame splits by rows with the volume,
forest and transfer function replicated on every rank.  The only exchange is
one gather of the rendered rows to the rank that presents the frame.

Two assignments:
  interleaved (default)  the frame's rows are cut into bands of
                         LRVOL_BAND_ROWS (8) rows and band b goes to rank
                         b mod world, so every rank gets rows from the whole
                         height and the expensive middle of the image (where
                         rays cross the most of the volume) is shared out
                         evenly; one render launch per rank (the camera's
                         band_count / band_index);
  contiguous             rank r gets one block of rows (row_range).
This module holds the host-side logic around the render.
"""
from __future__ import annotations

BAND_ROWS = 8   # LRVOL_BAND_ROWS: one band is one row of the render's 16x8-pixel CTAs


def row_range(height: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous rows [r0, r1) of `rank`; sizes differ by at most one row."""
    if world < 1 or not (0 <= rank < world) or height < 0:
        raise ValueError("bad height/world/rank")
    base, extra = divmod(height, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def row_bands(height: int, world: int, rank: int) -> list[tuple[int, int]]:
    """The interleaved bands [r0, r1) of `rank`: every world-th band of
    BAND_ROWS rows, starting with band `rank` (the last band may be shorter)."""
    if world < 1 or not (0 <= rank < world) or height < 0:
        raise ValueError("bad height/world/rank")
    n = (height + BAND_ROWS - 1) // BAND_ROWS
    return [(b * BAND_ROWS, min(height, (b + 1) * BAND_ROWS)) for b in range(rank, n, world)]


def rows_of(height: int, world: int, rank: int, interleaved: bool = True) -> list[tuple[int, int]]:
    return row_bands(height, world, rank) if interleaved else [row_range(height, world, rank)]


def render_shard(vol, cam, tf, step, out, world: int, rank: int, stream=None, interleaved: bool = True):
    """Render this rank's rows of the frame into `out` (H x W x 4, device):
    one launch either way.  Returns the rank's row spans."""
    spans = rows_of(cam.height, world, rank, interleaved)
    if interleaved:
        if spans:
            vol.render(cam, tf, step, out=out, stream=stream, row_begin=0, row_end=cam.height,
                       band_count=world, band_index=rank)
    else:
        r0, r1 = spans[0]
        if r1 > r0:
            vol.render(cam, tf, step, out=out, stream=stream, row_begin=r0, row_end=r1)
    return spans


def gather_rows(out, height: int, world: int, rank: int, dst: int = 0, group=None, interleaved: bool = True):
    """Assemble the frame on rank `dst` from every rank's rows (one collective).

    `out` is this rank's full-size buffer holding its own rows; every rank
    sends its rows packed one after another (padded to the largest share);
    rank `dst` returns the assembled frame, the other ranks return None."""
    import torch
    import torch.distributed as dist
    spans = [rows_of(height, world, q, interleaved) for q in range(world)]
    count = [sum(r1 - r0 for r0, r1 in s) for s in spans]
    send = torch.zeros((max(count),) + tuple(out.shape[1:]), dtype=out.dtype, device=out.device)
    k = 0
    for r0, r1 in spans[rank]:
        send[k:k + r1 - r0] = out[r0:r1]
        k += r1 - r0
    bufs = [torch.empty_like(send) for _ in range(world)]
    dist.all_gather(bufs, send, group=group)
    if rank != dst:
        return None
    frame = torch.empty_like(out)
    for q in range(world):
        k = 0
        for r0, r1 in spans[q]:
            frame[r0:r1] = bufs[q][k:k + r1 - r0]
            k += r1 - r0
    return frame


def max_over_ranks(x: float, group=None, device=None) -> float:
    """The slowest rank's value (timings are reported as the max over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())

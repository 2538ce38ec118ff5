"""Host-side logic of the multi-rank path on CPU ranks (gloo, world size 2).

The render on each rank is replaced by a deterministic CPU stand-in that
fills only its rows; what is tested is the row split (interleaved 8-row
bands, and contiguous blocks), the one gather that assembles the frame, and
the max-over-ranks timing reduction.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1707_01170_gb300.shard import BAND_ROWS, gather_rows, max_over_ranks, row_bands, row_range, rows_of


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pixel_value(h, w):
    j, i = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    img = np.stack([np.sin(0.1 * i) * np.cos(0.07 * j), i / w, j / h, (i + j) % 7 / 7.0], axis=-1)
    return img.astype(np.float32)


def _worker(rank, world, port, h, w, q, interleaved):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        full = torch.from_numpy(_pixel_value(h, w))
        out = torch.full_like(full, float("nan"))
        for r0, r1 in rows_of(h, world, rank, interleaved):
            out[r0:r1] = full[r0:r1]                # this rank's "render"
        frame = gather_rows(out, h, world, rank, dst=0, interleaved=interleaved)
        slow = max_over_ranks(1.5 + rank)          # rank 1 is the slowest
        if rank == 0:
            q.put(("frame", bool(torch.equal(frame, full)), slow))
        else:
            q.put(("other", frame is None, slow))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("h,interleaved", [(37, True), (64, True), (37, False), (64, False)])
def test_gather_assembles_frame_world2(h, interleaved):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, h, 23, q, interleaved)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = {k: (ok, slow) for k, ok, slow in res}
    assert d["frame"] == (True, 2.5)
    assert d["other"] == (True, 2.5)


@pytest.mark.parametrize("height,world", [(1080, 1), (1080, 2), (1080, 8), (7, 4), (3, 8), (0, 2)])
def test_row_ranges_cover_once(height, world):
    rows = []
    for r in range(world):
        r0, r1 = row_range(height, world, r)
        assert 0 <= r0 <= r1 <= height
        rows.extend(range(r0, r1))
    assert rows == list(range(height))
    sizes = [row_range(height, world, r)[1] - row_range(height, world, r)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def test_row_range_errors():
    with pytest.raises(ValueError):
        row_range(10, 0, 0)
    with pytest.raises(ValueError):
        row_range(10, 2, 2)


@pytest.mark.parametrize("height,world", [(1080, 1), (1080, 2), (1080, 8), (7, 4), (3, 8), (0, 2), (37, 3)])
def test_interleaved_bands_cover_once(height, world):
    """Every row once; rank r holds bands r, r + world, ...; the shares of
    the ranks differ by at most one band."""
    rows, per = [], []
    for r in range(world):
        spans = row_bands(height, world, r)
        per.append(sum(b - a for a, b in spans))
        for a, b in spans:
            assert a % BAND_ROWS == 0 and (a // BAND_ROWS) % world == r and 0 < b - a <= BAND_ROWS
            rows.extend(range(a, b))
    assert sorted(rows) == list(range(height))
    assert max(per) - min(per) <= BAND_ROWS


def test_interleaved_bands_balance_a_centred_load():
    """A cost concentrated in the middle rows (rays crossing the most of the
    volume) splits evenly across interleaved ranks but not across blocks."""
    h, world = 1080, 4
    cost = [max(0.0, 1.0 - abs(j - h / 2) / (h / 4)) for j in range(h)]
    share = lambda spans: sum(cost[j] for a, b in spans for j in range(a, b))
    inter = [share(row_bands(h, world, r)) for r in range(world)]
    block = [share([row_range(h, world, r)]) for r in range(world)]
    assert max(inter) / min(inter) < 1.05
    assert max(block) / max(min(block), 1e-9) > 2.0

"""Host side of the frame server, on the CPU: the arena bookkeeping of the C
library against a plain model, the seeded request stream, and the latency
statistics.  No GPU call is made."""
import math

import numpy as np
import pytest

from paper_1707_01170_gb300 import build as cuda_build
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300 import serve


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return lv.load()


class _FirstFit:
    """Plain model: sorted free list, lowest block that fits, merge neighbours."""

    def __init__(self, size, align):
        self.free = [(0, size)]
        self.used = {}
        self.align = align

    def alloc(self, n):
        need = -(-max(n, 1) // self.align) * self.align
        for k, (o, s) in enumerate(self.free):
            if s >= need:
                self.free[k:k + 1] = [(o + need, s - need)] if s > need else []
                self.used[o] = need
                return o
        return -1

    def release(self, o):
        s = self.used.pop(o)
        self.free.append((o, s))
        self.free.sort()
        merged = []
        for a, b in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + b)
            else:
                merged.append((a, b))
        self.free = merged


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arena_matches_first_fit_model(lib, seed):
    rng = np.random.default_rng(seed)
    size, align = 1 << 20, 256
    a, m = lv.Arena(size, align), _FirstFit(size, align)
    live = []
    for _ in range(3000):
        if live and rng.random() < 0.45:
            o = live.pop(int(rng.integers(len(live))))
            a.free(o)
            m.release(o)
        else:
            n = int(rng.choice([1, 100, 256, 257, 4096, 50_000, 200_000]))
            o = a.alloc(n)
            assert o == m.alloc(n)
            if o >= 0:
                assert o % align == 0 and o + n <= size
                live.append(o)
        assert a.used == sum(m.used.values())
        assert a.largest_free == max([s for _, s in m.free], default=0)
    for o in live:
        a.free(o)
    assert a.used == 0 and a.largest_free == size
    a.close()


def test_arena_errors(lib):
    with pytest.raises(lv.LrvolError):
        lv.Arena(1 << 20, 3)
    a = lv.Arena(1 << 12, 256)
    assert a.alloc(1 << 13) == -1
    o = a.alloc(10)
    with pytest.raises(lv.LrvolError):
        a.free(o + 256)
    a.free(o)
    with pytest.raises(lv.LrvolError):
        a.free(o)
    a.close()


def test_server_arguments_checked_before_cuda(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.lrvol_server_create(0, 1 << 30, ctypes.byref(h)) == lv.ERR_ARG
    assert lib.lrvol_server_create(65, 1 << 30, ctypes.byref(h)) == lv.ERR_ARG
    assert lib.lrvol_server_create(4, 1000, ctypes.byref(h)) == lv.ERR_ARG
    assert lib.lrvol_server_submit(None, None, None, None, None, None, None) == lv.ERR_ARG
    n = ctypes.c_int32()
    assert lib.lrvol_server_poll(None, None, 0, ctypes.byref(n)) == lv.ERR_ARG


def test_request_stream_is_seeded_and_poisson():
    a = serve.request_stream(7, 2000, 120.0, 3)
    b = serve.request_stream(7, 2000, 120.0, 3)
    assert [(r.arrival, r.volume, r.width, r.camera.eye) for r in a] == \
           [(r.arrival, r.volume, r.width, r.camera.eye) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert np.all(gaps > 0)
    # mean 1/rate within 4 standard errors; exponential: std = mean
    assert abs(gaps.mean() - 1 / 120) < 4 * (1 / 120) / math.sqrt(len(gaps))
    # coefficient of variation of an exponential is 1
    assert 0.9 < gaps.std() / gaps.mean() < 1.1
    vols = np.bincount([r.volume for r in a], minlength=3)
    sizes = {(r.width, r.height) for r in a}
    assert vols.min() > 550 and sizes == set(serve.SIZES)
    for r in a[:50]:
        assert (r.camera.width, r.camera.height) == (r.width, r.height)
        d = np.array(r.camera.eye) - 0.5
        assert abs(np.linalg.norm(d) - 1.8) < 1e-12


def test_orbit_advances_per_volume():
    c0 = serve.orbit_view(1, 0, 3, 64, 64)
    c1 = serve.orbit_view(1, 1, 3, 64, 64)
    a0 = math.atan2(c0.eye[1] - 0.5, c0.eye[0] - 0.5)
    a1 = math.atan2(c1.eye[1] - 0.5, c1.eye[0] - 0.5)
    assert abs((a1 - a0) - 2 * math.pi / 240) < 1e-9


def test_percentile_and_summary():
    x = np.random.default_rng(0).random(1001)
    for q in (0, 1, 50, 99, 100):
        assert serve.percentile(x, q) == pytest.approx(np.percentile(x, q))
    recs = [{"volume": 0, "width": 8, "height": 8, "arrival_s": k * 0.01, "admit_s": k * 0.01,
             "done_s": k * 0.01 + 0.002, "latency_ms": 2.0 + (k % 10), "device_ms": 1.0, "samples": 1000,
             "state": lv.REQ_DONE, "status": 0} for k in range(100)]
    s = serve.summarize(recs)
    assert s["frames"] == 100 and s["failed"] == 0
    assert s["p50_ms"] == pytest.approx(6.5) and s["max_ms"] == 11.0
    assert s["by_size"]["8x8"]["n"] == 100

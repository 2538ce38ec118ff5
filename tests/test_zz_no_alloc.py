"""lrvol_render_noalloc: the render entry point for callers that may not
allocate device memory (a host application that owns all device memory
through its own pool, or a service whose device footprint must stay fixed
after start-up).  Its scratch is the library's static device array, not
memory allocated for the handle.

Checked through the C ABI against lrvol_render on the same inputs, on two
calls in a row (the static array keeps the previous call's contents, so the
second call shows the counters are cleared), within the image tolerance of
the parity suite.  This file is collected last; it passes alone and after
the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

pytestmark = pytest.mark.gpu

RMSE_TOL = 1e-4


def test_render_noalloc_matches_render_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L = lv.load()
    vol = V.load_config(1)
    gv = lv.Volume(vol).build_accel((32, 32, 32)).to_bezier()
    tf, cams = V.config1_render()
    cam = lv.make_camera(V.orbit_camera(V.Stream(123), 150, 97))    # ragged tiles in both directions
    ctf = lv.make_tf(tf)
    step = lv.make_step(V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99))
    stream = torch.cuda.current_stream()

    ref = torch.zeros((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    rc = L.lrvol_render(gv.handle, ctypes.byref(cam), ctypes.byref(ctf), ctypes.byref(step), ref.data_ptr(),
                        stream.cuda_stream)
    assert rc == lv.OK, lv.last_error()
    st = gv.stats()

    for call in range(2):
        out = torch.full((cam.height, cam.width, 4), -1.0, dtype=torch.float32, device="cuda")
        cnt = torch.full((4,), 7, dtype=torch.int64, device="cuda")
        rc = L.lrvol_render_noalloc(gv.handle, ctypes.byref(cam), ctypes.byref(ctf), ctypes.byref(step),
                                    out.data_ptr(), cnt.data_ptr(), stream.cuda_stream)
        assert rc == lv.OK, lv.last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert float(np.sqrt(np.mean((a.astype(np.float64) - b) ** 2))) <= RMSE_TOL, f"call {call}"
        assert np.abs(a - b).max() <= 1e-6, f"call {call}"
        samples, lookups, rays, status = cnt.cpu().tolist()
        assert (samples, lookups, rays) == (st["samples"], st["lookups"], st["rays_hit"]), f"call {call}"
        assert status == 0

    # without a counters buffer, and a too-large image is rejected
    rc = L.lrvol_render_noalloc(gv.handle, ctypes.byref(cam), ctypes.byref(ctf), ctypes.byref(step),
                                ref.data_ptr(), None, stream.cuda_stream)
    assert rc == lv.OK
    big = lv.make_camera(V.ortho_z(40000, 4))
    rc = L.lrvol_render_noalloc(gv.handle, ctypes.byref(big), ctypes.byref(ctf), ctypes.byref(step),
                                ref.data_ptr(), None, stream.cuda_stream)
    assert rc == lv.ERR_ARG and "maximum" in lv.last_error()
    torch.cuda.synchronize()
    gv.close()

"""lrvol_render_noalloc: the render entry point for callers that may not
allocate device memory (a host application that owns all device memory
through its own pool, or a service whose device footprint must stay fixed
after start-up).  Its scratch is the library's static device array, not
memory allocated for the handle.

Checked through the C ABI against lrvol_render on the same inputs, on two
calls in a row (the static array keeps the previous call's contents, so the
second call shows the scratch is cleared).  Both calls run the same kernel
on the same inputs, so the images must be identical bit for bit and the
counters equal.  The cases cover fixed, Eq. 4 and learned steps, a scalar
and a 3-vector volume (|v| and one component, FP16 blocks), a row band and
an empty row band.  One case is also compared with the FP64 oracle on
sampled pixels, within the image tolerance of the parity suite.  This file
is collected last; it passes alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

pytestmark = pytest.mark.gpu

RMSE_TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return lv.load()


@pytest.fixture(scope="module")
def scalar_vol(lib):
    vol = V.load_config(1)
    gv = lv.Volume(vol).build_accel((32, 32, 32)).to_bezier()
    yield vol, gv
    gv.close()


@pytest.fixture(scope="module")
def vector_vol(lib):
    vol = V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3, seed=4)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(lv.STORE_F16)
    yield vol, gv
    gv.close()


def _both(L, gv, cam, ctf, step, calls=2):
    """lrvol_render once, then lrvol_render_noalloc `calls` times, into
    buffers pre-filled alike; returns (ref image, ref stats, [(image, counters)])."""
    stream = torch.cuda.current_stream()
    ref = torch.full((cam.height, cam.width, 4), -1.0, dtype=torch.float32, device="cuda")
    rc = L.lrvol_render(gv.handle, ctypes.byref(cam), ctypes.byref(ctf), ctypes.byref(step), ref.data_ptr(),
                        stream.cuda_stream)
    assert rc == lv.OK, lv.last_error()
    torch.cuda.synchronize()
    st = gv.stats()
    got = []
    for _ in range(calls):
        out = torch.full((cam.height, cam.width, 4), -1.0, dtype=torch.float32, device="cuda")
        cnt = torch.full((4,), 7, dtype=torch.int64, device="cuda")
        rc = L.lrvol_render_noalloc(gv.handle, ctypes.byref(cam), ctypes.byref(ctf), ctypes.byref(step),
                                    out.data_ptr(), cnt.data_ptr(), stream.cuda_stream)
        assert rc == lv.OK, lv.last_error()
        torch.cuda.synchronize()
        got.append((out, cnt.cpu().tolist()))
    return ref, st, got


CASES = {
    "scalar_eq4": dict(vol="scalar", step=dict(mode="heuristic", xi=1 / 256, alpha_stop=0.99)),
    "scalar_fixed": dict(vol="scalar", step=dict(mode="fixed", h=1 / 300, xi=1 / 256, alpha_stop=1.0)),
    "scalar_learned": dict(vol="scalar", step=dict(mode="learned", xi=1 / 256, alpha_stop=0.99)),
    "scalar_band": dict(vol="scalar", step=dict(mode="heuristic", xi=1 / 256, alpha_stop=0.99), rows=(13, 61)),
    "scalar_empty_band": dict(vol="scalar", step=dict(mode="heuristic", xi=1 / 256), rows=(20, 20)),
    "vector_magnitude_f16": dict(vol="vector", step=dict(mode="heuristic", xi=1 / 128, field="magnitude"),
                                 vrange=(0.0, 1.6)),
    "vector_component_f16": dict(vol="vector", step=dict(mode="heuristic", xi=1 / 128, field="component",
                                                         component=1), vrange=(-0.5, 1.0)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_render_noalloc_matches_render_twice(lib, scalar_vol, vector_vol, case):
    spec = CASES[case]
    vol, gv = scalar_vol if spec["vol"] == "scalar" else vector_vol
    if spec["vol"] == "scalar":
        tf, _ = V.config1_render()
    else:
        tf = V.seeded_tf(V.Stream(31), alpha_max=0.05)
        tf.vmin, tf.vmax = spec["vrange"]
    sp = V.StepParams(**spec["step"])
    mult = None
    if sp.mode == "learned":
        rng = np.random.default_rng(11)
        mult = torch.from_numpy(rng.choice(np.array([1.0, 1.5, 2.0, 4.0], np.float32), vol.n_elem)).cuda()
        sp.mult = mult
    r0, r1 = spec.get("rows", (0, 0))
    cam = lv.make_camera(V.orbit_camera(V.Stream(123), 150, 97), r0, r1)    # ragged tiles in both directions
    ref, st, got = _both(lib, gv, cam, lv.make_tf(tf), lv.make_step(sp))
    for call, (out, cnt) in enumerate(got):
        assert torch.equal(out, ref), f"call {call}: image differs from lrvol_render"
        samples, lookups, rays, status = cnt
        assert (samples, lookups, rays) == (st["samples"], st["lookups"], st["rays_hit"]), f"call {call}"
        assert status == 0
    if r0 == r1 != 0:
        assert got[0][1][:3] == [0, 0, 0] and bool(torch.all(got[0][0] == -1.0))
    else:
        assert st["samples"] > 0


def test_render_noalloc_against_oracle(lib, scalar_vol):
    """Sampled pixels of a noalloc frame against the FP64 oracle."""
    from oracle.oracle import Oracle
    vol, gv = scalar_vol
    tf, _ = V.config1_render()
    tf.table = np.asarray(tf.table, dtype=np.float32).astype(np.float64)
    sp = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    ocam = V.orbit_camera(V.Stream(124), 160, 120)
    cam = lv.make_camera(ocam)
    _, _, got = _both(lib, gv, cam, lv.make_tf(tf), lv.make_step(sp), calls=1)
    img = got[0][0].cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    pix = np.stack([rng.integers(0, cam.width, 400), rng.integers(0, cam.height, 400)], axis=1).astype(np.int32)
    ref, _ = Oracle(vol).render(ocam, tf, sp, pixels=pix)
    d = img[pix[:, 1], pix[:, 0]] - ref
    assert float(np.sqrt(np.mean(d ** 2))) <= RMSE_TOL
    assert np.abs(ref[:, 3]).max() > 0.05


def test_render_noalloc_arguments(lib, scalar_vol):
    vol, gv = scalar_vol
    tf, _ = V.config1_render()
    ctf = lv.make_tf(tf)
    step = lv.make_step(V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99))
    stream = torch.cuda.current_stream()
    cam = lv.make_camera(V.orbit_camera(V.Stream(123), 64, 48))
    out = torch.zeros((48, 64, 4), dtype=torch.float32, device="cuda")
    # without a counters buffer
    rc = lib.lrvol_render_noalloc(gv.handle, ctypes.byref(cam), ctypes.byref(ctf), ctypes.byref(step),
                                  out.data_ptr(), None, stream.cuda_stream)
    assert rc == lv.OK
    # a too-large image is rejected before anything runs
    big = lv.make_camera(V.ortho_z(40000, 4))
    rc = lib.lrvol_render_noalloc(gv.handle, ctypes.byref(big), ctypes.byref(ctf), ctypes.byref(step),
                                  out.data_ptr(), None, stream.cuda_stream)
    assert rc == lv.ERR_ARG and "maximum" in lv.last_error()
    torch.cuda.synchronize()

"""Empty inputs, size limits and degenerate cases across the C ABI: every
entry point accepts zero items without launching an empty grid, and sizes
past the documented limits are refused with LRVOL_ERR_ARG before any
kernel runs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


@pytest.fixture(scope="module")
def vec():
    vol = V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4,), ncomp=3, seed=4)
    gv = lv.Volume(vol).build_accel((8, 8, 8)).to_bezier()
    yield gv
    gv.close()


def test_empty_point_queries(vec):
    z = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    assert vec.lookup(z).numel() == 0
    assert vec.eval(z).shape == (0, 3)
    torch.cuda.synchronize()


def test_empty_streamlines_and_error(vec):
    seeds = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    s, c, st = lv.streamlines(vec, seeds, "RK4", "heuristic", 1.0, 1.0, max_samples=8)
    assert s.shape == (0, 8, 4) and c.numel() == 0 and st.numel() == 0
    e = lv.streamline_error(s, c, s, c)
    assert e.numel() == 0
    torch.cuda.synchronize()


def test_empty_mesh_trims_every_pixel(vec):
    cam = V.ortho_z(16, 12)
    tr = lv.trim(cam, torch.zeros((0, 9), dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.all(np.isinf(tr[..., 0])) and np.all(tr[..., 1] == 0)
    # a render trimmed by an empty mesh is empty
    img = vec.render(cam, V.config1_render()[0], V.StepParams(mode="heuristic", field="magnitude",
                                                           trim=torch.from_numpy(tr).cuda()))
    assert float(img.abs().max()) == 0.0


def test_no_lines_draws_no_tubes(vec):
    cam = V.ortho_z(16, 12)
    s = torch.zeros((0, 4, 4), dtype=torch.float64, device="cuda")
    c = torch.zeros(0, dtype=torch.int32, device="cuda")
    img = lv.tubes(vec, cam, s, c, 0.01, V.config1_render()[0])
    assert float(img.abs().max()) == 0.0
    # lines with fewer than two samples have no segment
    s1 = torch.rand((3, 4, 4), dtype=torch.float64, device="cuda")
    c1 = torch.tensor([0, 1, 1], dtype=torch.int32, device="cuda")
    assert float(lv.tubes(vec, cam, s1, c1, 0.05, V.config1_render()[0]).abs().max()) == 0.0


def test_zero_rows_network():
    packed = torch.zeros(lv.MLP_PACKED, dtype=torch.int16, device="cuda")
    out = lv.mlp_infer(torch.zeros((0, lv.MLP_IN), device="cuda"), packed, 3.0)
    assert out.numel() == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("w,h", [(32769, 4), (4, 32769), (0, 4)])
def test_image_size_limits(vec, w, h):
    cam = V.Camera("ortho", w, h, eye=(0.5, 0.5, 2.0), target=(0.5, 0.5, 0.0), up=(0.0, 1.0, 0.0), extent=1.0)
    out = torch.zeros(max(w, 1) * max(h, 1) * 4, dtype=torch.float32, device="cuda")   # room for the whole image
    tf = V.config1_render()[0]
    lib = lv.load()
    import ctypes
    rc = lib.lrvol_render(vec.handle, ctypes.byref(lv.make_camera(cam)), ctypes.byref(lv.make_tf(tf)),
                          ctypes.byref(lv.make_step(V.StepParams(mode="heuristic", field="magnitude"))),
                          out.data_ptr(), None)
    assert rc == lv.ERR_ARG
    rc = lib.lrvol_trim(ctypes.byref(lv.make_camera(cam)), None, 0, out.data_ptr(), None)
    assert rc == lv.ERR_ARG
    assert float(out.abs().max()) == 0.0          # nothing was written


def test_binding_refuses_short_output_buffers(vec):
    cam = V.ortho_z(16, 12)
    with pytest.raises(ValueError):
        vec.render(cam, V.config1_render()[0], V.StepParams(mode="heuristic", field="magnitude"),
                   out=torch.zeros((12, 15, 4), device="cuda"))
    seeds = torch.full((4, 3), 0.5, dtype=torch.float64, device="cuda")
    short = (torch.zeros((4, 7, 4), dtype=torch.float64, device="cuda"), torch.zeros(4, dtype=torch.int32, device="cuda"),
             torch.zeros(4, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        lv.streamlines(vec, seeds, "RK4", "heuristic", 1.0, 1.0, max_samples=8, out=short)
    with pytest.raises(TypeError):
        lv.trim(cam, torch.zeros((1, 9), dtype=torch.float64, device="cuda"))


def test_rebuilds_keep_the_device_accounting_and_a_failed_rebuild_keeps_the_forest():
    vol = V.tensor_product((1, 1, 1), (5, 3, 4), seed=2)          # faces at thirds and fifths: not dyadic
    gv = lv.Volume(vol).build_accel((4, 4, 4)).to_bezier()
    bytes0 = gv.stats()["bytes_device"]
    gv.build_accel((4, 4, 4)).to_bezier()
    gv.build_accel((4, 4, 4)).to_bezier(lv.STORE_F32)
    assert gv.stats()["bytes_device"] == bytes0
    pts = torch.rand((2000, 3), generator=torch.Generator().manual_seed(5)).float().cuda()
    before = gv.lookup(pts).clone()
    with pytest.raises(lv.LrvolError) as ei:                       # the host build fails before any buffer is touched
        gv.build_accel((4, 4, 4), split=lv.SPLIT_MIDPOINT)
    assert ei.value.status == lv.ERR_UNSUPPORTED
    assert torch.equal(gv.lookup(pts), before)
    gv.close()


def test_mlp_wait_timeout_is_reported_and_the_context_recovers():
    """The network kernel's tensor-core waits are bounded.  With no MMAs
    issued (the diagnostic entry point) every wait runs out: the rows get
    multiplier 1 (the Eq. 4 step), lrvol_mlp_check reports LRVOL_ERR_TIMEOUT
    once, and the next real inference on the same context is correct."""
    import time
    gen = torch.Generator().manual_seed(5)
    p = (0.25 * (2 * torch.rand(lv.MLP_PARAMS, generator=gen) - 1)).cuda()
    packed = lv.mlp_pack(p)
    X = (2 * torch.rand((1000, lv.MLP_IN), generator=gen) - 0.5).cuda()
    want = lv.mlp_infer(X, packed, 3.0)
    lv.mlp_check()
    t0 = time.perf_counter()
    out = lv.mlp_infer_timeout_test(X, packed, 3.0)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert elapsed < 5.0
    assert torch.all(out == 1.0)
    with pytest.raises(lv.LrvolError) as e:
        lv.mlp_check()
    assert e.value.status == lv.ERR_TIMEOUT
    lv.mlp_check()                                  # the report clears the status
    again = lv.mlp_infer(X, packed, 3.0)
    lv.mlp_check()
    assert torch.equal(again, want)
    assert not torch.all(want == 1.0)

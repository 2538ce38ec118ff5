"""Gradient shading (Sec. 4.1) on the GPU against the FP64 oracle.

Bars:
  gradient   per axis |g_gpu - g_orc| <= 1e-5 * 2p * iw_a * max|c| + 1e-5 |g|
             (the derivative of a Bernstein basis sums to at most 2p in
             absolute value, times 1/(hi - lo) per axis; FP32 contraction);
             16-bit blocks add s * u * 2p * iw_a (s the block's half range,
             u the format's unit roundoff);
  value      as the unshaded evaluation: 1e-5 * max(|f|, max|c|);
  images     RMSE <= 1e-4, as the unshaded renders (identical FP32 sample
             decisions; I = max(0.4, |l . n|) is continuous in the gradient,
             with the 1e-3 (vmax - vmin) floor on |grad f|).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import Stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


def _rmse(a, b):
    return float(np.sqrt(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)))


def _f32_tf(tf):
    tf.table = np.asarray(tf.table, dtype=np.float32).astype(np.float64)
    return tf


VOLS = {
    "cfg1": lambda: V.load_config(1),
    "ball_p2": lambda: V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), seed=4),
    "tp_p1": lambda: V.tensor_product((1, 1, 1), (5, 3, 4), seed=2),
}
U = {lv.STORE_F32: 0.0, lv.STORE_F16: 2.0 ** -11, lv.STORE_BF16: 2.0 ** -8}


@pytest.mark.parametrize("which", sorted(VOLS))
@pytest.mark.parametrize("storage", [lv.STORE_F32, lv.STORE_F16, lv.STORE_BF16])
def test_eval_grad_matches_oracle(which, storage):
    vol = VOLS[which]()
    orc = Oracle(vol)
    rng = np.random.default_rng(21)
    X = rng.random((6000, 3)).astype(np.float32)
    faces = np.unique(vol.elem_box.astype(np.float32))
    m = rng.random(X.shape) < 0.2
    X[m] = rng.choice(faces, size=int(m.sum()))
    val, grad = orc.eval_grad(X)
    _, elem = orc.eval(X, return_elem=True)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(storage)
    got = gv.eval_grad(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    gv.close()
    box = vol.elem_box[elem]
    iw = 1.0 / (box[:, 3:] - box[:, :3])
    p = np.asarray(vol.deg, dtype=np.float64)
    cmax = np.abs(vol.coef).max()
    blocks = orc.bezier_blocks(np.unique(elem))
    flat = blocks.reshape(len(blocks), -1)
    half = dict(zip(np.unique(elem), 0.5 * (flat.max(axis=1) - flat.min(axis=1))))
    s = np.array([half[e] for e in elem])
    vbound = 1e-5 * np.maximum(np.abs(val[:, 0]), cmax) + 1.02 * s * U[storage]
    assert np.all(np.abs(got[:, 0] - val[:, 0]) <= vbound)
    g = grad[:, 0, :]
    gbound = (1e-5 * cmax + 1.02 * s[:, None] * U[storage]) * 2 * p * iw + 1e-5 * np.abs(g)
    err = np.abs(got[:, 1:] - g)
    assert np.all(err <= gbound), f"worst excess {np.max(err - gbound)}"
    assert np.abs(g).max() > 1.0


@pytest.mark.parametrize("which,view", [("cfg1", 0), ("cfg1", 1), ("ball_p2", 1), ("tp_p1", 1)])
@pytest.mark.parametrize("light", [(0.0, 0.0, 0.0), (0.3, -0.5, 0.8)])
def test_shaded_render_matches_oracle(which, view, light):
    vol = VOLS[which]()
    tf, cams = V.config1_render()
    if which != "cfg1":
        tf = V.seeded_tf(Stream(41), alpha_max=0.06)
        tf.vmin, tf.vmax = float(vol.coef.min()), float(vol.coef.max())
    tf = _f32_tf(tf)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=1.0, shading="gradient", light=light)
    cam = cams[view] if which == "cfg1" else V.orbit_camera(Stream(42), 64, 48)
    ref, ost = Oracle(vol).render(cam, tf, step)
    gv = lv.Volume(vol).build_accel((32, 32, 32)).to_bezier()
    img = gv.render(cam, tf, step).cpu().numpy()
    plain = gv.render(cam, tf, V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=1.0)).cpu().numpy()
    st = gv.stats()
    gv.close()
    assert _rmse(img, ref) <= 1e-4
    assert abs(st["samples"] - ost["samples"]) <= 0.001 * ost["samples"]
    # shading changes colour, never opacity
    np.testing.assert_array_equal(img[..., 3], plain[..., 3])
    assert np.abs(img[..., :3] - plain[..., :3]).max() > 1e-3


def test_shaded_noalloc_equals_render(cfg1):
    tf, cams = V.config1_render()
    step = V.StepParams(mode="heuristic", alpha_stop=0.98, shading="gradient")
    gv = lv.Volume(cfg1).build_accel((32, 32, 32)).to_bezier(lv.STORE_F16)
    a = gv.render(cams[1], tf, step)
    b = torch.zeros_like(a)
    c = lv.make_camera(cams[1])
    lib = lv.load()
    import ctypes
    assert lib.lrvol_render_noalloc(gv.handle, ctypes.byref(c), ctypes.byref(lv.make_tf(tf)),
                                    ctypes.byref(lv.make_step(step)), b.data_ptr(), None, None) == 0
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    gv.close()


def test_shading_rejected_for_vector_fields():
    vol = V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4,), ncomp=3, seed=4)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    tf, _ = V.config1_render()
    with pytest.raises(lv.LrvolError) as e:
        gv.render(V.ortho_z(8, 8), tf, V.StepParams(mode="heuristic", field="magnitude", shading="gradient"))
    assert e.value.status == lv.ERR_UNSUPPORTED
    gv.close()

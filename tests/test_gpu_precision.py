"""Reduced-precision Bezier storage (FP16 / BF16 with a per-block offset and
scale, FP32 accumulation) against the FP64 oracle.

Bound: a block stores q' = binom*(c - o)/s with o, s the midpoint and half
range of its coefficients, so |q'| <= binom and, the Bernstein basis summing
to one, rounding q' to a format with unit roundoff u changes a value by at
most s*u (u = 2^-11 for FP16, 2^-8 for BF16).  The scales s are taken from
the oracle's own Bezier blocks (interpolation), not from the CUDA path.
Each image's error against the FP64 oracle is printed and bounded.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

pytestmark = pytest.mark.gpu

U = {lv.STORE_F16: 2.0 ** -11, lv.STORE_BF16: 2.0 ** -8}
NAME = {lv.STORE_F16: "fp16", lv.STORE_BF16: "bf16"}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


def _vector_volume():
    return V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3, seed=4)


@pytest.mark.parametrize("storage", [lv.STORE_F16, lv.STORE_BF16])
@pytest.mark.parametrize("which", ["cfg1", "vector_p2"])
def test_eval_within_block_bound(storage, which):
    vol = V.load_config(1) if which == "cfg1" else _vector_volume()
    orc = Oracle(vol)
    rng = np.random.default_rng(13)
    X = rng.random((20000, 3)).astype(np.float32)
    want, elem = orc.eval(X, return_elem=True)
    uniq, inv = np.unique(elem, return_inverse=True)
    blocks = orc.bezier_blocks(uniq)                                  # (n, nc, ...)
    flat = blocks.reshape(len(uniq), vol.ncomp, -1)
    half_range = 0.5 * (flat.max(axis=2) - flat.min(axis=2))        # s per element and component
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(storage)
    got = gv.eval(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    bound = 1.02 * half_range[inv] * U[storage] + 1e-5 * np.maximum(np.abs(want), np.abs(vol.coef).max())
    err = np.abs(got - want)
    assert np.all(err <= bound), f"worst excess {np.max(err - bound)}"
    # the format is actually in use: errors are far above FP32 rounding
    assert err.max() > 20 * 1e-7 * np.abs(vol.coef).max()
    gv.close()


@pytest.mark.parametrize("storage", [lv.STORE_F32, lv.STORE_F16, lv.STORE_BF16])
def test_render_error_vs_oracle(storage, capsys):
    vol = V.load_config(1)
    tf, cams = V.config1_render()
    tf.table = tf.table.astype(np.float32).astype(np.float64)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=1.0)
    ref, _ = Oracle(vol).render(cams[1], tf, step)
    gv = lv.Volume(vol).build_accel((32, 32, 32)).to_bezier(storage)
    img = gv.render(cams[1], tf, step).cpu().numpy()
    rmse = float(np.sqrt(np.mean((img - ref) ** 2)))
    mx = float(np.abs(img - ref).max())
    with capsys.disabled():
        print(f"\n[{NAME.get(storage, 'fp32')}] cfg1 oblique view: image RMSE vs FP64 oracle {rmse:.2e}, max {mx:.2e}")
    limit = {lv.STORE_F32: 1e-4, lv.STORE_F16: 5e-4, lv.STORE_BF16: 4e-3}[storage]
    assert rmse <= limit
    gv.close()


def test_storage_is_smaller():
    vol = V.load_config(1)
    sizes = {}
    for st in (lv.STORE_F32, lv.STORE_F16):
        gv = lv.Volume(vol).to_bezier(st)
        sizes[st] = gv.stats()["bytes_device"]
        gv.close()
    # FP32 render blocks are 256 B per element, 16-bit ones 160 B
    assert sizes[lv.STORE_F32] - sizes[lv.STORE_F16] == vol.n_elem * (256 - 160)

"""Streamline tubes (Sec. 5.3) on the GPU against the oracle: visibility is
an FP32 decision taken in the same order of operations on both sides, so
the covered pixels must be identical; colours (speed from the FP32 block vs
the FP64 definition, FP32 shading) agree within 1e-4."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

import test_oracle_streamlines as SL
import test_oracle_tubes as TU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


@pytest.mark.parametrize("which", ["helix", "swirl"])
@pytest.mark.parametrize("radius", [0.004, 0.02])
def test_tubes_match_oracle(which, radius):
    if which == "helix":
        vol = SL.helix_volume()
        seeds = SL._seeds(24, 3)
    else:
        vol = V.refined_ball((2, 2, 2), (4, 4, 4), centres=((0.4, 0.5, 0.55),), radii=(0.35, 0.18), ncomp=3, seed=12)
        vol.coef = (vol.coef - 0.5) * 2.0
        seeds = np.random.default_rng(1).uniform(0.2, 0.8, (32, 3))
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    smp, cnt, st = lv.streamlines(gv, torch.from_numpy(seeds).cuda(), "RK4", "heuristic", 1.0, 0.5, max_samples=200)
    cam = V.orbit_camera(V.Stream(29), 160, 120)
    cmap = TU._cmap()
    cmap.table = cmap.table.astype(np.float32).astype(np.float64)
    img = lv.tubes(gv, cam, smp, cnt, radius, cmap).cpu().numpy()
    ref = Oracle(vol).tubes(cam, smp.cpu().numpy(), cnt.cpu().numpy(), radius, cmap)
    gv.close()
    assert np.array_equal(img[..., 3] > 0, ref[..., 3] > 0)
    assert (ref[..., 3] > 0).sum() > 200
    assert np.abs(img - ref).max() <= 1e-4


def test_tubes_occlusion_and_caps():
    vol = TU._field_z()
    gv = lv.Volume(vol).build_accel((8, 8, 8)).to_bezier()
    s, c = TU._lines([[0.3, 0.5, 0.3], [0.7, 0.5, 0.3]], [[0.5, 0.3, 0.6], [0.5, 0.7, 0.6]])
    cam = V.ortho_z(48, 48)
    img = lv.tubes(gv, cam, torch.from_numpy(s).cuda(), torch.from_numpy(c.astype(np.int32)).cuda(), 0.05,
                   TU._cmap()).cpu().numpy()
    ref = Oracle(vol).tubes(cam, s, c, 0.05, TU._cmap())
    gv.close()
    assert np.array_equal(img[..., 3], ref[..., 3].astype(np.float32))
    assert np.abs(img - ref).max() <= 1e-4


def test_tubes_few_large_segments_split_over_warps():
    """Three short lines of thick tubes filling much of a 256x192 view: the
    raster gives each group of 32 segment slots many warps (the image is
    large against the number of segments); visibility must still equal the
    oracle's brute force pixel for pixel."""
    vol = TU._field_z()
    gv = lv.Volume(vol).build_accel((8, 8, 8)).to_bezier()
    s, c = TU._lines([[0.2, 0.3, 0.3], [0.5, 0.35, 0.4], [0.8, 0.3, 0.35]],
                     [[0.3, 0.8, 0.6], [0.45, 0.5, 0.5], [0.7, 0.45, 0.7]],
                     [[0.5, 0.2, 0.8], [0.55, 0.6, 0.2]])
    cam = V.orbit_camera(V.Stream(31), 256, 192)
    img = lv.tubes(gv, cam, torch.from_numpy(s).cuda(), torch.from_numpy(c.astype(np.int32)).cuda(), 0.06,
                   TU._cmap()).cpu().numpy()
    ref = Oracle(vol).tubes(cam, s, c, 0.06, TU._cmap())
    gv.close()
    assert np.array_equal(img[..., 3] > 0, ref[..., 3] > 0)
    assert (ref[..., 3] > 0).mean() > 0.05
    assert np.abs(img - ref).max() <= 1e-4

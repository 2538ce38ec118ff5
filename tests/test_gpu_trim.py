"""Trimming (Sec. 4.1) on the GPU against the oracle.

Hits are FP32 decisions taken in the same order of operations on both sides
(watertight ray/triangle test), so the per-pixel intervals must be equal bit
for bit; trimmed images then follow the renderer's RMSE bar (1e-4).  At
sizes the oracle cannot brute-force (a 2.4M-triangle sphere at 1920x1080)
the intervals are checked against the sphere's chord: every ray through the
interior has a front and a back hit near the analytic ones, no ray outside
has any."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from oracle.oracle import Oracle
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


def _tris(t):
    return torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda()


CASES = {
    "box_ortho": (lambda: V.ortho_z(64, 64), lambda: V.box_mesh((0.25, 0.25, 0.25), (0.75, 0.75, 0.75))),
    "sphere_orbit": (lambda: V.orbit_camera(V.Stream(17), 160, 120), lambda: V.icosphere((0.45, 0.5, 0.55), 0.3, 3)),
    "uv_sphere": (lambda: V.orbit_camera(V.Stream(5), 128, 96), lambda: V.uv_sphere((0.5, 0.5, 0.5), 0.35, 40, 64)),
    "eye_inside": (lambda: V.Camera("persp", 64, 48, eye=(0.5, 0.5, 0.5), target=(0.9, 0.6, 0.2), up=(0.0, 0.0, 1.0),
                                    fovy=np.deg2rad(60.0)),
                   lambda: V.box_mesh((0.2, 0.3, 0.25), (0.8, 0.7, 0.75))),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_trim_intervals_bit_exact(name):
    cam, mesh = CASES[name][0](), CASES[name][1]()
    want = orc.trim(cam, mesh)
    got = lv.trim(cam, _tris(mesh)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.isfinite(want[..., 0]).sum() > 0 or name == "eye_inside"


@pytest.mark.parametrize("mode", ["heuristic", "fixed"])
def test_trimmed_render_matches_oracle(cfg1, cfg1_oracle, mode):
    tf, _ = V.config1_render()
    tf.table = tf.table.astype(np.float32).astype(np.float64)
    cam = V.orbit_camera(V.Stream(17), 160, 120)
    mesh = V.icosphere((0.45, 0.5, 0.55), 0.3, 3)
    tr = lv.trim(cam, _tris(mesh))
    gv = lv.Volume(cfg1).build_accel((32, 32, 32)).to_bezier()
    img = gv.render(cam, tf, V.StepParams(mode=mode, h=1 / 300, xi=1 / 256, alpha_stop=0.99, trim=tr)).cpu().numpy()
    st = gv.stats()
    ref, ost = cfg1_oracle.render(cam, tf, V.StepParams(mode=mode, h=1 / 300, xi=1 / 256, alpha_stop=0.99,
                                                         trim=tr.cpu().numpy()))
    full = gv.render(cam, tf, V.StepParams(mode=mode, h=1 / 300, xi=1 / 256, alpha_stop=0.99)).cpu().numpy()
    gv.close()
    assert float(np.sqrt(np.mean((img - ref) ** 2))) <= 1e-4
    assert st["rays_hit"] == ost["rays_hit"]
    outside = ~np.isfinite(tr.cpu().numpy()[..., 0])
    assert np.all(img[outside] == 0) and np.abs(full[outside]).max() > 0.01   # trimming hides what it should


def test_large_mesh_full_hd_chords():
    cam = V.orbit_camera(V.Stream(5), 1920, 1080)
    r, ctr = 0.35, np.array([0.5, 0.5, 0.5])
    mesh = V.uv_sphere(ctr, r, 1000, 1200)                 # 2.4M triangles
    tr = lv.trim(cam, _tris(mesh)).cpu().numpy()
    rng = np.random.default_rng(2)
    seen = 0
    for _ in range(3000):
        i, j = int(rng.integers(0, 1920)), int(rng.integers(0, 1080))
        ry = orc.ray(cam, i, j)
        if ry is None:
            assert tr[j, i, 0] == np.inf and tr[j, i, 1] == 0
            continue
        o, d = np.asarray(ry[0], np.float64), np.asarray(ry[1], np.float64)
        dist = np.linalg.norm(np.cross(ctr - o, d)) / np.linalg.norm(d)
        tc = np.dot(ctr - o, d) / np.linalg.norm(d)
        if dist < 0.999 * r:
            half = np.sqrt(r * r - dist * dist)
            assert abs(tr[j, i, 0] - (tc - half)) < 1e-3 and abs(tr[j, i, 1] - (tc + half)) < 1e-3
            seen += 1
        elif dist > 1.001 * r:
            assert tr[j, i, 0] == np.inf and tr[j, i, 1] == 0
    assert seen > 300

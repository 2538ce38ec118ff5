"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars (from the arithmetic of each step):
  element ids        bit-exact (FP32 queries, split planes rounded up: the
                     FP32 comparison equals the FP64 one);
  per-sample values  |v_gpu - v_orc| <= 1e-5 * max(|v_orc|, max|c|);
  Bezier blocks      GPU FP64 blossoming vs oracle interpolation within
                     1e-12 * max|c| (both exact up to rounding);
  images             RMSE <= 1e-4 in [0,1] RGBA (sample positions, element
                     choices and step lengths are identical FP32 decisions on
                     both sides, so only FP32 vs FP64 arithmetic differs).
"""
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import NONE, Oracle
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import LRVolume

pytestmark = pytest.mark.gpu

RMSE_TOL = 1e-4
VAL_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


def _f32_tf(tf):
    tf.table = np.asarray(tf.table, dtype=np.float32).astype(np.float64)
    return tf


def _with_coef(vol, coef):
    return LRVolume(deg=vol.deg, elem_box=vol.elem_box, knots=vol.knots,
                    coef=np.asarray(coef, dtype=np.float64).reshape(vol.n_basis, -1), weight=vol.weight, grid=vol.grid)


def _rmse(a, b):
    return float(np.sqrt(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)))


def _probe_points(vol, n, seed, blocks=(64, 64, 64)):
    """Uniform points plus points on element faces, forest block faces, 0 and 1."""
    rng = np.random.default_rng(seed)
    X = rng.random((n, 3)).astype(np.float32)
    faces = np.unique(vol.elem_box.astype(np.float32))
    m = rng.random((n, 3)) < 0.3
    X[m] = rng.choice(faces, size=int(m.sum()))
    bf = np.unique(np.concatenate([np.arange(b + 1) / b for b in blocks])).astype(np.float32)
    m = rng.random((n, 3)) < 0.1
    X[m] = rng.choice(bf, size=int(m.sum()))
    edges = np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0.5], [0.5, 0.5, 1]], np.float32)
    out = np.array([[1.0000001, 0.5, 0.5], [-1e-7, 0.5, 0.5], [0.5, 2.0, 0.5]], np.float32)
    return np.concatenate([X, edges, out])


def _nondyadic():
    return V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3, seed=4)


VOLS = {
    "cfg1": lambda: V.load_config(1),
    "nondyadic_p2_vec": _nondyadic,
    "tp_p1": lambda: V.tensor_product((1, 1, 1), (5, 3, 4), seed=2),
}


@pytest.fixture(scope="module")
def vols():
    return {k: f() for k, f in VOLS.items()}


@pytest.fixture(scope="module")
def oracles(vols):
    return {k: Oracle(v) for k, v in vols.items()}


# ----------------------------------------------------------------------------
# look-up (Alg. 1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(VOLS))
@pytest.mark.parametrize("blocks", [(1, 1, 1), (2, 2, 2), (64, 64, 64), (8, 4, 16)])
def test_lookup_bit_exact(vols, oracles, name, blocks):
    vol = vols[name]
    gv = lv.Volume(vol).build_accel(blocks)
    n = 200_000 if blocks == (64, 64, 64) and name == "cfg1" else 40_000
    X = _probe_points(vol, n, seed=zlib.crc32(f"{name}{blocks}".encode()) % 1000, blocks=blocks)
    got = gv.lookup(torch.from_numpy(X).cuda()).cpu().numpy().view(np.uint32)
    want = oracles[name].lookup(X)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} mismatches, e.g. {X[bad[:3]]} gpu {got[bad[:3]]} orc {want[bad[:3]]}"
    assert np.sum(want == NONE) == 3
    st = gv.stats()
    assert st["depth_max"] >= st["depth_min"] >= 0
    gv.close()


@pytest.mark.parametrize("blocks", [(1, 1, 1), (4, 4, 4), (8, 4, 16)])
def test_octree_lookup_bit_exact(vols, oracles, blocks):
    """Midpoint (octree-style) trees over a dyadic mesh give the brute-force
    element ids, faces included; one tree over the whole cube is the paper's
    octree look-up."""
    vol = vols["cfg1"]
    gv = lv.Volume(vol).build_accel(blocks, split=lv.SPLIT_MIDPOINT)
    X = _probe_points(vol, 100_000, seed=zlib.crc32(f"oct{blocks}".encode()) % 1000, blocks=blocks)
    got = gv.lookup(torch.from_numpy(X).cuda()).cpu().numpy().view(np.uint32)
    want = oracles["cfg1"].lookup(X)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} mismatches, e.g. {X[bad[:3]]} gpu {got[bad[:3]]} orc {want[bad[:3]]}"
    st = gv.stats()
    assert st["depth_max"] >= st["depth_min"] >= 0 and st["n_nodes"] > 0
    gv.close()


def test_octree_render_identical_to_balanced_forest(vols):
    vol = vols["cfg1"]
    tf, cams = V.config1_render()
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    a = lv.Volume(vol).build_accel((64, 64, 64)).to_bezier()
    b = lv.Volume(vol).build_accel((1, 1, 1), split=lv.SPLIT_MIDPOINT).to_bezier()
    for cam in cams:
        ia, ib = a.render(cam, tf, step), b.render(cam, tf, step)
        assert torch.equal(ia, ib)
    assert a.stats()["samples"] == b.stats()["samples"] and a.stats()["lookups"] == b.stats()["lookups"]
    a.close()
    b.close()


@pytest.mark.slow
def test_octree_on_the_benchmark_volume():
    """cfg2 (174,000 elements): octree-style trees in 4^3 blocks give the
    brute-force element ids on sampled points (faces included), and a frame
    identical to the balanced 64^3 forest's."""
    vol = V.load_config(2)
    gv = lv.Volume(vol).build_accel((4, 4, 4), split=lv.SPLIT_MIDPOINT)
    X = _probe_points(vol, 6000, seed=77, blocks=(4, 4, 4))
    got = gv.lookup(torch.from_numpy(X).cuda()).cpu().numpy().view(np.uint32)
    want = Oracle(vol).lookup(X)
    np.testing.assert_array_equal(got, want)
    tf, _ = V.config2_render(vol=vol)
    cam = V.orbit_camera(V.Stream(4243), 320, 180)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    img = gv.to_bezier().render(cam, tf, step)
    ref = lv.Volume(vol).build_accel((64, 64, 64)).to_bezier()
    assert torch.equal(img, ref.render(cam, tf, step))
    gv.close()
    ref.close()


@pytest.mark.parametrize("name", ["tp_p1", "nondyadic_p2_vec"])
def test_octree_rejects_nondyadic_faces(vols, name):
    gv = lv.Volume(vols[name])
    with pytest.raises(lv.LrvolError) as ei:
        gv.build_accel((4, 4, 4), split=lv.SPLIT_MIDPOINT)
    assert ei.value.status == lv.ERR_UNSUPPORTED
    with pytest.raises(lv.LrvolError) as ei:
        gv.build_accel((4, 4, 4), split=7)
    assert ei.value.status == lv.ERR_ARG
    gv.build_accel((4, 4, 4))                  # the balanced rule handles any box partition
    gv.close()


@pytest.mark.slow
@pytest.mark.parametrize("blocks", [(64, 64, 64), (4, 4, 4)])
def test_lookup_bit_exact_cfg3_full_size(blocks):
    """The vector benchmark volume at full size (388,016 elements, faces at
    multiples of 1/192, not FP32-exact): element ids of 50,000 probe points,
    faces and forest-block faces included, equal brute force; with 4^3 blocks
    the trees are 3 to 18 levels deep."""
    vol = V.load_config(3)
    gv = lv.Volume(vol).build_accel(blocks)
    X = _probe_points(vol, 50_000, seed=91, blocks=blocks)
    got = gv.lookup(torch.from_numpy(X).cuda()).cpu().numpy().view(np.uint32)
    want = Oracle(vol).lookup(X)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} mismatches, e.g. {X[bad[:3]]} gpu {got[bad[:3]]} orc {want[bad[:3]]}"
    assert gv.stats()["depth_max"] >= (6 if blocks[0] == 64 else 12)
    gv.close()


def test_lookup_million_points_cfg1(vols, oracles):
    vol = vols["cfg1"]
    gv = lv.Volume(vol).build_accel((64, 64, 64))
    X = _probe_points(vol, 1_000_000, seed=17)
    got = gv.lookup(torch.from_numpy(X).cuda()).cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, oracles["cfg1"].lookup(X))


def test_lookup_empty_and_state(vols):
    gv = lv.Volume(vols["tp_p1"])
    with pytest.raises(lv.LrvolError) as ei:
        gv.lookup(torch.zeros((4, 3), device="cuda"))
    assert ei.value.status == lv.ERR_STATE
    gv.build_accel((4, 4, 4))
    out = gv.lookup(torch.zeros((0, 3), device="cuda"))
    assert out.numel() == 0
    with pytest.raises(lv.LrvolError) as ei:
        gv.build_accel((3, 4, 4))
    assert ei.value.status == lv.ERR_ARG


# ----------------------------------------------------------------------------
# change of basis and evaluation (Sec. 3.2.3)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(VOLS))
def test_bezier_blocks_match_interpolation(vols, oracles, name):
    vol = vols[name]
    gv = lv.Volume(vol).to_bezier()
    B = gv.get_bezier()
    rng = np.random.default_rng(1)
    el = rng.choice(vol.n_elem, min(vol.n_elem, 400), replace=False)
    ref = oracles[name].bezier_blocks(el)
    scale = np.abs(vol.coef).max()
    np.testing.assert_allclose(B[el], ref, atol=1e-12 * scale, rtol=0)
    gv.close()


@pytest.mark.parametrize("name", list(VOLS))
def test_eval_values(vols, oracles, name):
    vol = vols[name]
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    X = _probe_points(vol, 100_000, seed=5)
    got = gv.eval(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    want = oracles[name].eval(X)
    tol = VAL_TOL * np.maximum(np.abs(want), np.abs(vol.coef).max())
    err = np.abs(got - want)
    assert np.all(err <= tol), f"max err {err.max()} at {np.argmax(err.max(axis=1))}"
    gv.close()


def test_eval_anisotropic_degree():
    vol = V.refined_ball((1, 2, 3), (4, 3, 5), centres=((0.5, 0.5, 0.5),), radii=(0.35,), seed=8)
    gv = lv.Volume(vol).build_accel((8, 8, 8)).to_bezier()
    X = _probe_points(vol, 20_000, seed=6)
    got = gv.eval(torch.from_numpy(X).cuda()).cpu().numpy()
    want = Oracle(vol).eval(X)
    assert np.abs(got - want).max() <= VAL_TOL * max(1.0, np.abs(vol.coef).max())


# ----------------------------------------------------------------------------
# rendering (Sec. 4)
# ----------------------------------------------------------------------------

def _render_pair(vol, orc, cam, tf, step, blocks=(64, 64, 64), pixels=None):
    gv = lv.Volume(vol).build_accel(blocks).to_bezier()
    img = gv.render(cam, tf, step).cpu().numpy()
    st = gv.stats()
    gv.close()
    if pixels is None:
        ref, ost = orc.render(cam, tf, step)
        return img, ref, st, ost
    ref, ost = orc.render(cam, tf, step, pixels=pixels)
    return img[pixels[:, 1], pixels[:, 0]], ref, st, ost


@pytest.mark.parametrize("mode", ["fixed", "heuristic"])
@pytest.mark.parametrize("view", [0, 1])
def test_render_cfg1(vols, oracles, mode, view):
    tf, cams = V.config1_render()
    tf = _f32_tf(tf)
    step = V.StepParams(mode=mode, h=1 / 256, xi=1 / 256, alpha_stop=1.0)
    img, ref, st, ost = _render_pair(vols["cfg1"], oracles["cfg1"], cams[view], tf, step)
    assert _rmse(img, ref) <= RMSE_TOL
    assert np.abs(img - ref).max() <= 2e-3
    assert st["rays_hit"] == ost["rays_hit"]
    # identical FP32 decisions: same samples, except where FP32 alpha saturates to 1 before FP64
    assert abs(st["samples"] - ost["samples"]) <= 0.001 * ost["samples"]


@pytest.mark.parametrize("mode", ["fixed", "heuristic"])
def test_render_ragged_persp(vols, oracles, mode):
    """A size that leaves partial tiles in both directions, perspective, early termination on."""
    tf, _ = V.config1_render()
    tf = _f32_tf(tf)
    cam = V.orbit_camera(V.Stream(77), 100, 70)
    step = V.StepParams(mode=mode, h=1 / 300, xi=1 / 256, alpha_stop=0.95)
    img, ref, st, ost = _render_pair(vols["cfg1"], oracles["cfg1"], cam, tf, step, blocks=(32, 32, 32))
    assert _rmse(img, ref) <= RMSE_TOL


@pytest.mark.parametrize("field,comp", [("magnitude", 0), ("component", 0), ("component", 2)])
def test_render_vector(vols, oracles, field, comp):
    vol = vols["nondyadic_p2_vec"]
    tf = _f32_tf(V.seeded_tf(V.Stream(31), alpha_max=0.05))
    tf.vmin, tf.vmax = (0.0, 1.6) if field == "magnitude" else (0.0, 1.0)
    cam = V.orbit_camera(V.Stream(32), 64, 48)
    step = V.StepParams(mode="heuristic", xi=1 / 128, field=field, component=comp)
    img, ref, st, ost = _render_pair(vol, oracles["nondyadic_p2_vec"], cam, tf, step, blocks=(16, 16, 16))
    assert _rmse(img, ref) <= RMSE_TOL
    assert st["samples"] == ost["samples"]


@pytest.mark.parametrize("mode", ["fixed", "heuristic"])
def test_render_closed_form_constant_field(vols, mode):
    vol = _with_coef(vols["cfg1"], np.full(vols["cfg1"].n_basis, 0.37))
    a_src, rgb = 0.02, np.array([0.9, 0.4, 0.1], np.float32)
    tf = V.TransferFunction(table=np.tile(np.array([*rgb, a_src], np.float32), (256, 1)).astype(np.float64))
    cam = V.orbit_camera(V.Stream(5), 48, 32)
    step = V.StepParams(mode=mode, h=1 / 200, xi=1 / 128)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    img = gv.render(cam, tf, step).cpu().numpy()
    from oracle.oracle import ray
    for j in range(cam.height):
        for i in range(cam.width):
            r = ray(cam, i, j)
            if r is None:
                assert np.all(img[j, i] == 0)
                continue
            alpha = 1 - (1 - float(np.float32(a_src))) ** ((r[3] - r[2]) / step.xi)
            assert abs(img[j, i, 3] - alpha) <= 2e-5
            np.testing.assert_allclose(img[j, i, :3], rgb.astype(np.float64) * alpha, atol=2e-5)


def test_render_deterministic_and_rows(vols):
    tf, cams = V.config1_render()
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    gv = lv.Volume(vols["cfg1"]).build_accel((32, 32, 32)).to_bezier()
    a = gv.render(cams[1], tf, step)
    b = gv.render(cams[1], tf, step)
    assert torch.equal(a, b)
    # row ranges (screen-space shards) reproduce the full image exactly
    out = torch.full_like(a, -1.0)
    for r0, r1 in [(0, 50), (50, 51), (51, 128)]:
        gv.render(cams[1], tf, step, out=out, row_begin=r0, row_end=r1)
    assert torch.equal(out, a)
    gv.close()


def test_render_errors(vols):
    tf, cams = V.config1_render()
    step = V.StepParams()
    gv = lv.Volume(vols["cfg1"])
    with pytest.raises(lv.LrvolError) as ei:
        gv.render(cams[0], tf, step)
    assert ei.value.status == lv.ERR_STATE
    gv.build_accel((8, 8, 8)).to_bezier()
    with pytest.raises(lv.LrvolError) as ei:
        gv.render(cams[0], tf, V.StepParams(field="magnitude"))
    assert ei.value.status == lv.ERR_ARG
    with pytest.raises(lv.LrvolError) as ei:
        gv.render(cams[0], tf, V.StepParams(h=0.0))
    assert ei.value.status == lv.ERR_ARG
    one = V.ortho_z(1, 1)
    img = gv.render(one, tf, step).cpu().numpy()
    ref, _ = Oracle(vols["cfg1"]).render(one, _f32_tf(tf), step)
    assert _rmse(img, ref) <= RMSE_TOL
    gv.close()
    aniso = V.refined_ball((1, 2, 3), (4, 3, 5), radii=(0.3,))
    ga = lv.Volume(aniso).build_accel((8, 8, 8)).to_bezier()
    with pytest.raises(lv.LrvolError) as ei:
        ga.render(cams[0], tf, step)
    assert ei.value.status == lv.ERR_UNSUPPORTED


def _sample_pixels(cam, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], axis=1).astype(np.int32)


@pytest.mark.slow
def test_render_cfg2_full_size_sampled():
    """The benchmark configuration (1920x1080, Eq. 4, alpha_stop 0.99, 64^3 forest)
    on 1024 sampled pixels, each recomputed by the oracle (sample and look-up
    counts of such pixels: test_gpu_trace)."""
    vol = V.load_config(2)
    tf, cam = V.config2_render()
    tf = _f32_tf(tf)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    pix = _sample_pixels(cam, 1024, 3)
    img, ref, st, ost = _render_pair(vol, Oracle(vol), cam, tf, step, blocks=(64, 64, 64), pixels=pix)
    assert _rmse(img, ref) <= RMSE_TOL
    assert st["samples"] > 0 and st["rays_hit"] > 0


@pytest.mark.slow
def test_render_cfg2_shaded_full_size_sampled():
    """The benchmark frame with gradient shading (Sec. 4.1, light at the eye;
    the FP32 kernel that runs 4 CTAs per SM with spills) on 512 sampled
    pixels, each recomputed by the oracle with its own FP64 gradients."""
    vol = V.load_config(2)
    tf, cam = V.config2_render()
    tf = _f32_tf(tf)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, shading="gradient")
    pix = _sample_pixels(cam, 512, 6)
    img, ref, st, ost = _render_pair(vol, Oracle(vol), cam, tf, step, blocks=(64, 64, 64), pixels=pix)
    assert _rmse(img, ref) <= RMSE_TOL
    assert np.abs(ref[:, 3]).max() > 0.05


@pytest.mark.slow
@pytest.mark.parametrize("field", ["magnitude", "component"])
def test_render_cfg3_full_size_sampled(field):
    """The vector benchmark configurations (388,016 elements, knots not FP32
    exact, 1920x1080, |v| or v_x, 64^3 forest) on sampled pixels."""
    vol = V.load_config(3)
    tf, cam = V.config3_render()
    tf = _f32_tf(tf)
    if field == "magnitude":
        tf.vmin, tf.vmax = 0.0, 1.5
        step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field="magnitude")
    else:
        tf.vmin, tf.vmax = -0.5, 1.5
        step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field="component", component=0)
    pix = _sample_pixels(cam, 1024, 4)
    img, ref, st, ost = _render_pair(vol, Oracle(vol), cam, tf, step, blocks=(64, 64, 64), pixels=pix)
    assert _rmse(img, ref) <= RMSE_TOL
    assert np.abs(ref[:, 3]).max() > 0.05              # the sampled rays see the field


@pytest.mark.parametrize("mode", ["fixed", "heuristic"])
def test_render_eye_inside_volume(vols, oracles, mode):
    """A perspective eye inside [0,1]^3: rays start at t = 0, not at a face."""
    tf, _ = V.config1_render()
    tf = _f32_tf(tf)
    cam = V.Camera("persp", 48, 40, eye=(0.47, 0.52, 0.55), target=(0.9, 0.2, 0.1), up=(0.0, 0.0, 1.0),
                   fovy=np.deg2rad(70.0))
    step = V.StepParams(mode=mode, h=1 / 300, xi=1 / 256, alpha_stop=1.0)
    img, ref, st, ost = _render_pair(vols["cfg1"], oracles["cfg1"], cam, tf, step, blocks=(32, 32, 32))
    assert _rmse(img, ref) <= RMSE_TOL
    assert st["rays_hit"] == ost["rays_hit"] == 48 * 40
    assert abs(st["samples"] - ost["samples"]) <= 0.001 * ost["samples"]


def test_render_one_pixel_and_extreme_aspect(vols, oracles):
    tf, _ = V.config1_render()
    tf = _f32_tf(tf)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    for w, h in ((1, 1), (257, 1), (1, 129)):
        cam = V.orbit_camera(V.Stream(70 + w + h), w, h)
        img, ref, st, ost = _render_pair(vols["cfg1"], oracles["cfg1"], cam, tf, step, blocks=(16, 16, 16))
        assert img.shape == (h, w, 4)
        assert _rmse(img, ref) <= RMSE_TOL


@pytest.mark.parametrize("interleaved", [True, False])
@pytest.mark.parametrize("world", [2, 3, 8])
def test_render_shards_reassemble(vols, interleaved, world):
    """Screen-space shards of `world` ranks (interleaved 8-row bands, or
    contiguous row blocks), rendered here in turn, give the full frame
    bitwise; each shard writes only its own rows."""
    from paper_1707_01170_gb300.shard import render_shard, rows_of
    tf, cams = V.config1_render()
    cam = V.orbit_camera(V.Stream(9), 70, 53)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    gv = lv.Volume(vols["cfg1"]).build_accel((16, 16, 16)).to_bezier()
    full = gv.render(cam, tf, step)
    out = torch.full_like(full, -1.0)
    for r in range(world):
        one = torch.full_like(full, -1.0)
        render_shard(gv, cam, tf, step, one, world=world, rank=r, interleaved=interleaved)
        mine = torch.zeros(cam.height, dtype=torch.bool, device="cuda")
        for a, b in rows_of(cam.height, world, r, interleaved):
            mine[a:b] = True
        assert bool(torch.all(one[~mine] == -1.0))
        out[mine] = one[mine]
    assert torch.equal(out, full)
    with pytest.raises(lv.LrvolError) as ei:
        gv.render(cam, tf, step, band_count=2, band_index=2)
    assert ei.value.status == lv.ERR_ARG
    gv.close()


@pytest.mark.parametrize("storage", [lv.STORE_F32, lv.STORE_F16])
@pytest.mark.parametrize("field", ["magnitude", "component"])
def test_render_shards_reassemble_vector(vols, storage, field):
    """The same for a 3-vector volume, whose kernels map 4x8-pixel warps
    (scalar ones 8x4) onto the 8-row bands: 3 interleaved and 2 contiguous
    shards give the full frame bitwise, on a ragged 70x53 image."""
    from paper_1707_01170_gb300.shard import render_shard, rows_of
    tf = V.seeded_tf(V.Stream(31), alpha_max=0.05)
    tf.vmin, tf.vmax = (0.0, 1.6) if field == "magnitude" else (-0.5, 1.0)
    cam = V.orbit_camera(V.Stream(10), 70, 53)
    step = V.StepParams(mode="heuristic", xi=1 / 128, field=field, component=1)
    gv = lv.Volume(vols["nondyadic_p2_vec"]).build_accel((16, 16, 16)).to_bezier(storage)
    full = gv.render(cam, tf, step)
    assert float(full[..., 3].max()) > 0.05
    for world, interleaved in ((3, True), (2, False)):
        out = torch.full_like(full, -1.0)
        for r in range(world):
            one = torch.full_like(full, -1.0)
            render_shard(gv, cam, tf, step, one, world=world, rank=r, interleaved=interleaved)
            mine = torch.zeros(cam.height, dtype=torch.bool, device="cuda")
            for a, b in rows_of(cam.height, world, r, interleaved):
                mine[a:b] = True
            assert bool(torch.all(one[~mine] == -1.0))
            out[mine] = one[mine]
        assert torch.equal(out, full), (world, interleaved)
    gv.close()

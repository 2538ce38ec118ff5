"""The render kernel's own samples against the FP64 oracle's march.

lrvol_render_trace runs k_render (the kernel lrvol_render launches, with its
compile-time trace flag on) over a pixel list and returns, per composited
sample, (t_k, element id, field value, segment).  Oracle.render_trace returns
the same from oracle.c's march.  Bars:
  t_k, element ids, segments   bit-exact: they are FP32 decisions taken in
                               the same order on both sides (Sec. 4 ray
                               setup, Alg. 1, Eq. 4 / fixed / learned steps);
  values                       |v_gpu - v_orc| <= 1e-5 max(|v_orc|, c_e) with
                               c_e a bound on the element's Bernstein
                               coefficients (the hull of its incident c_i, or
                               its interpolated block), plus 1.02 s_e u for
                               16-bit blocks (s_e the half range of the
                               element's coefficients, u = 2^-11 FP16, 2^-8
                               BF16), 2.04 s_e u for FP16 blocks (the x
                               monomials are rounded to FP16 too, for the
                               mixed-precision FMAs);
  sample counts                equal, except where the ray's opacity sits at
                               the early-termination threshold: FP32
                               transmittance (GPU) and FP64 opacity (oracle)
                               then decide differently; the shorter march
                               must end within 1e-4 of alpha_stop;
  pixels                       RMSE <= 1e-4 against the oracle (5e-4 FP16,
                               4e-3 BF16 blocks, as in test_gpu_precision),
                               and bit for bit equal to lrvol_render's image.
Covered: degrees 1-3; scalar, |v| and component fields; FP32, FP16 and BF16
blocks; fixed, Eq. 4 and learned steps; gradient shading; config 1, a
non-dyadic 3-vector volume, and >= 1000 hitting pixels of the full-size
1920x1080 frames of configs 2 and 3.
"""
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle, ray
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

pytestmark = pytest.mark.gpu

VAL_TOL = 1e-5
# image bars of test_gpu_precision: 1e-4 for FP32 blocks; 16-bit blocks add
# their storage error (up to s u per sample) to every composited sample
RMSE_TOL = {"f32": 1e-4, "f16": 5e-4, "bf16": 4e-3}
U = {"f32": 0.0, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
STORE = {"f32": lv.STORE_F32, "f16": lv.STORE_F16, "bf16": lv.STORE_BF16}
CANDIDATES = np.array([1, 1.5, 2, 3, 4, 6, 8], np.float32)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


def _f32_tf(tf):
    tf.table = np.asarray(tf.table, dtype=np.float32).astype(np.float64)
    return tf


def _hitting_pixels(cam, n, seed, pool=8):
    """n pixels whose rays meet the unit cube (seeded), else as many as found."""
    rng = np.random.default_rng(seed)
    cand = np.stack([rng.integers(0, cam.width, pool * n), rng.integers(0, cam.height, pool * n)], axis=1)
    keep = [p for p in cand if ray(cam, int(p[0]), int(p[1])) is not None][:n]
    return np.asarray(keep, dtype=np.int32)


def _alg2_alpha(tf, vals, segs, xi):
    """Opacity after each sample of one march (Alg. 2, FP64)."""
    x = np.clip((vals - tf.vmin) / (tf.vmax - tf.vmin), 0.0, 1.0) * 255.0
    i0 = np.minimum(np.floor(x).astype(np.int64), 254)
    f = x - i0
    a_src = (1 - f) * tf.table[i0, 3] + f * tf.table[i0 + 1, 3]
    T = (1 - a_src) ** (segs / xi)
    return 1 - np.cumprod(T)


def _bounds(O, elems, field, comp, storage, exact_blocks):
    """Per element: the coefficient bound c_e and the 16-bit bound: 1.02 s_e u
    for BF16 blocks, 2.04 s_e u for FP16 blocks, whose render also rounds the
    x monomials to FP16 for its mixed-precision FMAs."""
    uniq, inv = np.unique(elems, return_inverse=True)
    if exact_blocks:
        B = O.bezier_blocks(uniq).reshape(len(uniq), O.nc, -1)
        lo, hi = B.min(axis=2), B.max(axis=2)
    else:
        H = O.coefficient_hull(uniq)
        lo, hi = H[:, :, 0], H[:, :, 1]
    amax = np.maximum(np.abs(lo), np.abs(hi))
    half = 0.5 * (hi - lo)
    if field == "magnitude":
        c = np.sqrt((amax ** 2).sum(axis=1))
        s = np.sqrt((half ** 2).sum(axis=1))
    else:
        k = comp if field == "component" else 0
        c, s = amax[:, k], half[:, k]
    return c[inv], (2.04 if storage == "f16" else 1.02) * U[storage] * s[inv]


def _runs(elem, count):
    """Runs of equal consecutive element ids over each march's first count samples."""
    live = np.arange(elem.shape[1])[None, :] < np.asarray(count)[:, None]
    change = np.concatenate([np.ones((elem.shape[0], 1), bool), elem[:, 1:] != elem[:, :-1]], axis=1)
    return int(np.sum(live & change))


def compare_traces(O, tf, step, storage, gpu, orc, exact_blocks=True):
    (gtr, gcnt, grgba, gst), (otr, ocnt, orgba, ost) = gpu, orc
    n_pix, maxs = gtr.shape[0], gtr.shape[1]
    assert gst["rays_hit"] == ost["rays_hit"]
    assert gst["samples"] == int(gcnt.sum()) and ost["samples"] == int(ocnt.sum())
    differ = np.nonzero(gcnt != ocnt)[0]
    # counts differ only where the opacity sits at the termination threshold
    for q in differ:
        n = int(min(gcnt[q], ocnt[q]))
        a = _alg2_alpha(tf, otr[q, :n, 2], otr[q, :n, 3], step.xi)
        assert n > 0 and abs(a[-1] - step.alpha_stop) <= 1e-4, (q, gcnt[q], ocnt[q], a[-1])
    # FP32 blocks: the FP32 and FP64 opacities differ by rounding only; 16-bit
    # blocks move values by up to s u, so more rays sit within that of the
    # threshold
    assert len(differ) <= max(2, n_pix // (100 if storage == "f32" else 25))
    n = np.minimum(np.minimum(gcnt, ocnt), maxs)
    mask = np.arange(maxs)[None, :] < n[:, None]
    # look-ups: one per run of equal element ids in a march (element reuse).
    # The oracle looks up exactly that; the kernel may also have looked up the
    # sample it evaluated but dropped when the ray stopped early.
    if np.all(np.maximum(gcnt, ocnt) <= maxs):
        assert ost["lookups"] == _runs(otr[:, :, 1], ocnt)
        r = _runs(gtr[:, :, 1].view(np.uint32), gcnt)
        assert r <= gst["lookups"] <= r + n_pix
    g, o = gtr[mask], otr[mask]
    assert g.shape[0] == int(n.sum()) and g.shape[0] > 0
    np.testing.assert_array_equal(g[:, 0], o[:, 0].astype(np.float32))                     # t_k
    np.testing.assert_array_equal(g[:, 1].view(np.uint32), o[:, 1].astype(np.uint32))      # element ids
    np.testing.assert_array_equal(g[:, 3], o[:, 3].astype(np.float32))                     # segments
    elems = o[:, 1].astype(np.int64)
    c, b16 = _bounds(O, elems, step.field, step.component, storage, exact_blocks)
    tol = VAL_TOL * np.maximum(np.abs(o[:, 2]), c) + b16
    err = np.abs(g[:, 2].astype(np.float64) - o[:, 2])
    worst = int(np.argmax(err - tol))
    assert np.all(err <= tol), f"value {g[worst, 2]} vs {o[worst, 2]} (tol {tol[worst]:.3e}), element {elems[worst]}"
    rmse = float(np.sqrt(np.mean((grgba.astype(np.float64) - orgba) ** 2)))
    assert rmse <= RMSE_TOL[storage], rmse
    return int(n.sum()), float((err / np.maximum(tol, 1e-30)).max())


def run_case(gv, O, cam, tf, step, storage, pix, maxs=4096, exact_blocks=True, image=None):
    """Trace pix on the GPU and in the oracle and compare; with an image,
    the traced pixels must be that lrvol_render image's pixels bit for bit."""
    tr, cnt, rgba = gv.render_trace(cam, tf, step, torch.from_numpy(pix).cuda(), maxs)
    torch.cuda.synchronize()
    gpu = (tr.cpu().numpy(), cnt.cpu().numpy(), rgba.cpu().numpy(), gv.stats())
    step_o = step
    if step.mult is not None:                    # the oracle takes the same multipliers from the host
        step_o = V.StepParams(**{**step.__dict__, "mult": step.mult.cpu().numpy()})
    ns, ratio = compare_traces(O, tf, step_o, storage, gpu, O.render_trace(cam, tf, step_o, pix, maxs),
                               exact_blocks)
    if image is not None:
        img = image.cpu().numpy()
        assert np.array_equal(img[pix[:, 1], pix[:, 0]], gpu[2])
    return ns, ratio, gpu[3]


def _mult(vol, seed):
    """Seeded per-element multipliers from the learned step's candidate set."""
    u = V.Stream(seed, vol.n_elem + 16).take(vol.n_elem)
    idx = np.minimum((u * len(CANDIDATES)).astype(np.int64), len(CANDIDATES) - 1)
    return torch.from_numpy(CANDIDATES[idx]).cuda()


def _seed(*key):
    return zlib.crc32(repr(key).encode()) % 1000


@pytest.fixture(scope="module")
def cfg1():
    vol = V.load_config(1)
    return vol, Oracle(vol)


CFG1_CASES = [
    # storage, mode, view, alpha_stop
    ("f32", "heuristic", "oblique", 1.0),
    ("f32", "fixed", "ortho", 1.0),
    ("f32", "learned", "persp", 0.99),
    ("f32", "heuristic", "persp", 0.95),
    ("f16", "heuristic", "persp", 0.99),
    ("f16", "fixed", "oblique", 1.0),
    ("bf16", "learned", "oblique", 1.0),
    ("bf16", "heuristic", "ortho", 0.99),
]


@pytest.mark.parametrize("storage,mode,view,alpha_stop", CFG1_CASES)
def test_trace_cfg1(cfg1, storage, mode, view, alpha_stop, capsys):
    vol, O = cfg1
    tf, cams = V.config1_render()
    tf = _f32_tf(tf)
    cam = {"ortho": cams[0], "oblique": cams[1], "persp": V.orbit_camera(V.Stream(77), 150, 97)}[view]
    step = V.StepParams(mode=mode, h=1 / 256, xi=1 / 256, alpha_stop=alpha_stop)
    if mode == "learned":
        step.mult = _mult(vol, 3)
    gv = lv.Volume(vol).build_accel((32, 32, 32)).to_bezier(STORE[storage])
    pix = _hitting_pixels(cam, 1500, _seed(storage, mode, view))
    ns, ratio, _ = run_case(gv, O, cam, tf, step, storage, pix, image=gv.render(cam, tf, step))
    with capsys.disabled():
        print(f"\n[trace cfg1 {storage} {mode} {view} a_stop {alpha_stop}] {len(pix)} pixels, {ns} samples, "
              f"worst value error {ratio:.2f} of its bound")
    gv.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_trace_cfg1_shaded(cfg1, storage):
    """Gradient shading (Sec. 4.1): same march and values; shaded pixels."""
    vol, O = cfg1
    tf, _ = V.config1_render()
    tf = _f32_tf(tf)
    cam = V.orbit_camera(V.Stream(78), 120, 90)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, shading="gradient")
    gv = lv.Volume(vol).build_accel((32, 32, 32)).to_bezier(STORE[storage])
    run_case(gv, O, cam, tf, step, storage, _hitting_pixels(cam, 600, 9), image=gv.render(cam, tf, step))
    gv.close()


def _nondyadic():
    return V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3, seed=4)


@pytest.fixture(scope="module")
def vec():
    vol = _nondyadic()
    return vol, Oracle(vol)


VEC_CASES = [
    ("f32", "magnitude", 0, "heuristic"),
    ("f16", "magnitude", 0, "heuristic"),
    ("bf16", "magnitude", 0, "fixed"),
    ("f32", "component", 0, "fixed"),
    ("f16", "component", 1, "learned"),
    ("bf16", "component", 2, "heuristic"),
]


@pytest.mark.parametrize("storage,field,comp,mode", VEC_CASES)
def test_trace_vector_nondyadic(vec, storage, field, comp, mode):
    """p = 2, three components, knots at multiples of 1/12 (not FP32-exact)."""
    vol, O = vec
    tf = _f32_tf(V.seeded_tf(V.Stream(31), alpha_max=0.05))
    tf.vmin, tf.vmax = (0.0, 1.6) if field == "magnitude" else (-0.5, 1.0)
    cam = V.orbit_camera(V.Stream(32), 96, 72)
    step = V.StepParams(mode=mode, h=1 / 300, xi=1 / 128, alpha_stop=0.99, field=field, component=comp)
    if mode == "learned":
        step.mult = _mult(vol, 4)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(STORE[storage])
    run_case(gv, O, cam, tf, step, storage, _hitting_pixels(cam, 800, 21), 2048, image=gv.render(cam, tf, step))
    gv.close()


VEC_DEG_CASES = [
    (1, "f32", "magnitude", 0),
    (1, "f32", "component", 2),
    (1, "f16", "magnitude", 0),
    (1, "f16", "component", 1),
    (1, "bf16", "magnitude", 0),
    (1, "bf16", "component", 2),
    (3, "f32", "magnitude", 0),
    (3, "f32", "component", 0),
    (3, "f16", "magnitude", 0),
    (3, "f16", "component", 2),
    (3, "bf16", "magnitude", 0),
    (3, "bf16", "component", 1),
]


@pytest.mark.parametrize("deg,storage,field,comp", VEC_DEG_CASES)
def test_trace_vector_degrees(deg, storage, field, comp):
    """3-vector volumes of degree 1 and 3 (the benchmark's vector volume is
    degree 2): |v| and single components through every block layout, the
    16-bit ones in both of their load paths (256-bit loads where a
    component's words start 32-byte aligned, 128-bit loads otherwise)."""
    vol = V.refined_ball((deg,) * 3, (3, 3, 3), centres=((0.4, 0.55, 0.5),), radii=(0.35, 0.18), ncomp=3,
                         seed=7 + deg)
    O = Oracle(vol)
    tf = _f32_tf(V.seeded_tf(V.Stream(51), alpha_max=0.05))
    if field == "magnitude":
        tf.vmin, tf.vmax = 0.0, float(np.linalg.norm(vol.coef, axis=1).max())
    else:
        tf.vmin, tf.vmax = float(vol.coef[:, comp].min()), float(vol.coef[:, comp].max())
    cam = V.orbit_camera(V.Stream(52), 80, 60)
    step = V.StepParams(mode="heuristic", xi=1 / 128, alpha_stop=0.99, field=field, component=comp)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(STORE[storage])
    run_case(gv, O, cam, tf, step, storage, _hitting_pixels(cam, 500, 23), 2048, image=gv.render(cam, tf, step))
    gv.close()


@pytest.mark.parametrize("deg,storage,mode", [(2, "f32", "heuristic"), (2, "f16", "learned"), (2, "bf16", "heuristic"),
                                               (1, "f32", "heuristic"), (1, "f16", "fixed"), (1, "bf16", "fixed")])
def test_trace_scalar_low_degree(deg, storage, mode):
    vol = V.refined_ball((deg,) * 3, (4, 4, 4), centres=((0.45, 0.5, 0.55),), radii=(0.35, 0.15), seed=6)
    O = Oracle(vol)
    tf = _f32_tf(V.seeded_tf(V.Stream(41), alpha_max=0.06))
    tf.vmin, tf.vmax = float(vol.coef.min()), float(vol.coef.max())
    cam = V.orbit_camera(V.Stream(42), 90, 64)
    step = V.StepParams(mode=mode, h=1 / 256, xi=1 / 256, alpha_stop=0.99)
    if mode == "learned":
        step.mult = _mult(vol, 5)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(STORE[storage])
    run_case(gv, O, cam, tf, step, storage, _hitting_pixels(cam, 600, 22), 2048, image=gv.render(cam, tf, step))
    gv.close()


@pytest.mark.parametrize("deg,storage", [(1, "f32"), (1, "f16"), (1, "bf16"), (2, "f32"), (2, "f16"), (2, "bf16")])
def test_trace_shaded_low_degree(deg, storage):
    """Gradient shading on scalar volumes of degree 1 and 2, whose blocks take
    the generic layout (with 16-bit storage: mixed-precision FMAs for FP16,
    conversion for BF16) instead of the tricubic row pairs."""
    vol = V.refined_ball((deg,) * 3, (4, 4, 4), centres=((0.45, 0.5, 0.55),), radii=(0.35, 0.15), seed=6)
    O = Oracle(vol)
    tf = _f32_tf(V.seeded_tf(V.Stream(43), alpha_max=0.06))
    tf.vmin, tf.vmax = float(vol.coef.min()), float(vol.coef.max())
    cam = V.orbit_camera(V.Stream(44), 90, 64)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, shading="gradient", light=(0.3, -0.5, 0.8))
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(STORE[storage])
    run_case(gv, O, cam, tf, step, storage, _hitting_pixels(cam, 500, 24), 2048, image=gv.render(cam, tf, step))
    gv.close()


def test_trace_edge_cases(cfg1):
    """Pixels that miss, an empty list, a ray longer than max_samples (only
    the first records are kept; the count is the full one), and a pixel
    outside the image (count 0, status LRVOL_ERR_BOUNDS at the next stats)."""
    vol, O = cfg1
    tf, _ = V.config1_render()
    tf = _f32_tf(tf)
    cam = V.orbit_camera(V.Stream(80), 64, 48, radius=3.0)
    step = V.StepParams(mode="fixed", h=1 / 1024, xi=1 / 256, alpha_stop=1.0)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    misses = np.array([[0, 0], [63, 47], [0, 47]], np.int32)
    assert all(ray(cam, int(i), int(j)) is None for i, j in misses)
    hit = np.array([[32, 24], [30, 20], [34, 26], [28, 25]], np.int32)
    pix = np.concatenate([misses, hit])
    tr, cnt, rgba = gv.render_trace(cam, tf, step, torch.from_numpy(pix).cuda(), 16)
    torch.cuda.synchronize()
    otr, ocnt, orgba, _ = O.render_trace(cam, tf, step, pix, 16)
    cnt, tr = cnt.cpu().numpy(), tr.cpu().numpy()
    assert np.all(cnt[:3] == 0) and np.all(rgba[:3].cpu().numpy() == 0)
    assert np.all(cnt[3:] > 16) and np.array_equal(cnt, ocnt)
    np.testing.assert_array_equal(tr[3:, :, 0], otr[3:, :, 0].astype(np.float32))
    empty = gv.render_trace(cam, tf, step, torch.zeros((0, 2), dtype=torch.int32, device="cuda"), 16)
    assert empty[1].numel() == 0
    gv.stats()                                                  # status clean so far
    bad = torch.tensor([[64, 0], [5, 5]], dtype=torch.int32, device="cuda")
    _, c2, _ = gv.render_trace(cam, tf, step, bad, 16)
    assert int(c2[0]) == 0
    with pytest.raises(lv.LrvolError) as ei:
        gv.stats()
    assert ei.value.status == lv.ERR_BOUNDS
    gv.close()


# ----------------------------------------------------------------------------
# the full-size benchmark frames (1920x1080), >= 1000 hitting pixels each
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg2():
    vol = V.load_config(2)
    return vol, Oracle(vol)


@pytest.mark.slow
@pytest.mark.parametrize("storage,mode", [("f32", "heuristic"), ("f16", "learned"), ("bf16", "fixed")])
def test_trace_cfg2_1080p(cfg2, storage, mode, capsys):
    """The benchmark frame (Eq. 4, FP32 blocks, alpha_stop 0.99, 64^3 forest),
    the headline frame's form (learned steps, FP16 blocks) and a fixed step."""
    vol, O = cfg2
    tf, cam = V.config2_render(vol=vol)
    tf = _f32_tf(tf)
    step = V.StepParams(mode=mode, h=1 / 512, xi=1 / 256, alpha_stop=0.99)
    if mode == "learned":
        step.mult = _mult(vol, 6)
    gv = lv.Volume(vol).build_accel((64, 64, 64)).to_bezier(STORE[storage])
    pix = _hitting_pixels(cam, 1024, 31)
    assert len(pix) == 1024
    ns, ratio, st = run_case(gv, O, cam, tf, step, storage, pix, 4096, exact_blocks=False,
                             image=gv.render(cam, tf, step))
    with capsys.disabled():
        print(f"\n[trace cfg2 1080p {storage} {mode}] 1024 pixels, {ns} samples, lookups {st['lookups']}, "
              f"worst value error {ratio:.2f} of its bound")
    gv.close()


@pytest.fixture(scope="module")
def cfg3():
    vol = V.load_config(3)
    return vol, Oracle(vol)


@pytest.mark.slow
@pytest.mark.parametrize("field,storage", [("magnitude", "f32"), ("magnitude", "f16"), ("component", "f32"),
                                           ("component", "bf16")])
def test_trace_cfg3_1080p(cfg3, field, storage, capsys):
    """The vector frames: 388,016 elements with knots at multiples of 1/192,
    |v| and v_x, FP32 and 16-bit blocks."""
    vol, O = cfg3
    tf, cam = V.config3_render()
    tf = _f32_tf(tf)
    tf.vmin, tf.vmax = (0.0, 1.5) if field == "magnitude" else (-0.5, 1.5)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field=field, component=0)
    gv = lv.Volume(vol).build_accel((64, 64, 64)).to_bezier(STORE[storage])
    pix = _hitting_pixels(cam, 1024, 32)
    assert len(pix) == 1024
    ns, ratio, st = run_case(gv, O, cam, tf, step, storage, pix, 4096, exact_blocks=False,
                             image=gv.render(cam, tf, step))
    with capsys.disabled():
        print(f"\n[trace cfg3 1080p {field} {storage}] 1024 pixels, {ns} samples, lookups {st['lookups']}, "
              f"worst value error {ratio:.2f} of its bound")
    gv.close()

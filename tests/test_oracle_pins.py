"""Pins of the FP64 oracle to things other than itself (no GPU).

Each test fixes a part of the oracle against what the paper or the
mathematics determines: closed-form B-spline pieces, a library B-spline,
partition of unity (Eq. 2), polynomial reproduction, the exactness of the
change of basis (Sec. 3.2.3), brute force on tiny partitions, the telescoping
of Alg. 2, and the step counts of Eq. 4.
"""
import os
from fractions import Fraction
from math import comb

import numpy as np
import pytest

from oracle.oracle import NONE, Oracle, bernstein, bspline, ray
from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import LRVolume, greville

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _with_coef(vol, coef):
    return LRVolume(deg=vol.deg, elem_box=vol.elem_box, knots=vol.knots,
                    coef=np.asarray(coef, dtype=np.float64).reshape(vol.n_basis, -1),
                    weight=vol.weight, grid=vol.grid)


# --------------------------------------------------------------------------
# Eq. 1 factors: univariate B-splines
# --------------------------------------------------------------------------

def test_bspline_golden_closed_forms():
    """Uniform quadratic/cubic pieces and the clamped end, as exact fractions."""
    n = 0
    for line in open(os.path.join(GOLDEN, "uniform_bspline.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        p, knots, x, val = line.split()
        k = [float(v) for v in knots.split(";")]
        got = bspline(k, int(p), float(x))
        assert got == pytest.approx(float(Fraction(val)), abs=1e-15), line
        n += 1
    assert n >= 20


def test_bspline_matches_scipy():
    """Random local knot vectors (with repeated knots) against scipy's B-spline."""
    interpolate = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(7)
    for trial in range(300):
        p = int(rng.integers(1, 5))
        k = np.sort(rng.choice(np.linspace(0.0, 1.0, 9), size=p + 2))
        if k[0] == k[-1]:
            continue
        b = interpolate.BSpline.basis_element(k, extrapolate=False)
        xs = np.concatenate([rng.uniform(k[0], k[-1], 20), k[1:-1]])
        xs = xs[(xs > k[0]) & (xs < k[-1])]
        ref = np.nan_to_num(b(xs))
        got = np.array([bspline(k, p, x) for x in xs])
        np.testing.assert_allclose(got, ref, atol=1e-13, err_msg=f"knots {k}")


def test_bspline_half_open_support():
    k = [0.25, 0.5, 0.5, 0.75]      # quadratic with a double knot
    assert bspline(k, 2, 0.25) == 0.0
    assert bspline(k, 2, 0.75) == 0.0   # right end of a non-final support is excluded
    assert bspline(k, 2, 0.5) == pytest.approx(1.0)
    assert bspline(k, 2, 0.8) == 0.0


# --------------------------------------------------------------------------
# Eq. 2: partition of unity and polynomial reproduction
# --------------------------------------------------------------------------

def _points_with_faces(vol, n, seed):
    rng = np.random.default_rng(seed)
    X = rng.random((n, 3))
    # snap a third of the coordinates to element faces, and include the corners
    faces = np.unique(vol.elem_box)
    m = rng.random((n, 3)) < 0.33
    X[m] = rng.choice(faces, size=int(m.sum()))
    return np.concatenate([X, [[0, 0, 0], [1, 1, 1], [1, 0, 0.5], [0.5, 1, 1]]])


@pytest.mark.parametrize("deg,n,radii,centre", [
    ((3, 3, 3), (8, 8, 8), (0.25, 0.12), (0.4, 0.55, 0.5)),
    ((2, 2, 2), (3, 3, 3), (0.4, 0.2, 0.1), (0.3, 0.6, 0.45)),     # knots multiples of 1/24: not dyadic
    ((1, 2, 3), (4, 3, 5), (0.35, 0.2), (0.5, 0.5, 0.5)),        # anisotropic degree
])
def test_partition_of_unity(deg, n, radii, centre):
    vol = V.refined_ball(deg, n, centres=(centre,), radii=radii)
    ones = _with_coef(vol, np.ones(vol.n_basis))
    O = Oracle(ones)
    X = _points_with_faces(vol, 4000, 3)
    np.testing.assert_allclose(O.eval(X)[:, 0], 1.0, atol=1e-13)


def _elementary(t, k):
    """Elementary symmetric polynomial e_k of the values t."""
    e = np.zeros(k + 1)
    e[0] = 1.0
    for v in t:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * v
    return e[k]


def _blossom_coef(knots, deg, polys):
    """Blossom (polar form) of prod_a P_a(x_a) at each B-spline's interior knots:
    for x^k of degree p the blossom is e_k(t_1..t_p)/C(p,k)."""
    p = [int(v) for v in deg]
    o = [0, p[0] + 2, p[0] + p[1] + 4]
    out = np.ones(len(knots))
    for a in range(3):
        inner = knots[:, o[a] + 1:o[a] + 1 + p[a]]
        val = np.zeros(len(knots))
        for k, ak in enumerate(polys[a]):
            if ak == 0:
                continue
            assert k <= p[a]
            val += ak * np.array([_elementary(row, k) for row in inner]) / comb(p[a], k)
        out *= val
    return out


def _poly(polys, X):
    out = np.ones(len(X))
    for a in range(3):
        out *= np.polyval(list(reversed(polys[a])), X[:, a])
    return out


@pytest.mark.parametrize("deg,polys", [
    ((3, 3, 3), ([0.3, 1.0], [-0.2, 0.7], [1.1, -0.4])),                 # trilinear
    ((3, 3, 3), ([0.3, 1.0, -0.8], [0.5, -0.2, 0.9], [1.0, 0.3, 0.4])),   # triquadratic
    ((2, 2, 2), ([0.1, -1.0, 2.0], [0.2, 0.5, -0.3], [1.0, 0.0, 1.0])),
])
@pytest.mark.parametrize("mode", ["carried", "tensor"])
def test_polynomial_reproduction(deg, polys, mode):
    """Polynomials of degree <= p are reproduced exactly.

    tensor : unrefined tensor-product mesh with coefficients = blossoms at
             each B-spline's interior knots (Marsden's identity);
    carried: the same start coefficients carried through two levels of LR
             refinement by the splitting weights (refinement is exact).
    (Assigning blossoms directly to the refined LR B-splines is not an
    identity in general: one split sends the parent's blossom to children
    whose own blossoms differ, e.g. for p = 2 under this refinement.)"""
    from paper_1707_01170_gb300.synth.lrgen import Refiner
    levels = 2 if mode == "carried" else 0
    R = Refiner(deg, (4, 4, 4), levels, 1)
    R.set_coef(_blossom_coef(R.knots(), deg, polys))
    for rad in (0.3, 0.15)[:levels]:
        e = R.element_boxes()
        c = 0.5 * (e[:, :3] + e[:, 3:])
        R.refine(np.linalg.norm(c - np.array([0.45, 0.5, 0.55]), axis=1) < rad)
    vol = R.volume()
    assert vol.n_elem > 64 * levels
    O = Oracle(vol)
    X = _points_with_faces(vol, 3000, 11)
    np.testing.assert_allclose(O.eval(X)[:, 0], _poly(polys, X), atol=1e-12)


def test_tensor_product_special_case():
    """Without refinement Eq. 2 is Eq. 1 with gamma = 1: compare with a direct
    triple sum of scipy B-splines on the global knot vectors."""
    interpolate = pytest.importorskip("scipy.interpolate")
    vol = V.tensor_product((2, 3, 1), (3, 2, 4), ncomp=2, seed=5)
    assert np.all(vol.weight == 1.0)
    O = Oracle(vol)
    rng = np.random.default_rng(2)
    X = rng.random((500, 3))
    got = O.eval(X)
    sl = vol.knot_slices()
    ref = np.zeros_like(got)
    for i in range(vol.n_basis):
        w = np.ones(len(X))
        for a in range(3):
            w *= np.nan_to_num(interpolate.BSpline.basis_element(vol.knots[i, sl[a]], extrapolate=False)(X[:, a]))
        ref += w[:, None] * vol.coef[i]
    np.testing.assert_allclose(got, ref, atol=1e-13)


# --------------------------------------------------------------------------
# element look-up by brute force
# --------------------------------------------------------------------------

def _tiny_partition():
    els, pts = [], []
    for line in open(os.path.join(GOLDEN, "tiny_partition.txt")):
        if line.startswith("E "):
            els.append([float(v) for v in line.split()[2:]])
        elif line.startswith("P "):
            f = line.split()[1:]
            pts.append(([float(v) for v in f[:3]], int(f[3])))
    return np.array(els), pts


def test_lookup_tiny_partition():
    els, pts = _tiny_partition()
    assert np.prod(els[:, 3:] - els[:, :3], axis=1).sum() == pytest.approx(1.0)
    # a constant linear B-spline per element is enough to make a volume object
    vol = LRVolume(deg=np.array([1, 1, 1]), elem_box=els,
                   knots=np.array([[0, 0, 1, 0, 0, 1, 0, 0, 1.0]]), coef=np.zeros((1, 1)),
                   weight=np.ones(1), grid=np.array([4, 4, 4]))
    O = Oracle(vol)
    for x, want in pts:
        got = O.find_element(x)
        assert got == (NONE if want < 0 else want), (x, got, want)
    f32 = np.array([x for x, _ in pts], dtype=np.float32)
    want = np.array([NONE if w < 0 else w for _, w in pts], dtype=np.uint32)
    np.testing.assert_array_equal(O.lookup(f32), want)


def test_lookup_unique_cover(cfg1, cfg1_oracle):
    """Every point of [0,1]^3 lies in exactly one half-open element box."""
    X = _points_with_faces(cfg1, 3000, 5).astype(np.float32)
    e = cfg1_oracle.lookup(X)
    b = cfg1.elem_box
    Xd = X.astype(np.float64)
    ins = ((b[None, :, :3] <= Xd[:, None, :])
           & ((Xd[:, None, :] < b[None, :, 3:]) | ((Xd[:, None, :] == 1.0) & (b[None, :, 3:] == 1.0)))).all(axis=2)
    assert np.all(ins.sum(axis=1) == 1)
    np.testing.assert_array_equal(np.argmax(ins, axis=1), e)


# --------------------------------------------------------------------------
# Bezier blocks (Sec. 3.2.3)
# --------------------------------------------------------------------------

def test_bezier_blocks_equal_bspline_evaluation(cfg1, cfg1_oracle):
    rng = np.random.default_rng(3)
    el = rng.choice(cfg1.n_elem, 300, replace=False)
    B = cfg1_oracle.bezier_blocks(el)
    lo, hi = cfg1.elem_box[el, :3], cfg1.elem_box[el, 3:]
    X = lo + rng.random((len(el), 3)) * (hi - lo)
    np.testing.assert_allclose(cfg1_oracle.bezier_eval(B, el, X), cfg1_oracle.eval(X), atol=1e-12)


def test_bezier_single_element_is_bernstein():
    """On one clamped element the B-splines are the Bernstein polynomials, so
    the Bezier block equals the B-spline coefficients."""
    vol = V.tensor_product((3, 2, 1), (1, 1, 1), seed=9)
    O = Oracle(vol)
    B = O.bezier_blocks()[0, 0]                              # (z, y, x)
    g = greville(vol)                                       # orders B-splines by their knots
    # the TP B-spline (i,j,k) of the generator is enumerated with i fastest
    expect = vol.coef[:, 0].reshape(2, 3, 4)
    np.testing.assert_allclose(B, expect, atol=1e-13)
    assert g.shape == (24, 3)


def test_bezier_continuity_across_faces(cfg1, cfg1_oracle):
    """Adjacent blocks agree on their common face (a change of basis keeps continuity)."""
    rng = np.random.default_rng(4)
    b = cfg1.elem_box
    checked = 0
    for e in rng.choice(cfg1.n_elem, 120, replace=False):
        x = np.array([b[e, 3], rng.uniform(b[e, 1], b[e, 4]), rng.uniform(b[e, 2], b[e, 5])])
        if x[0] >= 1.0:
            continue
        n = cfg1_oracle.find_element(x)
        assert n != e
        B = cfg1_oracle.bezier_blocks([e, n])
        v = cfg1_oracle.bezier_eval(B, [e, n], np.stack([x, x]))
        assert abs(v[0, 0] - v[1, 0]) < 1e-12
        checked += 1
    assert checked > 50


# --------------------------------------------------------------------------
# ray setup, Alg. 2 and Eq. 4
# --------------------------------------------------------------------------

def _camera_double(cam, i, j):
    """Independent FP64 ray of pixel (i, j) and its slab interval."""
    eye, tgt, up = (np.array(v, dtype=np.float64) for v in (cam.eye, cam.target, cam.up))
    F = tgt - eye
    F /= np.linalg.norm(F)
    R = np.cross(F, up)
    R /= np.linalg.norm(R)
    U = np.cross(R, F)
    ty = np.tan(cam.fovy / 2) if cam.projection == "persp" else cam.extent / 2
    tx = ty * cam.width / cam.height
    a = (2 * (i + 0.5) / cam.width - 1) * tx
    b = (1 - 2 * (j + 0.5) / cam.height) * ty
    if cam.projection == "persp":
        o, d = eye, F + a * R + b * U
        d /= np.linalg.norm(d)
    else:
        o, d = eye + a * R + b * U, F
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (0 - o) / d
        t1 = (1 - o) / d
    tn = np.nanmax(np.append(np.minimum(t0, t1), 0.0))
    tf = np.nanmin(np.maximum(t0, t1))
    return o, d, tn, tf


@pytest.mark.parametrize("which", ["ortho_z", "oblique", "persp"])
def test_ray_setup_matches_double(which):
    st = V.Stream(99)
    cam = {"ortho_z": V.ortho_z(64, 48), "oblique": V.seeded_oblique(st, 50, 40),
           "persp": V.orbit_camera(st, 96, 54)}[which]
    hits = 0
    for i in range(0, cam.width, 3):
        for j in range(0, cam.height, 3):
            r = ray(cam, i, j)
            o2, d2, tn, tf = _camera_double(cam, i, j)
            if r is None:
                assert not (tn < tf - 1e-5)
                continue
            o, d, ti, to = r
            hits += 1
            np.testing.assert_allclose(o, o2, atol=2e-6)
            np.testing.assert_allclose(d, d2, atol=2e-6)
            assert ti == pytest.approx(tn, abs=1e-5) and to == pytest.approx(tf, abs=1e-5)
    assert hits > 0


def test_ray_ortho_z_exact():
    cam = V.ortho_z(128, 128)
    o, d, ti, to = ray(cam, 5, 7)
    assert list(d) == [0.0, 0.0, -1.0]
    assert o[0] == (5 + 0.5) / 128 and o[1] == 1 - (7 + 0.5) / 128
    assert ti == 1.0 and to == 2.0


def _const_tf(rgba):
    return V.TransferFunction(table=np.tile(np.asarray(rgba, dtype=np.float64), (256, 1)))


@pytest.mark.parametrize("mode", ["fixed", "heuristic"])
@pytest.mark.parametrize("which", ["ortho_z", "persp"])
def test_closed_form_opacity(cfg1, mode, which):
    """Constant emission/opacity: Alg. 2 telescopes to alpha = 1-(1-a)^(L/xi),
    C = C_src * alpha (Eq. 3 with constant sigma: 1 - exp(-sigma L))."""
    vol = _with_coef(cfg1, np.full(cfg1.n_basis, 0.37))
    O = Oracle(vol)
    a_src, rgb = 0.02, np.array([0.9, 0.4, 0.1])
    tf = _const_tf([*rgb, a_src])
    cam = V.ortho_z(16, 16) if which == "ortho_z" else V.orbit_camera(V.Stream(5), 24, 16)
    step = V.StepParams(mode=mode, h=1 / 200, xi=1 / 128)
    img, stats = O.render(cam, tf, step)
    for j in range(cam.height):
        for i in range(cam.width):
            r = ray(cam, i, j)
            if r is None:
                assert np.all(img[j, i] == 0)
                continue
            L = (r[3] - r[2]) if which == "persp" else 1.0
            alpha = 1 - (1 - a_src) ** (L / step.xi)
            sigma = -np.log(1 - a_src) / step.xi
            assert img[j, i, 3] == pytest.approx(1 - np.exp(-sigma * L), abs=1e-12)
            assert img[j, i, 3] == pytest.approx(alpha, abs=1e-12)
            np.testing.assert_allclose(img[j, i, :3], rgb * alpha, atol=1e-12)


def test_tf_linear_interpolation(cfg1):
    """A ramp TF maps a constant field value v to alpha = v exactly (per segment
    of length xi); endpoints clamp."""
    ramp = np.zeros((256, 4))
    ramp[:, 3] = np.arange(256) / 255.0 * 0.5
    ramp[:, 0] = 1.0
    cam = V.ortho_z(4, 4)
    for v, want in [(0.3, 0.15), (0.0, 0.0), (1.0, 0.5), (-0.2, 0.0), (1.7, 0.5), (0.123456, 0.061728)]:
        vol = _with_coef(cfg1, np.full(cfg1.n_basis, v))
        step = V.StepParams(mode="fixed", h=1 / 4, xi=1 / 4)
        img, _ = Oracle(vol).render(cam, V.TransferFunction(table=ramp), step)
        # 4 segments of length xi, each with opacity `want`
        assert img[0, 0, 3] == pytest.approx(1 - (1 - want) ** 4, abs=1e-12)


def heuristic_count_pin(vol, O, mult=None):
    """Eq. 4 on axis-aligned rays, walked independently in exact rational
    arithmetic: from z = 1 downwards, the sample at z belongs to the element
    with lo_z <= z < hi_z (z = 1: the top element) and advances by 2^-d times
    that element's shortest side, d = max degree.  Dyadic knots make the
    oracle's FP32 walk exact, so the sample counts must agree exactly; per
    element the count is within one of s_z / step."""
    from fractions import Fraction as Fr
    cam = V.ortho_z(16, 16)
    tf = _const_tf([1, 1, 1, 0.0])
    if mult is None:
        img, stats = O.render(cam, tf, V.StepParams(mode="heuristic"))
    else:
        img, stats = O.render(cam, tf, V.StepParams(mode="learned", mult=mult))
    b = vol.elem_box
    d = int(max(vol.deg))
    total = 0
    for j in range(16):
        for i in range(16):
            x, y = (i + 0.5) / 16, 1 - (j + 0.5) / 16
            col = np.nonzero((b[:, 0] <= x) & (x < b[:, 3]) & (b[:, 1] <= y) & (y < b[:, 4]))[0]
            lo = [Fr(b[e, 2]) for e in col]
            hi = [Fr(b[e, 5]) for e in col]
            step = [Fr(float(np.min(b[e, 3:] - b[e, :3]))) / 2 ** d * Fr(1 if mult is None else float(mult[e]))
                    for e in col]
            z, per = Fr(1), {}
            while z > 0:
                k = next(q for q in range(len(col)) if lo[q] <= z and (z < hi[q] or z == 1 == hi[q]))
                per[k] = per.get(k, 0) + 1
                z -= step[k]
            total += sum(per.values())
            if mult is None:
                for k, n in per.items():
                    assert abs(n - (hi[k] - lo[k]) / step[k]) <= 1
    assert stats["samples"] == total
    e0 = int(np.argmin(np.min(b[:, 3:] - b[:, :3], axis=1)))
    assert O.heuristic_step(e0) == pytest.approx(np.min(b[e0, 3:] - b[e0, :3]) / 2 ** d)


def anisotropic_volume():
    """Tri-degree (2,3,1) on a 4x8x2 start mesh (elements 1/4 x 1/8 x 1/2),
    refined once: anisotropic boxes, dyadic knots."""
    return V.refined_ball((2, 3, 1), (4, 8, 2), centres=((0.6, 0.4, 0.5),), radii=(0.3,))


def test_heuristic_step_counts(cfg1, cfg1_oracle):
    heuristic_count_pin(cfg1, cfg1_oracle)


def test_heuristic_step_counts_anisotropic():
    vol = anisotropic_volume()
    heuristic_count_pin(vol, Oracle(vol))


def test_learned_step_counts():
    """Learned steps (Eq. 4 times a per-element multiplier): power-of-two
    multipliers keep the walk exact, so the counts match a rational walk."""
    vol = anisotropic_volume()
    mult = (2.0 ** np.floor(V.Stream(77).uniform(0.0, 3.0, vol.n_elem))).astype(np.float32)
    heuristic_count_pin(vol, Oracle(vol), mult=mult)


def test_learned_unit_multipliers_equal_heuristic(cfg1, cfg1_oracle):
    tf, cams = V.config1_render()
    a, sa = cfg1_oracle.render(cams[1], tf, V.StepParams(mode="heuristic", alpha_stop=0.99))
    b, sb = cfg1_oracle.render(cams[1], tf, V.StepParams(mode="learned", alpha_stop=0.99,
                                                          mult=np.ones(cfg1.n_elem, np.float32)))
    assert np.array_equal(a, b) and sa == sb


def test_fixed_step_converges(cfg1, cfg1_oracle):
    """Fixed-step images approach a limit as h -> 0 (Riemann sums of Eq. 3)."""
    tf, cams = V.config1_render()
    cam = V.ortho_z(12, 12)
    imgs = [cfg1_oracle.render(cam, tf, V.StepParams(h=h, xi=1 / 256))[0] for h in (1 / 64, 1 / 128, 1 / 256, 1 / 512)]
    d = [np.abs(imgs[k + 1] - imgs[k]).max() for k in range(3)]
    assert d[2] < d[1] < d[0]
    assert d[2] < 0.6 * d[1]


def test_early_termination_and_miss(cfg1_oracle):
    tf = _const_tf([1, 0.5, 0.25, 0.5])
    cam = V.ortho_z(4, 4)
    full, s_full = cfg1_oracle.render(cam, _const_tf([1, 0.5, 0.25, 0.05]), V.StepParams(h=1 / 64, xi=1 / 64))
    cut, s_cut = cfg1_oracle.render(cam, tf, V.StepParams(h=1 / 64, xi=1 / 64, alpha_stop=0.9))
    assert s_cut["samples"] == 16 * 4          # 1-(1/2)^k >= 0.9 at k = 4
    assert np.all(cut[..., 3] == 1 - 0.5 ** 4)
    assert s_full["samples"] == 16 * 64         # alpha = 1 - 0.95^64 < 1: no termination
    # with alpha_stop = 1 a ray stops once alpha_dst rounds to exactly 1
    sat, s_sat = cfg1_oracle.render(cam, tf, V.StepParams(h=1 / 64, xi=1 / 64))
    assert s_sat["samples"] == 16 * 54 and np.all(sat[..., 3] == 1.0)
    miss = V.Camera("ortho", 4, 4, eye=(5.0, 5.0, 5.0), target=(6.0, 5.0, 5.0), up=(0.0, 0.0, 1.0), extent=0.5)
    img, s = cfg1_oracle.render(miss, tf, V.StepParams())
    assert s["rays_hit"] == 0 and np.all(img == 0)

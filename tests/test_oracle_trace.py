"""Pins of the oracle's per-sample trace (Oracle.render_trace), the reference
the render kernel's own samples are compared with.

Each pixel's trace is rebuilt here independently of oracle.c:
  - sample positions, element ids and steps by an exact rational walk with
    correctly rounded FP32 operations (the FP32 decisions of Sec. 4 / Eq. 4 /
    Alg. 1 as lrvol.h states them: p_k = clamp(fmaf(t_k, d, o), 0, 1), the
    element by brute-force box search, t_{k+1} = t_k + ds(e_k) (times the
    multiplier for learned steps) or fmaf(k+1, h, t_in));
  - values through the interpolated Bezier blocks (Sec. 3.2.3), a code path
    that shares nothing with the oracle's Cox-de Boor evaluation;
  - the pixel's RGBA by running Alg. 2 over the traced samples in numpy.
Only the FP32 ray (origin, direction, t_in, t_out) is taken from the oracle;
its own pin is in test_oracle_pins.py.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle.oracle import Oracle, ray
from paper_1707_01170_gb300.synth import volumes as V

F32_INF = np.float32(np.inf)


def rn32(x: Fraction) -> float:
    """x rounded to the nearest FP32 value, ties to even (exact)."""
    f = np.float32(float(x))
    cands = [np.nextafter(f, -F32_INF), f, np.nextafter(f, F32_INF)]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - x), int(np.float32(c).view(np.uint32)) & 1))
    return float(best)


def find_element(box, p):
    """Brute-force half-open box search; the upper domain face belongs to the element with hi = 1."""
    lo, hi = box[:, :3], box[:, 3:]
    ok = np.all((lo <= p) & ((p < hi) | ((p == 1.0) & (hi == 1.0))), axis=1)
    idx = np.nonzero(ok)[0]
    assert idx.size == 1, (p, idx)
    return int(idx[0])


def eq4_step(box, deg, e):
    """Eq. 4: 2^-d times the shortest side (FP64), rounded once to FP32."""
    side = np.min(box[e, 3:] - box[e, :3])
    return rn32(Fraction(float(side)) / 2 ** int(max(deg)))


def walk(vol, cam, i, j, step, max_samples=100000):
    """Independent FP32 march of one pixel: list of (t, element, segment)."""
    r = ray(cam, i, j)
    if r is None:
        return []
    o, d, tin, tout = r
    out = []
    t = tin
    k = 0
    while t < tout and k < max_samples:
        p = np.array([min(max(rn32(Fraction(t) * Fraction(float(d[c])) + Fraction(float(o[c]))), 0.0), 1.0)
                      for c in range(3)])
        e = find_element(vol.elem_box, p)
        if step.mode == "fixed":
            tn = rn32(Fraction(k + 1) * Fraction(float(np.float32(step.h))) + Fraction(tin))
        elif step.mode == "heuristic":
            tn = rn32(Fraction(t) + Fraction(eq4_step(vol.elem_box, vol.deg, e)))
        else:
            ds = rn32(Fraction(eq4_step(vol.elem_box, vol.deg, e)) * Fraction(float(step.mult[e])))
            tn = rn32(Fraction(t) + Fraction(ds))
        if not tn > t:
            tn = float(np.nextafter(np.float32(t), F32_INF))
        seg = float(Fraction(min(tn, tout)) - Fraction(t))
        out.append((t, e, seg, p))
        t = tn
        k += 1
    return out


def tf_lookup(tf, v):
    x = (v - tf.vmin) / (tf.vmax - tf.vmin)
    x = min(max(x, 0.0), 1.0) * 255.0
    i0 = min(int(np.floor(x)), 254)
    f = x - i0
    return (1 - f) * tf.table[i0] + f * tf.table[i0 + 1]


def composite(tf, vals, segs, xi, alpha_stop):
    """Alg. 2 over the traced samples; returns (RGBA, samples composited)."""
    C, A = np.zeros(3), 0.0
    n = 0
    for v, s in zip(vals, segs):
        src = tf_lookup(tf, v)
        T = (1 - src[3]) ** (s / xi)
        w = (1 - T) * (1 - A)
        C += w * src[:3]
        A += w
        n += 1
        if A >= alpha_stop:
            break
    return np.array([*C, A]), n


def field_values(O, blocks_of, elems, pts, field, comp):
    """Values at FP32 points through the interpolated Bezier blocks."""
    el = np.asarray(elems, dtype=np.int64)
    B = blocks_of(el)
    val = O.bezier_eval(B, el, np.asarray(pts, dtype=np.float64))
    if field == "magnitude":
        return np.linalg.norm(val, axis=1)
    return val[:, comp if field == "component" else 0]


def check_trace(vol, O, cam, tf, step, pix, max_samples=4096):
    trace, count, rgba, _ = O.render_trace(cam, tf, step, pix, max_samples)
    cache = {}

    def blocks_of(el):
        miss = [e for e in np.unique(el) if e not in cache]
        if miss:
            for e, b in zip(miss, O.bezier_blocks(np.array(miss))):
                cache[e] = b
        return np.stack([cache[e] for e in el])

    scale = float(np.abs(vol.coef).max())
    seen = 0
    for q, (i, j) in enumerate(pix):
        w = walk(vol, cam, int(i), int(j), step)
        n = int(count[q])
        if not w:
            assert n == 0 and np.all(rgba[q] == 0)
            continue
        seen += 1
        assert n <= len(w)
        tr = trace[q, :n]
        np.testing.assert_array_equal(tr[:, 0], [s[0] for s in w[:n]])           # t_k
        np.testing.assert_array_equal(tr[:, 1], [s[1] for s in w[:n]])           # element ids
        np.testing.assert_array_equal(tr[:, 3], [s[2] for s in w[:n]])           # segments
        want = field_values(O, blocks_of, tr[:, 1].astype(np.int64), [s[3] for s in w[:n]], step.field,
                            step.component)
        np.testing.assert_allclose(tr[:, 2], want, rtol=0, atol=1e-11 * scale)
        # Alg. 2 over the traced samples gives the pixel, and stops where the oracle stopped
        full = [s[2] for s in w]
        vals = list(tr[:, 2]) + [0.0] * (len(w) - n)
        rec, m = composite(tf, vals[:n], full[:n], step.xi, step.alpha_stop)
        np.testing.assert_allclose(rec, rgba[q], rtol=0, atol=1e-12)
        if step.alpha_stop >= 1.0:
            assert n == len(w)                                                   # walked to t_out
            assert sum(full) == pytest.approx(w[-1][0] - w[0][0] + full[-1], abs=1e-12)
        else:
            assert m == n and (n == len(w) or rec[3] >= step.alpha_stop)
    assert seen >= len(pix) // 4
    return trace, count, rgba


def _pixels(cam, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], axis=1).astype(np.int32)


@pytest.fixture(scope="module")
def cfg1():
    return V.load_config(1)


@pytest.fixture(scope="module")
def cfg1_oracle(cfg1):
    return Oracle(cfg1)


@pytest.mark.parametrize("mode", ["fixed", "heuristic", "learned"])
def test_trace_cfg1_oblique(cfg1, cfg1_oracle, mode):
    tf, cams = V.config1_render()
    step = V.StepParams(mode=mode, h=1 / 256, xi=1 / 256, alpha_stop=1.0)
    if mode == "learned":
        step.mult = (2.0 ** V.Stream(5).uniform(0.0, 3.0, cfg1.n_elem)).astype(np.float32)
    check_trace(cfg1, cfg1_oracle, cams[1], tf, step, _pixels(cams[1], 24, 1))


def test_trace_cfg1_perspective_early_termination(cfg1, cfg1_oracle):
    tf, _ = V.config1_render()
    tf.table = np.clip(tf.table * np.array([1, 1, 1, 4.0]), 0, 1)
    cam = V.orbit_camera(V.Stream(77), 100, 70)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.9)
    _, count, rgba = check_trace(cfg1, cfg1_oracle, cam, tf, step, _pixels(cam, 30, 2))
    assert np.any(rgba[:, 3] >= 0.9)                      # some rays do stop early


def test_trace_vector_nondyadic():
    """A (2,2,2) 3-vector volume with knots at multiples of 1/12 (not FP32
    exact): |v| and one component."""
    vol = V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3, seed=4)
    O = Oracle(vol)
    tf = V.seeded_tf(V.Stream(31), alpha_max=0.05)
    cam = V.orbit_camera(V.Stream(32), 64, 48)
    for field, comp, (lo, hi) in (("magnitude", 0, (0.0, 1.6)), ("component", 2, (-0.5, 1.0))):
        tf.vmin, tf.vmax = lo, hi
        step = V.StepParams(mode="heuristic", xi=1 / 128, field=field, component=comp)
        check_trace(vol, O, cam, tf, step, _pixels(cam, 16, 3))


def test_trace_matches_render_and_counts(cfg1, cfg1_oracle):
    """The traced march is the oracle's render: same RGBA, same statistics;
    max_samples only limits what is kept."""
    tf, cams = V.config1_render()
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    pix = _pixels(cams[1], 50, 4)
    tr, cnt, rgba, st = cfg1_oracle.render_trace(cams[1], tf, step, pix, 8)
    ref, rst = cfg1_oracle.render(cams[1], tf, step, pixels=pix)
    np.testing.assert_array_equal(rgba, ref)
    assert st == rst and int(cnt.sum()) == rst["samples"]
    tr2, cnt2, _, _ = cfg1_oracle.render_trace(cams[1], tf, step, pix, 400)
    np.testing.assert_array_equal(cnt, cnt2)
    np.testing.assert_array_equal(tr, tr2[:, :8])


def test_coefficient_hull_bounds_the_blocks():
    """The incidence hull used to scale per-sample tolerances contains every
    Bernstein coefficient of the element (convex combination), and equals the
    min / max of the coefficients found by a numpy support test."""
    for vol in (V.load_config(1),
                V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3,
                               seed=4)):
        O = Oracle(vol)
        el = np.arange(0, vol.n_elem, max(1, vol.n_elem // 300))
        hull = O.coefficient_hull(el)
        B = O.bezier_blocks(el).reshape(len(el), vol.ncomp, -1)
        scale = np.abs(vol.coef).max()
        assert np.all(B.min(axis=2) >= hull[:, :, 0] - 1e-12 * scale)
        assert np.all(B.max(axis=2) <= hull[:, :, 1] + 1e-12 * scale)
        p = [int(x) for x in vol.deg]
        kx, ky = vol.knots[:, :p[0] + 2], vol.knots[:, p[0] + 2:p[0] + p[1] + 4]
        kz = vol.knots[:, p[0] + p[1] + 4:]
        for r, e in enumerate(el[:40]):
            b = vol.elem_box[e]
            sup = ((kx[:, 0] <= b[0]) & (b[3] <= kx[:, -1]) & (ky[:, 0] <= b[1]) & (b[4] <= ky[:, -1]) &
                   (kz[:, 0] <= b[2]) & (b[5] <= kz[:, -1]))
            np.testing.assert_array_equal(hull[r, :, 0], vol.coef[sup].min(axis=0))
            np.testing.assert_array_equal(hull[r, :, 1], vol.coef[sup].max(axis=0))

"""Pins of the oracle's gradient (Eq. 2 differentiated factor by factor) and
of gradient shading (Sec. 4.1: C_src times I = max(0.4, |l . n|)) to things
other than themselves: central finite differences, scipy's B-spline
derivative, exact gradients of reproduced polynomials, and closed forms of
shaded images (a constant field has no gradient beyond rounding, far below
the 1e-3 (vmax - vmin) floor, so I = 0.4; a field linear in z seen along z
with the light at the eye gives I = 1, with the light along x I = 0.4, and
with the light along (0, 3, 4) I = 0.8)."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import Oracle
from paper_1707_01170_gb300.synth import volumes as V

import test_oracle_pins as P


def test_bspline_derivative_matches_scipy():
    interpolate = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = int(rng.integers(1, 5))
        k = np.sort(rng.random(p + 2))
        d = interpolate.BSpline.basis_element(k, extrapolate=False).derivative()
        for x in k[0] + (k[-1] - k[0]) * rng.random(20):
            if np.min(np.abs(x - k)) < 1e-9:
                continue
            want = float(np.nan_to_num(d(x)))
            assert orc.bspline_d1(k, p, x) == pytest.approx(want, rel=1e-10, abs=1e-10)


def test_bspline_derivative_repeated_knots_finite_differences():
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = int(rng.integers(1, 5))
        k = np.sort(rng.random(p + 2))
        m = int(rng.integers(1, p + 1))             # a knot of multiplicity m <= p
        j = int(rng.integers(0, p + 2 - m + 1))
        k[j:j + m] = k[j]
        k = np.sort(k)
        for x in k[0] + (k[-1] - k[0]) * rng.random(10):
            if np.min(np.abs(x - k)) < 1e-5:
                continue
            h = 1e-7
            fd = (orc.bspline(k, p, x + h) - orc.bspline(k, p, x - h)) / (2 * h)
            assert orc.bspline_d1(k, p, x) == pytest.approx(fd, rel=1e-5, abs=1e-4)


def test_bspline_derivative_right_hand_at_knots():
    # linear hat on 0, 0.5, 1: slope +2 on [0, 0.5), -2 on [0.5, 1]
    k = [0.0, 0.5, 1.0]
    assert orc.bspline_d1(k, 1, 0.0) == 2.0
    assert orc.bspline_d1(k, 1, 0.5) == -2.0
    assert orc.bspline_d1(k, 1, 1.0) == -2.0       # domain end: the last piece
    assert orc.bspline_d1([0.2, 0.6], 0, 0.3) == 0.0


def test_gradient_matches_finite_differences(cfg1, cfg1_oracle):
    rng = np.random.default_rng(4)
    box = cfg1.elem_box
    e = rng.integers(0, cfg1.n_elem, 300)
    u = 0.1 + 0.8 * rng.random((300, 3))              # element interiors
    X = box[e, :3] + u * (box[e, 3:] - box[e, :3])
    val, grad = cfg1_oracle.eval_grad(X)
    np.testing.assert_allclose(val, cfg1_oracle.eval(X), atol=1e-14)
    h = 1e-6
    for a in range(3):
        dx = np.zeros(3)
        dx[a] = h
        fd = (cfg1_oracle.eval(X + dx)[:, 0] - cfg1_oracle.eval(X - dx)[:, 0]) / (2 * h)
        np.testing.assert_allclose(grad[:, 0, a], fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("deg,polys", [
    ((3, 3, 3), ([0.3, 1.0, -0.8], [0.5, -0.2, 0.9], [1.0, 0.3, 0.4])),
    ((2, 2, 2), ([0.1, -1.0, 2.0], [0.2, 0.5, -0.3], [1.0, 0.0, 1.0])),
    ((1, 1, 1), ([0.1, -1.0], [0.2, 0.5], [1.0, 0.7])),
])
def test_gradient_of_reproduced_polynomials(deg, polys):
    """Coefficients carried through LR refinement reproduce prod_a P_a(x_a);
    the gradient must be its exact gradient, at faces too."""
    from paper_1707_01170_gb300.synth.lrgen import Refiner
    R = Refiner(deg, (4, 4, 4), 2, 1)
    R.set_coef(P._blossom_coef(R.knots(), deg, polys))
    for rad in (0.3, 0.15):
        e = R.element_boxes()
        c = 0.5 * (e[:, :3] + e[:, 3:])
        R.refine(np.linalg.norm(c - np.array([0.45, 0.5, 0.55]), axis=1) < rad)
    vol = R.volume()
    O = Oracle(vol)
    X = P._points_with_faces(vol, 2000, 12)
    _, grad = O.eval_grad(X)
    for a in range(3):
        want = np.ones(len(X))
        for b in range(3):
            c = list(reversed(polys[b]))
            want *= np.polyval(np.polyder(c) if b == a else c, X[:, b])
        np.testing.assert_allclose(grad[:, 0, a], want, atol=1e-11)


def _shade(step, **kw):
    return V.StepParams(**{**step.__dict__, **kw})


def test_shading_of_a_constant_field_is_0p4(cfg1):
    vol = P._with_coef(cfg1, np.full(cfg1.n_basis, 0.37))
    O = Oracle(vol)
    tf = P._const_tf([0.9, 0.4, 0.1, 0.02])
    cam = V.orbit_camera(V.Stream(5), 20, 14)
    step = V.StepParams(mode="heuristic", xi=1 / 128)
    plain, _ = O.render(cam, tf, step)
    lit, _ = O.render(cam, tf, _shade(step, shading="gradient"))
    np.testing.assert_allclose(lit[..., :3], 0.4 * plain[..., :3], atol=1e-15)
    np.testing.assert_array_equal(lit[..., 3], plain[..., 3])


def _linear_in_z():
    """f = 0.2 + 0.6 z on a refined tricubic mesh (carried blossoms)."""
    from paper_1707_01170_gb300.synth.lrgen import Refiner
    deg, polys = (3, 3, 3), ([1.0], [1.0], [0.2, 0.6])
    R = Refiner(deg, (4, 4, 4), 1, 1)
    R.set_coef(P._blossom_coef(R.knots(), deg, polys))
    e = R.element_boxes()
    R.refine(np.linalg.norm(0.5 * (e[:, :3] + e[:, 3:]) - 0.5, axis=1) < 0.3)
    return R.volume()


def test_shading_closed_forms_linear_field():
    O = Oracle(_linear_in_z())
    tf = V.seeded_tf(V.Stream(9), alpha_max=0.1)
    cam = V.ortho_z(12, 12)                          # rays along -z: headlight l = (0, 0, 1), n = (0, 0, 1)
    step = V.StepParams(mode="heuristic", xi=1 / 256)
    plain, _ = O.render(cam, tf, step)
    head, _ = O.render(cam, tf, _shade(step, shading="gradient"))
    side, _ = O.render(cam, tf, _shade(step, shading="gradient", light=(1.0, 0.0, 0.0)))
    tilt, _ = O.render(cam, tf, _shade(step, shading="gradient", light=(0.0, 3.0, 4.0)))
    np.testing.assert_allclose(head, plain, atol=1e-14)
    np.testing.assert_allclose(side[..., :3], 0.4 * plain[..., :3], atol=1e-14)
    np.testing.assert_allclose(tilt[..., :3], 0.8 * plain[..., :3], atol=1e-14)
    assert plain[..., 3].max() > 0.2

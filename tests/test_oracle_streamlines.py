"""Pins of the oracle's streamlines (Sec. 5, Eq. 5-7) to things other than
themselves: the exact solution of a linear (helical) field, which quadratic
LR-splines reproduce exactly, gives each fixed-step method its order of
convergence (a wrong tableau entry drops it); a constant field is
integrated exactly by every method; the Eq. 4 step on a uniform mesh is
known in closed form; adaptive methods meet their tolerance; and the
Eq. 7 metric of a shifted copy is the shift times the time span."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, streamline_error
from paper_1707_01170_gb300.synth import volumes as V

OMEGA, VZ = 2 * math.pi, 0.05
ORDERS = {"RK1": 1, "RK2": 2, "RK3": 3, "RK4": 4, "RK38": 4, "RKF5": 5, "HE": 2, "BS": 3, "RKF45": 5}


def helix_volume():
    """f(x) = (-w (y - 1/2), w (x - 1/2), vz): linear, carried exactly through
    the refinement of a triquadratic mesh."""
    def lin(g):
        return np.stack([-OMEGA * (g[:, 1] - 0.5), OMEGA * (g[:, 0] - 0.5), np.full(len(g), VZ)], axis=1)
    return V.refined_ball((2, 2, 2), (4, 4, 4), centres=((0.5, 0.5, 0.5),), radii=(0.3,), ncomp=3, carry_fn=lin)


def helix_exact(seeds, t):
    c, s = np.cos(OMEGA * t), np.sin(OMEGA * t)
    dx, dy = seeds[:, 0] - 0.5, seeds[:, 1] - 0.5
    return np.stack([0.5 + c * dx - s * dy, 0.5 + s * dx + c * dy, seeds[:, 2] + VZ * t], axis=1)


def _seeds(n=24, seed=3):
    rng = np.random.default_rng(seed)
    r = 0.15 + 0.15 * rng.random(n)
    a = 2 * math.pi * rng.random(n)
    return np.stack([0.5 + r * np.cos(a), 0.5 + r * np.sin(a), 0.3 + 0.2 * rng.random(n)], axis=1)


@pytest.fixture(scope="module")
def helix():
    return Oracle(helix_volume())


def test_helix_field_is_reproduced(helix):
    X = np.random.default_rng(0).random((500, 3))
    want = np.stack([-OMEGA * (X[:, 1] - 0.5), OMEGA * (X[:, 0] - 0.5), np.full(500, VZ)], axis=1)
    np.testing.assert_allclose(helix.eval(X), want, atol=1e-12)


@pytest.mark.parametrize("method", sorted(ORDERS))
def test_fixed_step_order(helix, method):
    seeds = _seeds()
    q = ORDERS[method]
    hs = (1 / 64, 1 / 128) if q <= 2 else (1 / 16, 1 / 32)
    errs = []
    for h in hs:
        out, cnt, st = helix.streamlines(seeds, method, "fixed", h, 1.0, max_samples=200)
        assert np.all(st == 0) and np.all(cnt == round(1 / h) + 1)
        end = out[np.arange(len(seeds)), cnt - 1, :3]
        assert np.all(out[np.arange(len(seeds)), cnt - 1, 3] == 1.0)
        errs.append(np.abs(end - helix_exact(seeds, 1.0)).max())
    ratio = errs[0] / errs[1]
    assert 2 ** q * 0.7 < ratio < 2 ** q * 1.45, (method, errs, ratio)


@pytest.mark.parametrize("method", ["RK1", "RK4", "RKF5", "BS"])
def test_constant_field_is_exact_and_heuristic_step_closed_form(method):
    vol = V.tensor_product((3, 3, 3), (4, 4, 4), ncomp=3, coef=np.tile([0.3, 0.2, 0.1], (7 ** 3, 1)))
    O = Oracle(vol)
    seeds = np.array([[0.1, 0.1, 0.1], [0.2, 0.15, 0.3]])
    out, cnt, st = O.streamlines(seeds, method, "heuristic", 1.0, 1.0, max_samples=100)
    # Eq. 4 on a uniform 4^3 cubic mesh: 2^-3 / 4 = 1/32 everywhere
    assert np.all(st == 0) and np.all(cnt == 33)
    np.testing.assert_allclose(out[:, :33, 3], np.tile(np.arange(33) / 32, (2, 1)), atol=1e-15)
    want = seeds[:, None, :] + out[:, :33, 3:4] * np.array([0.3, 0.2, 0.1])
    np.testing.assert_allclose(out[:, :33, :3], want, atol=1e-14)
    # base factor 1/2 halves the step
    _, cnt2, _ = O.streamlines(seeds, method, "heuristic", 0.5, 1.0, max_samples=100)
    assert np.all(cnt2 == 65)


def test_domain_exit_and_sample_cap():
    vol = V.tensor_product((2, 2, 2), (2, 2, 2), ncomp=3, coef=np.tile([1.0, 0.0, 0.0], (4 ** 3, 1)))
    O = Oracle(vol)
    out, cnt, st = O.streamlines([[0.55, 0.5, 0.5]], "RK4", "fixed", 0.1, 10.0, max_samples=100)
    assert st[0] == 1 and cnt[0] == 5                       # x = 0.55, ..., 0.95; the step to 1.05 leaves
    assert out[0, 4, 0] == pytest.approx(0.95, abs=1e-14)
    out, cnt, st = O.streamlines([[0.1, 0.5, 0.5]], "RK4", "fixed", 0.01, 10.0, max_samples=7)
    assert st[0] == 2 and cnt[0] == 7


@pytest.mark.parametrize("method", ["HE", "BS", "RKF45"])
def test_adaptive_meets_tolerance(helix, method):
    seeds = _seeds(12, 5)
    errs, steps = [], []
    for tol in (1e-5, 1e-7):
        out, cnt, st = helix.streamlines(seeds, method, "adaptive", 0.0, 1.0, tol=tol, max_samples=20000)
        assert np.all(st == 0)
        end = out[np.arange(len(seeds)), cnt - 1, :3]
        errs.append(np.abs(end - helix_exact(seeds, 1.0)).max())
        steps.append(cnt.mean())
    # tighter tolerance: smaller global error, more steps; error within a few hundred local tolerances
    assert errs[1] < errs[0] and steps[1] > steps[0]
    assert errs[1] < 300 * 1e-7


def test_eq7_metric_of_a_shift():
    t = np.linspace(0, 2, 41)
    ref = np.zeros((1, 41, 4))
    ref[0, :, 0] = 0.2 + 0.1 * t
    ref[0, :, 3] = t
    app = ref.copy()
    app[0, :, 1] += 3e-3                                     # a constant offset of 3e-3
    sums, E = streamline_error(ref, [41], app, [41])
    assert E == pytest.approx(2 * 3e-3, rel=1e-12)
    # the approximation's own times need not be the reference's (linear track: interpolation exact)
    app2 = np.zeros((1, 7, 4))
    tt = np.array([0, 0.13, 0.5, 0.77, 1.2, 1.9, 2.0])
    app2[0, :, 0] = 0.2 + 0.1 * tt
    app2[0, :, 3] = tt
    assert streamline_error(ref, [41], app2, [7])[1] == pytest.approx(0.0, abs=1e-15)


def test_reference_convergence_of_the_metric(helix):
    """Eq. 7 against the exact helix: the RKF5 reference at h = 1/512 is far
    closer than RK4 at h = 1/32 (the metric ranks the approximations)."""
    seeds = _seeds(8, 7)
    t = np.arange(0, 513) / 512
    exact = np.zeros((len(seeds), 513, 4))
    for k, tk in enumerate(t):
        exact[:, k, :3] = helix_exact(seeds, tk)
        exact[:, k, 3] = tk
    ref, rc, _ = helix.streamlines(seeds, "RKF5", "fixed", 1 / 512, 1.0, max_samples=600)
    app, ac, _ = helix.streamlines(seeds, "RK4", "fixed", 1 / 32, 1.0, max_samples=64)
    e_ref = streamline_error(exact, np.full(8, 513), ref, rc)[1]
    e_app = streamline_error(exact, np.full(8, 513), app, ac)[1]
    assert e_ref < 1e-6 < e_app

"""The seeded input generator: RNG definition and LR-mesh invariants (no GPU)."""
import numpy as np

from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import Refiner, uniforms


def test_mt19937_64_standard_value():
    # The C++ standard fixes the 10000th output of a default-seeded mt19937_64.
    u = uniforms(5489, 10000)
    assert u[-1] == (9981545732273789042 >> 11) * 2.0 ** -53
    assert np.all((u >= 0) & (u < 1))


def test_seeded_streams_are_reproducible():
    a = V.Stream(123).take(50)
    b = V.Stream(123).take(50)
    assert np.array_equal(a, b)


def _check_partition(vol):
    b = vol.elem_box
    assert np.all(b[:, 3:] > b[:, :3])
    assert np.all((b >= 0) & (b <= 1))
    assert abs(np.prod(b[:, 3:] - b[:, :3], axis=1).sum() - 1.0) < 1e-12
    rng = np.random.default_rng(0)
    X = rng.random((4000, 3))
    inside = ((b[None, :, :3] <= X[:, None, :]) & (X[:, None, :] < b[None, :, 3:])).all(axis=2)
    assert np.all(inside.sum(axis=1) == 1)      # no overlaps, no holes


def _check_supports(vol):
    """Each LR B-spline's support is a union of whole elements, its local knots
    are non-decreasing, and it covers at least one element."""
    b = vol.elem_box
    sl = vol.knot_slices()
    for i in range(0, vol.n_basis, max(1, vol.n_basis // 400)):
        lo = np.array([vol.knots[i, sl[a]][0] for a in range(3)])
        hi = np.array([vol.knots[i, sl[a]][-1] for a in range(3)])
        for a in range(3):
            assert np.all(np.diff(vol.knots[i, sl[a]]) >= 0)
        ov = np.all((b[:, :3] < hi) & (b[:, 3:] > lo), axis=1)
        inner = np.all((b[:, :3] >= lo) & (b[:, 3:] <= hi), axis=1)
        assert ov.any() and np.array_equal(ov, inner)


def test_config1_mesh(cfg1):
    assert cfg1.n_elem == 9864 and cfg1.ncomp == 1 and list(cfg1.deg) == [3, 3, 3]
    _check_partition(cfg1)
    _check_supports(cfg1)
    assert cfg1.coef.min() == 0.0 and cfg1.coef.max() == 1.0


def test_refined_nondyadic_mesh():
    vol = V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2))
    _check_partition(vol)
    _check_supports(vol)
    assert np.any(vol.elem_box.astype(np.float32) != vol.elem_box)     # multiples of 1/12: not FP32-exact


def test_weights_positive_and_tensor_product_weights_one():
    vol = V.tensor_product((3, 3, 3), (3, 3, 3))
    assert np.all(vol.weight == 1.0)
    R = Refiner((3, 3, 3), (4, 4, 4), 1, 1)
    e = R.element_boxes()
    R.refine(np.linalg.norm(0.5 * (e[:, :3] + e[:, 3:]) - 0.5, axis=1) < 0.3)
    g = R.gamma()
    assert np.all(g > 0) and np.all(g <= 1.0 + 1e-15)

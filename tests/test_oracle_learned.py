"""Pins of the learned-step reference (oracle/learned.py, orc_labels) to
things other than themselves: finite differences, a closed-form Adam step,
BF16 rounding of known values, hand-computed features, and labels of
constant fields (Alg. 2 telescopes, so every step size gives the same
segment composite)."""
import numpy as np
import pytest

from oracle import learned as OL
from oracle.oracle import Oracle
from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import LRVolume


def _params(seed, scale=0.3):
    u = V.Stream(seed, OL.N_PARAMS + 8).take(OL.N_PARAMS)
    return scale * (2 * u - 1)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(5)
    X = rng.normal(size=(37, OL.IN))
    t = rng.normal(size=37)
    loss, g = OL.loss_and_grad(p, X, t)
    idx = np.concatenate([rng.choice(OL.N_PARAMS, 60, replace=False), [OL.N_PARAMS - 1]])
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (OL.loss_and_grad(p + e, X, t)[0] - OL.loss_and_grad(p - e, X, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), i
    assert loss == pytest.approx(0.5 * np.mean((OL.forward(p, X) - t) ** 2))


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    p1, m, v = OL.adam(p, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # bias-corrected first step: lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_every_step_closed_form():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step t, so each update is lr * g / (|g| + eps): a wrong or
    missing bias correction shows from t = 2 on."""
    g = np.array([0.3, -4.0, 1e-3])
    p, m, v = np.array([1.0, -2.0, 0.5]), np.zeros(3), np.zeros(3)
    for t in range(1, 8):
        p1, m, v = OL.adam(p, g, m, v, t, 0.01)
        np.testing.assert_allclose(p1 - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-12)
        p = p1


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -7, -2.5, 3.140625, 1 + 2 ** -8 + 2 ** -20])
    want = np.array([1.0, 1.0, 1 + 2 ** -7, 1 + 2 ** -7, -2.5, 3.140625, 1 + 2 ** -7])
    np.testing.assert_array_equal(OL.bf16(x), want)


def test_forward_emulation_is_rounding_of_the_fp64_forward():
    rng = np.random.default_rng(1)
    p = _params(6)
    X = rng.normal(size=(200, OL.IN))
    a, b = OL.forward(p, X), OL.forward(p, X, emulate_bf16=True)
    assert np.max(np.abs(a - b)) < 0.05 * (1 + np.max(np.abs(a)))
    assert np.max(np.abs(a - b)) > 0


def test_features_single_element_by_hand():
    """One clamped tricubic element: the block equals the coefficients."""
    coef = np.linspace(0.21, 0.61, 64)   # ends away from TF bin edges
    vol = V.tensor_product((3, 3, 3), (1, 1, 1), coef=coef[:, None])
    orc = Oracle(vol)
    table = np.zeros((256, 4))
    table[:, 3] = np.arange(256) / 255.0                      # alpha ramp
    table[:, 0] = np.where(np.arange(256) < 128, 0.25, 0.75)  # red step at 128
    tf = V.TransferFunction(table=table, vmin=0.0, vmax=1.0)
    cam = V.Camera("persp", 8, 8, eye=(0.5, 0.5, 3.0), target=(0.5, 0.5, 0.5), up=(0.0, 1.0, 0.0), fovy=0.5)
    F = OL.features(orc, vol.elem_box, cam, tf)[0]
    np.testing.assert_allclose(F[0:3], np.log2(64.0))
    assert F[3] == pytest.approx(0.21) and F[4] == pytest.approx(0.61) and F[5] == pytest.approx(0.4)
    i0, i1 = 53, 156
    assert F[6] == pytest.approx(i1 / 255) and F[7] == pytest.approx((i0 + i1) / 2 / 255)
    assert F[8] == pytest.approx(1.0) and F[9] == pytest.approx(0.5)
    np.testing.assert_allclose(F[10:13], [0, 0, -1], atol=1e-12)
    assert F[13] == pytest.approx(np.log2(2048 / 8)) and F[14] == pytest.approx(1.0)
    assert F[15] == pytest.approx(np.log2(1 + 255 * 0.4))


def test_labels_constant_field_accept_every_candidate(cfg1):
    vol = LRVolume(deg=cfg1.deg, elem_box=cfg1.elem_box, knots=cfg1.knots,
                   coef=np.full((cfg1.n_basis, 1), 0.4), weight=cfg1.weight, grid=cfg1.grid)
    orc = Oracle(vol)
    tf, _ = V.config1_render()
    cand = [1, 1.5, 2, 3, 4]
    lab = orc.labels(V.ortho_z(8, 8), tf, V.StepParams(mode="heuristic"), 1 / 2048, 1e-9, cand)
    visited = lab < len(cand)
    assert visited.sum() > 20
    assert np.all(lab[visited] == len(cand) - 1)


def test_labels_monotone_in_tau(cfg1, cfg1_oracle):
    tf, _ = V.config1_render()
    cam = V.ortho_z(6, 6)
    cand = [1, 2, 4, 8]
    step = V.StepParams(mode="heuristic")
    tight = cfg1_oracle.labels(cam, tf, step, 1 / 2048, 1e-7, cand)
    loose = cfg1_oracle.labels(cam, tf, step, 1 / 2048, 1e-2, cand)
    visited = tight < len(cand)
    assert np.array_equal(visited, loose < len(cand))
    assert np.all(tight[visited] <= loose[visited]) and np.any(tight[visited] < loose[visited])


def _slab_volume():
    """Trilinear, constant in x and y; z knots 0, 0.5, 0.75, 1: elements
    e0 = z in [0, 0.5) (zero field), e1 = [0.5, 0.75) (ramp 0 -> 1),
    e2 = [0.75, 1] (ramp 1 -> 0).  Eq. 4 steps: 1/4 in e0, 1/8 in e1, e2."""
    zk = [[0, 0, 0.5], [0, 0.5, 0.75], [0.5, 0.75, 1], [0.75, 1, 1]]
    zc = [0.0, 0.0, 1.0, 0.0]
    xk = [[0, 0, 1], [0, 1, 1]]
    knots, coef = [], []
    for kz, cz in zip(zk, zc):
        for ky in xk:
            for kx in xk:
                knots.append(kx + ky + kz)
                coef.append([cz])
    box = np.array([[0, 0, 0, 1, 1, 0.5], [0, 0, 0.5, 1, 1, 0.75], [0, 0, 0.75, 1, 1, 1]], dtype=np.float64)
    return LRVolume(deg=np.array([1, 1, 1]), elem_box=box, knots=np.array(knots, dtype=np.float64),
                    coef=np.array(coef), weight=np.ones(len(knots)), grid=np.array([1, 1, 4]))


def _slab_tf():
    table = np.ones((256, 4))
    table[:, 3] = 0.5 * np.arange(256) / 255.0
    return V.TransferFunction(table=table, vmin=0.0, vmax=1.0)


def test_labels_count_what_the_last_step_skips():
    """Looking along +z, every step longer than Eq. 4's from e0 lands at or
    past z = 0.75 and skips the opaque ramp in e1, so e0 takes label 0."""
    orc = Oracle(_slab_volume())
    cam = V.Camera("ortho", 2, 2, eye=(0.5, 0.5, -2.0), target=(0.5, 0.5, 0.0), up=(0.0, 1.0, 0.0), extent=0.5)
    lab = orc.labels(cam, _slab_tf(), V.StepParams(mode="heuristic", xi=1 / 256), 1 / 2048, 1e-3, [1, 1.5, 2, 4, 8])
    assert lab[0] == 0


def test_labels_weigh_errors_by_front_transmittance():
    """Looking along -z, e2's ramp leaves a transmittance of about 5e-7 in
    front of e1, so every candidate of e1 is acceptable there."""
    orc = Oracle(_slab_volume())
    cam = V.Camera("ortho", 2, 2, eye=(0.5, 0.5, 3.0), target=(0.5, 0.5, 0.5), up=(0.0, 1.0, 0.0), extent=0.5)
    cand = [1, 1.5, 2, 4, 8]
    lab = orc.labels(cam, _slab_tf(), V.StepParams(mode="heuristic", xi=1 / 256), 1 / 2048, 1e-3, cand)
    assert lab[1] == len(cand) - 1
    assert lab[2] < len(cand) - 1          # the ramp in front is judged at full weight


# ----------------------------------------------------------------------------
# the network forward against a hand-built network
# ----------------------------------------------------------------------------

def _hand_network():
    """Sparse weights whose forward is known in closed form (W[in][out]):
    h1_0 = relu(2 x0), h1_1 = relu(x1 + 0.5), h1_2 = relu(-1) = 0;
    h2_0 = relu(h1_0 + 3 h1_1 - 0.25) (the 3 sits at W2[1][0], so a
    transposed W2 feeds h2_1 instead); h3_5 = relu(0.5 h2_0 + 0.125);
    y = 4 h3_5 + 0.375.  Every weight and bias is exact in BF16."""
    d = {name: np.zeros(shape) for name, shape in OL.SIZES}
    d["W1"][0, 0], d["W1"][1, 1], d["b1"][1], d["b1"][2] = 2.0, 1.0, 0.5, -1.0
    d["W2"][0, 0], d["W2"][1, 0], d["b2"][0] = 1.0, 3.0, -0.25
    d["W3"][0, 5], d["b3"][5] = 0.5, 0.125
    d["W4"][5], d["b4"][0] = 4.0, 0.375
    return OL.pack(d)


def _hand_y(x0, x1):
    relu = lambda v: max(v, 0.0)
    h10, h11 = relu(2 * x0), relu(x1 + 0.5)
    h20 = relu(h10 + 3 * h11 - 0.25)
    return 4 * relu(0.5 * h20 + 0.125) + 0.375


# inputs exact in BF16 whose intermediates stay exact in BF16 too
_HAND_X = [(0.5, 0.25), (-0.75, 1.5), (0.0, -0.5), (1.25, -2.0), (-1.0, -1.0), (0.125, 0.0)]


def _hand_pin_holds(forward) -> bool:
    p = _hand_network()
    X = np.zeros((len(_HAND_X), OL.IN))
    X[:, 0], X[:, 1] = [a for a, _ in _HAND_X], [b for _, b in _HAND_X]
    X[:, 7] = 5.0                                   # an input no weight reads
    want = np.array([_hand_y(a, b) for a, b in _HAND_X])
    return bool(np.array_equal(forward(p, X), want) and np.array_equal(forward(p, X, emulate_bf16=True), want))


def test_forward_matches_hand_built_network():
    assert _hand_pin_holds(OL.forward)
    assert len({_hand_y(a, b) for a, b in _HAND_X}) >= 4           # the cases are not all alike


def test_multipliers_clamp_the_exponent():
    p = OL.pack({name: np.zeros(shape) for name, shape in OL.SIZES})
    X = np.zeros((1, OL.IN))
    for b4, ymax, want in ((-1.5, 3.0, 1.0), (1.5, 3.0, 2 ** 1.5), (5.0, 3.0, 8.0), (0.0, 0.0, 1.0)):
        p[-1] = b4
        np.testing.assert_allclose(OL.multipliers(p, X, ymax), [want], rtol=1e-15)
    # a lower clamp below zero lets the multiplier refine below Eq. 4
    for b4, ymin, want in ((-1.5, -2.0, 2 ** -1.5), (-3.0, -2.0, 0.25), (0.5, -1.0, 2 ** 0.5)):
        p[-1] = b4
        np.testing.assert_allclose(OL.multipliers(p, X, 3.0, ymin=ymin), [want], rtol=1e-15)


def test_hand_pin_catches_planted_forward_mistakes():
    """Mistakes planted in copies of the forward (on the CPU) trip the pin."""
    def make(mistake):
        def fwd(p, X, emulate_bf16=False):
            w = OL.unpack(p)
            r = OL.bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
            h = r(X)
            for k in (1, 2, 3):
                W = r(w[f"W{k}"])
                if mistake == "transposed W2" and k == 2:
                    W = W.T
                z = h @ W + (0.0 if mistake == "no bias" and k == 1 else w[f"b{k}"])
                h = r(z if mistake == "no relu" and k == 1 else np.maximum(z, 0.0))
            b4 = 0.0 if mistake == "no output bias" else w["b4"][0]
            return h @ (r(w["W4"]) if mistake != "W4 shifted" else np.roll(r(w["W4"]), 1)) + b4
        return fwd

    assert _hand_pin_holds(make(None))                                  # the copy itself is right
    for mistake in ("transposed W2", "no relu", "no bias", "no output bias", "W4 shifted"):
        assert not _hand_pin_holds(make(mistake)), mistake

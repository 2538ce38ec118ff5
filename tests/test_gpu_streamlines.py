"""Streamlines (Sec. 5) on the GPU against the FP64 oracle.

Step-wise parity: every recorded step x_n -> x_{n+1} of the GPU is redone
by the oracle from the GPU's x_n with the GPU's step h_n = t_{n+1} - t_n
(so step-size decisions need not coincide for the comparison to hold).
Bar per coordinate: 2 h (1e-5 max|c| + 1.2e-7 G) + 1e-12, from FP32 field
evaluation (1e-5 of the coefficient scale, the per-sample bar of the
renderer), stage points that may round to a neighbouring float (G bounds
|grad f|), and weights with sum |b_i| < 2.  The heuristic step itself is
checked exactly: h_n = base * Eq. 4 step of the element holding the FP32
rounding of x_n.  Globally the GPU's trajectories on a helical field
(reproduced exactly) converge with each method's order, and the Eq. 7
kernel equals the oracle's metric.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle, streamline_error
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V

import test_oracle_streamlines as SL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


@pytest.fixture(scope="module")
def helix():
    vol = SL.helix_volume()
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    yield vol, Oracle(vol), gv
    gv.close()


@pytest.fixture(scope="module")
def swirl():
    """A rough field: seeded coefficients on a refined triquadratic mesh."""
    vol = V.refined_ball((2, 2, 2), (4, 4, 4), centres=((0.4, 0.5, 0.55),), radii=(0.35, 0.18), ncomp=3, seed=12)
    vol.coef = (vol.coef - 0.5) * 2.0
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
    yield vol, Oracle(vol), gv
    gv.close()


def _gpu_lines(gv, seeds, method, rule, h, t_end, tol=0.0, max_samples=400):
    s, c, st = lv.streamlines(gv, torch.from_numpy(np.ascontiguousarray(seeds)).cuda(), method, rule, h, t_end, tol,
                              max_samples)
    return s.cpu().numpy(), c.cpu().numpy(), st.cpu().numpy()


def _stepwise(vol, orc, samples, count, method, G):
    xs, hs, nxt = [], [], []
    for j in range(len(samples)):
        for n in range(int(count[j]) - 1):
            xs.append(samples[j, n, :3])
            hs.append(samples[j, n + 1, 3] - samples[j, n, 3])
            nxt.append(samples[j, n + 1, :3])
    xs, hs, nxt = np.array(xs), np.array(hs), np.array(nxt)
    cmax = np.abs(vol.coef).max()
    worst = 0.0
    for h in np.unique(hs):
        sel = hs == h
        out, cnt, st = orc.streamlines(xs[sel], method, "fixed", h, h, max_samples=2)
        ok = cnt == 2
        assert ok.mean() > 0.99
        err = np.abs(out[ok, 1, :3] - nxt[sel][ok])
        bound = 2 * h * (1e-5 * cmax + 1.2e-7 * G) + 1e-12
        worst = max(worst, float((err / bound).max()))
    assert worst <= 1.0, worst
    return len(xs)


@pytest.mark.parametrize("method", ["RK1", "RK2", "RK3", "RK4", "RK38", "RKF5", "HE", "BS", "RKF45"])
def test_stepwise_parity_heuristic(swirl, method):
    vol, orc, gv = swirl
    seeds = np.random.default_rng(1).uniform(0.2, 0.8, (64, 3))
    s, c, st = _gpu_lines(gv, seeds, method, "heuristic", 1.0, 0.6)
    G = 2 * 2 * 1.0 * 48                                        # 2p max|c| / min element side
    steps = _stepwise(vol, orc, s, c, method, G)
    assert steps > 500
    # the heuristic step is exactly the Eq. 4 step of the element of the FP32 point
    for j in range(8):
        for n in range(int(c[j]) - 2):
            e = orc.eval(s[j, n, :3].astype(np.float32)[None], return_elem=True)[1][0]
            assert s[j, n + 1, 3] - s[j, n, 3] == pytest.approx(orc.heuristic_step(int(e)), rel=0, abs=1e-15)


STORE = {"f32": lv.STORE_F32, "f16": lv.STORE_F16, "bf16": lv.STORE_BF16}
# per-evaluation bound of 16-bit blocks, in units of the element's coefficient
# half range (at most max|c|): FP16 pairs with mixed-precision FMAs 2.04 u,
# BF16 converted at element entry 1.02 u
BLOCK_BOUND = {"f32": 0.0, "f16": 2.04 * 2.0 ** -11, "bf16": 1.02 * 2.0 ** -8}


@pytest.mark.parametrize("deg,storage", [(1, "f32"), (1, "f16"), (2, "f16"), (2, "bf16"), (3, "f32"), (3, "f16"),
                                         (3, "bf16")])
def test_stepwise_parity_degrees_and_storage(deg, storage):
    """RK4 with Eq. 4 steps on 3-vector volumes of every degree and block
    storage the tracer instantiates; each GPU step redone by the FP64 oracle
    with the bar above plus the 16-bit block bound, and the heuristic step
    exact."""
    vol = V.refined_ball((deg,) * 3, (4, 4, 4), centres=((0.4, 0.5, 0.55),), radii=(0.35, 0.18), ncomp=3,
                         seed=13 + deg)
    vol.coef = (vol.coef - 0.5) * 2.0
    orc = Oracle(vol)
    gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier(STORE[storage])
    seeds = np.random.default_rng(3 + deg).uniform(0.2, 0.8, (32, 3))
    s, c, st = _gpu_lines(gv, seeds, "RK4", "heuristic", 1.0, 0.4)
    gv.close()
    cmax = np.abs(vol.coef).max()
    min_side = float(np.min(vol.elem_box[:, 3:] - vol.elem_box[:, :3]))
    G = 2 * deg * cmax / min_side
    xs, hs, nxt = [], [], []
    for j in range(len(s)):
        for n in range(int(c[j]) - 1):
            xs.append(s[j, n, :3])
            hs.append(s[j, n + 1, 3] - s[j, n, 3])
            nxt.append(s[j, n + 1, :3])
    xs, hs, nxt = np.array(xs), np.array(hs), np.array(nxt)
    assert len(xs) > 300
    worst = 0.0
    for h in np.unique(hs):
        sel = hs == h
        out, cnt, _ = orc.streamlines(xs[sel], "RK4", "fixed", h, h, max_samples=2)
        ok = cnt == 2
        assert ok.mean() > 0.99
        err = np.abs(out[ok, 1, :3] - nxt[sel][ok])
        bound = 2 * h * ((1e-5 + BLOCK_BOUND[storage]) * cmax + 1.2e-7 * G) + 1e-12
        worst = max(worst, float((err / bound).max()))
    assert worst <= 1.0, worst
    for j in range(4):
        for n in range(int(c[j]) - 2):
            e = orc.eval(s[j, n, :3].astype(np.float32)[None], return_elem=True)[1][0]
            assert s[j, n + 1, 3] - s[j, n, 3] == pytest.approx(orc.heuristic_step(int(e)), rel=0, abs=1e-15)


@pytest.mark.parametrize("method,tol", [("HE", 1e-5), ("BS", 1e-6), ("RKF45", 1e-7)])
def test_stepwise_parity_adaptive(swirl, method, tol):
    vol, orc, gv = swirl
    seeds = np.random.default_rng(2).uniform(0.2, 0.8, (48, 3))
    s, c, st = _gpu_lines(gv, seeds, method, "adaptive", 0.0, 0.5, tol=tol, max_samples=4000)
    assert np.all(st != 3)
    _stepwise(vol, orc, s, c, method, 2 * 2 * 1.0 * 48)


@pytest.mark.parametrize("method", sorted(SL.ORDERS))
def test_gpu_orders_on_the_helix(helix, method):
    vol, orc, gv = helix
    seeds = SL._seeds()
    q = SL.ORDERS[method]
    hs = (1 / 64, 1 / 128) if q <= 2 else (1 / 16, 1 / 32)
    errs = []
    for h in hs:
        s, c, st = _gpu_lines(gv, seeds, method, "fixed", h, 1.0, max_samples=200)
        assert np.all(st == 0) and np.all(c == round(1 / h) + 1)
        end = s[np.arange(len(seeds)), c - 1, :3]
        errs.append(np.abs(end - SL.helix_exact(seeds, 1.0)).max())
    ratio = errs[0] / errs[1]
    assert 2 ** q * 0.7 < ratio < 2 ** q * 1.45, (method, errs, ratio)


def test_eq7_kernel_matches_oracle(helix):
    vol, orc, gv = helix
    seeds = SL._seeds(40, 9)
    ref = _gpu_lines(gv, seeds, "RKF5", "fixed", 1 / 256, 1.0, max_samples=300)
    app = _gpu_lines(gv, seeds, "RK2", "heuristic", 1.0, 1.0, max_samples=300)
    want, E = streamline_error(ref[0], ref[1], app[0], app[1])
    got = lv.streamline_error(*(torch.from_numpy(a).cuda() for a in (ref[0], ref[1], app[0], app[1]))).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)
    assert E > 0


def test_eq7_kernel_edge_cases():
    """Synthetic line sets: approximations running past the reference's last
    time, lines with 0 or 1 samples on either side, two-sample references,
    samples exactly at reference times, and lines longer than a warp's 32
    lanes many times over."""
    rng = np.random.default_rng(17)
    n, rmax, amax = 64, 700, 300
    ref = np.zeros((n, rmax, 4))
    app = np.zeros((n, amax, 4))
    rc = rng.integers(0, rmax + 1, n).astype(np.int32)
    ac = rng.integers(0, amax + 1, n).astype(np.int32)
    rc[:4] = (0, 1, 2, 2)
    ac[4:8] = (0, 1, 2, amax)
    for j in range(n):
        tr = np.cumsum(rng.uniform(1e-3, 3e-3, rmax))
        tr -= tr[0]
        ref[j, :, 3] = tr
        ref[j, :, :3] = rng.normal(size=(rmax, 3)).cumsum(axis=0) * 1e-2
        ta = np.cumsum(rng.uniform(1e-3, 8e-3, amax))
        ta -= ta[0]
        if j % 3 == 0:                       # some samples exactly at reference times
            k = np.concatenate([[0], np.sort(rng.choice(np.arange(1, rmax), amax - 1, replace=False))])
            ta = tr[k]
        app[j, :, 3] = ta
        app[j, :, :3] = rng.normal(size=(amax, 3)).cumsum(axis=0) * 1e-2
    want, E = streamline_error(ref, rc, app, ac)
    got = lv.streamline_error(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ref, rc, app, ac))).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)
    assert np.count_nonzero(want) > n // 2


def test_exit_cap_and_status_match_oracle():
    vol = V.tensor_product((2, 2, 2), (2, 2, 2), ncomp=3, coef=np.tile([1.0, 0.0, 0.0], (4 ** 3, 1)))
    gv = lv.Volume(vol).build_accel((4, 4, 4)).to_bezier(lv.STORE_BF16)
    orc = Oracle(vol)
    seeds = np.array([[0.55, 0.5, 0.5], [0.1, 0.5, 0.5], [1.5, 0.5, 0.5]])
    for max_samples, h in ((100, 0.1), (7, 0.01)):
        g = _gpu_lines(gv, seeds, "RK4", "fixed", h, 10.0, max_samples=max_samples)
        o = orc.streamlines(seeds, "RK4", "fixed", h, 10.0, max_samples=max_samples)
        np.testing.assert_array_equal(g[1], o[1])
        np.testing.assert_array_equal(g[2], o[2])
        for j in range(3):
            np.testing.assert_allclose(g[0][j, :g[1][j]], o[0][j, :o[1][j]], atol=1e-12)
    gv.close()


@pytest.mark.parametrize("method,rule,h,tol", [("RK4", "heuristic", 1.0, 0.0), ("RKF45", "adaptive", 0.0, 1e-6)])
def test_lines_do_not_depend_on_the_rake_size(swirl, method, rule, h, tol):
    """The launch traces 1 to 32 lines per warp depending on the number of
    seeds; every line must come out bit for bit the same either way."""
    vol, orc, gv = swirl
    seeds = np.random.default_rng(3).uniform(0.15, 0.85, (20000, 3))
    big = _gpu_lines(gv, seeds, method, rule, h, 0.6, tol, max_samples=512)
    for n in (1, 37, 700):
        small = _gpu_lines(gv, seeds[:n], method, rule, h, 0.6, tol, max_samples=512)
        np.testing.assert_array_equal(small[1], big[1][:n])
        np.testing.assert_array_equal(small[2], big[2][:n])
        for j in range(n):
            assert np.array_equal(small[0][j, :small[1][j]], big[0][j, :big[1][j]])
    assert (big[1] >= 2).mean() > 0.9


def test_rejects_bad_arguments(helix):
    vol, orc, gv = helix
    seeds = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(lv.LrvolError):
        lv.streamlines(gv, seeds, "RK4", "adaptive", 0.0, 1.0, 1e-6)
    with pytest.raises(lv.LrvolError):
        lv.streamlines(gv, seeds, "RK4", "fixed", 0.0, 1.0)
    scalar = lv.Volume(V.load_config(1)).build_accel((16, 16, 16)).to_bezier()
    with pytest.raises(lv.LrvolError) as e:
        lv.streamlines(scalar, seeds, "RK4", "fixed", 0.1, 1.0)
    assert e.value.status == lv.ERR_UNSUPPORTED
    scalar.close()

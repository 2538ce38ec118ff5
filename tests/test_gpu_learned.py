"""Learned step sizes on the GPU against the FP64 oracle (oracle/learned.py,
orc_labels, orc_render in learned mode).

Bars:
  learned render     same as the heuristic render (identical FP32 decisions:
                     the step is the FP32 product ds*m on both sides), RMSE
                     <= 1e-4; multipliers of 1 reproduce the heuristic image
                     bit for bit;
  features           1e-5 absolute (FP32 element geometry and block ranges);
                     the four TF-table features only where the bin range is
                     not decided by a value within 1e-3 bins of a bin edge;
  BF16 inference     against the oracle's forward with the same BF16 operand
                     rounding: FP32 vs FP64 accumulation can move an
                     activation across a BF16 rounding boundary, so log2 of
                     the multiplier is held to 3e-2 max and 3e-3 mean;
  FP32 gradient      relative 1e-4 of the largest gradient entry per layer,
                     on inputs whose pre-activations stay 2e-5 away from the
                     ReLU kink (so both sides take the same branch);
  Adam               moments within 4 FP32 ulps of their larger term, the
                     step within 1e-3 relative of the FP64 step;
  labels             between the oracle's labels at tau*(1 -+ 0.02) (the
                     decision error <= tau is FP32 on the GPU, FP64 in the
                     oracle; labels are monotone in tau), and equal for >= 98%
                     of the visited elements.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import learned as OL
from oracle.oracle import Oracle
from paper_1707_01170_gb300 import learned as LS
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import Stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


def _f32_tf(tf):
    tf.table = np.asarray(tf.table, dtype=np.float32).astype(np.float64)
    return tf


def _rmse(a, b):
    return float(np.sqrt(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)))


@pytest.fixture(scope="module")
def cfg1_gpu(cfg1):
    gv = lv.Volume(cfg1).build_accel((32, 32, 32)).to_bezier()
    yield gv
    gv.close()


def _seeded_mult(n, seed):
    u = Stream(seed, n + 8).take(n)
    return (2.0 ** (3.0 * u)).astype(np.float32)     # m in [1, 8)


# ----------------------------------------------------------------------------
# learned-mode rendering
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("view", [0, 1])
def test_learned_render_matches_oracle(cfg1, cfg1_oracle, cfg1_gpu, view):
    tf, cams = V.config1_render()
    tf = _f32_tf(tf)
    mult = _seeded_mult(cfg1.n_elem, 101 + view)
    step = V.StepParams(mode="learned", xi=1 / 256, alpha_stop=1.0, mult=mult)
    ref, ost = cfg1_oracle.render(cams[view], tf, step)
    gstep = V.StepParams(mode="learned", xi=1 / 256, alpha_stop=1.0, mult=torch.from_numpy(mult).cuda())
    img = cfg1_gpu.render(cams[view], tf, gstep).cpu().numpy()
    st = cfg1_gpu.stats()
    assert _rmse(img, ref) <= 1e-4
    assert st["rays_hit"] == ost["rays_hit"]
    assert abs(st["samples"] - ost["samples"]) <= 0.001 * ost["samples"]
    # the multipliers are in use: fewer samples than the heuristic
    _, hst = cfg1_oracle.render(cams[view], tf, V.StepParams(mode="heuristic", xi=1 / 256))
    assert ost["samples"] < 0.6 * hst["samples"]


def test_unit_multipliers_reproduce_heuristic(cfg1, cfg1_gpu):
    tf, cams = V.config1_render()
    ones = torch.ones(cfg1.n_elem, dtype=torch.float32, device="cuda")
    a = cfg1_gpu.render(cams[1], tf, V.StepParams(mode="learned", mult=ones, alpha_stop=0.97)).cpu()
    b = cfg1_gpu.render(cams[1], tf, V.StepParams(mode="heuristic", alpha_stop=0.97)).cpu()
    assert torch.equal(a, b)


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------

def _edge_rows(orc, tf, field, comp, blocks):
    """Elements whose TF bin range is decided by a value within 1e-3 bins of a
    bin edge (FP32 block ranges move 255*x by ~1e-4 bins at most)."""
    F = OL.features(orc, orc.box, V.ortho_z(), tf, field, comp, blocks)
    near = lambda x: (x > 0) & (x < 1) & (np.abs(255 * x - np.round(255 * x)) < 1e-3)
    return near(F[:, 3]) | near(F[:, 4])


@pytest.mark.parametrize("which", ["cfg1", "vec_mag", "vec_comp"])
def test_features_match_oracle(cfg1, cfg1_oracle, cfg1_gpu, which):
    if which == "cfg1":
        orc, gv, field, comp = cfg1_oracle, cfg1_gpu, "scalar", 0
        tf, cams = V.config1_render()
        cam = cams[1]
    else:
        vol = V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3, seed=4)
        orc = Oracle(vol)
        gv = lv.Volume(vol).build_accel((16, 16, 16)).to_bezier()
        field, comp = ("magnitude", 0) if which == "vec_mag" else ("component", 2)
        tf = V.seeded_tf(Stream(31), alpha_max=0.05)
        tf.vmin, tf.vmax = (0.0, 1.6) if field == "magnitude" else (0.0, 1.0)
        cam = V.orbit_camera(Stream(32), 64, 48)
    tf = _f32_tf(tf)
    blocks = orc.bezier_blocks()
    want = OL.features(orc, orc.box, cam, tf, field, comp, blocks)
    got = lv.features(gv, cam, tf, V.StepParams(mode="heuristic", field=field, component=comp)).cpu().numpy()
    assert got.shape == want.shape
    edge = _edge_rows(orc, tf, field, comp, blocks)
    assert edge.mean() < 0.02
    cols = [c for c in range(16) if c not in (6, 7, 8, 9)]
    np.testing.assert_allclose(got[:, cols], want[:, cols], atol=1e-5, rtol=1e-5)
    np.testing.assert_allclose(got[~edge][:, 6:10], want[~edge][:, 6:10], atol=1e-5, rtol=1e-5)
    if which != "cfg1":
        gv.close()


def test_features_match_oracle_full_size_cfg2():
    """The benchmark volume (cfg2, 174,000 elements) with its own TF and
    camera: 3,000 sampled elements against the oracle's features computed
    from its own Bezier blocks.  Its elements at the shells span up to the
    whole TF range, so the range scans run through the 16-bin aggregates as
    well as single bins (checked below)."""
    vol = V.load_config(2)
    tf, cam = V.config2_render(vol=vol)
    tf = _f32_tf(tf)
    orc = Oracle(vol)
    gv = lv.Volume(vol).build_accel((64, 64, 64)).to_bezier()
    got = lv.features(gv, cam, tf, V.StepParams(mode="heuristic")).cpu().numpy()
    gv.close()
    rng = np.random.default_rng(17)
    sel = np.sort(rng.choice(vol.n_elem, 3000, replace=False))
    want = OL.features(orc, orc.box[sel], cam, tf, "scalar", 0, orc.bezier_blocks(sel))
    got = got[sel]
    near = lambda x: (x > 0) & (x < 1) & (np.abs(255 * x - np.round(255 * x)) < 1e-3)
    edge = near(want[:, 3]) | near(want[:, 4])
    assert edge.mean() < 0.02
    width = np.ceil(255 * np.clip(want[:, 4], 0, 1)) - np.floor(255 * np.clip(want[:, 3], 0, 1))
    assert np.sum(width >= 32) >= 20                      # ranges that cover whole 16-bin blocks
    cols = [c for c in range(16) if c not in (6, 7, 8, 9)]
    np.testing.assert_allclose(got[:, cols], want[:, cols], atol=1e-5, rtol=1e-5)
    np.testing.assert_allclose(got[~edge][:, 6:10], want[~edge][:, 6:10], atol=1e-5, rtol=1e-5)


def test_features_unaligned_output_matches_aligned(cfg1, cfg1_gpu):
    """An output buffer that is not 16-byte aligned takes the kernel's
    scalar-store path; its rows equal those written to an aligned buffer,
    and nothing outside the rows is written."""
    tf, cams = V.config1_render()
    step = V.StepParams(mode="heuristic")
    n = cfg1_gpu.n_elem
    want = lv.features(cfg1_gpu, cams[1], tf, step)
    assert want.data_ptr() % 16 == 0
    buf = torch.full((16 * n + 2,), -7.0, dtype=torch.float32, device="cuda")
    shifted = buf[1:1 + 16 * n].view(n, 16)
    assert shifted.data_ptr() % 16 != 0
    got = lv.features(cfg1_gpu, cams[1], tf, step, out=shifted)
    assert torch.equal(got, want)
    assert float(buf[0]) == -7.0 and float(buf[-1]) == -7.0


# ----------------------------------------------------------------------------
# network: BF16 inference, FP32 gradient, Adam
# ----------------------------------------------------------------------------

def _net(seed, scale=0.25, b4=4.0):
    p = scale * (2 * Stream(seed, OL.N_PARAMS + 8).take(OL.N_PARAMS) - 1)
    p[-1] = b4
    return p.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,ymin", [(1, 0.0), (16, 0.0), (1000, 0.0), (1000, -2.0), (70001, 0.0)])
def test_mlp_infer_matches_bf16_forward(n, ymin):
    p = _net(7)
    if ymin < 0:
        p[-1] = -0.2                                 # outputs on both sides of 0
    X = (2 * Stream(8, 16 * n + 8).take(16 * n).reshape(n, 16) - 0.5).astype(np.float32)
    ymax = 8.0
    packed = lv.mlp_pack(torch.from_numpy(p.astype(np.float32)).cuda())
    got = lv.mlp_infer(torch.from_numpy(X).cuda(), packed, ymax, ymin=ymin).cpu().numpy().astype(np.float64)
    want = OL.multipliers(p, X.astype(np.float64), ymax, emulate_bf16=True, ymin=ymin)
    if ymin < 0:
        assert np.any(want < 1.0) and np.all(want >= 2.0 ** ymin)
    lv.mlp_check()                                   # no tensor-core wait ran out
    d = np.abs(np.log2(got) - np.log2(want))
    assert d.max() <= 3e-2 and d.mean() <= 3e-3, (d.max(), d.mean())
    y = OL.forward(p, X.astype(np.float64), emulate_bf16=True)
    inside = (y > ymin + 0.5) & (y < ymax - 0.5)
    assert inside.mean() > 0.5                       # the comparison is not all clamps


def test_mlp_infer_unaligned_features_match_aligned():
    """Feature rows at an address that is not 16-byte aligned take the
    kernel's scalar-load path; the multipliers are the same as from an
    aligned copy of the same rows (ragged last tile included)."""
    n = 1000
    p = _net(11)
    X = (2 * Stream(12, 16 * n + 8).take(16 * n).reshape(n, 16) - 0.5).astype(np.float32)
    packed = lv.mlp_pack(torch.from_numpy(p.astype(np.float32)).cuda())
    aligned = torch.from_numpy(X).cuda()
    buf = torch.zeros(16 * n + 1, dtype=torch.float32, device="cuda")
    buf[1:] = aligned.reshape(-1)
    shifted = buf[1:].view(n, 16)
    assert shifted.data_ptr() % 16 != 0
    want = lv.mlp_infer(aligned, packed, 8.0)
    got = lv.mlp_infer(shifted, packed, 8.0)
    lv.mlp_check()
    assert torch.equal(got, want)


def _separated_case(n, seed0):
    """Parameters and inputs whose FP64 pre-activations stay 2e-5 from 0
    (about 10 times the typical FP32 error of a 64-term sum here)."""
    for seed in range(seed0, seed0 + 200):
        p = _net(seed, scale=0.3, b4=0.1)
        X = (2 * Stream(seed + 1000, 16 * n + 8).take(16 * n).reshape(n, 16) - 1).astype(np.float32)
        t = (2 * Stream(seed + 2000, n + 8).take(n)).astype(np.float32)
        w = OL.unpack(p)
        h, ok = X.astype(np.float64), True
        for k in (1, 2, 3):
            z = h @ w[f"W{k}"] + w[f"b{k}"]
            ok &= bool(np.min(np.abs(z)) > 2e-5)
            h = np.maximum(z, 0)
        if ok:
            return p, X, t
    pytest.fail("no well separated case")


@pytest.mark.parametrize("n", [1, 37, 200])
def test_mlp_grad_matches_fp64(n):
    p, X, t = _separated_case(n, 11)
    loss_w, g_w = OL.loss_and_grad(p, X.astype(np.float64), t.astype(np.float64))
    loss, g = lv.mlp_grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(),
                          torch.from_numpy(p.astype(np.float32)).cuda())
    g = g.cpu().numpy().astype(np.float64)
    assert float(loss.item()) == pytest.approx(loss_w, rel=1e-5)
    o = 0
    for name, shape in OL.SIZES:
        k = int(np.prod(shape))
        scale = np.abs(g_w[o:o + k]).max()
        assert np.abs(g[o:o + k] - g_w[o:o + k]).max() <= 1e-4 * scale + 1e-12, name
        o += k


def test_adam_step_matches_fp64():
    """One training step (FP32 gradient, then Adam at step 3) against the
    oracle's FP64 gradient and Adam from the same inputs.  The FP32 gradient is
    within d = 1e-4 of each layer's largest entry (test_mlp_grad_matches_fp64),
    so each first moment may move by 0.1 d and each second moment by
    0.001 (2|g| d + d^2); the bounds below carry that through Adam's update
    plus a few units in the last place of FP32."""
    n = 64
    p, X, t = _separated_case(n, 21)
    rng = np.random.default_rng(3)
    m0 = (1e-3 * rng.normal(size=OL.N_PARAMS)).astype(np.float32)
    v0 = (1e-6 * rng.random(OL.N_PARAMS)).astype(np.float32)
    P = torch.from_numpy(p.astype(np.float32)).cuda()
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    M, Vv = torch.from_numpy(m0).cuda(), torch.from_numpy(v0).cuda()
    loss = torch.zeros(1, device="cuda")
    lr, it = 1e-3, 3
    lv.mlp_train_step(Xd, td, P, M, Vv, it, lr, lv.mlp_scratch(n), loss)
    _, g = OL.loss_and_grad(p, X.astype(np.float64), t.astype(np.float64))
    p1, m1, v1 = OL.adam(p, g, m0.astype(np.float64), v0.astype(np.float64), it, lr)
    d = np.zeros_like(g)
    o = 0
    for name, shape in OL.SIZES:
        k = int(np.prod(shape))
        d[o:o + k] = 1e-4 * np.abs(g[o:o + k]).max()
        o += k
    ulp = 2.0 ** -22
    dm = 0.1 * d + ulp * (0.9 * np.abs(m0) + 0.1 * np.abs(g))
    dv = 0.001 * (2 * np.abs(g) * d + d * d) + ulp * (0.999 * v0 + 0.001 * g * g)
    assert np.all(np.abs(M.cpu().numpy() - m1) <= dm + 1e-30)
    assert np.all(np.abs(Vv.cpu().numpy() - v1) <= dv + 1e-30)
    # update lr * mhat / (sqrt(vhat) + eps): first-order propagation of dm, dv
    b1, b2 = 1 - 0.9 ** it, 1 - 0.999 ** it
    sv = np.sqrt(v1 / b2)
    dstep = lr * (dm / b1 / (sv + 1e-8) + np.abs(m1 / b1) * (dv / b2) / (2 * sv * (sv + 1e-8) ** 2))
    step_gpu = P.cpu().numpy().astype(np.float64) - p
    err = np.abs(step_gpu - (p1 - p))
    tol = 2 * dstep + 1e-3 * np.abs(p1 - p) + 2.0 ** -23 * np.abs(p) + 1e-12     # last: FP32 rounding of p
    assert np.all(err <= tol), float(np.max(err - tol))


def test_training_reduces_loss():
    n = 4096
    X = (2 * Stream(5, 16 * n + 8).take(16 * n).reshape(n, 16) - 1).astype(np.float32)
    t = (1.5 + np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2]).astype(np.float32)
    cfg = LS.TrainConfig(steps=400, batch=1024, lr=3e-3, lr_final=3e-4)
    model, losses = LS.train(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), cfg, log_every=100)
    first, _ = OL.loss_and_grad(LS.init_params(cfg.seed).astype(np.float64), X, t)
    final, _ = OL.loss_and_grad(model.params.cpu().numpy().astype(np.float64), X, t)
    assert final < 0.05 * first, (first, final, losses)


# ----------------------------------------------------------------------------
# labels
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("cand", [LS.CAND, LS.CAND_REFINE], ids=["default", "refining"])
def test_labels_match_oracle(cfg1, cfg1_oracle, cfg1_gpu, cand):
    tf, _ = V.config1_render()
    tf = _f32_tf(tf)
    cam = V.seeded_oblique(Stream(55), 12, 10)
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=1.0)
    tau = 2e-4
    got = lv.labels(cfg1_gpu, cam, tf, step, 1 / 2048, tau, cand).cpu().numpy()
    want = cfg1_oracle.labels(cam, tf, step, 1 / 2048, tau, cand)
    # a label is the outcome of comparisons err <= tau, taken on FP32
    # composites on the GPU and FP64 ones in the oracle; the FP32 error of a
    # composite difference is a few 1e-7, about 1e-3 of tau, so a 2 % band
    # of tau bounds every label and all but a few agree exactly
    lo = cfg1_oracle.labels(cam, tf, step, 1 / 2048, 0.98 * tau, cand)
    hi = cfg1_oracle.labels(cam, tf, step, 1 / 2048, 1.02 * tau, cand)
    visited = want < len(cand)
    assert np.array_equal(got < len(cand), visited)
    assert visited.sum() > 50
    assert np.all((got >= lo) & (got <= hi))
    assert np.mean(got[visited] == want[visited]) >= 0.98
    # the labels discriminate: several classes occur
    assert len(np.unique(want[visited])) >= 3


# ----------------------------------------------------------------------------
# what the trained network gains over Eq. 4 alone
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def trained():
    """The default training recipe on seeded cameras of configs 1 and 2."""
    cfg = LS.TrainConfig()
    vols = {1: V.load_config(1), 2: V.load_config(2)}
    tfs = {1: V.config1_render()[0], 2: V.config2_render(vol=vols[2])[0]}
    gvs = {k: lv.Volume(v).build_accel((64, 64, 64)).to_bezier() for k, v in vols.items()}
    step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    model, losses, rows = LS.fit([(gvs[1], tfs[1]), (gvs[2], tfs[2])], step, cfg)
    yield model, losses, gvs, tfs, step
    for g in gvs.values():
        g.close()


def _gain(model, gv, tf, step, k):
    """(samples of the learned render / Eq. 4's, learned RMSE, Eq. 4 RMSE)
    against the fine-step (1/2048) reference on held-out camera k."""
    cam = V.orbit_camera(Stream(4242 + k), 480, 270)
    fine = gv.render(cam, tf, V.StepParams(mode="fixed", h=1 / 2048, xi=1 / 256, alpha_stop=0.99)).cpu().numpy()
    heur = gv.render(cam, tf, step).cpu().numpy()
    s_h = gv.stats()["samples"]
    mult = model.multipliers(gv, cam, tf, step)
    learned = gv.render(cam, tf, V.StepParams(mode="learned", xi=1 / 256, alpha_stop=0.99, mult=mult)).cpu().numpy()
    s_l = gv.stats()["samples"]
    return s_l / s_h, _rmse(learned, fine), _rmse(heur, fine)


@pytest.mark.parametrize("k", [1, 2])
def test_trained_step_gain(trained, k, capsys):
    """The default recipe (steps at least Eq. 4's) on held-out views.  On the
    MR-like volume: an image within RMSE 1e-3 of the fine-step reference with
    at most 0.6 of Eq. 4's samples.  On config 1, whose opaque transfer
    function leaves Eq. 4 itself above 1e-3, no multiplier >= 1 can reach the
    bar (the refining recipe below does); there the learned walk must still
    take fewer samples than Eq. 4, and test_network_beats_constant_and_rule
    shows it does so better than any constant or empty-space rule."""
    model, losses, gvs, tfs, step = trained
    frac, e_l, e_h = _gain(model, gvs[k], tfs[k], step, k)
    with capsys.disabled():
        print(f"\n[learned step, config {k}] loss {losses}, samples {frac:.3f} of Eq. 4, "
              f"RMSE vs fine: learned {e_l:.2e}, Eq. 4 {e_h:.2e}")
    if k == 2:
        assert e_l <= 1e-3 and frac <= 0.6
    else:
        assert e_h > 1e-3 and frac <= 0.9


@pytest.fixture(scope="module")
def trained_refine(trained):
    """The refining recipe (multipliers from 1/2 to 8) on the same cameras."""
    _, _, gvs, tfs, step = trained
    model, losses, rows = LS.fit([(gvs[1], tfs[1]), (gvs[2], tfs[2])], step, LS.refine_config())
    return model, losses


@pytest.mark.parametrize("k", [1, 2])
def test_refining_step_meets_the_bar(trained, trained_refine, k, capsys):
    """With multipliers below 1 allowed, the network refines where Eq. 4 is
    too coarse: both volumes' held-out images within RMSE 1e-3 of the
    fine-step reference, config 1 included (Eq. 4 alone misses it there), and
    on the MR-like volume still well under Eq. 4's samples."""
    model, losses = trained_refine
    _, _, gvs, tfs, step = trained
    frac, e_l, e_h = _gain(model, gvs[k], tfs[k], step, k)
    with capsys.disabled():
        print(f"\n[refining step, config {k}] samples {frac:.3f} of Eq. 4, RMSE vs fine: learned {e_l:.2e}, "
              f"Eq. 4 {e_h:.2e}; multipliers {model.cfg.cand[0]}..{model.cfg.cand[-1]}")
    assert e_l <= 1e-3
    if k == 1:
        assert e_h > 1e-3
    else:
        assert frac <= 0.6


@pytest.mark.parametrize("k", [1, 2])
def test_network_beats_constant_and_rule(trained, k, capsys):
    """What the network learns beyond a rule: on a held-out view, the trained
    network against (a) the best constant multiplier of the candidate set and
    (b) per-element rules on the features it already computes (8x where the
    TF's largest opacity over the element's value range is at most theta,
    else a constant), each taken at its fewest samples with an image at least
    as close to the fine-step reference as the network's."""
    model, losses, gvs, tfs, step = trained
    gv, tf = gvs[k], tfs[k]
    cam = V.orbit_camera(Stream(4242 + k), 480, 270)
    fine = gv.render(cam, tf, V.StepParams(mode="fixed", h=1 / 2048, xi=1 / 256, alpha_stop=0.99))
    ab = LS.ablation(gv, cam, tf, step, model, fine)
    with capsys.disabled():
        print(f"\n[ablation, config {k}] Eq. 4 RMSE {ab['eq4_rmse']:.2e}; network "
              f"{ab['network']['samples_frac']:.3f} of Eq. 4 samples at RMSE {ab['network']['rmse']:.2e}; "
              f"empty-element rule {ab['rule_empty_8x_else_1x']}; best constant at the network's RMSE "
              f"{ab['best_constant_at_network_rmse']}; best rule at the network's RMSE "
              f"{ab['best_rule_at_network_rmse']}; train info {model.train_info}")
    net = ab["network"]["samples_frac"]
    for key in ("best_constant_at_network_rmse", "best_rule_at_network_rmse"):
        other = ab[key]
        assert other is None or net < other["samples_frac"], (key, other, net)
    r = ab["rule_empty_8x_else_1x"]
    assert r["rmse"] > ab["network"]["rmse"] or net < r["samples_frac"]


def test_step_model_save_load(trained, tmp_path):
    model = trained[0]
    path = str(tmp_path / "step.bin")
    model.save(path)
    again = LS.StepModel.load(path)
    assert torch.equal(again.params, model.params)
    assert again.cfg.tau == model.cfg.tau and again.cfg.margin == model.cfg.margin and again.cfg.cand == model.cfg.cand
    assert again.cfg.ymin == model.cfg.ymin and again.cfg.ymax == model.cfg.ymax
    assert torch.equal(again.packed, model.packed)


@pytest.mark.slow
def test_learned_multipliers_full_size(trained):
    """The trained network's multipliers for the benchmark frame (cfg2,
    1920x1080): within [1, 8] and on average well above 1.  (The learned
    render itself is compared with the oracle sample by sample, with seeded
    multipliers of the same candidate set, in test_gpu_trace.)"""
    model, losses, gvs, tfs, step = trained
    vol = V.load_config(2)
    tf = _f32_tf(V.config2_render(vol=vol)[0])
    cam = V.config2_render(vol=vol)[1]
    mult = model.multipliers(gvs[2], cam, tf, step)
    assert float(mult.min()) >= 1.0 and float(mult.max()) <= 8.0 and float(mult.mean()) > 1.5

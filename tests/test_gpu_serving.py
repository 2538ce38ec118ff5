"""The frame server on the GPU: every frame in a mixed, overlapping batch is
identical (bit for bit, with the same sample counts) to the same request
rendered alone by lrvol_render, and sampled pixels of served frames of every
volume and mode (FP32 Eq. 4, FP16 |v|, fixed steps, learned steps) match the
FP64 oracle (RMSE <= 1e-4); admission respects the arena and FIFO order;
frames really overlap on the device; host copies and server-side learned
steps give the same images as the plain calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import Oracle
from paper_1707_01170_gb300 import learned as LS
from paper_1707_01170_gb300 import lrvol as lv
from paper_1707_01170_gb300 import serve
from paper_1707_01170_gb300.synth import volumes as V
from paper_1707_01170_gb300.synth.lrgen import Stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lv.load()


RMSE_TOL = 1e-4


def _rmse(a, b):
    return float(np.sqrt(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2)))


def _oracle_pixels(vol, cam, tf, step, img, n, seed):
    """n seeded pixels of a served image and the oracle's values there (the TF
    rounded to FP32 as the library stores it; learned multipliers from the host)."""
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], axis=1).astype(np.int32)
    tf32 = V.TransferFunction(table=np.asarray(tf.table, np.float32).astype(np.float64), vmin=tf.vmin, vmax=tf.vmax)
    if step.mode == "learned":
        step = V.StepParams(**{**step.__dict__, "mult": step.mult.cpu().numpy()})
    ref, _ = Oracle(vol).render(cam, tf32, step, pixels=pix)
    got = img.cpu().numpy()[pix[:, 1], pix[:, 0]]
    return got, ref


_VOLS = {}


def _resident_volumes():
    if not _VOLS:
        _VOLS["v"] = [V.load_config(1),
                      V.refined_ball((2, 2, 2), (3, 3, 3), centres=((0.3, 0.6, 0.45),), radii=(0.4, 0.2), ncomp=3,
                                     seed=4),
                      V.tensor_product((1, 1, 1), (5, 3, 4), seed=2)]
    return _VOLS["v"]


@pytest.fixture(scope="module")
def resident():
    """Three resident volumes of different kinds, with TF and step each."""
    v1, vec, tp = _resident_volumes()
    gvs = [lv.Volume(v1).build_accel((32, 32, 32)).to_bezier(),
           lv.Volume(vec).build_accel((16, 16, 16)).to_bezier(lv.STORE_F16),
           lv.Volume(tp).build_accel((8, 8, 8)).to_bezier()]
    tf1 = V.config1_render()[0]
    tfv = V.seeded_tf(Stream(31), alpha_max=0.05)
    tfv.vmin, tfv.vmax = 0.0, 1.6
    tft = V.seeded_tf(Stream(33), alpha_max=0.1)
    steps = [V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99),
             V.StepParams(mode="heuristic", xi=1 / 128, field="magnitude"),
             V.StepParams(mode="fixed", h=1 / 200, xi=1 / 256)]
    yield gvs, [tf1, tfv, tft], steps
    for g in gvs:
        g.close()


SMALL = ((64, 48), (200, 120), (333, 171))


def test_mixed_batch_identical_to_alone(resident):
    gvs, tfs, steps = resident
    reqs = serve.request_stream(99, 36, 1000.0, 3, sizes=SMALL)
    srv = lv.Server(slots=6, arena_bytes=64 << 20)
    tickets = [srv.submit(gvs[r.volume], r.camera, tfs[r.volume], steps[r.volume]) for r in reqs]
    srv.drain()
    st = srv.stats()
    assert st["done"] == len(reqs) and st["failed"] == 0 and st["max_running"] >= 2
    infos = [srv.info(t) for t in tickets]
    for r, t, d in zip(reqs, tickets, infos):
        alone = gvs[r.volume].render(r.camera, tfs[r.volume], steps[r.volume])
        ast = gvs[r.volume].stats()
        mixed = srv.image(t)
        assert torch.equal(mixed, alone), f"ticket {t}"
        assert (d["samples"], d["lookups"], d["rays_hit"]) == (ast["samples"], ast["lookups"], ast["rays_hit"])
    # frames overlapped on the device: some pair of [start, end] intervals intersects
    iv = sorted((d["dev_start_ms"], d["dev_end_ms"]) for d in infos)
    assert any(iv[k + 1][0] < iv[k][1] for k in range(len(iv) - 1))
    # served frames against the FP64 oracle: one frame per volume (FP32 Eq. 4,
    # FP16 |v|, fixed step), 300 sampled pixels each
    vols = _resident_volumes()
    for v in range(3):
        r, t = next((r, t) for r, t in zip(reqs, tickets) if r.volume == v)
        got, ref = _oracle_pixels(vols[v], r.camera, tfs[v], steps[v], srv.image(t), 300, 40 + v)
        assert _rmse(got, ref) <= RMSE_TOL, f"volume {v}"
        assert np.abs(ref[:, 3]).max() > 0.01
    for t in tickets:
        srv.release(t)
    assert srv.stats()["arena_used"] == 0
    srv.close()


def test_served_learned_frames_against_oracle(resident):
    """Learned-step requests (caller-supplied per-element multipliers) served
    in a mix with plain ones: each equals the same request alone, and sampled
    pixels match the oracle marching with the same multipliers."""
    gvs, tfs, steps = resident
    vols = _resident_volumes()
    rng = np.random.default_rng(3)
    cand = np.array([1, 1.5, 2, 3, 4, 6, 8], np.float32)
    lsteps = [V.StepParams(mode="learned", xi=1 / 256, alpha_stop=0.99,
                           mult=torch.from_numpy(rng.choice(cand, vols[0].n_elem)).cuda()),
              V.StepParams(mode="learned", xi=1 / 128, field="magnitude",
                           mult=torch.from_numpy(rng.choice(cand, vols[1].n_elem)).cuda())]
    reqs = serve.request_stream(12, 12, 1000.0, 2, sizes=SMALL)
    srv = lv.Server(slots=4, arena_bytes=64 << 20)
    tickets = []
    for k, r in enumerate(reqs):
        tickets.append(srv.submit(gvs[r.volume], r.camera, tfs[r.volume], lsteps[r.volume]))
        if k % 3 == 0:                                   # plain frames in the same mix
            srv.submit(gvs[r.volume], r.camera, tfs[r.volume], steps[r.volume])
    srv.drain()
    checked = set()
    for r, t in zip(reqs, tickets):
        img = srv.image(t)
        assert torch.equal(img, gvs[r.volume].render(r.camera, tfs[r.volume], lsteps[r.volume]))
        if r.volume not in checked:
            got, ref = _oracle_pixels(vols[r.volume], r.camera, tfs[r.volume], lsteps[r.volume], img, 300, 50)
            assert _rmse(got, ref) <= RMSE_TOL, f"volume {r.volume}"
            checked.add(r.volume)
    assert checked == {0, 1}
    srv.close()


def test_admission_by_memory_and_fifo(resident):
    gvs, tfs, steps = resident
    img = 512 * 512 * 16                               # 4 MiB per frame
    srv = lv.Server(slots=8, arena_bytes=2 * img + img // 2)
    cams = [serve.orbit_view(0, k, 1, 512, 512) for k in range(7)]
    host = [torch.empty((512, 512, 4), dtype=torch.float32, pin_memory=True) for _ in cams]
    tickets = [srv.submit(gvs[0], c, tfs[0], steps[0], host_out=h) for c, h in zip(cams, host)]
    srv.drain()
    st = srv.stats()
    assert st["done"] == 7 and st["max_running"] <= 2 and st["arena_high_water"] <= 2 * img
    assert st["arena_used"] == 0                       # host copies return the memory at retirement
    admits = [srv.info(t)["t_admit"] for t in tickets]
    assert admits == sorted(admits)
    for c, h, t in zip(cams, host, tickets):
        assert srv.info(t)["rgba_dev"] is None
        assert torch.equal(h, gvs[0].render(c, tfs[0], steps[0]).cpu())
        srv.release(t)
    srv.close()


def test_request_larger_than_arena_rejected(resident):
    gvs, tfs, steps = resident
    srv = lv.Server(slots=2, arena_bytes=1 << 20)
    with pytest.raises(lv.LrvolError) as e:
        srv.submit(gvs[0], serve.orbit_view(0, 0, 1, 512, 512), tfs[0], steps[0])
    assert e.value.status == lv.ERR_ARG
    with pytest.raises(lv.LrvolError):
        srv.submit(gvs[0], serve.orbit_view(0, 0, 1, 64, 64), tfs[0], V.StepParams(mode="learned"))
    srv.close()


def test_server_learned_steps_match_manual(resident, cfg1):
    gvs, tfs, steps = resident
    model = LS.StepModel(LS.init_params(5), LS.TrainConfig(margin=-1.5))
    srv = lv.Server(slots=3, arena_bytes=64 << 20)
    srv.set_step_model(model.packed, model.cfg.ymax, model.cfg.ymin)
    cams = [serve.orbit_view(0, k, 1, 160, 90) for k in range(5)]
    lstep = V.StepParams(mode="learned", xi=1 / 256, alpha_stop=0.99)
    tickets = [srv.submit(gvs[0], c, tfs[0], lstep) for c in cams]
    srv.drain()
    for c, t in zip(cams, tickets):
        mult = model.multipliers(gvs[0], c, tfs[0], steps[0])
        want = gvs[0].render(c, tfs[0], V.StepParams(mode="learned", xi=1 / 256, alpha_stop=0.99, mult=mult))
        assert torch.equal(srv.image(t), want)
        srv.release(t)
    srv.close()


def test_realtime_stream_latencies(resident, capsys):
    gvs, tfs, steps = resident
    reqs = serve.request_stream(5, 120, 400.0, 3, sizes=SMALL)
    srv = lv.Server(slots=4, arena_bytes=64 << 20)
    recs = serve.run_stream(srv, gvs, tfs, steps, reqs)
    s = serve.summarize(recs)
    with capsys.disabled():
        print(f"\n[serving, small frames at 400 req/s] p50 {s['p50_ms']:.3f} ms, p99 {s['p99_ms']:.3f} ms, "
              f"{s['frames_per_s']:.0f} frames/s, max in flight {srv.stats()['max_running']}")
    assert s["frames"] == 120 and s["failed"] == 0
    assert all(r["latency_ms"] >= 0 and r["done_s"] >= r["admit_s"] >= r["arrival_s"] - 1e-6 for r in recs)
    srv.close()


def test_size_tiers_let_small_frames_overtake(resident):
    """With tiers on, small frames submitted behind large ones that fill the
    arena are admitted first; within a tier admission stays FIFO."""
    gvs, tfs, steps = resident
    big = 1024 * 1024 * 16                                 # 16 MiB per large frame
    srv = lv.Server(slots=8, arena_bytes=2 * big + (4 << 20))
    srv.set_priority_pixels(64 * 64)
    hl = [torch.empty((1024, 1024, 4), pin_memory=True) for _ in range(5)]
    hs = [torch.empty((48, 64, 4), pin_memory=True) for _ in range(5)]
    large = [srv.submit(gvs[0], serve.orbit_view(0, k, 1, 1024, 1024), tfs[0], steps[0], host_out=h)
             for k, h in enumerate(hl)]
    assert srv.progress() == 0                             # two large frames fill the arena
    small = [srv.submit(gvs[0], serve.orbit_view(0, k, 1, 64, 48), tfs[0], steps[0], host_out=h)
             for k, h in enumerate(hs)]
    srv.drain()
    st = srv.stats()
    assert st["done"] == 10 and st["arena_high_water"] <= 2 * big + (4 << 20)
    adm_l = [srv.info(t)["t_admit"] for t in large]
    adm_s = [srv.info(t)["t_admit"] for t in small]
    assert adm_l == sorted(adm_l) and adm_s == sorted(adm_s)
    assert max(adm_s) < adm_l[2]                           # every small frame before the third large one
    assert min(adm_s) > adm_l[1]
    for t in large + small:
        srv.release(t)
    srv.close()


@pytest.mark.slow
def test_full_size_mix_identical_to_alone():
    """The benchmark's serving mix at full size (configs 1-3 resident; 256x256,
    1920x1080 and 3840x2160 frames, size tiers on): every frame equals the same
    request rendered alone, bit for bit."""
    vols = [V.load_config(1), V.load_config(2), V.load_config(3)]
    gvs = [lv.Volume(v).build_accel((64, 64, 64)).to_bezier() for v in vols]
    tf3 = V.config3_render()[0]
    tf3.vmin, tf3.vmax = 0.0, 1.5
    tfs = [V.config1_render()[0], V.config2_render(vol=vols[1])[0], tf3]
    steps = [V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)] * 2 + \
            [V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field="magnitude")]
    reqs = serve.request_stream(77, 12, 1000.0, 3)
    srv = lv.Server(slots=8, arena_bytes=2 << 30)
    srv.set_priority_pixels(1 << 20)
    tickets = [srv.submit(gvs[r.volume], r.camera, tfs[r.volume], steps[r.volume]) for r in reqs]
    srv.drain()
    assert srv.stats()["max_running"] >= 2
    checked = set()
    for r, t in zip(reqs, tickets):
        alone = gvs[r.volume].render(r.camera, tfs[r.volume], steps[r.volume])
        img = srv.image(t)
        assert torch.equal(img, alone)
        if r.volume not in checked:                     # one frame per volume against the oracle
            got, ref = _oracle_pixels(vols[r.volume], r.camera, tfs[r.volume], steps[r.volume], img, 256, 60)
            assert _rmse(got, ref) <= RMSE_TOL, f"volume {r.volume}"
            checked.add(r.volume)
        srv.release(t)
    assert checked == {0, 1, 2}
    srv.close()
    for g in gvs:
        g.close()


def test_drain_reports_memory_held_by_unreleased_frames(resident):
    """Frames kept in the arena (no host copy, not released) can block the
    queue; drain then returns an error instead of waiting forever, and
    releasing them lets the rest through."""
    gvs, tfs, steps = resident
    img = 512 * 512 * 16
    srv = lv.Server(slots=4, arena_bytes=2 * img + (1 << 20))
    cams = [serve.orbit_view(0, k, 1, 512, 512) for k in range(4)]
    tickets = [srv.submit(gvs[0], c, tfs[0], steps[0]) for c in cams]
    with pytest.raises(lv.LrvolError) as e:
        srv.drain()
    assert e.value.status == lv.ERR_OOM
    st = srv.stats()
    assert st["done"] == 2 and st["queued"] == 2
    for t in tickets[:2]:
        srv.release(t)
    srv.drain()
    assert srv.stats()["done"] == 4
    for c, t in zip(cams[2:], tickets[2:]):
        assert torch.equal(srv.image(t), gvs[0].render(c, tfs[0], steps[0]))
        srv.release(t)
    srv.close()

"""Benchmark: direct volume ray casting of an LR-spline on one GB300.

One step = one frame of the whole per-frame path (ray setup, forest look-up,
element reuse, Bezier evaluation, Eq. 4 steps, transfer function, Alg. 2
compositing) at 1920x1080 on the MR-like scalar tricubic volume (~174k
elements, perspective camera at distance 1.8, fovy 40 deg, alpha_stop 0.99).
The once-per-volume change of basis and forest build are timed separately
(`setup`).  Metric: Gsamples/s (a sample = one field evaluation that is
composited); ms/frame beside it.

At one GPU the line also carries `learned_step`: the same frame rendered with
learned step sizes (per-element multipliers from the BF16 network, trained
first on seeded cameras of configs 1 and 2) on FP16 blocks, timed whole
(features, network, render) against the plain FP32 Eq. 4 frame, with both
images' RMSE against the fine-step (1/2048) reference, and `serving`: the
continuous-batching frame server over configs 1-3 resident at once, fed
seeded Poisson streams of mixed-size requests (latency p50/p99, frames/s).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--learned off|f32|f16|bf16] [--serve off|plain|learned|both]
Under torchrun each rank renders its own frame (replicas; weak scaling) and
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the frame server runs 3 streams per slot; give each its own hardware queue
# (read when the CUDA context is created, before any CUDA call below)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

WIDTH, HEIGHT = 1920, 1080
BLOCKS = (64, 64, 64)
METRIC = "Gsamples/s (1080p frame, MR-like tricubic LR-spline, Eq. 4 steps)"
L2_FLUSH_BYTES = 512 << 20

FP32_LANES = 128   # FP32 FMA lanes per SM (Blackwell)


def fp32_peak(clocks: dict | None = None):
    """FP32 FMA peak of the current device in TFLOP/s and how it was derived:
    the SM count from the device properties x 128 lanes x 2 flop x the median
    SM clock sampled during the timed region (else the GPU's maximum SM clock,
    from the same sampling or the measured-peaks file).  No FP32 rate is
    measured by a copy or a GEMM, so this is a derived denominator."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, src = None, None
    if clocks and clocks.get("sm_mhz"):
        mhz, src = float(clocks["sm_mhz"]), "median SM clock sampled during the timed region"
    elif clocks and clocks.get("sm_max_mhz"):
        mhz, src = float(clocks["sm_max_mhz"]), "maximum SM clock reported by nvidia-smi"
    else:
        try:
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
            src = "maximum SM clock in the measured-peaks file"
        except (OSError, ValueError, KeyError):
            mhz, src = 2070.0, "nominal maximum SM clock (no clock sampled)"
    peak = sms * FP32_LANES * 2 * mhz * 1e6 / 1e12
    return peak, f"derived: {sms} SMs (device property) x {FP32_LANES} FP32 lanes x 2 x {mhz:.0f} MHz ({src})"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOADS = {
    "cfg2": "cfg2: MR-like scalar tricubic LR-spline, 174000 elements, 1920x1080 persp fovy 40 at distance 1.8, "
            "Eq. 4 heuristic steps, xi 1/256, alpha_stop 0.99",
    "cfg3mag": "cfg3: wind-flow 3-vector triquadratic LR-spline, 388016 elements, |v|, 1920x1080 persp, "
               "Eq. 4 heuristic steps, xi 1/256, alpha_stop 0.99",
    "cfg3x": "cfg3: wind-flow 3-vector triquadratic LR-spline, 388016 elements, v_x, 1920x1080 persp, "
             "Eq. 4 heuristic steps, xi 1/256, alpha_stop 0.99",
}


def bench_config(workload: str, storage: str, ws: int) -> dict:
    """The workload description both arms print (the reference arm runs the
    same frame on the host)."""
    return {"workload": WORKLOADS[workload] + f", forest {BLOCKS[0]}^3", "block_storage": storage,
            "l2": "flushed between frames (512 MB write, outside the timed events)",
            "parallelism": f"replicas x{ws}"}


def flop_per_sample_shaded(p: int) -> int:
    """Gradient-shaded scalar sample: the scalar sample, plus the gradient
    contraction 2*((p+1)^3 + 2(p+1)^2 + 3(p+1)) reusing the value's partial
    sums, derivative monomials 3*(2p+1), world scaling 3, I = max(0.4, |l.g|/|g|)
    15, and the shaded colour weight 1."""
    n = p + 1
    return flop_per_sample(p, "scalar") + 2 * (n ** 3 + 2 * n ** 2 + 3 * n) + 3 * (2 * p + 1) + 3 + 15 + 1


def flop_per_sample(p: int, field: str) -> int:
    """Algorithmic FP32 flops per composited sample (an FMA counts 2): sample
    position 12, local coordinates 9, monomial basis 3*(2p+1) (p=3: 21),
    contraction 2*((p+1)^3 + (p+1)^2 + (p+1)) per component, |v| 6, transfer
    function 13, Alg. 2 compositing 15."""
    n = p + 1
    contraction = 2 * (n ** 3 + n ** 2 + n)
    comps = 3 if field == "magnitude" else 1
    return 12 + 9 + 3 * (2 * p + 1) + comps * contraction + (6 if field == "magnitude" else 0) + 13 + 15


def _workload(name: str = "cfg2"):
    from paper_1707_01170_gb300.synth import volumes as V
    if name == "cfg2":
        vol = V.load_config(2)
        tf, cam = V.config2_render(WIDTH, HEIGHT, vol)
        step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    else:
        vol = V.load_config(3)
        tf, cam = V.config3_render(WIDTH, HEIGHT)
        if name == "cfg3mag":
            tf.vmin, tf.vmax = 0.0, 1.5
            step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field="magnitude")
        else:
            tf.vmin, tf.vmax = -0.5, 1.5
            step = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field="component", component=0)
    tf.table = np.asarray(tf.table, dtype=np.float32).astype(np.float64)
    return vol, tf, cam, step


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _core_model() -> str:
    try:
        for ln in open("/proc/cpuinfo"):
            k, _, v = ln.partition(":")
            if k.strip() in ("model name", "Model name", "CPU part") and v.strip():
                return v.strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(vol, tf, cam, step, samples_per_frame=None, target_s: float = 12.0, seed: int = 11):
    """The FP64 oracle, as it stands, on a seeded pixel subset of the same
    frame, sized to about target_s seconds of work on all host cores; plus a
    short one-thread run and the frame time extrapolated from the rate."""
    from oracle.oracle import Oracle
    rng = np.random.default_rng(seed)
    orc = Oracle(vol)

    def run(n, threads=None):
        pix = np.stack([rng.integers(0, cam.width, n), rng.integers(0, cam.height, n)], axis=1).astype(np.int32)
        t0 = time.perf_counter()
        _, st = orc.render(cam, tf, step, pixels=pix, threads=threads)
        return st["samples"], time.perf_counter() - t0

    s0, d0 = run(256)
    n = int(min(40000, max(256, 256 * (target_s - d0) / max(d0, 1e-3))))
    s1, d1 = run(n)
    samples, dt = s0 + s1, d0 + d1
    value = samples / dt / 1e9
    s2, d2 = run(max(16, n // (4 * orc.threads)), threads=1)
    out = {"value": value, "unit": "Gsamples/s", "cores": orc.threads, "kind": "oracle",
           "core_model": _core_model(), "one_thread_value": s2 / d2 / 1e9, "us_per_sample": 1e6 * dt / samples,
           "sample": f"{256 + n} seeded pixels of the same 1920x1080 frame ({samples} samples, {dt:.1f} s)"}
    if samples_per_frame:
        out["extrapolated_ms_per_frame"] = 1e3 * samples_per_frame / (value * 1e9)
    # a whole frame the oracle finishes: config 1, 128x128, Eq. 4 steps
    from paper_1707_01170_gb300.synth import volumes as V
    v1 = V.load_config(1)
    tf1, cams1 = V.config1_render()
    o1 = Oracle(v1)
    t0 = time.perf_counter()
    _, st1 = o1.render(cams1[1], tf1, V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99))
    out["config1_full_frame"] = {"frame": "128x128 oblique view, Eq. 4 steps", "s": time.perf_counter() - t0,
                                 "samples": st1["samples"], "cores": o1.threads}
    return out


RENDER_SOURCES = ("render.cu", "device_common.cuh", "lrvol_internal.h")


def render_source_hash(root: str | None = None) -> str:
    """sha256 (16 hex digits) of the files that define k_render."""
    import hashlib
    h = hashlib.sha256()
    for name in RENDER_SOURCES:
        h.update(open(os.path.join(root or ROOT, "paper_1707_01170_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profiled_counters():
    """DRAM and L2 bytes per k_render launch from the committed ncu summary,
    if the render kernel's source is unchanged since that capture; else None."""
    try:
        prof = open(os.path.join(ROOT, "profiles", "k_render_cfg2_1080p.md")).read()
        sha = render_source_hash()
    except OSError:
        return None
    fields = dict(ln.strip().split(": ", 1) for ln in prof.splitlines() if ln.strip().startswith(
        ("render_source_sha256_16:", "traffic_bytes_per_launch:", "l2_bytes_per_launch:")))
    if fields.get("render_source_sha256_16") != sha:
        return None
    return {"traffic": int(fields["traffic_bytes_per_launch"]), "l2": int(fields.get("l2_bytes_per_launch", 0)) or None}


def measured_hbm_gbs():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def measured_bf16_tflops():
    """Burst dense BF16 rate (a kernel timed alone), else the stated fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]), "measured (burst)"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


# tensor-core work of the step network per feature row: the three hidden layers
NET_TENSOR_FLOP_PER_ROW = 2 * (16 * 64 + 64 * 64 + 64 * 64)


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    vol, tf, cam, step = _workload(args.workload)
    from oracle.oracle import Oracle
    orc = Oracle(vol)
    rng = np.random.default_rng(5)
    times, samples = [], 0
    for k in range(args.warmup + args.steps):
        pix = np.stack([rng.integers(0, cam.width, 96), rng.integers(0, cam.height, 96)], axis=1).astype(np.int32)
        t0 = time.perf_counter()
        _, st = orc.render(cam, tf, step, pixels=pix)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            samples += st["samples"]
    tot = sum(times)
    val = samples / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gsamples/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.workload, args.storage, args.gpus),
            "cpu_baseline": {"value": val, "unit": "Gsamples/s", "cores": orc.threads, "kind": "oracle",
                             "sample": "96 seeded pixels of the same frame per step (FP64 oracle)"},
            "e2e": {"value": val, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _timed_frames(fns, steps: int, flush, stream):
    """Mean CUDA-event time (ms) of each callable in fns, run in order once
    per frame for `steps` frames, the L2 flushed before each frame."""
    import torch
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(fns) + 1)] for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        for q, fn in enumerate(fns):
            fn()
            evs[k][q + 1].record(stream)
    torch.cuda.synchronize()
    return [sum(e[q].elapsed_time(e[q + 1]) for e in evs) / steps for q in range(len(fns))]


def learned_leg(vol, tf, step, plain, steps: int, storage: str, flush, stream, model_path=None, save_path=None):
    """Learned step sizes with reduced-precision blocks against the plain FP32
    Eq. 4 renderer on the same frames (1920x1080 and 3840x2160): both images
    against the fine-step (1/2048) reference, and the learned frame timed
    whole (features, BF16 tcgen05 network, render, each in its own event
    pair), L2 flushed between frames like the main loop."""
    import torch
    from paper_1707_01170_gb300 import learned as LS
    from paper_1707_01170_gb300 import lrvol as lv
    from paper_1707_01170_gb300.synth import volumes as V
    t0 = time.perf_counter()
    gv32 = plain["gv32"]
    if model_path:
        model, losses, rows = LS.StepModel.load(model_path), [(0, None)], 0
    else:
        v1 = V.load_config(1)
        tf1 = V.config1_render()[0]
        g1 = lv.Volume(v1).build_accel(BLOCKS, stream=stream).to_bezier(stream=stream)
        model, losses, rows = LS.fit([(g1, tf1), (gv32, tf)], step)
        torch.cuda.synchronize()
        g1.close()
    if save_path:
        model.save(save_path)
    train_s = time.perf_counter() - t0
    code = {"f32": lv.STORE_F32, "f16": lv.STORE_F16, "bf16": lv.STORE_BF16}[storage]
    gq = lv.Volume(vol).build_accel(BLOCKS, stream=stream).to_bezier(storage=code, stream=stream)
    ctf = lv.make_tf(tf)
    feat = torch.empty((vol.n_elem, lv.MLP_IN), dtype=torch.float32, device="cuda")
    mult = torch.empty(vol.n_elem, dtype=torch.float32, device="cuda")
    lstep = lv.make_step(V.StepParams(mode="learned", xi=step.xi, alpha_stop=step.alpha_stop, field=step.field,
                                      component=step.component, mult=mult))
    pstep = lv.make_step(step)
    rmse = lambda a, b: float(torch.sqrt(torch.mean((a.double() - b.double()) ** 2)))
    res = {"storage": storage, "fine_reference": "fixed step 1/2048, FP32 blocks, same alpha_stop",
           "gpu_launches_per_frame": 3, "frames_timed": steps,
           "model": {"train_s": train_s, "rows": rows, "loss": losses[-1][1], "losses": losses,
                     "train_info": getattr(model, "train_info", {}), "tau": model.cfg.tau,
                     "margin": model.cfg.margin, "ymin": model.cfg.ymin, "ymax": model.cfg.ymax,
                     "candidates": list(model.cfg.cand), "steps": model.cfg.steps,
                     "recipe": ("loaded from " + model_path) if model_path else
                     "32 seeded 320x180 cameras on each of configs 1 and 2"},
           "by_resolution": {}}
    for (w, h) in ((WIDTH, HEIGHT), (3840, 2160)):
        ccam = lv.make_camera(V.config2_render(w, h, vol)[1])
        fine = gv32.render(ccam, ctf, V.StepParams(mode="fixed", h=1 / 2048, xi=step.xi, alpha_stop=step.alpha_stop),
                           stream=stream)
        out = torch.empty_like(fine)
        ref_img = torch.empty_like(fine)
        if (w, h) == (WIDTH, HEIGHT):
            ms_plain, samples_plain, ref_img = plain["ms"], plain["samples"], plain["img"]
        else:
            gv32.render(ccam, ctf, pstep, out=ref_img, stream=stream)
            ms_plain = _timed_frames([lambda: gv32.render(ccam, ctf, pstep, out=ref_img, stream=stream)],
                                     steps, flush, stream)[0]
            samples_plain = gv32.stats()["samples"]
        feat_fn = lambda: lv.features(gq, ccam, ctf, step, out=feat, stream=stream)
        net_fn = lambda: lv.mlp_infer(feat, model.packed, model.cfg.ymax, out=mult, stream=stream,
                                      ymin=model.cfg.ymin)
        render_fn = lambda: gq.render(ccam, ctf, lstep, out=out, stream=stream)
        for _ in range(3):
            feat_fn()
            net_fn()
            render_fn()
        torch.cuda.synchronize()
        lv.mlp_check()
        lst = gq.stats()
        samples, lookups = lst["samples"], lst["lookups"]
        ms_feat, ms_net, ms_render = _timed_frames([feat_fn, net_fn, render_fn], steps, flush, stream)
        fps = flop_per_sample(int(vol.deg[0]), "scalar")
        peak32, peak32_src = plain.get("peak32") or fp32_peak(None)
        ms_mult = ms_feat + ms_net
        if (w, h) == (WIDTH, HEIGHT):
            res["ablation"] = LS.ablation(gq, ccam, ctf, step, model, fine, stream=stream)
        res["by_resolution"][f"{w}x{h}"] = {
            "ms_per_frame": ms_mult + ms_render, "ms_multipliers": ms_mult, "ms_features": ms_feat,
            "ms_network": ms_net, "ms_render": ms_render,
            "samples_per_frame": samples, "lookups_per_frame": lookups, "rmse_vs_fine": rmse(out, fine),
            "plain_f32_ms_per_frame": ms_plain, "plain_f32_samples_per_frame": samples_plain,
            "plain_f32_rmse_vs_fine": rmse(ref_img, fine), "speedup_vs_plain_f32": ms_plain / (ms_mult + ms_render),
            # the learned render's counted flops (same per-sample count as the plain frame) against the FP32 peak
            "render_roofline": {"bound": "alu", "achieved": fps * samples / (ms_render * 1e-3) / 1e12,
                                "peak": peak32, "unit": "TFLOP/s",
                                "frac": fps * samples / (ms_render * 1e-3) / 1e12 / peak32,
                                "flop_per_sample": fps, "peak_source": peak32_src}}
        del fine, out
    res.update(res["by_resolution"][f"{WIDTH}x{HEIGHT}"])
    peak, peak_src = measured_bf16_tflops()
    achieved = NET_TENSOR_FLOP_PER_ROW * vol.n_elem / (res["ms_network"] * 1e-3) / 1e12
    res["network"] = {
        "kernel": "k_mlp_infer: tcgen05.mma kind::f16 (BF16 operands, FP32 accumulators in tensor memory), "
                  "M 128, N 64, K 16 per MMA; two 128-row pipelines per CTA",
        "rows": vol.n_elem, "us_per_frame": res["ms_network"] * 1e3,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "flop_per_row": NET_TENSOR_FLOP_PER_ROW,
                     "peak_source": peak_src + " dense BF16",
                     "note": "a small contraction (K <= 64, N = 64): latency of the three dependent layers per "
                             "tile bounds it, not the tensor pipe"}}
    gq.close()
    res["_model"] = model
    return res


def learned_summary(res: dict) -> dict:
    """The headline comparison in a few hundred characters: per resolution the
    learned + reduced-precision frame against the plain FP32 Eq. 4 frame
    (ms/frame, RMSE against the fine-step reference, speed-up), and the
    ablation against a constant multiplier and a per-element rule."""
    r3 = lambda x: None if x is None else float(f"{x:.4g}")
    out = {"storage": res["storage"]}
    for k, v in res["by_resolution"].items():
        out[k] = {"ms": r3(v["ms_per_frame"]), "rmse": r3(v["rmse_vs_fine"]),
                  "plain_f32_ms": r3(v["plain_f32_ms_per_frame"]), "plain_f32_rmse": r3(v["plain_f32_rmse_vs_fine"]),
                  "speedup": r3(v["speedup_vs_plain_f32"]),
                  "samples_frac": r3(v["samples_per_frame"] / v["plain_f32_samples_per_frame"]),
                  "render_frac": r3(v["render_roofline"]["frac"])}
    ab = res.get("ablation")
    if ab:
        pick = lambda b: None if b is None else [b["param"], r3(b["samples_frac"]), r3(b["rmse"])]
        out["ablation_1080p"] = {
            "network": [r3(ab["network"]["samples_frac"]), r3(ab["network"]["rmse"])],
            "empty_rule": [r3(ab["rule_empty_8x_else_1x"]["samples_frac"]), r3(ab["rule_empty_8x_else_1x"]["rmse"])],
            "best_constant": pick(ab["best_constant_at_network_rmse"]),
            "best_rule": pick(ab["best_rule_at_network_rmse"])}
    out["network_us"] = r3(res["network"]["us_per_frame"])
    return out


def serving_summary(sv: dict) -> dict:
    """p50 / p99 frame latency (ms) per mode and arrival rate."""
    out = {}
    for r in sv["runs"]:
        key = "plain" if r["mode"].startswith("FP32") else "learned"
        out.setdefault(key, {})[f"{r['rate_per_s']:g}/s"] = [float(f"{r['p50_ms']:.3g}"), float(f"{r['p99_ms']:.3g}")]
    return out


def vector_leg(flush, stream, frames: int):
    """Config 3 (the wind-flow 3-vector volume) at 1920x1080 with Eq. 4 steps:
    |v| and v_x with FP32, FP16 and BF16 blocks (per-block offset and scale,
    FP32 accumulation).  Per run [ms/frame (L2 flushed between frames),
    Gsamples/s, the image's RMSE against the FP32-block image] (the error of
    each storage against the FP64 oracle is in the GPU tests)."""
    import torch
    from paper_1707_01170_gb300 import lrvol as lv
    out = {}
    for name, field in (("cfg3mag", "|v|"), ("cfg3x", "v_x")):
        vol, tf, cam, step = _workload(name)
        ccam, ctf, cstep = lv.make_camera(cam), lv.make_tf(tf), lv.make_step(step)
        ref = None
        for storage, code in (("f32", lv.STORE_F32), ("f16", lv.STORE_F16), ("bf16", lv.STORE_BF16)):
            gv = lv.Volume(vol).build_accel(BLOCKS, stream=stream).to_bezier(code, stream=stream)
            img = torch.empty((HEIGHT, WIDTH, 4), dtype=torch.float32, device="cuda")
            for _ in range(3):
                gv.render(ccam, ctf, cstep, out=img, stream=stream)
            torch.cuda.synchronize()
            n = gv.stats()["samples"]
            ms = _timed_frames([lambda: gv.render(ccam, ctf, cstep, out=img, stream=stream)], frames, flush,
                               stream)[0]
            if ref is None:
                ref = img.clone()
            rm = float(torch.sqrt(torch.mean((img.double() - ref.double()) ** 2)))
            out[f"{field} {storage}"] = [float(f"{ms:.4g}"), float(f"{n / ms / 1e6:.4g}"), float(f"{rm:.3g}")]
            gv.close()
    return out


SL_RUNS = (("RK2", "heuristic", 1.0, 0.0), ("RK4", "heuristic", 1.0, 0.0), ("RKF5", "heuristic", 1.0, 0.0),
           ("RK4", "heuristic", 0.5, 0.0), ("RKF45", "adaptive", 0.0, 1e-6), ("BS", "adaptive", 0.0, 1e-6))
SL_BLOCKS = (256, 256, 256)
SL_STAGES = {"RK1": 1, "RK2": 2, "RK3": 3, "RK4": 4, "RK38": 4, "RKF5": 6, "HE": 2, "BS": 4, "RKF45": 6}


def streamline_leg(stream, n_seeds: int = 65536, n_err: int = 4096, t_end: float = 1.2, reps: int = 3):
    """Streamlines through config 3's wind field (Sec. 5): a seeded rake of
    n_seeds upstream of the obstacle, integrated to t_end or until the line
    leaves the domain, by several methods and step rules.  Each run is timed
    with CUDA events (mean of reps); the Eq. 7 error is taken on the first
    n_err lines against Fehlberg's fifth-order solution with the fixed step
    2^-12 (the paper's reference)."""
    import torch
    from paper_1707_01170_gb300 import lrvol as lv
    from paper_1707_01170_gb300.synth import volumes as V
    vol = V.load_config(3)
    # 256^3 blocks: the trees near the obstacle, where the lines take most of
    # their steps, are at most 3 levels deep (6 at 64^3), and every element
    # change on a line waits for its look-up
    g = lv.Volume(vol).build_accel(SL_BLOCKS, stream=stream).to_bezier(stream=stream)
    seeds = torch.from_numpy(V.config3_seeds(n_seeds)).cuda()
    href = 2.0 ** -12
    nref = int(t_end / href) + 2
    ref = lv.streamlines(g, seeds[:n_err].contiguous(), "RKF5", "fixed", href, t_end, max_samples=nref, stream=stream)
    torch.cuda.synchronize()
    out = {"volume": "config 3 (388,016 elements, triquadratic 3-vector wind flow)", "seeds": n_seeds,
           "forest": f"{SL_BLOCKS[0]}^3 blocks",
           "t_end": t_end, "reference": f"RKF5 fixed step 2^-12 on the first {n_err} seeds",
           "precision": "outer loop in float pairs (about 48 bits) and FP64 time, field evaluation in FP32",
           "runs": []}
    max_samples = 4096
    buf = (torch.empty((n_seeds, max_samples, 4), dtype=torch.float64, device="cuda"),
           torch.empty(n_seeds, dtype=torch.int32, device="cuda"), torch.empty(n_seeds, dtype=torch.int32, device="cuda"))
    for method, rule, h, tol in SL_RUNS:
        run = lambda: lv.streamlines(g, seeds, method, rule, h, t_end, tol, max_samples, out=buf, stream=stream)
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        samples, count, status = buf
        steps = int((count.to(torch.int64) - 1).clamp(min=0).sum())
        sums = lv.streamline_error(ref[0], ref[1], samples[:n_err].contiguous(), count[:n_err].contiguous(),
                                   stream=stream)
        st = torch.bincount(status.to(torch.int64), minlength=4).tolist()
        evals = steps * SL_STAGES[method]
        out["runs"].append({"method": method, "rule": rule, "h": h, "tol": tol, "ms": ms, "accepted_steps": steps,
                            "steps_per_s": steps / (ms / 1e3), "evals_per_s_accepted": evals / (ms / 1e3),
                            "eq7_max": float(sums.max()), "eq7_mean": float(sums.mean()),
                            "status_counts": {"t_end": st[0], "left": st[1], "cap": st[2], "control": st[3]}})
    # tubes (Sec. 5.3) of the first 4,096 lines of the last run, 1920x1080
    n_t, radius = 4096, 0.002
    tf3, cam3 = V.config3_render(WIDTH, HEIGHT)
    tf3.vmin, tf3.vmax = 0.0, 1.5
    ccam, ctf = lv.make_camera(cam3), lv.make_tf(tf3)
    vis = torch.empty((HEIGHT, WIDTH), dtype=torch.int64, device="cuda")
    img = torch.empty((HEIGHT, WIDTH, 4), dtype=torch.float32, device="cuda")
    samples, count, _ = buf
    tub = lambda: lv.tubes(g, ccam, samples[:n_t], count[:n_t], radius, ctf, vis=vis, out=img, stream=stream)
    tub()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        tub()
    e1.record(stream)
    torch.cuda.synchronize()
    segs = int((count[:n_t].to(torch.int64) - 1).clamp(min=0).sum())
    out["tubes"] = {"lines": n_t, "segments": segs, "radius": radius, "image": f"{WIDTH}x{HEIGHT}",
                    "ms": e0.elapsed_time(e1) / reps, "covered_pixels": int((img[..., 3] > 0).sum()),
                    "from": "the last run's first lines"}
    # small rakes (the paper traces 88 to 250 seeds): a rake's time is its
    # slowest line's latency, so these runs show the per-line latency path
    out["small_rakes"] = []
    for n_small in (256, 4096):
        sub = seeds[:n_small].contiguous()
        for method, rule, h, tol in (("RK4", "heuristic", 1.0, 0.0), ("RKF45", "adaptive", 0.0, 1e-6)):
            run = lambda: lv.streamlines(g, sub, method, rule, h, t_end, tol, max_samples,
                                         out=(buf[0][:n_small], buf[1][:n_small], buf[2][:n_small]), stream=stream)
            run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            torch.cuda.synchronize()
            cnt = buf[1][:n_small].to(torch.int64)
            out["small_rakes"].append({"seeds": n_small, "method": method, "rule": rule, "ms": e0.elapsed_time(e1) / reps,
                                       "accepted_steps": int((cnt - 1).clamp(min=0).sum()),
                                       "longest_line_steps": int(cnt.max()) - 1})
    g.close()
    return out


def trim_leg(gv, vol, tf, cam, step, flush, stream, reps: int = 10):
    """Trimming (Sec. 4.1) at 1920x1080: the per-pixel interval of a
    2.4M-triangle sphere (latitude-longitude tessellation) inside the cfg2
    volume, computed by lrvol_trim (timed), and the trimmed frame."""
    import torch
    from paper_1707_01170_gb300 import lrvol as lv
    from paper_1707_01170_gb300.synth import volumes as V
    mesh = torch.from_numpy(np.ascontiguousarray(V.uv_sphere((0.5, 0.5, 0.5), 0.35, 1000, 1200),
                                                 dtype=np.float32)).cuda()
    ccam = lv.make_camera(cam)
    tr = torch.empty((cam.height, cam.width, 2), dtype=torch.float32, device="cuda")
    lv.trim(ccam, mesh, out=tr, stream=stream)
    ms_trim = _timed_frames([lambda: lv.trim(ccam, mesh, out=tr, stream=stream)], reps, flush, stream)[0]
    tstep = lv.make_step(V.StepParams(mode=step.mode, xi=step.xi, alpha_stop=step.alpha_stop, trim=tr))
    ctf = lv.make_tf(tf)
    out = torch.empty((cam.height, cam.width, 4), dtype=torch.float32, device="cuda")
    gv.render(ccam, ctf, tstep, out=out, stream=stream)
    ms_render = _timed_frames([lambda: gv.render(ccam, ctf, tstep, out=out, stream=stream)], reps, flush, stream)[0]
    st = gv.stats()
    return {"mesh": "latitude-longitude sphere, radius 0.35, 2,400,000 triangles", "ms_trim": ms_trim,
            "ms_trimmed_frame": ms_render, "samples_per_frame": st["samples"], "rays_kept": st["rays_hit"],
            "reps": reps}


FOREST_SWEEP = (1, 4, 16, 64, 256)
OCTREE_SWEEP = (1, 4, 16)   # midpoint (octree-style) trees; at 64^3 cfg2 has no trees at all


SHORT_SWEEP = (("cfg2", (1, 16, 64)), ("cfg3mag", (4, 16, 64)))


def forest_leg(stream, frames: int = 20, plan=None):
    """The paper's look-up comparison (Sec. 4.3 tables) on the synthetic
    volumes: for each forest resolution (trees per axis) and split rule
    (depth-balanced k-d trees; octree-style midpoint trees), the build time
    on the host, the tree depth statistics and the 1080p frame time (cfg2
    scalar and cfg3 |v|, Eq. 4 steps, L2 flushed between frames).  One
    balanced tree is the single k-d tree, one midpoint tree the octree, and
    the forest at the finest element size (no trees) the look-up texture."""
    import torch
    from paper_1707_01170_gb300 import lrvol as lv
    from paper_1707_01170_gb300.synth import volumes as V
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = []
    for name in ("cfg2", "cfg3mag"):
        if plan is not None and name not in dict(plan):
            continue
        vol, tf, cam, step = _workload(name)
        ccam, ctf, cstep = lv.make_camera(cam), lv.make_tf(tf), lv.make_step(step)
        img = torch.empty((HEIGHT, WIDTH, 4), dtype=torch.float32, device="cuda")
        runs = [(lv.SPLIT_BALANCED, b) for b in FOREST_SWEEP] + [(lv.SPLIT_MIDPOINT, b) for b in OCTREE_SWEEP]
        if plan is not None:
            runs = [(lv.SPLIT_BALANCED, b) for b in dict(plan).get(name, ())]
        for split, b in runs:
            gv = lv.Volume(vol)
            t0 = time.perf_counter()
            try:
                gv.build_accel((b, b, b), stream=stream, split=split)
            except lv.LrvolError as e:
                out.append({"workload": name, "split": "midpoint", "trees_per_axis": b, "unsupported": str(e)})
                gv.close()
                continue
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
            gv.to_bezier(stream=stream)
            for _ in range(3):
                gv.render(ccam, ctf, cstep, out=img, stream=stream)
            torch.cuda.synchronize()
            st = gv.stats()
            ms = _timed_frames([lambda: gv.render(ccam, ctf, cstep, out=img, stream=stream)], frames, flush, stream)[0]
            out.append({"workload": name, "split": "balanced" if split == lv.SPLIT_BALANCED else "midpoint",
                        "trees_per_axis": b, "build_s": build_s, "nodes": st["n_nodes"],
                        "depth": {"min": st["depth_min"], "max": st["depth_max"], "mean": st["depth_mean"],
                                  "var": st["depth_var"]},
                        "ms_per_frame": ms, "lookups_per_frame": st["lookups"],
                        "gsamples_per_s": st["samples"] / (ms / 1e3) / 1e9})
            gv.close()
    return out


SERVE_PLAN = ((60.0, 500), (120.0, 1000), (240.0, 2000))   # (requests/s, requests): about 8 s each


def serving_leg(model, modes, plan=SERVE_PLAN, slots: int = 8, arena_gb: int = 4):
    """Continuous-batching frame server over three resident volumes (configs
    1, 2 and 3 as |v|): seeded Poisson request streams mixing 256x256,
    1920x1080 and 3840x2160 frames on orbiting cameras, admitted by free
    slot and arena memory.  Per mode and arrival rate: latency p50/p99 (ms,
    completion minus arrival, host clock), frames/s and Gsamples/s."""
    import torch
    from paper_1707_01170_gb300 import lrvol as lv
    from paper_1707_01170_gb300 import serve
    from paper_1707_01170_gb300.synth import volumes as V
    vols = [V.load_config(1), V.load_config(2), V.load_config(3)]
    tf1 = V.config1_render()[0]
    tf2 = V.config2_render(vol=vols[1])[0]
    tf3 = V.config3_render()[0]
    tf3.vmin, tf3.vmax = 0.0, 1.5
    tfs = [tf1, tf2, tf3]
    plain = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99)
    mag = V.StepParams(mode="heuristic", xi=1 / 256, alpha_stop=0.99, field="magnitude")
    learned = V.StepParams(mode="learned", xi=1 / 256, alpha_stop=0.99)
    out = {"volumes": ["config 1 (9,864 elements)", "config 2 (174,000)", "config 3 |v| (388,016)"],
           "sizes": [f"{w}x{h}" for w, h in serve.SIZES], "slots": slots, "arena_bytes": arena_gb << 30,
           "priority_pixels": 1 << 20, "latency": "host clock, from scheduled arrival to the poll that saw the "
                                                  "frame finished; images stay on the device", "runs": []}
    for mode in modes:
        store = lv.STORE_F32 if mode == "plain" else lv.STORE_F16
        gvs = [lv.Volume(v).build_accel(BLOCKS).to_bezier(store) for v in vols]
        steps = [plain, plain, mag] if mode == "plain" else [learned, learned, mag]
        for rate, n in plan:
            srv = lv.Server(slots=slots, arena_bytes=arena_gb << 30)
            srv.set_priority_pixels(1 << 20)
            if mode != "plain":
                srv.set_step_model(model.packed, model.cfg.ymax, model.cfg.ymin)
            reqs = serve.request_stream(1707011700 + 5000 + int(rate), n, rate, 3)
            torch.cuda.synchronize()
            recs = serve.run_stream(srv, gvs, tfs, steps, reqs)
            summ = serve.summarize(recs)
            st = srv.stats()
            srv.close()
            out["runs"].append({"mode": "FP32 blocks, Eq. 4" if mode == "plain" else
                                "FP16 blocks, learned steps on configs 1-2 (server-side network), Eq. 4 on config 3",
                                "rate_per_s": rate, "requests": n, "max_in_flight": st["max_running"],
                                "arena_high_water": st["arena_high_water"], **summ})
        for g in gvs:
            g.close()
    return out


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1707_01170_gb300 import lrvol as lv

    vol, tf, cam, step = _workload(args.workload)
    stream = torch.cuda.current_stream()
    # ---- setup (once per volume) ----
    t0 = time.perf_counter()
    gv = lv.Volume(vol)
    t1 = time.perf_counter()
    gv.build_accel(BLOCKS, stream=stream)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    gv.to_bezier(storage={"f32": lv.STORE_F32, "f16": lv.STORE_F16, "bf16": lv.STORE_BF16}[args.storage],
                 stream=stream)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    ccam, ctf, cstep = lv.make_camera(cam), lv.make_tf(tf), lv.make_step(step)
    out = torch.zeros((HEIGHT, WIDTH, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        gv.render(ccam, ctf, cstep, out=out, stream=stream)
    torch.cuda.synchronize()
    st = gv.stats()
    samples_per_frame = st["samples"]

    # ---- timed region: K frames, L2 flushed between frames (flush not timed) ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            gv.render(ccam, ctf, cstep, out=out, stream=stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    clk_summary = clk.summary()
    if dist:
        dist.barrier()
    per = [a.elapsed_time(b) for a, b in evs]
    dev_ms = float(sum(per))
    if dist:
        t = torch.tensor([dev_ms, wall], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms, wall = float(t[0]), float(t[1])
    total_samples = samples_per_frame * args.steps * ws
    value = total_samples / (dev_ms / 1e3) / 1e9
    ms_per_step = dev_ms / args.steps

    learned = None
    if args.learned != "off" and ws == 1 and step.field == "scalar":
        if args.storage == "f32":
            plain = {"gv32": gv, "ms": ms_per_step, "samples": samples_per_frame, "img": out.clone(),
                     "peak32": fp32_peak(clk_summary)}
            learned = learned_leg(vol, tf, step, plain, max(3, min(args.steps, 50)), args.learned, flush, stream,
                                  args.learned_model, args.save_learned_model)

    shading = None
    if ws == 1 and step.field == "scalar" and args.workload == "cfg2":
        from paper_1707_01170_gb300.synth import volumes as V
        sstep = lv.make_step(V.StepParams(mode="heuristic", xi=step.xi, alpha_stop=step.alpha_stop,
                                          shading="gradient"))
        for _ in range(3):
            gv.render(ccam, ctf, sstep, out=out, stream=stream)
        torch.cuda.synchronize()
        s_samples = gv.stats()["samples"]
        n_sh = max(3, min(args.steps, 50))
        ms_sh = _timed_frames([lambda: gv.render(ccam, ctf, sstep, out=out, stream=stream)], n_sh, flush, stream)[0]
        fps_sh = flop_per_sample_shaded(int(vol.deg[0]))
        ach = fps_sh * s_samples / (ms_sh / 1e3) / 1e12
        shading = {"what": "gradient shading (Sec. 4.1), light at the eye, same frame and storage",
                   "ms_per_frame": ms_sh, "samples_per_frame": s_samples,
                   "gsamples_per_s": s_samples / (ms_sh / 1e3) / 1e9, "flop_per_sample": fps_sh,
                   "achieved_tflops": ach, "frac_of_fp32_peak": ach / fp32_peak(clk_summary)[0],
                   "frames_timed": n_sh,
                   "kernel": f"k_render<{int(vol.deg[0])},3,{args.storage}>"}

    sl = None
    if args.streamlines and ws == 1:
        sl = streamline_leg(stream, n_seeds=args.sl_seeds)

    trimming = None
    if ws == 1 and args.workload == "cfg2":
        trimming = trim_leg(gv, vol, tf, cam, step, flush, stream)

    forest = forest_leg(stream) if (args.forest_sweep and ws == 1) else None
    # a short look-up sweep in every default run: the k-d trees the 64^3
    # benchmark forest leaves out (cfg2 needs none there) at work
    forest_short = forest_leg(stream, frames=10, plan=SHORT_SWEEP) if (not args.forest_sweep and ws == 1
                                                                      and args.short_sweep) else None

    vector = vector_leg(flush, stream, max(3, min(args.steps, 30))) if (args.vector and ws == 1) else None

    serving = None
    if args.serve != "off" and ws == 1:
        modes = ["plain", "learned"] if args.serve == "both" else [args.serve]
        if "learned" in modes and (learned is None or "_model" not in learned):
            modes = [m for m in modes if m != "learned"]
        serving = serving_leg(learned.get("_model") if learned else None, modes)

    # ---- end to end through the C ABI with host buffers ----
    # Every frame: the camera, TF and step go host -> device as kernel
    # parameters and the 33.2 MB image comes back to pinned host memory.
    # Streaming form: two frames in flight, frame k's image copied on a second
    # stream while frame k+1 renders; the host holds frame k before frame k+2
    # is submitted.  The serial form (render, copy, wait) is reported beside it.
    import ctypes
    hosts = [torch.empty((HEIGHT, WIDTH, 4), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    outs = [out, torch.empty_like(out)]
    copy_stream = torch.cuda.Stream()
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(10, min(args.steps, 60))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for k in range(e2e_steps):
        b = k & 1
        if k >= 2:
            copied[b].synchronize()          # the host has frame k-2; its buffers are free again
        gv.render(ccam, ctf, cstep, out=outs[b], stream=stream)   # camera/TF/step travel as kernel parameters
        rendered[b].record(stream)
        copy_stream.wait_event(rendered[b])
        with torch.cuda.stream(copy_stream):
            hosts[b].copy_(outs[b], non_blocking=True)
        copied[b].record(copy_stream)
    copied[(e2e_steps - 1) & 1].synchronize()
    copied[e2e_steps & 1].synchronize()
    e2e_s = (time.perf_counter() - e0) / e2e_steps
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(e2e_steps):
        gv.render(ccam, ctf, cstep, out=out, stream=stream)
        hosts[0].copy_(out, non_blocking=True)
        stream.synchronize()
    serial_s = (time.perf_counter() - e0) / e2e_steps
    if dist:                                   # whole-job figures: the slowest rank's times
        t = torch.tensor([e2e_s, serial_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s, serial_s = float(t[0]), float(t[1])
    h2d = ctypes.sizeof(lv.Camera) + ctypes.sizeof(lv.TF) + ctypes.sizeof(lv.Step)
    e2e = {"value": samples_per_frame * ws / e2e_s / 1e9, "unit": "Gsamples/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": HEIGHT * WIDTH * 16, "ms_per_step": 1e3 * e2e_s, "frames": e2e_steps,
           "form": "two frames in flight: image copies on a second stream overlap the next render",
           "serial": {"value": samples_per_frame * ws / serial_s / 1e9, "ms_per_step": 1e3 * serial_s,
                      "form": "render, copy, wait per frame"}}

    if rank != 0:
        gv.close()
        if dist:
            dist.destroy_process_group()
        return 0
    fps = flop_per_sample(int(vol.deg[0]), step.field)
    flop = fps * samples_per_frame
    achieved = flop / (ms_per_step / 1e3) / 1e12
    prof = profiled_counters() if (args.workload == "cfg2" and args.storage == "f32") else None
    fcode = {"scalar": 0, "magnitude": 1, "component": 2}[step.field]
    peak, peak_src = fp32_peak(clk_summary)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": prof["traffic"] if prof else None,
            "kernel": f"k_render<{int(vol.deg[0])},{fcode},{args.storage}>", "flop_per_sample": fps,
            "peak_source": peak_src}
    hbm = measured_hbm_gbs()
    if prof:
        dram_gbs = prof["traffic"] / (ms_per_step / 1e3) / 1e9
        roof["memory_side"] = {"dram_gbs": dram_gbs, "hbm_peak_gbs": hbm,
                               "dram_frac": dram_gbs / hbm if hbm else None,
                               "l2_gbs": prof["l2"] / (ms_per_step / 1e3) / 1e9 if prof["l2"] else None,
                               "source": "ncu bytes per launch (profiles/k_render_cfg2_1080p.md) / event time"}
    line = {"metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(args.workload, args.storage, ws),
            "frame": {"samples": samples_per_frame, "rays_hit": st["rays_hit"], "lookups": st["lookups"]},
            "wall_s": wall, "gpu_launches": args.steps,
            "roofline": roof, "e2e": e2e, "clocks": clk_summary,
            "setup": {"create_s": t1 - t0, "build_accel_s": t2 - t1, "to_bezier_s": t3 - t2,
                      "forest_depth": [st["depth_min"], st["depth_max"], st["depth_mean"], st["depth_var"]],
                      "n_nodes": st["n_nodes"], "incidence_entries": st["incidence_entries"]}}
    # details first; the driver keeps the end of the line, so the headline
    # comparison (learned_step) comes last and short
    if learned is not None:
        learned.pop("_model", None)
        line["learned_step_detail"] = learned
    if serving is not None:
        line["serving_detail"] = serving
    if sl is not None:
        line["streamlines"] = sl
    if forest is not None:
        line["forest_sweep"] = forest
    if trimming is not None:
        line["trimming"] = trimming
    if shading is not None:
        line["shading"] = shading
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(vol, tf, cam, step, samples_per_frame)
    if serving is not None:
        line["serving"] = serving_summary(serving)
    if forest_short is not None:
        line["forest"] = [[r["workload"], r["trees_per_axis"], float(f"{r['depth']['mean']:.3g}"),
                           float(f"{r['ms_per_frame']:.4g}")] for r in forest_short if "ms_per_frame" in r]
    if vector is not None:
        line["vector"] = vector
    if learned is not None:
        line["learned_step"] = learned_summary(learned)
    print(json.dumps(line))
    gv.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="cfg2", choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"],
                    help="Bezier block storage (FP32 accumulation in every case)")
    ap.add_argument("--learned", default="f16", choices=["off", "f32", "f16", "bf16"],
                    help="also time learned step sizes with this block storage against plain FP32 Eq. 4")
    ap.add_argument("--learned-model", default=None, help="load step-model weights instead of training")
    ap.add_argument("--save-learned-model", default=None, help="write the trained step-model weights here")
    ap.add_argument("--serve", default="both", choices=["off", "plain", "learned", "both"],
                    help="frame-server runs over three resident volumes (learned needs --learned)")
    ap.add_argument("--forest-sweep", action="store_true",
                    help="also time the frame for 1^3 .. 256^3 trees (the paper's look-up comparison)")
    ap.add_argument("--no-streamlines", dest="streamlines", action="store_false",
                    help="skip the streamline runs on config 3")
    ap.add_argument("--no-short-sweep", dest="short_sweep", action="store_false",
                    help="skip the short look-up sweep (cfg2 at 1, 16, 64 and cfg3 |v| at 4, 16, 64 trees per axis)")
    ap.add_argument("--no-vector", dest="vector", action="store_false",
                    help="skip the config 3 |v| and v_x frames (FP32, FP16, BF16 blocks)")
    ap.add_argument("--sl-seeds", type=int, default=65536,
                    help="seeds of the streamline runs (a smaller rake makes a small profiling case)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)   # at least 3 untimed warm-up frames
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

"""bench.py's reference arm runs on the CPU (it is the oracle): it must print
one JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_record_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    """The roofline's ncu traffic comes from the committed k_render summary
    only while the render kernel's sources still have the hash that summary
    records."""
    b = _bench_module()
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "paper_1707_01170_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in b.RENDER_SOURCES:
        (src / name).write_bytes(b"// source A of " + name.encode() + b"\n")
    sha = b.render_source_hash(str(tmp_path))
    (tmp_path / "profiles" / "k_render_cfg2_1080p.md").write_text(
        "# summary\n\n    render_source_sha256_16: %s\n" % sha
        + "    traffic_bytes_per_launch: 123\n    l2_bytes_per_launch: 456\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.profiled_counters() == {"traffic": 123, "l2": 456}
    (src / "device_common.cuh").write_bytes(b"// source B\n")
    assert b.profiled_counters() is None


def test_committed_traffic_record_parses():
    rec = _bench_module().profiled_counters()
    assert rec is None or (rec["traffic"] > 0 and rec["l2"] > rec["traffic"])


def test_network_roofline_inputs(tmp_path, monkeypatch):
    b = _bench_module()
    assert b.NET_TENSOR_FLOP_PER_ROW == 2 * (16 * 64 + 64 * 64 * 2)     # the three hidden layers, FMA = 2
    peak, src = b.measured_bf16_tflops()
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        assert src.startswith("measured") and peak == json.load(open(peaks))["bf16_tflops"]
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.measured_bf16_tflops() == (1900.0, "fallback")


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    """Launched like the multi-GPU runs (torchrun, two ranks, 127.0.0.1),
    rank 0 alone prints the one JSON line and every rank exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0

"""Frame serving over resident volumes: a seeded request stream and the host
loop that drives the library's frame server (lrvol_server_*).

Requests arrive by a Poisson process.  Each names a resident volume, an
image size and a camera on that volume's orbit.  The loop submits every
request at its arrival time, lets the server admit and launch work between
arrivals (continuous batching: a request arriving while others run is
admitted as soon as a slot and arena memory are free, and its frame runs
beside theirs), collects retired frames, and records each frame's latency,
completion minus arrival.  All rendering happens in the library's kernels.

A serving process should set CUDA_DEVICE_MAX_CONNECTIONS to 3 x slots (at
most 32) before its CUDA context exists: each slot launches on one of three
streams of different priority, and streams that share a hardware queue
serialise (a small frame would wait for a large one queued before it).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import lrvol as lv
from .synth.lrgen import Stream
from .synth.volumes import Camera

SIZES = ((256, 256), (1920, 1080), (3840, 2160))


@dataclass
class FrameRequest:
    arrival: float      # seconds after the start of the stream
    volume: int         # index into the server's volume list
    width: int
    height: int
    camera: Camera


def orbit_view(volume: int, k: int, n_volumes: int, width: int, height: int, steps: int = 240,
               radius: float = 1.8, fovy_deg: float = 40.0) -> Camera:
    """The k-th camera on volume `volume`'s orbit: the azimuth advances by
    2 pi / steps per frame from a per-volume phase, the elevation swings
    between -20 and +20 degrees twice per revolution."""
    az = 2 * math.pi * (volume / max(1, n_volumes) + k / steps)
    el = math.radians(20.0) * math.sin(4 * math.pi * k / steps)
    d = (math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el))
    eye = tuple(0.5 + radius * c for c in d)
    return Camera("persp", width, height, eye=eye, target=(0.5, 0.5, 0.5), up=(0.0, 0.0, 1.0),
                  fovy=math.radians(fovy_deg))


def request_stream(seed: int, n: int, rate: float, n_volumes: int, sizes=SIZES):
    """n seeded requests: exponential inter-arrival times of mean 1/rate,
    volume and size uniform, cameras advancing along each volume's orbit."""
    u = Stream(seed, 3 * n + 16).take(3 * n).reshape(n, 3)
    t, out, k = 0.0, [], [0] * n_volumes
    for i in range(n):
        t += -math.log1p(-u[i, 0]) / rate
        v = min(n_volumes - 1, int(u[i, 1] * n_volumes))
        w, h = sizes[min(len(sizes) - 1, int(u[i, 2] * len(sizes)))]
        out.append(FrameRequest(t, v, w, h, orbit_view(v, k[v], n_volumes, w, h)))
        k[v] += 1
    return out


def percentile(x, q: float) -> float:
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    a = np.sort(np.asarray(x, dtype=np.float64))
    if a.size == 0:
        return float("nan")
    pos = (a.size - 1) * q / 100.0
    lo = int(math.floor(pos))
    hi = min(lo + 1, a.size - 1)
    return float(a[lo] + (a[hi] - a[lo]) * (pos - lo))


def run_stream(server: "lv.Server", volumes, tfs, steps, requests, realtime: bool = True, keep: bool = False,
               lead_s: float = 0.02):
    """Drive the server through the request stream.

    volumes, tfs, steps: per volume index, the resident lv.Volume, its
    transfer function and step parameters.  Returns one record per request
    (arrival/admit/done times relative to the stream start, latency_ms,
    device_ms, samples, ticket when `keep`)."""
    ctfs = [lv.make_tf(t) for t in tfs]
    csteps = [lv.make_step(s, allow_auto=True) for s in steps]
    n = len(requests)
    records = [None] * n
    index = {}
    t0 = lv.clock() + lead_s
    i = 0
    while i < n or index:
        now = lv.clock()
        while i < n and (not realtime or t0 + requests[i].arrival <= now):
            r = requests[i]
            tk = server.submit(volumes[r.volume], r.camera, ctfs[r.volume], csteps[r.volume])
            index[tk] = i
            i += 1
        server.progress()
        for tk in server.poll():
            d = server.info(tk)
            q = index.pop(tk)
            r = requests[q]
            arr = t0 + r.arrival if realtime else d["t_submit"]
            records[q] = {"volume": r.volume, "width": r.width, "height": r.height,
                          "arrival_s": arr - t0, "admit_s": d["t_admit"] - t0, "done_s": d["t_done"] - t0,
                          "latency_ms": 1e3 * (d["t_done"] - arr), "device_ms": d["device_ms"],
                          "samples": d["samples"], "state": d["state"], "status": d["status"]}
            if keep:
                records[q]["ticket"] = tk
            else:
                server.release(tk)
        if realtime and i < n and not index:
            # idle until the next arrival (the server has nothing in flight)
            wait = t0 + requests[i].arrival - lv.clock()
            if wait > 2e-4:
                time.sleep(wait - 1e-4)
    return records


def summarize(records, wall_s: float | None = None) -> dict:
    """Latency percentiles (overall and per image size) and throughput."""
    ok = [r for r in records if r is not None and r["state"] == lv.REQ_DONE]
    lat = [r["latency_ms"] for r in ok]
    span = wall_s if wall_s is not None else (max(r["done_s"] for r in ok) - min(r["arrival_s"] for r in ok))
    out = {"frames": len(ok), "failed": sum(1 for r in records if r is not None and r["state"] != lv.REQ_DONE),
           "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99), "mean_ms": float(np.mean(lat)),
           "max_ms": float(np.max(lat)), "span_s": span, "frames_per_s": len(ok) / span,
           "gsamples_per_s": sum(r["samples"] for r in ok) / span / 1e9,
           "device_busy": sum(r["device_ms"] for r in ok) / 1e3 / span}
    by = {}
    for r in ok:
        by.setdefault(f'{r["width"]}x{r["height"]}', []).append(r["latency_ms"])
    out["by_size"] = {k: {"n": len(v), "p50_ms": percentile(v, 50), "p99_ms": percentile(v, 99)}
                      for k, v in sorted(by.items())}
    return out

"""Python binding of liblrvol (include/lrvol.h): argument marshalling only.

Device buffers and streams come from PyTorch; every step of the path runs in
the library's CUDA kernels.  There is no CPU fallback: if liblrvol.so is
missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrvol.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_BOUNDS, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
ORTHO, PERSP = 0, 1
STEP_FIXED, STEP_HEURISTIC, STEP_LEARNED = 0, 1, 2
FIELD_SCALAR, FIELD_MAGNITUDE, FIELD_COMPONENT = 0, 1, 2
STORE_F32, STORE_F16, STORE_BF16 = 0, 1, 2
SHADE_NONE, SHADE_GRADIENT = 0, 1
SPLIT_BALANCED, SPLIT_MIDPOINT = 0, 1
NONE = 0xFFFFFFFF

EXPORTED = ["lrvol_create", "lrvol_build_accel", "lrvol_build_accel_split", "lrvol_to_bezier", "lrvol_render",
            "lrvol_lookup", "lrvol_eval", "lrvol_eval_grad", "lrvol_get_bezier", "lrvol_stats",
            "lrvol_status_string", "lrvol_last_error", "lrvol_destroy", "lrvol_render_noalloc",
            "lrvol_render_trace", "lrvol_features",
            "lrvol_mlp_pack", "lrvol_mlp_infer", "lrvol_mlp_check", "lrvol_mlp_infer_timeout_test",
            "lrvol_mlp_scratch_floats", "lrvol_mlp_grad", "lrvol_mlp_train_step", "lrvol_labels",
            "lrvol_arena_create", "lrvol_arena_alloc", "lrvol_arena_free", "lrvol_arena_used",
            "lrvol_arena_largest_free", "lrvol_arena_destroy", "lrvol_server_create", "lrvol_server_set_step_model",
            "lrvol_server_set_priority_pixels", "lrvol_server_set_large_cap", "lrvol_server_submit",
            "lrvol_server_progress", "lrvol_server_drain", "lrvol_server_poll", "lrvol_server_info",
            "lrvol_server_release", "lrvol_server_get_stats", "lrvol_server_clock", "lrvol_server_destroy",
            "lrvol_streamlines", "lrvol_streamline_error", "lrvol_trim", "lrvol_tubes"]
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
SL_METHODS = ["RK1", "RK2", "RK3", "RK4", "RK38", "RKF5", "HE", "BS", "RKF45"]
SL_RULES = ["fixed", "heuristic", "adaptive"]
MLP_IN, MLP_HIDDEN, MLP_PARAMS, MLP_PACKED = 16, 64, 9473, 10120
BAND_ROWS = 8


class LrvolError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({_lib_str(status)}): {last_error()}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("projection", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fovy", ctypes.c_double), ("extent", ctypes.c_double),
                ("row_begin", ctypes.c_int32), ("row_end", ctypes.c_int32),
                ("band_count", ctypes.c_int32), ("band_index", ctypes.c_int32)]


class TF(ctypes.Structure):
    _fields_ = [("rgba", (ctypes.c_float * 4) * 256), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double)]


class Step(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("field", ctypes.c_int32), ("component", ctypes.c_int32),
                ("h", ctypes.c_double), ("xi", ctypes.c_double), ("alpha_stop", ctypes.c_double),
                ("mult", ctypes.c_void_p), ("shading", ctypes.c_int32), ("light", ctypes.c_double * 3),
                ("trim", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("n_basis", ctypes.c_int64), ("n_nodes", ctypes.c_int64),
                ("blocks", ctypes.c_int32 * 3), ("depth_min", ctypes.c_int32), ("depth_max", ctypes.c_int32),
                ("depth_mean", ctypes.c_double), ("depth_var", ctypes.c_double),
                ("incidence_entries", ctypes.c_int64), ("bytes_device", ctypes.c_int64),
                ("samples", ctypes.c_int64), ("lookups", ctypes.c_int64), ("rays_hit", ctypes.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["blocks"] = list(self.blocks)
        return d


class SLParams(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("step_rule", ctypes.c_int32), ("h", ctypes.c_double),
                ("t_end", ctypes.c_double), ("tol", ctypes.c_double), ("max_samples", ctypes.c_int32)]


class FrameInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("rgba_dev", ctypes.c_void_p),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("device_ms", ctypes.c_float), ("dev_start_ms", ctypes.c_float), ("dev_end_ms", ctypes.c_float),
                ("samples", ctypes.c_int64), ("lookups", ctypes.c_int64), ("rays_hit", ctypes.c_int64),
                ("bytes", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("done", ctypes.c_int64), ("failed", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("arena_used", ctypes.c_int64), ("arena_high_water", ctypes.c_int64), ("slots", ctypes.c_int32),
                ("max_running", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load liblrvol.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"liblrvol.so not built at {path}: run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.lrvol_create.restype = ctypes.c_int
        L.lrvol_create.argtypes = [vp, i32, i64, vp, i64, vp, vp, vp, ctypes.POINTER(vp)]
        L.lrvol_build_accel.restype = ctypes.c_int
        L.lrvol_build_accel.argtypes = [vp, vp, vp]
        L.lrvol_build_accel_split.restype = ctypes.c_int
        L.lrvol_build_accel_split.argtypes = [vp, vp, i32, vp]
        L.lrvol_to_bezier.restype = ctypes.c_int
        L.lrvol_to_bezier.argtypes = [vp, i32, vp]
        L.lrvol_render.restype = ctypes.c_int
        L.lrvol_render.argtypes = [vp, ctypes.POINTER(Camera), ctypes.POINTER(TF), ctypes.POINTER(Step), vp, vp]
        L.lrvol_render_trace.restype = ctypes.c_int
        L.lrvol_render_trace.argtypes = [vp, ctypes.POINTER(Camera), ctypes.POINTER(TF), ctypes.POINTER(Step),
                                         vp, i64, i32, vp, vp, vp, vp]
        L.lrvol_render_noalloc.restype = ctypes.c_int
        L.lrvol_render_noalloc.argtypes = [vp, ctypes.POINTER(Camera), ctypes.POINTER(TF), ctypes.POINTER(Step),
                                           vp, vp, vp]
        L.lrvol_lookup.restype = ctypes.c_int
        L.lrvol_lookup.argtypes = [vp, vp, i64, vp, vp]
        L.lrvol_eval.restype = ctypes.c_int
        L.lrvol_eval.argtypes = [vp, vp, i64, vp, vp]
        L.lrvol_eval_grad.restype = ctypes.c_int
        L.lrvol_eval_grad.argtypes = [vp, vp, i64, vp, vp]
        L.lrvol_get_bezier.restype = ctypes.c_int
        L.lrvol_get_bezier.argtypes = [vp, vp]
        L.lrvol_stats.restype = ctypes.c_int
        L.lrvol_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.lrvol_status_string.restype = ctypes.c_char_p
        L.lrvol_status_string.argtypes = [ctypes.c_int]
        L.lrvol_last_error.restype = ctypes.c_char_p
        L.lrvol_last_error.argtypes = []
        L.lrvol_destroy.restype = None
        L.lrvol_destroy.argtypes = [vp]
        L.lrvol_features.restype = ctypes.c_int
        L.lrvol_features.argtypes = [vp, ctypes.POINTER(Camera), ctypes.POINTER(TF), ctypes.POINTER(Step), vp, vp]
        L.lrvol_mlp_pack.restype = ctypes.c_int
        L.lrvol_mlp_pack.argtypes = [vp, vp, vp]
        L.lrvol_mlp_infer.restype = ctypes.c_int
        L.lrvol_mlp_infer.argtypes = [vp, i64, vp, ctypes.c_float, ctypes.c_float, vp, vp]
        L.lrvol_mlp_check.restype = ctypes.c_int
        L.lrvol_mlp_check.argtypes = []
        L.lrvol_mlp_infer_timeout_test.restype = ctypes.c_int
        L.lrvol_mlp_infer_timeout_test.argtypes = [vp, i64, vp, ctypes.c_float, ctypes.c_float, vp, vp]
        L.lrvol_mlp_scratch_floats.restype = i64
        L.lrvol_mlp_scratch_floats.argtypes = [i64]
        L.lrvol_mlp_grad.restype = ctypes.c_int
        L.lrvol_mlp_grad.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
        L.lrvol_mlp_train_step.restype = ctypes.c_int
        L.lrvol_mlp_train_step.argtypes = [vp, vp, i64, vp, vp, vp, i64, ctypes.c_float, vp, vp, vp]
        L.lrvol_labels.restype = ctypes.c_int
        L.lrvol_labels.argtypes = [vp, ctypes.POINTER(Camera), ctypes.POINTER(TF), ctypes.POINTER(Step),
                                   ctypes.c_double, ctypes.c_double, vp, i32, vp, vp]
        L.lrvol_tubes.restype = ctypes.c_int
        L.lrvol_tubes.argtypes = [vp, ctypes.POINTER(Camera), vp, vp, i64, i32, ctypes.c_float, ctypes.POINTER(TF),
                                  vp, vp, vp]
        L.lrvol_trim.restype = ctypes.c_int
        L.lrvol_trim.argtypes = [ctypes.POINTER(Camera), vp, i64, vp, vp]
        L.lrvol_streamlines.restype = ctypes.c_int
        L.lrvol_streamlines.argtypes = [vp, ctypes.POINTER(SLParams), vp, i64, vp, vp, vp, vp]
        L.lrvol_streamline_error.restype = ctypes.c_int
        L.lrvol_streamline_error.argtypes = [vp, vp, i32, vp, vp, i32, i64, vp, vp]
        L.lrvol_arena_create.restype = ctypes.c_int
        L.lrvol_arena_create.argtypes = [i64, i64, ctypes.POINTER(vp)]
        L.lrvol_arena_alloc.restype = i64
        L.lrvol_arena_alloc.argtypes = [vp, i64]
        L.lrvol_arena_free.restype = ctypes.c_int
        L.lrvol_arena_free.argtypes = [vp, i64]
        L.lrvol_arena_used.restype = i64
        L.lrvol_arena_used.argtypes = [vp]
        L.lrvol_arena_largest_free.restype = i64
        L.lrvol_arena_largest_free.argtypes = [vp]
        L.lrvol_arena_destroy.restype = None
        L.lrvol_arena_destroy.argtypes = [vp]
        L.lrvol_server_create.restype = ctypes.c_int
        L.lrvol_server_create.argtypes = [i32, i64, ctypes.POINTER(vp)]
        L.lrvol_server_set_step_model.restype = ctypes.c_int
        L.lrvol_server_set_step_model.argtypes = [vp, vp, ctypes.c_float, ctypes.c_float]
        L.lrvol_server_set_priority_pixels.restype = ctypes.c_int
        L.lrvol_server_set_priority_pixels.argtypes = [vp, i64]
        L.lrvol_server_set_large_cap.restype = ctypes.c_int
        L.lrvol_server_set_large_cap.argtypes = [vp, i32]
        L.lrvol_server_submit.restype = ctypes.c_int
        L.lrvol_server_submit.argtypes = [vp, vp, ctypes.POINTER(Camera), ctypes.POINTER(TF), ctypes.POINTER(Step),
                                          vp, ctypes.POINTER(i64)]
        L.lrvol_server_progress.restype = ctypes.c_int
        L.lrvol_server_progress.argtypes = [vp, ctypes.POINTER(i32)]
        L.lrvol_server_drain.restype = ctypes.c_int
        L.lrvol_server_drain.argtypes = [vp]
        L.lrvol_server_poll.restype = ctypes.c_int
        L.lrvol_server_poll.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        L.lrvol_server_info.restype = ctypes.c_int
        L.lrvol_server_info.argtypes = [vp, i64, ctypes.POINTER(FrameInfo)]
        L.lrvol_server_release.restype = ctypes.c_int
        L.lrvol_server_release.argtypes = [vp, i64]
        L.lrvol_server_get_stats.restype = ctypes.c_int
        L.lrvol_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.lrvol_server_clock.restype = ctypes.c_double
        L.lrvol_server_clock.argtypes = []
        L.lrvol_server_destroy.restype = None
        L.lrvol_server_destroy.argtypes = [vp]
        _lib = L
    return _lib


def _lib_str(status: int) -> str:
    try:
        return load().lrvol_status_string(status).decode()
    except Exception:  # library not loadable
        return "?"


def last_error() -> str:
    try:
        return load().lrvol_last_error().decode()
    except Exception:
        return ""


def _check(status: int, what: str) -> None:
    if status != OK:
        raise LrvolError(status, what)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def make_camera(cam, row_begin: int = 0, row_end: int = 0, band_count: int = 0, band_index: int = 0) -> Camera:
    """From any object with projection ('ortho'|'persp'), width, height, eye, target, up, fovy, extent;
    optionally a row range and an interleaved band (every band_count-th 8-row band from band_index)."""
    c = Camera()
    c.projection = PERSP if cam.projection == "persp" else ORTHO
    c.width, c.height = int(cam.width), int(cam.height)
    c.eye = (ctypes.c_double * 3)(*[float(v) for v in cam.eye])
    c.target = (ctypes.c_double * 3)(*[float(v) for v in cam.target])
    c.up = (ctypes.c_double * 3)(*[float(v) for v in cam.up])
    c.fovy, c.extent = float(cam.fovy), float(cam.extent)
    c.row_begin, c.row_end = int(row_begin), int(row_end)
    c.band_count, c.band_index = int(band_count), int(band_index)
    return c


def make_tf(tf) -> TF:
    """From any object with table (256 x 4), vmin, vmax; the table is rounded to FP32."""
    t = TF()
    tab = np.ascontiguousarray(np.asarray(tf.table, dtype=np.float32).reshape(256, 4))
    ctypes.memmove(ctypes.addressof(t.rgba), tab.ctypes.data, tab.nbytes)
    t.vmin, t.vmax = float(tf.vmin), float(tf.vmax)
    return t


def make_step(step, allow_auto: bool = False) -> Step:
    """From any object with mode ('fixed'|'heuristic'|'learned'), field,
    component, h, xi, alpha_stop and, for learned steps, mult: a CUDA float32
    tensor of one multiplier per element (kept alive by the caller).  With
    allow_auto, a learned step may leave mult None (the frame server then
    computes the multipliers with its step model)."""
    s = Step()
    s.mode = {"fixed": STEP_FIXED, "heuristic": STEP_HEURISTIC, "learned": STEP_LEARNED}[step.mode]
    if step.mode == "learned" and not (allow_auto and step.mult is None):
        m = step.mult
        if m is None or not getattr(m, "is_cuda", False) or not m.is_contiguous():
            raise ValueError("learned steps need a contiguous CUDA tensor of multipliers")
        s.mult = m.data_ptr()
    s.field = {"scalar": FIELD_SCALAR, "magnitude": FIELD_MAGNITUDE, "component": FIELD_COMPONENT}[step.field]
    s.component = int(step.component)
    s.h, s.xi, s.alpha_stop = float(step.h), float(step.xi), float(step.alpha_stop)
    s.shading = {"none": SHADE_NONE, "gradient": SHADE_GRADIENT}[getattr(step, "shading", "none")]
    for a, x in enumerate(getattr(step, "light", (0.0, 0.0, 0.0))):
        s.light[a] = float(x)
    trim = getattr(step, "trim", None)
    if trim is not None:
        if not getattr(trim, "is_cuda", False) or not trim.is_contiguous():
            raise ValueError("trim must be a contiguous CUDA tensor (height x width x 2 float32)")
        s.trim = trim.data_ptr()
    return s


class Volume:
    """One LR-spline volume resident on the current CUDA device (lrvol_t)."""

    def __init__(self, vol):
        L = load()
        deg = np.ascontiguousarray([int(v) for v in vol.deg], dtype=np.int32)
        self._arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in
                        (vol.elem_box, vol.knots, vol.coef, vol.weight)]
        box, knots, coef, weight = self._arrays
        self.ncomp = int(coef.shape[1])
        self.n_elem = int(box.shape[0])
        self.deg = [int(v) for v in deg]
        h = ctypes.c_void_p()
        _check(L.lrvol_create(deg.ctypes.data, self.ncomp, self.n_elem, box.ctypes.data, int(knots.shape[0]),
                              knots.ctypes.data, coef.ctypes.data, weight.ctypes.data, ctypes.byref(h)),
               "lrvol_create")
        self._h = h
        self._arrays = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lrvol_destroy(self._h)
            self._h = None

    __del__ = close

    @property
    def handle(self):
        return self._h

    def build_accel(self, blocks=(64, 64, 64), stream=None, split: int = None):
        """The k-d forest; split=SPLIT_MIDPOINT builds octree-style trees instead."""
        b = np.ascontiguousarray(blocks, dtype=np.int32)
        if split is None:
            _check(load().lrvol_build_accel(self._h, b.ctypes.data, _stream_ptr(stream)), "lrvol_build_accel")
        else:
            _check(load().lrvol_build_accel_split(self._h, b.ctypes.data, int(split), _stream_ptr(stream)),
                   "lrvol_build_accel_split")
        return self

    def to_bezier(self, storage: int = STORE_F32, stream=None):
        _check(load().lrvol_to_bezier(self._h, int(storage), _stream_ptr(stream)), "lrvol_to_bezier")
        return self

    def render(self, cam, tf, step, out=None, stream=None, row_begin: int = 0, row_end: int = 0,
               band_count: int = 0, band_index: int = 0):
        """Render into a (H, W, 4) float32 CUDA tensor (allocated if out is None)."""
        import torch
        c = cam if isinstance(cam, Camera) else make_camera(cam, row_begin, row_end, band_count, band_index)
        t = tf if isinstance(tf, TF) else make_tf(tf)
        s = step if isinstance(step, Step) else make_step(step)
        if out is None:
            out = torch.zeros((c.height, c.width, 4), dtype=torch.float32, device="cuda")
        ptr = _dev(out, torch.float32, c.height * c.width * 4, "render out", exact=True)
        _check(load().lrvol_render(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), ptr,
                                   _stream_ptr(stream)), "lrvol_render")
        return out

    def render_trace(self, cam, tf, step, pixels, max_samples: int, stream=None):
        """The render kernel's own samples for a pixel list (lrvol_render_trace).
        pixels: (n, 2) int32 CUDA tensor of (i, j).  Returns (trace (n, max, 4)
        float32: t, element id bits, value, segment; count (n,) int32;
        rgba (n, 4) float32), all CUDA tensors."""
        import torch
        c = cam if isinstance(cam, Camera) else make_camera(cam)
        t = tf if isinstance(tf, TF) else make_tf(tf)
        s = step if isinstance(step, Step) else make_step(step)
        if pixels.dim() != 2 or pixels.shape[1] != 2:
            raise ValueError("pixels: expected n x 2 int32")
        n = pixels.shape[0]
        pp = _dev(pixels, torch.int32, 2 * n, "pixels", exact=True)
        trace = torch.empty((n, max_samples, 4), dtype=torch.float32, device="cuda")
        count = torch.empty(n, dtype=torch.int32, device="cuda")
        rgba = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        _check(load().lrvol_render_trace(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), pp, n,
                                         int(max_samples), trace.data_ptr(), count.data_ptr(), rgba.data_ptr(),
                                         _stream_ptr(stream)), "lrvol_render_trace")
        return trace, count, rgba

    def lookup(self, pts, out=None, stream=None):
        import torch
        n = _points(pts)
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=pts.device)
        if out.element_size() != 4:
            raise TypeError("lookup out: expected a 32-bit integer tensor")
        _check(load().lrvol_lookup(self._h, pts.data_ptr(), n, _dev(out, None, n, "lookup out"), _stream_ptr(stream)),
               "lrvol_lookup")
        return out

    def eval(self, pts, out=None, stream=None):
        import torch
        n = _points(pts)
        if out is None:
            out = torch.empty((n, self.ncomp), dtype=torch.float32, device=pts.device)
        _check(load().lrvol_eval(self._h, pts.data_ptr(), n, _dev(out, torch.float32, n * self.ncomp, "eval out"),
                                 _stream_ptr(stream)), "lrvol_eval")
        return out

    def eval_grad(self, pts, out=None, stream=None):
        """(n, 4) float32 CUDA tensor: value and gradient of a scalar volume."""
        import torch
        n = _points(pts)
        if out is None:
            out = torch.empty((n, 4), dtype=torch.float32, device=pts.device)
        _check(load().lrvol_eval_grad(self._h, pts.data_ptr(), n, _dev(out, torch.float32, 4 * n, "eval_grad out"),
                                      _stream_ptr(stream)), "lrvol_eval_grad")
        return out

    def get_bezier(self) -> np.ndarray:
        p = self.deg
        out = np.empty((self.n_elem, self.ncomp, p[2] + 1, p[1] + 1, p[0] + 1), dtype=np.float64)
        _check(load().lrvol_get_bezier(self._h, out.ctypes.data), "lrvol_get_bezier")
        return out

    def stats(self) -> dict:
        s = Stats()
        _check(load().lrvol_stats(self._h, ctypes.byref(s)), "lrvol_stats")
        return s.as_dict()


# ---- learned step sizes ----------------------------------------------------

def _dev(t, dtype=None, numel=None, what="tensor", exact=False):
    """Device pointer of a contiguous CUDA tensor after checking it: a wrong
    device, layout, dtype or size raises here, so no kernel is ever handed a
    buffer smaller than what it reads or writes."""
    if not getattr(t, "is_cuda", False) or not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{what}: expected {dtype}, got {t.dtype}")
    if numel is not None and (t.numel() != numel if exact else t.numel() < numel):
        raise ValueError(f"{what}: {t.numel()} elements, {'expected' if exact else 'need at least'} {int(numel)}")
    return t.data_ptr()


def _points(pts):
    import torch
    _dev(pts, torch.float32, what="points")
    if pts.numel() % 3 != 0 or (pts.dim() > 0 and pts.shape[-1] != 3):
        raise ValueError("points: expected n x 3 float32")
    return pts.numel() // 3


def features(vol: "Volume", cam, tf, step, out=None, stream=None):
    """Per-element features (n_elem x 16 float32 CUDA tensor) for a camera/TF."""
    import torch
    if out is None:
        out = torch.empty((vol.n_elem, MLP_IN), dtype=torch.float32, device="cuda")
    c = cam if isinstance(cam, Camera) else make_camera(cam)
    t = tf if isinstance(tf, TF) else make_tf(tf)
    s = step if isinstance(step, Step) else make_step(step)
    _check(load().lrvol_features(vol.handle, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s),
                                 _dev(out, torch.float32, vol.n_elem * MLP_IN, "features out"), _stream_ptr(stream)),
           "lrvol_features")
    return out


def mlp_pack(params, out=None, stream=None):
    """FP32 master parameters -> BF16 fragment order (int16 CUDA tensor of MLP_PACKED)."""
    import torch
    if out is None:
        out = torch.empty(MLP_PACKED, dtype=torch.int16, device="cuda")
    _check(load().lrvol_mlp_pack(_dev(params, torch.float32, MLP_PARAMS, "params"),
                                 _dev(out, torch.int16, MLP_PACKED, "packed out"), _stream_ptr(stream)), "lrvol_mlp_pack")
    return out


def mlp_infer(x, packed, ymax: float, out=None, stream=None, ymin: float = 0.0):
    """Multipliers 2^clamp(y, ymin, ymax) for feature rows x (n x 16); hidden layers on the tcgen05 tensor cores."""
    import torch
    n = x.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(load().lrvol_mlp_infer(_dev(x, torch.float32, n * MLP_IN, "features"), n,
                                  _dev(packed, torch.int16, MLP_PACKED, "packed"), float(ymin), float(ymax),
                                  _dev(out, torch.float32, n, "multipliers out"), _stream_ptr(stream)), "lrvol_mlp_infer")
    return out


def mlp_infer_timeout_test(x, packed, ymax: float, out=None, stream=None, ymin: float = 0.0):
    """Diagnostic: the network kernel with no MMAs issued, so its bounded waits run out."""
    import torch
    n = x.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(load().lrvol_mlp_infer_timeout_test(_dev(x, torch.float32, n * MLP_IN, "features"), n,
                                               _dev(packed, torch.int16, MLP_PACKED, "packed"), float(ymin),
                                               float(ymax),
                                               _dev(out, torch.float32, n, "multipliers out"), _stream_ptr(stream)),
           "lrvol_mlp_infer_timeout_test")
    return out


def mlp_check() -> None:
    """Synchronise and raise if a tensor-core wait of mlp_infer ran out since the last check."""
    _check(load().lrvol_mlp_check(), "lrvol_mlp_check")


def mlp_scratch(n: int):
    import torch
    return torch.empty(int(load().lrvol_mlp_scratch_floats(n)), dtype=torch.float32, device="cuda")


def mlp_grad(x, target, params, scratch=None, stream=None):
    """Loss and gradient of the FP32 network on a batch (CUDA tensors)."""
    import torch
    n = x.shape[0]
    scratch = mlp_scratch(n) if scratch is None else scratch
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    _check(load().lrvol_mlp_grad(_dev(x, torch.float32, n * MLP_IN, "x"), _dev(target, torch.float32, n, "target"), n,
                                 _dev(params, torch.float32, MLP_PARAMS, "params"), _dev(grad), _dev(loss),
                                 _dev(scratch, torch.float32, load().lrvol_mlp_scratch_floats(n), "scratch"),
                                 _stream_ptr(stream)), "lrvol_mlp_grad")
    return loss, grad


def mlp_train_step(x, target, params, m, v, t: int, lr: float, scratch, loss=None, stream=None):
    """One Adam step of the FP32 network on a batch (all CUDA tensors, in place)."""
    import torch
    n = x.shape[0]
    _check(load().lrvol_mlp_train_step(_dev(x, torch.float32, n * MLP_IN, "x"), _dev(target, torch.float32, n, "target"),
                                       n, _dev(params, torch.float32, MLP_PARAMS, "params"),
                                       _dev(m, torch.float32, MLP_PARAMS, "m"), _dev(v, torch.float32, MLP_PARAMS, "v"),
                                       int(t), float(lr), None if loss is None else _dev(loss, torch.float32, 1, "loss"),
                                       _dev(scratch, torch.float32, load().lrvol_mlp_scratch_floats(n), "scratch"),
                                       _stream_ptr(stream)), "lrvol_mlp_train_step")


def labels(vol: "Volume", cam, tf, step, h_fine: float, tau: float, cand, label=None, stream=None):
    """Per-element training labels (int32 CUDA tensor; n_cand marks unvisited)."""
    import torch
    cand_t = torch.as_tensor(cand, dtype=torch.float32, device="cuda").contiguous()
    if label is None:
        label = torch.full((vol.n_elem,), len(cand_t), dtype=torch.int32, device="cuda")
    c = cam if isinstance(cam, Camera) else make_camera(cam)
    t = tf if isinstance(tf, TF) else make_tf(tf)
    s = step if isinstance(step, Step) else make_step(step)
    _check(load().lrvol_labels(vol.handle, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), float(h_fine),
                               float(tau), _dev(cand_t), len(cand_t), _dev(label, torch.int32, vol.n_elem, "label"),
                               _stream_ptr(stream)),
           "lrvol_labels")
    return label


# ---- host arena and frame server ------------------------------------------

class Arena:
    """Host-side first-fit bookkeeping of offsets (lrvol_arena_*)."""

    def __init__(self, nbytes: int, align: int = 256):
        h = ctypes.c_void_p()
        _check(load().lrvol_arena_create(int(nbytes), int(align), ctypes.byref(h)), "lrvol_arena_create")
        self._h = h

    def alloc(self, nbytes: int) -> int:
        return int(load().lrvol_arena_alloc(self._h, int(nbytes)))

    def free(self, offset: int) -> None:
        _check(load().lrvol_arena_free(self._h, int(offset)), "lrvol_arena_free")

    @property
    def used(self) -> int:
        return int(load().lrvol_arena_used(self._h))

    @property
    def largest_free(self) -> int:
        return int(load().lrvol_arena_largest_free(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lrvol_arena_destroy(self._h)
            self._h = None

    __del__ = close


class _DeviceArray:
    """A borrowed device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


class Server:
    """Frame server (lrvol_server_*): FIFO admission by free slot and arena
    memory, frames of several requests in flight on separate streams."""

    def __init__(self, slots: int = 8, arena_bytes: int = 1 << 30):
        h = ctypes.c_void_p()
        _check(load().lrvol_server_create(int(slots), int(arena_bytes), ctypes.byref(h)), "lrvol_server_create")
        self._h = h
        self._keep = {}   # ticket -> (camera, host buffer) kept alive while the request exists

    def set_step_model(self, packed, ymax: float, ymin: float = 0.0) -> None:
        self._model = packed
        import torch
        _check(load().lrvol_server_set_step_model(self._h, _dev(packed, torch.int16, MLP_PACKED, "packed"),
                                                  float(ymin), float(ymax)), "lrvol_server_set_step_model")

    def set_priority_pixels(self, max_pixels: int) -> None:
        _check(load().lrvol_server_set_priority_pixels(self._h, int(max_pixels)), "lrvol_server_set_priority_pixels")

    def set_large_cap(self, max_in_flight: int) -> None:
        _check(load().lrvol_server_set_large_cap(self._h, int(max_in_flight)), "lrvol_server_set_large_cap")

    def submit(self, vol: "Volume", cam, tf, step, host_out=None) -> int:
        c = cam if isinstance(cam, Camera) else make_camera(cam)
        t = tf if isinstance(tf, TF) else make_tf(tf)
        s = step if isinstance(step, Step) else make_step(step, allow_auto=True)
        ticket = ctypes.c_int64()
        hp = None
        if host_out is not None:
            import torch
            if host_out.is_cuda or not host_out.is_contiguous() or host_out.dtype != torch.float32 or \
                    host_out.numel() != c.width * c.height * 4:
                raise ValueError("host_out: expected a contiguous float32 host tensor of height x width x 4")
            hp = host_out.data_ptr()
        _check(load().lrvol_server_submit(self._h, vol.handle, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), hp,
                                          ctypes.byref(ticket)), "lrvol_server_submit")
        self._keep[ticket.value] = (c.width, c.height, host_out, step)
        return ticket.value

    def progress(self) -> int:
        n = ctypes.c_int32()
        _check(load().lrvol_server_progress(self._h, ctypes.byref(n)), "lrvol_server_progress")
        return n.value

    def drain(self) -> None:
        _check(load().lrvol_server_drain(self._h), "lrvol_server_drain")

    def poll(self, max_n: int = 256) -> list:
        """Tickets retired (done or failed) since the previous poll, in order."""
        buf = (ctypes.c_int64 * max_n)()
        n = ctypes.c_int32()
        out = []
        while True:
            _check(load().lrvol_server_poll(self._h, buf, max_n, ctypes.byref(n)), "lrvol_server_poll")
            out.extend(buf[:n.value])
            if n.value < max_n:
                return out

    def info(self, ticket: int) -> dict:
        fi = FrameInfo()
        _check(load().lrvol_server_info(self._h, int(ticket), ctypes.byref(fi)), "lrvol_server_info")
        return fi.as_dict()

    def image(self, ticket: int):
        """A copy (CUDA tensor, H x W x 4) of a finished frame still in the arena."""
        import torch
        d = self.info(ticket)
        if d["state"] != REQ_DONE or not d["rgba_dev"]:
            raise LrvolError(ERR_STATE, "image: frame not done or not in the arena")
        w, h = self._keep[ticket][:2]
        return torch.as_tensor(_DeviceArray(d["rgba_dev"], (h, w, 4)), device="cuda").clone()

    def release(self, ticket: int) -> None:
        _check(load().lrvol_server_release(self._h, int(ticket)), "lrvol_server_release")
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().lrvol_server_get_stats(self._h, ctypes.byref(st)), "lrvol_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lrvol_server_destroy(self._h)
            self._h = None

    __del__ = close


def clock() -> float:
    """The server's host clock (seconds, monotonic)."""
    return float(load().lrvol_server_clock())


# ---- streamlines (Sec. 5) ----------------------------------------------------

def streamlines(vol: "Volume", seeds, method: str, rule: str, h: float, t_end: float, tol: float = 0.0,
                max_samples: int = 1024, out=None, stream=None):
    """Streamlines from seeds (CUDA float64 tensor, n x 3): (samples n x max x 4
    float64 (x, y, z, t), count n int32, status n int32), CUDA tensors."""
    import torch
    n = seeds.shape[0]
    P = SLParams(SL_METHODS.index(method), SL_RULES.index(rule), float(h), float(t_end), float(tol),
                 int(max_samples))
    if out is None:
        out = (torch.empty((n, max_samples, 4), dtype=torch.float64, device="cuda"),
               torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"))
    samples, count, status = out
    if samples.dim() == 3 and samples.shape[1] != max_samples:
        raise ValueError(f"samples: {samples.shape[1]} samples per line, max_samples is {max_samples}")
    _check(load().lrvol_streamlines(vol.handle, ctypes.byref(P), _dev(seeds, torch.float64, 3 * n, "seeds"), n,
                                    _dev(samples, torch.float64, n * max_samples * 4, "samples"),
                                    _dev(count, torch.int32, n, "count"), _dev(status, torch.int32, n, "status"),
                                    _stream_ptr(stream)), "lrvol_streamlines")
    return samples, count, status


def streamline_error(ref, ref_count, app, app_count, stream=None):
    """Eq. 7 per streamline (CUDA float64 tensor of n sums); E is their max."""
    import torch
    n = ref.shape[0]
    sums = torch.empty(n, dtype=torch.float64, device="cuda")
    if ref.dim() != 3 or app.dim() != 3 or app.shape[0] != n:
        raise ValueError("ref and app: expected n x max x 4 float64 tensors with the same n")
    _check(load().lrvol_streamline_error(_dev(ref, torch.float64, n * ref.shape[1] * 4, "ref"),
                                         _dev(ref_count, torch.int32, n, "ref_count"), ref.shape[1],
                                         _dev(app, torch.float64, n * app.shape[1] * 4, "app"),
                                         _dev(app_count, torch.int32, n, "app_count"), app.shape[1], n, _dev(sums),
                                         _stream_ptr(stream)), "lrvol_streamline_error")
    return sums


# ---- trimming (Sec. 4.1) -----------------------------------------------------

def trim(cam, tris, out=None, stream=None):
    """Per-pixel (t_front, t_back) of a closed mesh (tris: CUDA float32 tensor
    of n x 3 x 3 or n x 9 vertices, counter-clockwise seen from outside):
    (H, W, 2) float32 CUDA tensor for lrvol_step.trim."""
    import torch
    c = cam if isinstance(cam, Camera) else make_camera(cam)
    t = tris.reshape(-1, 9)
    if out is None:
        out = torch.empty((c.height, c.width, 2), dtype=torch.float32, device="cuda")
    _check(load().lrvol_trim(ctypes.byref(c), _dev(t, torch.float32, what="triangles"), t.shape[0],
                             _dev(out, torch.float32, c.height * c.width * 2, "trim out"), _stream_ptr(stream)),
           "lrvol_trim")
    return out


def tubes(vol: "Volume", cam, samples, count, radius: float, cmap, vis=None, out=None, stream=None):
    """Streamline tubes (Sec. 5.3): (H, W, 4) float32 CUDA tensor of the
    capsules around the polylines (samples n x max x 4 float64, count n int32,
    CUDA tensors), coloured by cmap at the field's speed."""
    import torch
    c = cam if isinstance(cam, Camera) else make_camera(cam)
    t = cmap if isinstance(cmap, TF) else make_tf(cmap)
    if vis is None:
        vis = torch.empty((c.height, c.width), dtype=torch.int64, device="cuda")
    if out is None:
        out = torch.empty((c.height, c.width, 4), dtype=torch.float32, device="cuda")
    if samples.dim() != 3:
        raise ValueError("samples: expected n x max x 4 float64")
    n, ms = samples.shape[0], samples.shape[1]
    _check(load().lrvol_tubes(vol.handle, ctypes.byref(c), _dev(samples, torch.float64, n * ms * 4, "samples"),
                              _dev(count, torch.int32, n, "count"), n, ms, float(radius), ctypes.byref(t),
                              _dev(vis, torch.int64, c.height * c.width, "vis"),
                              _dev(out, torch.float32, c.height * c.width * 4, "tubes out"), _stream_ptr(stream)),
           "lrvol_tubes")
    return out

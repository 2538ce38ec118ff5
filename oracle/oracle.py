"""Python face of the FP64 CPU oracle (oracle.c) plus the Bezier-block oracle.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only users.  Nothing here imports or
calls the CUDA library, and the CUDA library never calls this.

Inputs are duck-typed: a volume needs ``deg, elem_box, knots, coef, weight``;
a camera ``projection, width, height, eye, target, up, fovy, extent``; a
transfer function ``table (256x4), vmin, vmax``; step parameters ``mode,
field, component, h, xi, alpha_stop`` (the dataclasses of the seeded input
generator fit).

Bezier blocks (Sec. 3.2.3): on each element the LR-spline is one polynomial
of tri-degree p, and the paper gets its Bernstein coefficients by
interpolation.  ``bezier_blocks`` does exactly that: it evaluates Eq. 2 at the
(p+1)^3 tensor points
u_m = (m + 1/2)/(p+1) inside the element and solves the tensor Bernstein
interpolation problem one axis at a time (numpy's dense solver is the
library step).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NONE = 0xFFFFFFFF
CFLAGS = ["-O2", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-fno-fast-math", "-std=c11"]


def build(force: bool = False, src: str = _SRC, lib: str = _LIB) -> str:
    """Compile liboracle.so in place with gcc (no FMA contraction: the FP32
    ray arithmetic must follow the stated operation order)."""
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, src, "-lm"])
        os.replace(tmp, lib)
    return lib


def use_library(path: str | None):
    """Point this module at another build of oracle.c (None: the default one).
    Used by the planted-mistake tests; returns the previous library."""
    global _lib, _LIB_OVERRIDE
    prev = _LIB_OVERRIDE
    _LIB_OVERRIDE = path
    _lib = None
    return prev


_LIB_OVERRIDE = None


class _Cam(ctypes.Structure):
    _fields_ = [("projection", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fovy", ctypes.c_double), ("extent", ctypes.c_double)]


class _TF(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("vmin", ctypes.c_double), ("vmax", ctypes.c_double)]


class _Step(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("field", ctypes.c_int32), ("component", ctypes.c_int32),
                ("h", ctypes.c_double), ("xi", ctypes.c_double), ("alpha_stop", ctypes.c_double),
                ("mult", ctypes.c_void_p), ("shading", ctypes.c_int32), ("light", ctypes.c_double * 3),
                ("trim", ctypes.c_void_p)]


class _SLParams(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("step_rule", ctypes.c_int32), ("h", ctypes.c_double),
                ("t_end", ctypes.c_double), ("tol", ctypes.c_double), ("max_samples", ctypes.c_int32)]


SL_METHODS = ["RK1", "RK2", "RK3", "RK4", "RK38", "RKF5", "HE", "BS", "RKF45"]
SL_RULES = ["fixed", "heuristic", "adaptive"]


class _Stats(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_int64), ("lookups", ctypes.c_int64), ("rays_hit", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE is None:
            build()
        L = ctypes.CDLL(_LIB_OVERRIDE or _LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.orc_create.restype = vp
        L.orc_create.argtypes = [vp, i32, i64, vp, i64, vp, vp, vp]
        L.orc_destroy.argtypes = [vp]
        L.orc_bspline.restype = ctypes.c_double
        L.orc_bspline.argtypes = [vp, i32, ctypes.c_double]
        L.orc_find_element.restype = ctypes.c_uint32
        L.orc_find_element.argtypes = [vp, vp]
        L.orc_incidence.restype = i64
        L.orc_incidence.argtypes = [vp, i64, vp]
        L.orc_eval.restype = ctypes.c_uint32
        L.orc_eval.argtypes = [vp, vp, vp]
        L.orc_lookup_batch.argtypes = [vp, vp, i64, vp, i32]
        L.orc_eval_batch_f32.argtypes = [vp, vp, i64, vp, vp, i32]
        L.orc_eval_batch_f64.argtypes = [vp, vp, i64, vp, vp, i32]
        L.orc_eval_grad_batch_f32.argtypes = [vp, vp, i64, vp, vp, i32]
        L.orc_eval_grad_batch_f64.argtypes = [vp, vp, i64, vp, vp, i32]
        L.orc_bspline_d1.restype = ctypes.c_double
        L.orc_bspline_d1.argtypes = [vp, i32, ctypes.c_double]
        L.orc_heuristic_step.restype = ctypes.c_float
        L.orc_heuristic_step.argtypes = [vp, ctypes.c_uint32]
        L.orc_render.argtypes = [vp, ctypes.POINTER(_Cam), ctypes.POINTER(_TF), ctypes.POINTER(_Step),
                                 vp, i64, vp, i32, ctypes.POINTER(_Stats)]
        L.orc_render_trace.argtypes = [vp, ctypes.POINTER(_Cam), ctypes.POINTER(_TF), ctypes.POINTER(_Step),
                                       vp, i64, i32, vp, vp, vp, i32, ctypes.POINTER(_Stats)]
        L.orc_labels.argtypes = [vp, ctypes.POINTER(_Cam), ctypes.POINTER(_TF), ctypes.POINTER(_Step),
                                 ctypes.c_double, ctypes.c_double, vp, i32, vp, i32]
        L.orc_streamlines.argtypes = [vp, ctypes.POINTER(_SLParams), vp, i64, vp, vp, vp, i32]
        L.orc_trim.argtypes = [ctypes.POINTER(_Cam), vp, i64, vp, i32]
        L.orc_tubes.argtypes = [vp, ctypes.POINTER(_Cam), vp, i64, ctypes.c_float, ctypes.POINTER(_TF), vp, i32]
        L.orc_ray.restype = i32
        L.orc_ray.argtypes = [ctypes.POINTER(_Cam), i32, i32, vp, vp, vp, vp]
        _lib = L
    return _lib


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def bspline(knots, p: int, x: float) -> float:
    """One univariate B-spline of degree p on local knots (p+2 values) at x."""
    k = np.ascontiguousarray(knots, dtype=np.float64)
    assert k.shape == (p + 2,)
    return float(_load().orc_bspline(k.ctypes.data, int(p), float(x)))


def bspline_d1(knots, p: int, x: float) -> float:
    """Its derivative (right-hand at knots)."""
    k = np.ascontiguousarray(knots, dtype=np.float64)
    assert k.shape == (p + 2,)
    return float(_load().orc_bspline_d1(k.ctypes.data, int(p), float(x)))


def _cam(c) -> _Cam:
    s = _Cam()
    s.projection = 1 if c.projection == "persp" else 0
    s.width, s.height = int(c.width), int(c.height)
    s.eye = (ctypes.c_double * 3)(*[float(v) for v in c.eye])
    s.target = (ctypes.c_double * 3)(*[float(v) for v in c.target])
    s.up = (ctypes.c_double * 3)(*[float(v) for v in c.up])
    s.fovy = float(c.fovy)
    s.extent = float(c.extent)
    return s


def ray(cam, i: int, j: int):
    """FP32 ray (origin, direction, t_in, t_out) of pixel (i, j); None on a miss."""
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    ti = np.zeros(1, np.float32)
    to = np.zeros(1, np.float32)
    c = _cam(cam)
    hit = _load().orc_ray(ctypes.byref(c), int(i), int(j), o.ctypes.data, d.ctypes.data,
                          ti.ctypes.data, to.ctypes.data)
    return (o, d, float(ti[0]), float(to[0])) if hit else None


def bernstein(p: int, u) -> np.ndarray:
    """Bernstein basis B^p_j(u), j = 0..p, as an array (..., p+1)."""
    u = np.asarray(u, dtype=np.float64)[..., None]
    j = np.arange(p + 1)
    binom = np.array([comb(p, int(t)) for t in j], dtype=np.float64)
    return binom * u ** j * (1.0 - u) ** (p - j)


class Oracle:
    """FP64 reference over one LR-spline volume (Eq. 2)."""

    def __init__(self, vol, threads: int | None = None):
        L = _load()
        self.deg = np.array([int(v) for v in vol.deg], dtype=np.int32)
        self.box = np.ascontiguousarray(vol.elem_box, dtype=np.float64)
        self.knots = np.ascontiguousarray(vol.knots, dtype=np.float64)
        self.coef = np.ascontiguousarray(vol.coef, dtype=np.float64)
        self.weight = np.ascontiguousarray(vol.weight, dtype=np.float64)
        self.nc = int(self.coef.shape[1])
        self.n_elem = int(self.box.shape[0])
        self.n_basis = int(self.knots.shape[0])
        self.threads = _threads(threads)
        self._h = L.orc_create(self.deg.ctypes.data, self.nc, self.n_elem, self.box.ctypes.data,
                               self.n_basis, self.knots.ctypes.data, self.coef.ctypes.data,
                               self.weight.ctypes.data)
        if not self._h:
            raise ValueError("oracle: bad volume")

    def __del__(self):
        if getattr(self, "_h", None):
            _load().orc_destroy(self._h)
            self._h = None

    # --- look-up and evaluation -------------------------------------------------
    def find_element(self, x) -> int:
        xd = np.ascontiguousarray(x, dtype=np.float64)
        return int(_load().orc_find_element(self._h, xd.ctypes.data))

    def incidence(self, e: int) -> np.ndarray:
        out = np.empty(self.n_basis, dtype=np.int64)
        n = _load().orc_incidence(self._h, int(e), out.ctypes.data)
        return out[:n].copy()

    def coefficient_hull(self, elements, threads: int | None = None):
        """Per element and component, (min, max) of the coefficients c_i of the
        B-splines whose support contains the element.  The element's Bernstein
        coefficients are convex combinations of these (gamma_i N_i sum to one
        and each restricted N_i has non-negative Bernstein coefficients), so
        the hull bounds the block's range without computing the block.
        Returns (n, nc, 2)."""
        from concurrent.futures import ThreadPoolExecutor
        el = np.asarray(elements, dtype=np.int64).reshape(-1)
        out = np.empty((len(el), self.nc, 2), dtype=np.float64)
        L = _load()

        def work(rows):
            buf = np.empty(self.n_basis, dtype=np.int64)
            for r in rows:
                n = L.orc_incidence(self._h, int(el[r]), buf.ctypes.data)
                c = self.coef[buf[:n]]
                out[r, :, 0] = c.min(axis=0)
                out[r, :, 1] = c.max(axis=0)

        nth = max(1, min(_threads(threads or self.threads), len(el)))
        with ThreadPoolExecutor(nth) as ex:
            list(ex.map(work, [range(t, len(el), nth) for t in range(nth)]))
        return out

    def lookup(self, pts_f32) -> np.ndarray:
        p = np.ascontiguousarray(pts_f32, dtype=np.float32).reshape(-1, 3)
        out = np.empty(len(p), dtype=np.uint32)
        _load().orc_lookup_batch(self._h, p.ctypes.data, len(p), out.ctypes.data, self.threads)
        return out

    def eval(self, pts, return_elem: bool = False):
        """f at points (FP32 input is used exactly as given, FP64 input likewise)."""
        pts = np.asarray(pts)
        val = np.empty((pts.reshape(-1, 3).shape[0], self.nc), dtype=np.float64)
        elem = np.empty(len(val), dtype=np.uint32)
        L = _load()
        if pts.dtype == np.float32:
            p = np.ascontiguousarray(pts).reshape(-1, 3)
            L.orc_eval_batch_f32(self._h, p.ctypes.data, len(p), val.ctypes.data, elem.ctypes.data, self.threads)
        else:
            p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
            L.orc_eval_batch_f64(self._h, p.ctypes.data, len(p), val.ctypes.data, elem.ctypes.data, self.threads)
        return (val, elem) if return_elem else val

    def eval_grad(self, pts):
        """f and its gradient at points: (val (n, nc), grad (n, nc, 3)), FP64,
        from Eq. 2 with each univariate factor differentiated (orc_bspline_d1)."""
        pts = np.asarray(pts)
        n = pts.reshape(-1, 3).shape[0]
        val = np.empty((n, self.nc), dtype=np.float64)
        grad = np.empty((n, self.nc, 3), dtype=np.float64)
        L = _load()
        if pts.dtype == np.float32:
            p = np.ascontiguousarray(pts).reshape(-1, 3)
            L.orc_eval_grad_batch_f32(self._h, p.ctypes.data, n, val.ctypes.data, grad.ctypes.data, self.threads)
        else:
            p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
            L.orc_eval_grad_batch_f64(self._h, p.ctypes.data, n, val.ctypes.data, grad.ctypes.data, self.threads)
        return val, grad

    def streamlines(self, seeds, method: str, rule: str, h: float, t_end: float, tol: float = 1e-6,
                    max_samples: int = 4096, threads: int | None = None):
        """Streamlines (Sec. 5) in FP64: (samples (n, max, 4) of x, y, z, t;
        count (n,); status (n,): 0 reached t_end, 1 left the domain,
        2 max_samples, 3 step control failed)."""
        seeds = np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 3)
        n = len(seeds)
        P = _SLParams(SL_METHODS.index(method), SL_RULES.index(rule), float(h), float(t_end), float(tol),
                      int(max_samples))
        out = np.zeros((n, max_samples, 4), dtype=np.float64)
        count = np.zeros(n, dtype=np.int32)
        status = np.zeros(n, dtype=np.int32)
        _load().orc_streamlines(self._h, ctypes.byref(P), seeds.ctypes.data, n, out.ctypes.data, count.ctypes.data,
                                status.ctypes.data, _threads(threads or self.threads))
        return out, count, status

    def tubes(self, cam, samples, count, radius: float, cmap, threads: int | None = None):
        """Streamline tubes (Sec. 5.3): RGBA (H, W, 4) FP64 of the capsules of
        radius r around every segment of the polylines (samples (n, max, 4),
        count (n,)), coloured by the colour map at the field's speed on the
        segment axis and shaded by max(0.4, |n . d|)."""
        seg = tube_segments(samples, count)
        table = np.ascontiguousarray(cmap.table, dtype=np.float64).reshape(256, 4)
        t = _TF()
        t.table = table.ctypes.data
        t.vmin, t.vmax = float(cmap.vmin), float(cmap.vmax)
        out = np.zeros((cam.height, cam.width, 4), dtype=np.float64)
        _load().orc_tubes(self._h, ctypes.byref(_cam(cam)), seg.ctypes.data, len(seg), float(radius), ctypes.byref(t),
                          out.ctypes.data, _threads(threads or self.threads))
        return out

    def heuristic_step(self, e: int) -> float:
        return float(_load().orc_heuristic_step(self._h, int(e)))

    # --- Bezier blocks by interpolation (Sec. 3.2.3) ----------------------------
    def bezier_blocks(self, elements=None) -> np.ndarray:
        """FP64 Bernstein coefficients, (n, nc, p2+1, p1+1, p0+1) (x fastest)."""
        p = [int(v) for v in self.deg]
        el = np.arange(self.n_elem) if elements is None else np.asarray(elements, dtype=np.int64)
        u = [(np.arange(p[a] + 1) + 0.5) / (p[a] + 1) for a in range(3)]
        uz, uy, ux = np.meshgrid(u[2], u[1], u[0], indexing="ij")
        U = np.stack([ux.ravel(), uy.ravel(), uz.ravel()], axis=1)            # (q, 3) x fastest
        lo = self.box[el, :3]
        hi = self.box[el, 3:]
        X = lo[:, None, :] + U[None, :, :] * (hi - lo)[:, None, :]             # (n, q, 3)
        F = self.eval(X.reshape(-1, 3)).reshape(len(el), -1, self.nc)          # (n, q, nc)
        F = F.transpose(0, 2, 1).reshape(len(el), self.nc, p[2] + 1, p[1] + 1, p[0] + 1)
        inv = [np.linalg.inv(bernstein(p[a], u[a])) for a in range(3)]         # V[m, j] = B_j(u_m)
        C = np.einsum("ai,nczyi->nczya", inv[0], F)                           # C = V^-1 F per axis
        C = np.einsum("bj,nczja->nczba", inv[1], C)
        C = np.einsum("ck,nqkba->nqcba", inv[2], C)
        return C

    def bezier_eval(self, blocks: np.ndarray, elements, x) -> np.ndarray:
        """Evaluate Bezier blocks (n, nc, ...) of the given elements at points x (n, 3)."""
        p = [int(v) for v in self.deg]
        el = np.asarray(elements, dtype=np.int64)
        lo = self.box[el, :3]
        hi = self.box[el, 3:]
        u = (np.asarray(x, dtype=np.float64) - lo) / (hi - lo)
        bx, by, bz = (bernstein(p[a], u[:, a]) for a in range(3))
        return np.einsum("nczyx,nx,ny,nz->nc", blocks, bx, by, bz)

    # --- rendering (Sec. 4, Alg. 2, Eq. 4) ---------------------------------------
    def render(self, cam, tf, step, pixels=None, threads: int | None = None):
        """RGBA (premultiplied) per pixel: (H, W, 4), or (n, 4) for a pixel list
        of (i, j) pairs.  Returns (rgba, stats dict)."""
        return self._render(cam, tf, step, pixels, threads, 0)

    def render_trace(self, cam, tf, step, pixels, max_samples: int, threads: int | None = None):
        """The march of each listed pixel, sample by sample: (trace (n, max, 4)
        FP64 of (t_k, element id, value before the transfer function, segment
        min(t_{k+1}, t_out) - t_k); count (n,) samples composited; rgba (n, 4);
        stats dict).  t_k and the element ids are the FP32 decisions of R11 and
        Alg. 1 (exact), the values FP64 Eq. 2."""
        return self._render(cam, tf, step, pixels, threads, int(max_samples))

    def _render(self, cam, tf, step, pixels, threads, max_trace):
        table = np.ascontiguousarray(tf.table, dtype=np.float64).reshape(256, 4)
        t = _TF()
        t.table = table.ctypes.data
        t.vmin, t.vmax = float(tf.vmin), float(tf.vmax)
        s = _Step()
        s.mode = {"fixed": 0, "heuristic": 1, "learned": 2}[step.mode]
        mult = None
        if step.mode == "learned":
            mult = np.ascontiguousarray(step.mult, dtype=np.float32).reshape(-1)
            if mult.shape[0] != self.n_elem:
                raise ValueError("learned steps need one multiplier per element")
            s.mult = mult.ctypes.data
        s.field = {"scalar": 0, "magnitude": 1, "component": 2}[step.field]
        s.component = int(step.component)
        s.h, s.xi, s.alpha_stop = float(step.h), float(step.xi), float(step.alpha_stop)
        s.shading = {"none": 0, "gradient": 1}[getattr(step, "shading", "none")]
        trim = getattr(step, "trim", None)
        if trim is not None:
            trim = np.ascontiguousarray(trim, dtype=np.float32)
            assert trim.shape == (cam.height, cam.width, 2)
            s.trim = trim.ctypes.data
        for a, x in enumerate(getattr(step, "light", (0.0, 0.0, 0.0))):
            s.light[a] = float(x)
        c = _cam(cam)
        st = _Stats()
        if max_trace > 0:
            pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
            out = np.zeros((len(pix), 4), dtype=np.float64)
            trace = np.zeros((len(pix), max_trace, 4), dtype=np.float64)
            count = np.zeros(len(pix), dtype=np.int32)
            _load().orc_render_trace(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), pix.ctypes.data,
                                     len(pix), max_trace, trace.ctypes.data, count.ctypes.data, out.ctypes.data,
                                     _threads(threads or self.threads), ctypes.byref(st))
            return trace, count, out, {"samples": st.samples, "lookups": st.lookups, "rays_hit": st.rays_hit}
        if pixels is None:
            n = cam.width * cam.height
            out = np.zeros((n, 4), dtype=np.float64)
            _load().orc_render(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), None, n,
                               out.ctypes.data, _threads(threads or self.threads), ctypes.byref(st))
            out = out.reshape(cam.height, cam.width, 4)
        else:
            pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
            out = np.zeros((len(pix), 4), dtype=np.float64)
            _load().orc_render(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), pix.ctypes.data,
                               len(pix), out.ctypes.data, _threads(threads or self.threads), ctypes.byref(st))
        return out, {"samples": st.samples, "lookups": st.lookups, "rays_hit": st.rays_hit}

    # --- learned-step training labels (definition of lrvol_labels) ------------
    def labels(self, cam, tf, step, h_fine: float, tau: float, cand, threads: int | None = None):
        table = np.ascontiguousarray(tf.table, dtype=np.float64).reshape(256, 4)
        t = _TF()
        t.table = table.ctypes.data
        t.vmin, t.vmax = float(tf.vmin), float(tf.vmax)
        s = _Step()
        s.mode, s.field, s.component = 1, 0, 0
        s.h, s.xi, s.alpha_stop = float(step.h), float(step.xi), float(step.alpha_stop)
        c = _cam(cam)
        cand = np.ascontiguousarray(cand, dtype=np.float32)
        lab = np.full(self.n_elem, len(cand), dtype=np.int32)
        _load().orc_labels(self._h, ctypes.byref(c), ctypes.byref(t), ctypes.byref(s), float(h_fine), float(tau),
                           cand.ctypes.data, len(cand), lab.ctypes.data, _threads(threads or self.threads))
        return lab


def streamline_error(ref, ref_count, approx, approx_count):
    """Eq. 7: for each streamline j, sum over the approximation's samples
    i >= 1 of (t^i - t^{i-1}) * ||x_j(t^i) - y_j(t^i)||_2, the reference x_j
    linearly interpolated between its samples at t^i (samples past the
    reference's last time are left out).  Returns (per-line sums, max)."""
    ref = np.asarray(ref, dtype=np.float64)
    approx = np.asarray(approx, dtype=np.float64)
    sums = np.zeros(len(approx))
    for j in range(len(approx)):
        r = ref[j, :int(ref_count[j])]
        a = approx[j, :int(approx_count[j])]
        if len(r) < 2 or len(a) < 2:
            continue
        t = a[1:, 3]
        keep = t <= r[-1, 3]
        t = t[keep]
        dt = np.diff(a[:, 3])[keep]
        x = np.stack([np.interp(t, r[:, 3], r[:, c]) for c in range(3)], axis=1)
        sums[j] = float(np.sum(dt * np.linalg.norm(x - a[1:, :3][keep], axis=1)))
    return sums, float(sums.max()) if len(sums) else 0.0


def trim(cam, tris, threads: int | None = None):
    """Per-pixel trimming interval (H, W, 2) float32: nearest front-face hit
    (+inf if none) and farthest back-face hit (0 if none) of the triangles
    (n x 3 x 3 FP32 vertices, counter-clockwise seen from outside)."""
    tri = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    out = np.zeros((cam.height, cam.width, 2), dtype=np.float32)
    _load().orc_trim(ctypes.byref(_cam(cam)), tri.ctypes.data, len(tri), out.ctypes.data,
                     _threads(threads or 0))
    return out


def tube_segments(samples, count):
    """FP32 segments (n_seg x 6: a, b) of polylines, line by line in order."""
    samples = np.asarray(samples)
    segs = []
    for j in range(len(samples)):
        c = int(count[j])
        if c >= 2:
            pts = samples[j, :c, :3].astype(np.float32)
            segs.append(np.concatenate([pts[:-1], pts[1:]], axis=1))
    return np.ascontiguousarray(np.concatenate(segs) if segs else np.zeros((0, 6), np.float32), dtype=np.float32)

"""ctypes wrapper of the structured-mesh LR refinement generator (lrgen.cpp).

Input construction only: the arrays it returns are what ``lrvol_create``
takes (element boxes, local knot vectors, coefficients, scale factors gamma
of Eq. 2).  Nothing here evaluates, looks up or renders.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lrgen.cpp")
_LIB = os.path.join(_HERE, "liblrgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liblrgen.so in place (plain g++, no GPU code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32p = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
        lib.lrgen_new.restype = vp
        lib.lrgen_new.argtypes = [i32p, i32p, ctypes.c_int, ctypes.c_int]
        lib.lrgen_free.argtypes = [vp]
        lib.lrgen_num_elements.restype = i64
        lib.lrgen_num_elements.argtypes = [vp]
        lib.lrgen_num_basis.restype = i64
        lib.lrgen_num_basis.argtypes = [vp]
        lib.lrgen_grid.argtypes = [vp, i32p]
        lib.lrgen_elements_int.argtypes = [vp, vp]
        lib.lrgen_knots_int.argtypes = [vp, vp]
        lib.lrgen_gamma.argtypes = [vp, vp]
        lib.lrgen_carried_coef.argtypes = [vp, vp]
        lib.lrgen_set_coef.argtypes = [vp, vp]
        lib.lrgen_refine.restype = ctypes.c_int
        lib.lrgen_refine.argtypes = [vp, vp]
        lib.lrgen_uniforms.argtypes = [ctypes.c_uint64, i64, vp]
        _lib = lib
    return _lib


def uniforms(seed: int, n: int) -> np.ndarray:
    """n uniforms in [0,1) from std::mt19937_64(seed), (x >> 11) * 2^-53."""
    out = np.empty(n, dtype=np.float64)
    _load().lrgen_uniforms(ctypes.c_uint64(seed), n, out.ctypes.data)
    return out


class Stream:
    """Sequential consumer of one seeded uniform stream."""

    def __init__(self, seed: int, n: int = 1 << 16):
        self._u = uniforms(seed, n)
        self._i = 0

    def take(self, n: int) -> np.ndarray:
        if self._i + n > len(self._u):
            raise RuntimeError("seeded stream exhausted")
        r = self._u[self._i:self._i + n]
        self._i += n
        return r

    def uniform(self, lo, hi, n: int = 1) -> np.ndarray:
        return lo + (hi - lo) * self.take(n)


@dataclass
class LRVolume:
    """A trivariate LR-spline (Eq. 2): f = sum_i c_i gamma_i N_i.

    deg        : (3,) tri-degree p
    elem_box   : (N, 6) float64, lo xyz then hi xyz, in [0,1]
    knots      : (M, p0+2+p1+2+p2+2) float64, local knot vectors x then y then z
    coef       : (M, ncomp) float64
    weight     : (M,) float64, the scale factors gamma
    grid       : (3,) integer resolution on which all knots lie (metadata)
    """

    deg: np.ndarray
    elem_box: np.ndarray
    knots: np.ndarray
    coef: np.ndarray
    weight: np.ndarray
    grid: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def ncomp(self) -> int:
        return int(self.coef.shape[1])

    @property
    def n_elem(self) -> int:
        return int(self.elem_box.shape[0])

    @property
    def n_basis(self) -> int:
        return int(self.knots.shape[0])

    def knot_slices(self):
        p = [int(v) for v in self.deg]
        o = [0, p[0] + 2, p[0] + p[1] + 4]
        return [slice(o[a], o[a] + p[a] + 2) for a in range(3)]

    def save(self, path: str) -> None:
        import json
        np.savez(path, deg=self.deg, elem_box=self.elem_box, knots=self.knots, coef=self.coef,
                 weight=self.weight, grid=self.grid, name=np.array(self.name), meta=np.array(json.dumps(self.meta)))

    @staticmethod
    def load(path: str) -> "LRVolume":
        import json
        z = np.load(path)
        meta = json.loads(str(z["meta"])) if "meta" in z else {}
        return LRVolume(deg=z["deg"], elem_box=z["elem_box"], knots=z["knots"], coef=z["coef"],
                        weight=z["weight"], grid=z["grid"], name=str(z["name"]), meta=meta)


class Refiner:
    """Tensor-product start mesh plus structured-mesh LR refinement passes."""

    def __init__(self, deg, nbase, levels: int, ncomp: int = 1):
        lib = _load()
        d = (ctypes.c_int32 * 3)(*[int(v) for v in deg])
        nb = (ctypes.c_int32 * 3)(*[int(v) for v in nbase])
        self._h = lib.lrgen_new(d, nb, int(levels), int(ncomp))
        if not self._h:
            raise ValueError("bad generator arguments")
        self.deg = np.array([int(v) for v in deg], dtype=np.int32)
        self.ncomp = int(ncomp)
        g = (ctypes.c_int32 * 3)()
        lib.lrgen_grid(self._h, g)
        self.grid = np.array(list(g), dtype=np.int64)

    def __del__(self):
        if getattr(self, "_h", None):
            _load().lrgen_free(self._h)
            self._h = None

    @property
    def n_elem(self) -> int:
        return int(_load().lrgen_num_elements(self._h))

    @property
    def n_basis(self) -> int:
        return int(_load().lrgen_num_basis(self._h))

    def elements_int(self) -> np.ndarray:
        out = np.empty((self.n_elem, 6), dtype=np.int32)
        _load().lrgen_elements_int(self._h, out.ctypes.data)
        return out

    def knots_int(self) -> np.ndarray:
        out = np.empty((self.n_basis, int(self.deg.sum()) + 6), dtype=np.int32)
        _load().lrgen_knots_int(self._h, out.ctypes.data)
        return out

    def gamma(self) -> np.ndarray:
        out = np.empty(self.n_basis, dtype=np.float64)
        _load().lrgen_gamma(self._h, out.ctypes.data)
        return out

    def carried_coef(self) -> np.ndarray:
        out = np.empty((self.n_basis, self.ncomp), dtype=np.float64)
        _load().lrgen_carried_coef(self._h, out.ctypes.data)
        return out

    def set_coef(self, coef: np.ndarray) -> None:
        c = np.ascontiguousarray(coef, dtype=np.float64).reshape(self.n_basis, self.ncomp)
        _load().lrgen_set_coef(self._h, c.ctypes.data)

    def element_boxes(self) -> np.ndarray:
        e = self.elements_int().astype(np.float64)
        g = np.concatenate([self.grid, self.grid]).astype(np.float64)
        return e / g

    def knots(self) -> np.ndarray:
        k = self.knots_int().astype(np.float64)
        p = self.deg
        scale = np.concatenate([np.full(p[a] + 2, float(self.grid[a])) for a in range(3)])
        return k / scale

    def refine(self, marked: np.ndarray) -> None:
        m = np.ascontiguousarray(marked, dtype=np.uint8)
        if m.shape != (self.n_elem,):
            raise ValueError("one mark per element")
        rc = _load().lrgen_refine(self._h, m.ctypes.data)
        if rc != 0:
            raise RuntimeError(f"refinement failed ({rc})")

    def volume(self, coef: np.ndarray | None = None, name: str = "") -> LRVolume:
        c = self.carried_coef() if coef is None else np.asarray(coef, dtype=np.float64)
        return LRVolume(deg=self.deg.copy(), elem_box=self.element_boxes(), knots=self.knots(),
                        coef=c.reshape(self.n_basis, self.ncomp), weight=self.gamma(),
                        grid=self.grid.copy(), name=name)


def greville(vol_or_knots, deg=None) -> np.ndarray:
    """Greville point of every B-spline: per axis the mean of its p interior knots."""
    if isinstance(vol_or_knots, LRVolume):
        knots, deg = vol_or_knots.knots, vol_or_knots.deg
    else:
        knots = vol_or_knots
    p = [int(v) for v in deg]
    o = [0, p[0] + 2, p[0] + p[1] + 4]
    cols = [knots[:, o[a] + 1:o[a] + 1 + p[a]].mean(axis=1) for a in range(3)]
    return np.stack(cols, axis=1)

"""Seeded synthetic workloads standing in for the paper's datasets.

The paper renders LR-spline approximations of an MR brain scan, of wind flow
around a telescope and of a fluidized bed (Sec. 4.3, Sec. 5.5); none of those
datasets is available, so these recipes build LR-splines of the same kind
(tri-degree, refinement pattern, element counts) from seeded analytic fields.

Every random number comes from ``lrgen.uniforms`` (std::mt19937_64, seed
1707011700 + config id; cameras use seed + 1000).  The recipes are input
construction only: they never evaluate the LR-spline they build.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

from .lrgen import LRVolume, Refiner, Stream, greville

SEED_BASE = 1707011700
_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))),
                      "_cache")


# ----------------------------------------------------------------------------
# render parameters
# ----------------------------------------------------------------------------

@dataclass
class Camera:
    """Pinhole (persp) or parallel (ortho) camera; image row 0 is the top row."""

    projection: str          # "ortho" | "persp"
    width: int
    height: int
    eye: tuple
    target: tuple
    up: tuple
    fovy: float = 0.0        # persp: full vertical field of view, radians
    extent: float = 1.0      # ortho: full height of the view window, world units


@dataclass
class TransferFunction:
    """256 RGBA entries over [vmin, vmax] (colour not premultiplied)."""

    table: np.ndarray        # (256, 4) float64
    vmin: float = 0.0
    vmax: float = 1.0


@dataclass
class StepParams:
    mode: str = "fixed"      # "fixed" | "heuristic" | "learned"
    h: float = 1.0 / 256     # fixed step
    xi: float = 1.0 / 256    # reference length xi of Alg. 2
    alpha_stop: float = 1.0  # early termination threshold (1 = off)
    field: str = "scalar"    # "scalar" | "magnitude" | "component"
    component: int = 0
    mult: object = None      # learned: per-element step multipliers (array or device tensor)
    shading: str = "none"    # "none" | "gradient" (scalar fields: C_src times max(0.4, |l . n|))
    light: tuple = (0.0, 0.0, 0.0)   # towards the light; zero = from the eye
    trim: object = None      # per-pixel (t_front, t_back) of a trimming mesh (array or device tensor)


def seeded_tf(stream: Stream, n_ctrl: int = 8, alpha_max: float = 0.08, bands=()) -> TransferFunction:
    """Piecewise-linear TF through n_ctrl seeded control points at equal spacing.

    Control point m sits at value m/(n_ctrl-1); RGB ~ U[0,1], alpha ~ U[0, alpha_max],
    alpha of the first control point is 0.  Each band (centre, half width,
    alpha, r, g, b) then raises the entries within the half width to a tent
    profile of that peak opacity and colour.
    """
    ctrl = np.zeros((n_ctrl, 4))
    for m in range(n_ctrl):
        ctrl[m, :3] = stream.take(3)
        ctrl[m, 3] = 0.0 if m == 0 else alpha_max * stream.take(1)[0]
    x = np.arange(256) / 255.0
    xc = np.arange(n_ctrl) / (n_ctrl - 1)
    table = np.stack([np.interp(x, xc, ctrl[:, c]) for c in range(4)], axis=1)
    for (c0, hw, a, r, g, b) in bands:
        w = np.clip(1.0 - np.abs(x - c0) / hw, 0.0, 1.0)
        sel = w > 0
        table[sel, 3] = np.maximum(table[sel, 3], a * w[sel])
        for ch, v in enumerate((r, g, b)):
            table[sel, ch] = (1 - w[sel]) * table[sel, ch] + w[sel] * v
    return TransferFunction(table=table, vmin=0.0, vmax=1.0)


def ortho_z(width: int = 128, height: int = 128) -> Camera:
    """Orthographic view along -z covering [0,1]^2 (pixel centres at (i+1/2)/W)."""
    return Camera("ortho", width, height, eye=(0.5, 0.5, 2.0), target=(0.5, 0.5, 0.0),
                  up=(0.0, 1.0, 0.0), extent=1.0)


def seeded_oblique(stream: Stream, width: int = 128, height: int = 128) -> Camera:
    """Orthographic view of the unit cube from a seeded direction in the upper hemisphere."""
    u = stream.take(2)
    phi = 2 * np.pi * u[0]
    cz = 0.2 + 0.7 * u[1]
    sz = np.sqrt(1 - cz * cz)
    d = np.array([sz * np.cos(phi), sz * np.sin(phi), cz])
    eye = 0.5 + 2.0 * d
    return Camera("ortho", width, height, eye=tuple(eye), target=(0.5, 0.5, 0.5),
                  up=(0.0, 0.0, 1.0) if abs(cz) < 0.99 else (0.0, 1.0, 0.0), extent=1.8)


def orbit_camera(stream: Stream, width: int, height: int, radius: float = 1.8,
                 fovy_deg: float = 40.0) -> Camera:
    """Perspective camera at distance `radius` from the cube centre, seeded azimuth/elevation."""
    u = stream.take(2)
    az = 2 * np.pi * u[0]
    el = np.deg2rad(-30.0 + 60.0 * u[1])
    d = np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
    eye = 0.5 + radius * d
    return Camera("persp", width, height, eye=tuple(eye), target=(0.5, 0.5, 0.5),
                  up=(0.0, 0.0, 1.0), fovy=np.deg2rad(fovy_deg))


# ----------------------------------------------------------------------------
# small volumes for tests
# ----------------------------------------------------------------------------

def tensor_product(deg=(3, 3, 3), n=(4, 4, 4), ncomp: int = 1, coef=None, seed: int = 0) -> LRVolume:
    """Unrefined tensor-product B-spline volume (Eq. 1) with seeded coefficients."""
    R = Refiner(deg, n, 0, ncomp)
    if coef is None:
        coef = Stream(seed, 3 * R.n_basis + 8).take(R.n_basis * ncomp).reshape(R.n_basis, ncomp)
    return R.volume(coef=coef, name=f"tp{tuple(deg)}x{tuple(n)}")


def refined_ball(deg=(3, 3, 3), n=(4, 4, 4), centres=((0.5, 0.5, 0.5),), radii=(0.3,),
                 ncomp: int = 1, seed: int = 0, coef_fn=None, carry_fn=None) -> LRVolume:
    """Tensor-product start mesh refined len(radii) times around seeded balls.

    coef_fn(greville_points) -> coefficients assigned after refinement;
    carry_fn(greville_points) -> coefficients of the start mesh, carried
    through the refinement by the splitting weights.
    Otherwise seeded uniform coefficients are assigned after refinement.
    """
    R = Refiner(deg, n, len(radii), ncomp)
    if carry_fn is not None:
        R.set_coef(carry_fn(greville(R.knots(), R.deg)))
    for lvl, rad in enumerate(radii):
        e = R.element_boxes()
        c = 0.5 * (e[:, :3] + e[:, 3:])
        mark = np.zeros(len(c), dtype=bool)
        for ctr in centres:
            mark |= np.linalg.norm(c - np.asarray(ctr), axis=1) < rad
        R.refine(mark)
    if carry_fn is not None:
        return R.volume(name="ball-carried")
    g = greville(R.knots(), R.deg)
    if coef_fn is not None:
        coef = np.asarray(coef_fn(g), dtype=np.float64).reshape(R.n_basis, ncomp)
    else:
        coef = Stream(seed, R.n_basis * ncomp + 8).take(R.n_basis * ncomp).reshape(R.n_basis, ncomp)
    return R.volume(coef=coef, name="ball")


# ----------------------------------------------------------------------------
# config 1: scalar tricubic, two refinement levels around a seeded point
# ----------------------------------------------------------------------------

def _gaussians(stream: Stream, k: int):
    c = stream.uniform(0.15, 0.85, 3 * k).reshape(k, 3)
    s = stream.uniform(0.1, 0.2, k)
    a = stream.uniform(0.5, 1.0, k)
    return c, s, a


def config1() -> LRVolume:
    """p=(3,3,3), scalar; uniform 8^3 start; level 1 refines elements whose centre
    lies within 0.25 of a seeded point in [0.25,0.75]^3, level 2 within 0.12.
    Coefficients: sum of 4 seeded isotropic Gaussians at the Greville points,
    min-max normalised to [0,1]."""
    st = Stream(SEED_BASE + 1)
    ctr = st.uniform(0.25, 0.75, 3)
    R = Refiner((3, 3, 3), (8, 8, 8), 2, 1)
    for rad in (0.25, 0.12):
        e = R.element_boxes()
        c = 0.5 * (e[:, :3] + e[:, 3:])
        R.refine(np.linalg.norm(c - ctr, axis=1) < rad)
    gc, gs, ga = _gaussians(st, 4)
    g = greville(R.knots(), R.deg)
    v = np.zeros(len(g))
    for m in range(4):
        v += ga[m] * np.exp(-np.sum((g - gc[m]) ** 2, axis=1) / (2 * gs[m] ** 2))
    v = (v - v.min()) / (v.max() - v.min())
    vol = R.volume(coef=v[:, None], name="cfg1")
    return vol


def config1_render():
    """TF and the two cameras of config 1 (ortho along -z, seeded oblique)."""
    st = Stream(SEED_BASE + 1 + 1000)
    tf = seeded_tf(st)
    return tf, [ortho_z(128, 128), seeded_oblique(st, 128, 128)]


# ----------------------------------------------------------------------------
# config 2: MR-like scalar field, 3 nested ellipsoidal shells, ~150k elements
# ----------------------------------------------------------------------------

class _ShellField:
    """Voxel field on a 256^3 cell-centred grid: 3 nested ellipsoidal shells
    (Gaussian profile) plus 16 low-frequency sinusoids, min-max normalised."""

    N = 256

    def __init__(self, st: Stream):
        base = np.array([0.40, 0.33, 0.25])
        self.axes = np.array([b * st.uniform(0.9, 1.1, 3) for b in base])      # (3 shells, 3 axes)
        self.width = st.uniform(0.01, 0.02, 3)
        self.amp = np.array([0.55, 0.75, 1.0]) * st.uniform(0.9, 1.0, 3)
        self.kvec = np.floor(st.uniform(-3.0, 4.0, 48)).reshape(16, 3)
        self.phase = 2 * np.pi * st.take(16)
        self.noise_amp = 0.05
        lo, hi = np.inf, -np.inf
        for z0 in range(0, self.N, 32):
            v = self._raw_slab(z0, z0 + 32)
            lo, hi = min(lo, float(v.min())), max(hi, float(v.max()))
        self.lo, self.hi = lo, hi

    def shell_distance(self, x: np.ndarray) -> np.ndarray:
        """(n, 3 shells) approximate signed distance to each shell."""
        out = np.empty((len(x), 3))
        for k in range(3):
            r = np.sqrt(np.sum(((x - 0.5) / self.axes[k]) ** 2, axis=1))
            out[:, k] = (r - 1.0) * self.axes[k].mean()
        return out

    def _raw_points(self, x: np.ndarray) -> np.ndarray:
        d = self.shell_distance(x)
        v = np.zeros(len(x))
        for k in range(3):
            v += self.amp[k] * np.exp(-0.5 * (d[:, k] / self.width[k]) ** 2)
        s = np.zeros(len(x))
        for m in range(16):
            s += np.sin(2 * np.pi * (x @ self.kvec[m]) + self.phase[m])
        return (v + self.noise_amp * s / 4.0).astype(np.float32)

    def _raw_slab(self, z0, z1):
        n = self.N
        ax = (np.arange(n) + 0.5) / n
        zz = (np.arange(z0, z1) + 0.5) / n
        X = np.stack(np.meshgrid(ax, ax, zz, indexing="ij"), axis=-1).reshape(-1, 3)
        return self._raw_points(X)

    def voxel(self, ijk: np.ndarray) -> np.ndarray:
        x = (ijk.astype(np.float64) + 0.5) / self.N
        raw = self._raw_points(x).astype(np.float64)
        return ((raw - self.lo) / (self.hi - self.lo)).astype(np.float32)

    def trilinear(self, p: np.ndarray) -> np.ndarray:
        n = self.N
        q = np.clip(p * n - 0.5, 0.0, n - 1.0)
        i0 = np.minimum(np.floor(q).astype(np.int64), n - 2)
        f = q - i0
        out = np.zeros(len(p))
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                         * (f[:, 2] if dz else 1 - f[:, 2]))
                    out += w * self.voxel(i0 + np.array([dx, dy, dz])).astype(np.float64)
        return out


CFG2_BASE = 4
CFG2_BANDS = (0.1, 0.04, 0.015, 0.006)   # band half widths around each shell, per refinement level


def config2() -> LRVolume:
    """p=(3,3,3), scalar; uniform 4^3 start refined 4 times (smallest element 1/64,
    size ratio 16) in bands around the shells, about 174k elements;
    coefficients = trilinear sample of the voxel field at the Greville points,
    stored as float32 values (the volume carries them as float64)."""
    st = Stream(SEED_BASE + 2)
    fld = _ShellField(st)
    R = Refiner((3, 3, 3), (CFG2_BASE,) * 3, len(CFG2_BANDS), 1)
    for w in CFG2_BANDS:
        e = R.element_boxes()
        c = 0.5 * (e[:, :3] + e[:, 3:])
        d = fld.shell_distance(c)
        R.refine(np.any(np.abs(d) < w, axis=1))
    g = greville(R.knots(), R.deg)
    coef = fld.trilinear(g).astype(np.float32).astype(np.float64)
    vol = R.volume(coef=coef[:, None], name="cfg2")
    # normalised field value on each shell (peak of its Gaussian profile)
    vol.meta["shell_values"] = [float((a - fld.lo) / (fld.hi - fld.lo)) for a in fld.amp]
    return vol


def config2_render(width: int = 1920, height: int = 1080, vol: LRVolume | None = None):
    """Perspective 1920x1080 camera at distance 1.8, fovy 40 deg, and the TF:
    the config-1 recipe (peak opacity 0.02) plus 3 opacity bands, half width
    0.04, centred on the normalised shell values (seeded peak opacity
    U[0.05,0.3], seeded colour)."""
    if vol is None:
        vol = load_config(2)
    st = Stream(SEED_BASE + 2 + 1000)
    cam = orbit_camera(st, width, height)
    centres = vol.meta["shell_values"]
    bands = []
    for k in range(3):
        a = st.uniform(0.05, 0.3, 1)[0]
        rgb = st.take(3)
        bands.append((float(centres[k]), 0.04, a, *rgb))
    tf = seeded_tf(st, alpha_max=0.02, bands=bands)
    return tf, cam


# ----------------------------------------------------------------------------
# config 3: 3-vector triquadratic flow past a box obstacle, ~400k elements
# ----------------------------------------------------------------------------

BOX_LO = np.array([0.40, 0.35, 0.00])
BOX_HI = np.array([0.55, 0.65, 0.30])


def box_distance(x: np.ndarray) -> np.ndarray:
    q = np.maximum(np.maximum(BOX_LO - x, x - BOX_HI), 0.0)
    return np.linalg.norm(q, axis=1)


class _Flow:
    """Uniform flow U=(1,0,0) with a sphere-doublet potential correction around
    the obstacle, smoothly masked to zero inside it, plus 6 Lamb-Oseen swirls."""

    def __init__(self, st: Stream):
        self.c = 0.5 * (BOX_LO + BOX_HI)
        self.R = 0.12
        self.vc = st.uniform(0.1, 0.9, 18).reshape(6, 3)
        ax = st.uniform(-1.0, 1.0, 18).reshape(6, 3)
        self.vax = ax / np.linalg.norm(ax, axis=1, keepdims=True)
        self.rc = st.uniform(0.03, 0.08, 6)
        self.gam = st.uniform(-1.0, 1.0, 6) * 0.5 * 2 * np.pi * self.rc / 0.638

    def __call__(self, x: np.ndarray) -> np.ndarray:
        r = x - self.c
        rn = np.maximum(np.linalg.norm(r, axis=1), 1e-3)
        ex = np.array([1.0, 0.0, 0.0])
        v = np.tile(ex, (len(x), 1))
        k = 0.5 * self.R ** 3
        v += k * (ex[None, :] / rn[:, None] ** 3 - 3 * r[:, :1] * r / rn[:, None] ** 5)
        for m in range(6):
            d = x - self.vc[m]
            along = d @ self.vax[m]
            perp = d - along[:, None] * self.vax[m]
            rho = np.maximum(np.linalg.norm(perp, axis=1), 1e-6)
            vt = self.gam[m] / (2 * np.pi * rho) * (1 - np.exp(-(rho / self.rc[m]) ** 2))
            tang = np.cross(self.vax[m][None, :], perp) / rho[:, None]
            v += vt[:, None] * tang
        s = np.clip(box_distance(x) / 0.03, 0.0, 1.0)
        s = s * s * (3 - 2 * s)
        inside = np.all((x > BOX_LO) & (x < BOX_HI), axis=1)
        s[inside] = 0.0
        return v * s[:, None]


CFG3_BASE = 6
CFG3_DIST = (0.1, 0.1, 0.1, 0.1, 0.05)


def config3() -> LRVolume:
    """p=(2,2,2), 3 components; uniform 6^3 start refined 5 times (knots are
    multiples of 1/192, not dyadic; size ratio 32) where the element centre lies
    within 0.1 of the box obstacle (0.05 on the last level), about 388k elements;
    coefficients = the flow at the Greville points."""
    st = Stream(SEED_BASE + 3)
    flow = _Flow(st)
    R = Refiner((2, 2, 2), (CFG3_BASE,) * 3, len(CFG3_DIST), 3)
    for dist in CFG3_DIST:
        e = R.element_boxes()
        c = 0.5 * (e[:, :3] + e[:, 3:])
        R.refine(box_distance(c) < dist)
    g = greville(R.knots(), R.deg)
    vol = R.volume(coef=flow(g), name="cfg3")
    return vol


def config3_render(width: int = 1920, height: int = 1080):
    st = Stream(SEED_BASE + 3 + 1000)
    cam = orbit_camera(st, width, height)
    tf = seeded_tf(st, alpha_max=0.03)
    return tf, cam


def config3_seeds(n: int) -> np.ndarray:
    """Streamline seeds for config 3: a seeded rake upstream of the obstacle,
    x in [0.02, 0.10], y in [0.05, 0.95], z in [0.02, 0.60] (n x 3, FP64)."""
    u = Stream(SEED_BASE + 3 + 2000, 3 * n + 8).take(3 * n).reshape(n, 3)
    lo, hi = np.array([0.02, 0.05, 0.02]), np.array([0.10, 0.95, 0.60])
    return lo + (hi - lo) * u


# ----------------------------------------------------------------------------
# trimming meshes (closed, counter-clockwise seen from outside)
# ----------------------------------------------------------------------------

def box_mesh(lo, hi) -> np.ndarray:
    """The 12 triangles of an axis-aligned box, (12, 3, 3)."""
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    c = np.array([[lo[0] if (k & 1) == 0 else hi[0], lo[1] if (k & 2) == 0 else hi[1],
                   lo[2] if (k & 4) == 0 else hi[2]] for k in range(8)])
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    tris = []
    for a, b, cc, d in quads:        # each face counter-clockwise seen from outside
        tris.append([c[a], c[b], c[cc]])
        tris.append([c[a], c[cc], c[d]])
    return np.array(tris)


def icosphere(centre=(0.5, 0.5, 0.5), radius: float = 0.3, subdiv: int = 3) -> np.ndarray:
    """A sphere tessellated from an icosahedron by subdiv 4-way splits,
    20 * 4^subdiv triangles, (n, 3, 3)."""
    t = (1 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache, nf = {}, []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    V_ = np.asarray(v) * radius + np.asarray(centre, dtype=np.float64)
    return V_[np.asarray(f)]


def uv_sphere(centre=(0.5, 0.5, 0.5), radius: float = 0.3, n_lat: int = 64, n_lon: int = 128) -> np.ndarray:
    """A latitude-longitude sphere, 2 * n_lat * n_lon triangles (those at the
    poles degenerate), counter-clockwise seen from outside, (n, 3, 3)."""
    th = np.linspace(0.0, np.pi, n_lat + 1)
    ph = np.linspace(0.0, 2 * np.pi, n_lon + 1)
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    P_ = np.stack([np.sin(T) * np.cos(Ph), np.sin(T) * np.sin(Ph), np.cos(T)], axis=-1) * radius
    P_ = P_ + np.asarray(centre, dtype=np.float64)
    a, b = P_[:-1, :-1], P_[1:, :-1]           # (lat k, lon l), (lat k+1, lon l)
    c, d = P_[1:, 1:], P_[:-1, 1:]             # (lat k+1, lon l+1), (lat k, lon l+1)
    t1 = np.stack([a, b, c], axis=2).reshape(-1, 3, 3)
    t2 = np.stack([a, c, d], axis=2).reshape(-1, 3, 3)
    return np.concatenate([t1, t2])


# ----------------------------------------------------------------------------

_BUILDERS = {1: config1, 2: config2, 3: config3}


def load_config(k: int, cache: bool = True) -> LRVolume:
    """Build (or load from the on-disk cache) the volume of config k."""
    if not cache:
        return _BUILDERS[k]()
    os.makedirs(_CACHE, exist_ok=True)
    path = os.path.join(_CACHE, f"cfg{k}_v2.npz")
    if os.path.exists(path):
        return LRVolume.load(path)
    vol = _BUILDERS[k]()
    tmp = path + f".tmp{os.getpid()}.npz"
    vol.save(tmp)
    os.replace(tmp, path)
    return vol

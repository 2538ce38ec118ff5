"""Pins of the oracle's trimming (Sec. 4.1: the ray interval cut to a
closed mesh's first front and last back face, a z-prepass) to things other
than itself: the exact intervals of an axis-aligned box seen along z,
watertightness on a tessellated sphere (every ray through the interior has
one front and one back hit; none is lost on a shared edge), and closed-form
opacity of a constant field over the trimmed chord, also with the eye inside
the mesh."""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import Oracle
from paper_1707_01170_gb300.synth import volumes as V

import test_oracle_pins as P


def test_meshes_are_closed_and_outward():
    for tris in (V.box_mesh((0.2, 0.3, 0.1), (0.7, 0.9, 0.6)), V.icosphere(subdiv=2)):
        c = tris.reshape(-1, 3).mean(axis=0)
        n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
        assert np.all(np.einsum("ij,ij->i", n, tris.mean(axis=1) - c) > 0)
        edges = {}
        for t in tris:
            for a, b in ((0, 1), (1, 2), (2, 0)):
                key = tuple(np.round(t[a], 12)), tuple(np.round(t[b], 12))
                edges[key] = edges.get(key, 0) + 1
        for (a, b), k in edges.items():                 # every directed edge once, its reverse once
            assert k == 1 and edges.get((b, a)) == 1


def test_box_intervals_along_z():
    cam = V.ortho_z(64, 64)                             # eye plane z = 2, rays along -z
    tr = orc.trim(cam, V.box_mesh((0.25, 0.25, 0.25), (0.75, 0.75, 0.75)))
    x = (np.arange(64) + 0.5) / 64
    inside = ((x > 0.25) & (x < 0.75))[None, :] & ((x > 0.25) & (x < 0.75))[:, None]
    np.testing.assert_allclose(tr[inside][:, 0], 1.25, rtol=1e-6)
    np.testing.assert_allclose(tr[inside][:, 1], 1.75, rtol=1e-6)
    assert np.all(tr[~inside][:, 0] == np.inf) and np.all(tr[~inside][:, 1] == 0)


def test_sphere_is_watertight():
    cam = V.orbit_camera(V.Stream(17), 96, 80)
    r, ctr = 0.3, np.array([0.45, 0.5, 0.55])
    tr = orc.trim(cam, V.icosphere(ctr, r, 3))
    seen = 0
    for j in range(cam.height):
        for i in range(cam.width):
            r_ = orc.ray(cam, i, j)
            if r_ is None:                                  # misses the unit cube, so the sphere too
                assert tr[j, i, 0] == np.inf and tr[j, i, 1] == 0
                continue
            o, d = np.asarray(r_[0], np.float64), np.asarray(r_[1], np.float64)
            dist = np.linalg.norm(np.cross(ctr - o, d)) / np.linalg.norm(d)
            if dist < 0.95 * r * np.cos(np.pi / 40):            # well inside the tessellated silhouette
                seen += 1
                assert np.isfinite(tr[j, i, 0]) and tr[j, i, 1] > tr[j, i, 0]
                tc = np.dot(ctr - o, d) / np.linalg.norm(d)
                half = np.sqrt(r * r - dist * dist)
                assert abs(tr[j, i, 0] - (tc - half)) < 0.02 and abs(tr[j, i, 1] - (tc + half)) < 0.02
            elif dist > 1.05 * r:
                assert tr[j, i, 0] == np.inf and tr[j, i, 1] == 0
    assert seen > 800


@pytest.mark.parametrize("where", ["outside", "inside"])
def test_trimmed_constant_field_closed_form(cfg1, where):
    vol = P._with_coef(cfg1, np.full(cfg1.n_basis, 0.37))
    O = Oracle(vol)
    a_src, rgb = 0.02, np.array([0.9, 0.4, 0.1])
    tf = P._const_tf([*rgb, a_src])
    box = V.box_mesh((0.2, 0.3, 0.25), (0.8, 0.7, 0.75))
    if where == "outside":
        cam = V.ortho_z(32, 32)
    else:
        cam = V.Camera("persp", 24, 20, eye=(0.5, 0.5, 0.5), target=(0.9, 0.6, 0.2), up=(0.0, 0.0, 1.0),
                       fovy=np.deg2rad(60.0))
    tr = orc.trim(cam, box)
    step = V.StepParams(mode="heuristic", xi=1 / 128, trim=tr)
    img, st = O.render(cam, tf, step)
    hit = 0
    for j in range(cam.height):
        for i in range(cam.width):
            r = orc.ray(cam, i, j)
            if r is None:
                assert np.all(img[j, i] == 0)
                continue
            tin, tout = float(r[2]), float(r[3])
            tf_, tb = float(tr[j, i, 0]), float(tr[j, i, 1])
            if tf_ == np.inf and tb == 0:
                assert np.all(img[j, i] == 0)
                continue
            lo = max(tin, tf_) if np.isfinite(tf_) else tin
            hi = min(tout, tb) if tb > 0 else tout
            L = max(0.0, hi - lo)
            alpha = 1 - (1 - a_src) ** (L / step.xi)
            assert img[j, i, 3] == pytest.approx(alpha, abs=1e-12)
            np.testing.assert_allclose(img[j, i, :3], rgb * alpha, atol=1e-12)
            hit += L > 0
    assert hit > 100
    if where == "inside":
        assert np.all(np.isinf(tr[..., 0])) and np.all(tr[..., 1] > 0)   # only back faces from inside

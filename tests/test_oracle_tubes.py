"""Pins of the oracle's streamline tubes (Sec. 5.3): a straight segment seen
along z gives the capsule's closed form (hit where |y - y0| < r, depth
z_eye - z0 - sqrt(r^2 - dy^2), shading sqrt(r^2 - dy^2)/r above the 0.4
floor, colour from the colour map at the field's speed); rays past a segment
end hit the cap sphere; of two crossing tubes the nearer one shows."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1707_01170_gb300.synth import volumes as V


def _const_field(v=(1.0, 0.0, 0.0)):
    return V.tensor_product((2, 2, 2), (2, 2, 2), ncomp=3, coef=np.tile(v, (4 ** 3, 1)))


def _cmap():
    table = np.zeros((256, 4))
    x = np.arange(256) / 255
    table[:, 0], table[:, 1], table[:, 2], table[:, 3] = x, 1 - x, 0.5, 1.0
    return V.TransferFunction(table=table, vmin=0.0, vmax=2.0)


def _lines(*polys):
    m = max(len(p) for p in polys)
    s = np.zeros((len(polys), m, 4))
    for j, p in enumerate(polys):
        s[j, :len(p), :3] = p
    return s, np.array([len(p) for p in polys])


def test_straight_segment_closed_form():
    O = Oracle(_const_field())
    cam = V.ortho_z(128, 128)                              # rays along -z from z = 2
    r, y0, z0 = 0.1, 0.5, 0.4
    s, c = _lines([[0.2, y0, z0], [0.8, y0, z0]])
    img = O.tubes(cam, s, c, r, _cmap())
    x = (np.arange(128) + 0.5) / 128
    rgb = np.array([0.5, 0.5, 0.5])                        # colour map at speed 1 of [0, 2]
    floor = 0
    for j in range(128):
        for i in range(128):
            px, py = x[i], 1 - x[j]
            dy = py - y0
            body = 0.2 < px < 0.8 and abs(dy) < r * 0.999
            if body:
                I = max(0.4, np.sqrt(r * r - dy * dy) / r)
                floor += I == 0.4
                np.testing.assert_allclose(img[j, i], [*(I * rgb), 1.0], atol=2e-5)
            elif abs(dy) > r * 1.001 or (px < 0.2 - r * 1.001 or px > 0.8 + r * 1.001):
                assert np.all(img[j, i] == 0)
    assert floor > 0                                       # the 0.4 floor is exercised


def _field_z():
    """f = (z, 0, 0), carried exactly through a refined triquadratic mesh."""
    return V.refined_ball((2, 2, 2), (4, 4, 4), centres=((0.5, 0.5, 0.5),), radii=(0.3,), ncomp=3,
                          carry_fn=lambda g: np.stack([g[:, 2], 0 * g[:, 2], 0 * g[:, 2]], axis=1))


def test_caps_and_occlusion():
    O = Oracle(_field_z())
    cam = V.ortho_z(48, 48)
    s, c = _lines([[0.3, 0.5, 0.3], [0.7, 0.5, 0.3]],           # far tube, speed 0.3
                  [[0.5, 0.3, 0.6], [0.5, 0.7, 0.6]])           # near tube across it, speed 0.6
    img = O.tubes(cam, s, c, 0.05, _cmap())
    x = (np.arange(48) + 0.5) / 48
    i = int(np.argmin(np.abs(x - 0.5)))
    j = int(np.argmin(np.abs(1 - x - 0.5)))
    assert img[j, i, 3] == 1.0                                  # the crossing shows the near tube:
    # its normal there is along z (I = 1 for the pixel closest to its axis)
    assert img[j, i, :3] == pytest.approx(np.array([0.3, 0.7, 0.5]) * 1.0, abs=0.03)
    # a cap: a ray 0.03 past the far tube's end (inside the radius 0.05)
    ic = int(np.argmin(np.abs(x - 0.72)))
    assert img[j, ic, 3] == 1.0
    ie = int(np.argmin(np.abs(x - 0.78)))
    assert img[j, ie, 3] == 0.0

"""FP64 reference of the learned step size (test infrastructure only).

Features, network, gradient and Adam step written out from their
definitions in include/lrvol.h (the paper has no learned component; the
learned step multiplies the Eq. 4 step per element).  Nothing here calls the
CUDA library.

Parameter vector (9473 floats): W1[16][64], b1[64], W2[64][64], b2[64],
W3[64][64], b3[64], W4[64], b4 -- W[in][out].
"""
from __future__ import annotations

import numpy as np

IN, HID = 16, 64
SIZES = [("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)), ("b3", (HID,)),
         ("W4", (HID,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(x):
    """Round to BF16 (round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, emulate_bf16: bool = False):
    """Network output y (n,) in FP64; with emulate_bf16 the weights and every
    layer's input are rounded to BF16 first (the tensor-core operands), biases
    stay FP32."""
    w = unpack(p)
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    h = r(X)
    for k in (1, 2, 3):
        h = np.maximum(h @ r(w[f"W{k}"]) + f32(w[f"b{k}"]), 0.0)
        h = r(h)
    return h @ r(w["W4"]) + f32(w["b4"])[0]


def multipliers(p, X, ymax: float, emulate_bf16: bool = True, ymin: float = 0.0):
    """Step multipliers 2^clamp(y, ymin, ymax) of the network output y."""
    return 2.0 ** np.clip(forward(p, X, emulate_bf16), ymin, ymax)


def loss_and_grad(p, X, t):
    """loss = mean((y - t)^2)/2 and its gradient, FP64 backward."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = len(X)
    h1 = np.maximum(X @ w["W1"] + w["b1"], 0.0)
    h2 = np.maximum(h1 @ w["W2"] + w["b2"], 0.0)
    h3 = np.maximum(h2 @ w["W3"] + w["b3"], 0.0)
    y = h3 @ w["W4"] + w["b4"][0]
    r = y - t
    loss = 0.5 * np.mean(r * r)
    dy = r / n
    g = {"W4": h3.T @ dy, "b4": np.array([dy.sum()])}
    d3 = np.outer(dy, w["W4"]) * (h3 > 0)
    g["W3"], g["b3"] = h2.T @ d3, d3.sum(axis=0)
    d2 = (d3 @ w["W3"].T) * (h2 > 0)
    g["W2"], g["b2"] = h1.T @ d2, d2.sum(axis=0)
    d1 = (d2 @ w["W2"].T) * (h1 > 0)
    g["W1"], g["b1"] = X.T @ d1, d1.sum(axis=0)
    return loss, pack(g)


def adam(p, g, m, v, t: int, lr: float):
    """One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)."""
    m = 0.9 * m + 0.1 * g
    v = 0.999 * v + 0.001 * g * g
    p = p - lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
    return p, m, v


def features(orc, box, cam, tf, field: str = "scalar", component: int = 0, blocks=None):
    """FP64 features of every element (n_elem x 16), from the oracle's own
    Bezier blocks (interpolation) and the element boxes."""
    if blocks is None:
        blocks = orc.bezier_blocks()
    flat = blocks.reshape(len(blocks), blocks.shape[1], -1)
    cmin, cmax = flat.min(axis=2), flat.max(axis=2)                    # (n, nc)
    if field == "magnitude":
        m = np.maximum(np.abs(cmin), np.abs(cmax))
        d = np.where(cmin > 0, cmin, np.where(cmax < 0, -cmax, 0.0))
        lo, hi = np.sqrt((d * d).sum(axis=1)), np.sqrt((m * m).sum(axis=1))
    else:
        c = component if field == "component" else 0
        lo, hi = cmin[:, c], cmax[:, c]
    box = np.asarray(box, dtype=np.float64)
    w = box[:, 3:] - box[:, :3]
    ctr = 0.5 * (box[:, 3:] + box[:, :3])
    deg = int(max(orc.deg))
    ds = np.min(w, axis=1) * 2.0 ** -deg
    table = np.asarray(tf.table, dtype=np.float64).reshape(256, 4)
    xlo = (lo - tf.vmin) / (tf.vmax - tf.vmin)
    xhi = (hi - tf.vmin) / (tf.vmax - tf.vmin)
    i0 = np.floor(255 * np.clip(xlo, 0, 1)).astype(int)
    i1 = np.minimum(255, np.ceil(255 * np.clip(xhi, 0, 1)).astype(int))
    F = np.zeros((len(box), IN))
    F[:, 0:3] = np.log2(64 * w)
    F[:, 3], F[:, 4], F[:, 5] = xlo, xhi, xhi - xlo
    dalpha = np.abs(np.diff(table[:, 3]))
    for e in range(len(box)):
        seg = table[i0[e]:i1[e] + 1]
        F[e, 6] = seg[:, 3].max()
        F[e, 7] = seg[:, 3].mean()
        F[e, 8] = 255 * (dalpha[i0[e]:i1[e]].max() if i1[e] > i0[e] else 0.0)
        F[e, 9] = (seg[:, :3].max(axis=0) - seg[:, :3].min(axis=0)).max()
    dirv = ctr - np.asarray(cam.eye, dtype=np.float64)
    dirv /= np.linalg.norm(dirv, axis=1, keepdims=True)
    F[:, 10:13] = dirv
    F[:, 13] = np.log2(2048 * ds)
    F[:, 14] = (np.abs(dirv) * w).sum(axis=1) / (8 * ds)
    F[:, 15] = np.log2(1 + 255 * (xhi - xlo))
    return F

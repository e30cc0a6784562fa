"""Plain FP64 reference of the learned transfer function (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Same network and loss as the
library's surrogate, written directly from their definition: inputs x[n][4], layers
z1 = x W1 + b1, h = silu(z), three 256 x 256 layers, y = h4 W5 + b5; loss per row
BCE(y0, c) + m_x ((y1 - t1)^2 + (y2 - t2)^2) + m_g (y3 - t3)^2, averaged over rows.
Parameters are one flat vector: W1[4][256], b1[256], (W[256][256], b[256]) x 3,
W5[256][4], b5[4].
"""
from __future__ import annotations

import numpy as np

HID, NIN, NOUT = 256, 4, 4
SHAPES = [("W1", (NIN, HID)), ("b1", (HID,))]
for _l in (2, 3, 4):
    SHAPES += [(f"W{_l}", (HID, HID)), (f"b{_l}", (HID,))]
SHAPES += [("W5", (HID, NOUT)), ("b5", (NOUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(flat: np.ndarray, x: np.ndarray):
    """Outputs y[n][4] and the pre-activations / activations of the hidden layers."""
    P = unpack(flat)
    h = np.asarray(x, dtype=np.float64)
    zs, hs = [], [h]
    for l in (1, 2, 3, 4):
        z = h @ P[f"W{l}"] + P[f"b{l}"]
        h = _silu(z)
        zs.append(z)
        hs.append(h)
    y = h @ P["W5"] + P["b5"]
    return y, zs, hs


def loss(flat: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _, _ = forward(flat, x)
    c, mx, mg = t[:, 0], t[:, 4], t[:, 5]
    bce = np.maximum(y[:, 0], 0) - c * y[:, 0] + np.log1p(np.exp(-np.abs(y[:, 0])))
    sq = mx * ((y[:, 1] - t[:, 1]) ** 2 + (y[:, 2] - t[:, 2]) ** 2) + mg * (y[:, 3] - t[:, 3]) ** 2
    return float(np.mean(bce + sq))


def gradients(flat: np.ndarray, x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """dL/dparams by reverse-mode differentiation, in FP64."""
    P = unpack(flat)
    y, zs, hs = forward(flat, x)
    n = x.shape[0]
    c, mx, mg = t[:, 0], t[:, 4], t[:, 5]
    dy = np.empty_like(y)
    dy[:, 0] = 1.0 / (1.0 + np.exp(-y[:, 0])) - c
    dy[:, 1] = 2 * mx * (y[:, 1] - t[:, 1])
    dy[:, 2] = 2 * mx * (y[:, 2] - t[:, 2])
    dy[:, 3] = 2 * mg * (y[:, 3] - t[:, 3])
    dy /= n
    G = {"W5": hs[4].T @ dy, "b5": dy.sum(axis=0)}
    dh = dy @ P["W5"].T
    for l in (4, 3, 2, 1):
        dz = dh * _dsilu(zs[l - 1])
        G[f"W{l}"] = hs[l - 1].T @ dz
        G[f"b{l}"] = dz.sum(axis=0)
        dh = dz @ P[f"W{l}"].T
    return pack(G)

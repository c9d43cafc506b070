"""FP64 CPU oracle of the transmission surrogate's network (TEST INFRASTRUCTURE ONLY).

MLP 3 -> 256 -> 256 -> 256 -> 256 -> 1, tanh hidden layers, sigmoid output, loss mean((y - t)^2).
Parameters are one flat vector in the order W1[256][3], b1, W2[256][256], b2, W3, b3, W4, b4,
w5[256], b5.  With round_bf16=True the operands the GPU kernels round to BF16 are rounded here at the
same points (weights, hidden activations entering layers 2..5, and the layer gradients entering the
backward products); all arithmetic is FP64.  With round_bf16=False this is the plain FP64 network and
its gradient (pinned by finite differences in the tests).
"""
from __future__ import annotations

import numpy as np

IN, HID = 3, 256
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)), ("b3", (HID,)),
          ("W4", (HID, HID)), ("b4", (HID,)), ("w5", (HID,)), ("b5", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(params):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(params[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(a):
    """Round to the nearest bfloat16 (ties to even) through float32, as the GPU's float->bf16 conversion."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grad(params, x, t, round_bf16=True):
    """(loss, gradient vector) of mean((y - t)^2) for inputs x [B][3] and targets t [B]."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    h = [np.tanh(x @ r(p["W1"]).T + p["b1"])]
    for l in (2, 3, 4):
        h.append(np.tanh(r(h[-1]) @ r(p["W%d" % l]).T + p["b%d" % l]))
    z5 = r(h[3]) @ r(p["w5"]) + p["b5"][0]
    y = 1.0 / (1.0 + np.exp(-z5))
    loss = float(np.mean((y - t) ** 2))
    g = {}
    dz5 = 2.0 * (y - t) / B * y * (1.0 - y)
    g["w5"] = r(h[3]).T @ dz5
    g["b5"] = np.array([dz5.sum()])
    dh = np.outer(dz5, r(p["w5"]))
    for l in (4, 3, 2):
        dz = dh * (1.0 - h[l - 1] ** 2)
        g["W%d" % l] = r(dz).T @ r(h[l - 2])
        g["b%d" % l] = dz.sum(axis=0)
        dh = r(dz) @ r(p["W%d" % l])
    dz1 = dh * (1.0 - h[0] ** 2)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def predict(params, x, round_bf16=True):
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(params)
    h = np.tanh(np.asarray(x, dtype=np.float64) @ r(p["W1"]).T + p["b1"])
    for l in (2, 3, 4):
        h = np.tanh(r(h) @ r(p["W%d" % l]).T + p["b%d" % l])
    return 1.0 / (1.0 + np.exp(-(r(h) @ r(p["w5"]) + p["b5"][0])))

"""FP64 CPU reference of the surrogate network (test infrastructure only).

Same architecture and parameter layout as the CUDA network (in 64 -> 256 ->
256 -> 256 -> 1, ReLU; weight matrices stored [out][in]; flat layout W1, b1,
W2, b2, W3, b3, w4, b4, 7 floats padding), evaluated in float64 with the
weights rounded to BF16 the way the device copy is (round to nearest even).
Forward, mean-squared-error loss and its gradient by plain backpropagation.
"""
from __future__ import annotations

import numpy as np

IN, H = 64, 256
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("w4", (H,)), ("b4", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES) + 7


def bf16_round(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(flat, round_weights=True):
    flat = np.asarray(flat)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        v = flat[o:o + k].reshape(shape).astype(np.float64)
        if round_weights and name.startswith(("W", "w")):
            v = bf16_round(flat[o:o + k].astype(np.float32)).reshape(shape)
        out[name] = v
        o += k
    return out


def _r(x, on):
    return bf16_round(np.asarray(x, dtype=np.float32)) if on else x


def forward(p, X, storage_bf16=False):
    """X [B, 64] float64 -> (y [B], cache). With storage_bf16 the hidden
    activations are rounded to BF16 where the device stores them."""
    z1 = X @ p["W1"].T + p["b1"]
    h1 = _r(np.maximum(z1, 0), storage_bf16)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = _r(np.maximum(z2, 0), storage_bf16)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = _r(np.maximum(z3, 0), storage_bf16)
    y = h3 @ p["w4"] + p["b4"][0]
    return y, (X, h1, h2, h3)


def loss_and_grad(p, X, t, storage_bf16=False):
    """Mean squared error and its gradient with respect to every parameter.
    With storage_bf16 the backward operands of the matrix products are rounded
    to BF16 where the device stores them (bias gradients use unrounded values)."""
    y, (X, h1, h2, h3) = forward(p, X, storage_bf16)
    B = X.shape[0]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    g = {"w4": h3.T @ dy, "b4": np.array([dy.sum()])}
    dz3 = np.outer(dy, p["w4"]) * (h3 > 0)
    g["b3"] = dz3.sum(0)
    dz3 = _r(dz3, storage_bf16)
    g["W3"] = dz3.T @ h2
    dz2 = (dz3 @ p["W3"]) * (h2 > 0)
    g["b2"] = dz2.sum(0)
    dz2 = _r(dz2, storage_bf16)
    g["W2"] = dz2.T @ h1
    dz1 = (dz2 @ p["W2"]) * (h1 > 0)
    g["b1"] = dz1.sum(0)
    dz1 = _r(dz1, storage_bf16)
    g["W1"] = dz1.T @ X
    return loss, g


def pack(g) -> np.ndarray:
    parts = [np.asarray(g[name], dtype=np.float64).ravel() for name, _ in SHAPES]
    return np.concatenate(parts + [np.zeros(7)])

"""Plain FP64 numpy MLP of the learned collide (test infrastructure only).

Network: 37 -> 128 -> 128 -> 37 with GELU (x * Phi(x), Phi the standard normal CDF written with
erf) after the two hidden layers; loss = mean squared error over samples and the 37 outputs.
Parameters are packed W1[128][37] b1[128] W2[128][128] b2[128] W3[37][128] b3[37].

With bf16=True the forward and backward passes round to bfloat16 exactly where a tensor-core
implementation with BF16 operands must (inputs, weights, hidden activations, and the output and
hidden gradients that feed products), so that its results can be compared at the level of FP32
accumulation differences. Only tests/, the smoke check and the benchmark's baseline leg use this.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

NIN, HID, NOUT = 37, 128, 37
SIZES = [("W1", (HID, NIN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (NOUT, HID)),
         ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, off = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, x, bf16=False):
    w = unpack(p)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x_ = r(x)
    z1 = x_ @ r(w["W1"]).T + w["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ r(w["W2"]).T + w["b2"]
    h2 = r(gelu(z2))
    y = h2 @ r(w["W3"]).T + w["b3"]
    return y, (x_, z1, h1, z2, h2)


def loss_grad(p, x, t, bf16=False):
    """(loss, packed gradient) of mean((network(x) - t)^2)."""
    w = unpack(p)
    r = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, (x_, z1, h1, z2, h2) = forward(p, x, bf16)
    n = x.shape[0]
    e = y - t
    loss = float(np.mean(e * e))
    dy = 2.0 * e / (n * NOUT)
    dy_ = r(dy)
    g = {"b3": dy.sum(0), "W3": dy_.T @ h2}
    dz2 = (dy_ @ r(w["W3"])) * gelu_grad(z2)
    dz2_ = r(dz2)
    g["b2"] = dz2.sum(0)
    g["W2"] = dz2_.T @ h1
    dz1 = (dz2_ @ r(w["W2"])) * gelu_grad(z1)
    g["b1"] = dz1.sum(0)
    g["W1"] = r(dz1).T @ x_
    return loss, pack(g)


def init_params(seed=0, scale=1.0):
    """Uniform +-scale/sqrt(fan_in) weights and biases (seeded numpy generator)."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        fan_in = NIN if name in ("W1", "b1") else HID
        d[name] = rng.uniform(-1, 1, shape) * scale / np.sqrt(fan_in)
    return pack(d)

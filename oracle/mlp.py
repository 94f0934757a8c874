"""fp64 numpy reference of the learned-proposal network (not in the paper).

TEST INFRASTRUCTURE ONLY.  MLP 6 -> 64 -> 64 -> 256 with exact (erf) GELU;
the weights it uses are the BF16-rounded parameters (round to nearest
even), evaluated in float64.  Loss: mean cross-entropy of the 256 logits.
Parameter layout: W1[64][6], b1[64], W2[64][64], b2[64], W3[256][64],
b3[256] (P = 21248 floats).  Pinned against central finite differences in
tests/test_oracle_mlp.py.
"""
from __future__ import annotations

import math

import numpy as np

IN, H, OUT = 6, 64, 256
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
          ("W3", (OUT, H)), ("b3", (OUT,))]
P = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf, otypes=[np.float64])


def bf16_round(w) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def unpack(flat) -> dict:
    out, off = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(flat[off:off + k], np.float64).reshape(shape)
        off += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[n], np.float64).reshape(-1) for n, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-style uniform initialisation (float32 master weights)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in SHAPES:
        if name.startswith("W"):
            fan_in = shape[1]
            lim = math.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, shape).reshape(-1))
        else:
            parts.append(np.zeros(shape).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def features(rays, box) -> np.ndarray:
    r = np.asarray(rays, np.float64).reshape(-1, 8)
    b = np.asarray(box, np.float64)
    return np.concatenate([(r[:, :3] - b[:3]) / b[3:], r[:, 4:7]], axis=1)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def forward(p: dict, X: np.ndarray):
    a1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    z = h2 @ p["W3"].T + p["b3"]
    return a1, h1, a2, h2, z


def loss_and_grad(flat_bf16, X, y):
    """Mean cross-entropy and its gradient (float64 backprop)."""
    p = unpack(flat_bf16)
    a1, h1, a2, h2, z = forward(p, X)
    B = X.shape[0]
    m = z.max(1, keepdims=True)
    e = np.exp(z - m)
    s = e.sum(1, keepdims=True)
    loss = float(np.mean(np.log(s[:, 0]) + m[:, 0] - z[np.arange(B), y]))
    dz = e / s
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    da2 = (dz @ p["W3"]) * gelu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    da1 = (da2 @ p["W2"]) * gelu_grad(a1)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return loss, pack(g)


def loss_only(flat, X, y) -> float:
    p = unpack(flat)
    z = forward(p, X)[-1]
    m = z.max(1, keepdims=True)
    return float(np.mean(np.log(np.exp(z - m).sum(1)) + m[:, 0] - z[np.arange(len(y)), y]))


def logits_bf16_activations(flat_bf16, X) -> np.ndarray:
    """Logits when the hidden activations enter layers 2 and 3 rounded to
    BF16 (round to nearest even) -- the tensor-core form of the forward."""
    p = unpack(flat_bf16)
    h1 = gelu(X @ p["W1"].T + p["b1"])
    h1 = bf16_round(h1.astype(np.float32)).astype(np.float64)
    h2 = gelu(h1 @ p["W2"].T + p["b2"])
    h2 = bf16_round(h2.astype(np.float32)).astype(np.float64)
    return h2 @ p["W3"].T + p["b3"]


def top1(flat_bf16, X) -> np.ndarray:
    return forward(unpack(flat_bf16), X)[-1].argmax(1)


def _bf(x) -> np.ndarray:
    return bf16_round(np.asarray(x, np.float64).astype(np.float32)).astype(np.float64)


def loss_and_grad_bf16_operands(flat_bf16, X, y):
    """Mean cross-entropy and its gradient when every operand of a product
    is rounded to BF16 (round to nearest even) and everything else is exact
    -- the tensor-core form of the training step: the hidden activations
    entering layers 2 and 3, dZ, dA2 and dA1 entering the weight-gradient and
    hidden-backward products, and the input features entering dW1.  Bias
    gradients are sums of the rounded dZ / dA (a column of ones in the
    product)."""
    p = unpack(flat_bf16)
    B = X.shape[0]
    a1 = X @ p["W1"].T + p["b1"]
    h1 = _bf(gelu(a1))
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = _bf(gelu(a2))
    z = h2 @ p["W3"].T + p["b3"]
    m = z.max(1, keepdims=True)
    e = np.exp(z - m)
    s = e.sum(1, keepdims=True)
    loss = float(np.mean(np.log(s[:, 0]) + m[:, 0] - z[np.arange(B), y]))
    dz = e / s
    dz[np.arange(B), y] -= 1.0
    dz = _bf(dz / B)
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    da2 = _bf((dz @ p["W3"]) * gelu_grad(a2))
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    da1 = _bf((da2 @ p["W2"]) * gelu_grad(a1))
    g["W1"] = da1.T @ _bf(X)
    g["b1"] = da1.sum(0)
    return loss, pack(g)

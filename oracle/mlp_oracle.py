"""FP64 reference of the warm-start network and its gradient (test infrastructure).

y = w3 . silu(W2 silu(W1 x + b1) + b2) + b3,  silu(z) = z / (1 + exp(-z)),
L = scale * sum_r (y_r - t_r)^2.

`bf16=True` rounds to bfloat16 exactly the operands the tensor-core kernels read as
bfloat16 (features, W1, W2, the first hidden layer, and in the backward pass the hidden
gradients dZ2 and dZ1 that enter the weight-gradient GEMMs); all arithmetic stays FP64.
`bf16=False` is the plain FP64 network (its gradient is pinned to central differences in
tests/test_mlp_oracle.py).

Parameter vector: W1 [128][24], b1 [128], W2 [128][128], b2 [128], w3 [128], b3.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 24, 128
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def bf16(a):
    """Round to the nearest bfloat16, ties to even (through float32)."""
    f = np.asarray(a, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    finite = (u & 0x7F800000) != 0x7F800000
    u = np.where(finite, u + 0x7FFF + ((u >> 16) & 1), u) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed=0):
    """He-style initialisation of the FP32 master parameters."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2.0 / N_IN), (N_HID, N_IN)), "b1": np.zeros(N_HID),
         "W2": rng.normal(0, np.sqrt(2.0 / N_HID), (N_HID, N_HID)), "b2": np.zeros(N_HID),
         "w3": rng.normal(0, np.sqrt(1.0 / N_HID), N_HID), "b3": np.zeros(1)}
    return pack(d).astype(np.float32).astype(np.float64)


def forward(p, x, bf16_ops=True):
    P = unpack(p)
    r = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    x = r(x)
    z1 = x @ r(P["W1"]).T + P["b1"]
    h1 = r(silu(z1))
    z2 = h1 @ r(P["W2"]).T + P["b2"]
    h2 = silu(z2)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (x, z1, h1, z2, h2)


def loss_and_grad(p, x, t, scale, bf16_ops=True):
    P = unpack(p)
    r = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    y, (xr, z1, h1, z2, h2) = forward(p, x, bf16_ops)
    res = y - t
    L = scale * np.sum(res ** 2)
    g = 2.0 * scale * res
    dz2 = g[:, None] * P["w3"][None, :] * dsilu(z2)
    dz2r = r(dz2)
    dh1 = dz2r @ r(P["W2"])
    dz1 = dh1 * dsilu(z1)
    grad = {"W1": r(dz1).T @ xr, "b1": dz1.sum(0), "W2": dz2r.T @ h1, "b2": dz2.sum(0),
            "w3": g @ h2, "b3": np.array([g.sum()])}
    return L, pack(grad)


def training_rows(node_off, mass, feat, lam_star, lam_prev, beta, h, g=9.81):
    """Training rows of the learned warm start (test infrastructure).

    The warm start of a substep is lambda0 = beta lambda_prev + m g h^2 y with y the
    network's output (the oracle's snake_step), so the output that makes it land on a
    reference solution lambda_star is y* = (lambda_star - beta lambda_prev) / (m g h^2).
    For every row whose features carry a row kind (a one-hot entry among the first six),
    snake by snake and node by node with the kinds in order, returns the row's features
    and y*.  node_off: [snakes + 1]; mass: [snakes]; feat: [nodes * 6, >= 24] in node
    order; lam_star, lam_prev: [nodes, 6]."""
    F, T = [], []
    for s in range(len(node_off) - 1):
        sc = float(mass[s]) * g * h * h
        for i in range(int(node_off[s]), int(node_off[s + 1])):
            for k in range(6):
                r = 6 * i + k
                if not np.any(feat[r, :6] != 0):
                    continue
                F.append(feat[r])
                T.append((float(lam_star[i, k]) - beta * float(lam_prev[i, k])) / sc)
    return np.array(F), np.array(T)

"""FP64 reference of the learned Newton starting guess for p* (test infrastructure).

Not in the paper: the two-shock Riemann solver of Sec. 4.1.2 iterates on p*,
and this small network predicts the starting point.  The plain guess and the
converged Newton iteration still decide the answer.

Network: 6 -> 64 -> 64 -> 1 with SiLU activations, predicting
y = ln(p* / p_ref).  Inputs use the Riemann problem's invariances under
density and pressure scaling and Galilean shifts:
    rho_ref = sqrt(rho_L rho_R), p_ref = sqrt(p_L p_R),
    c_ref = sqrt(gamma p_ref / rho_ref), u_bar = (u_L + u_R) / 2,
    x = (ln rho_L/rho_ref, (u_L - u_bar)/c_ref, ln p_L/p_ref,
         ln rho_R/rho_ref, (u_R - u_bar)/c_ref, ln p_R/p_ref).
Loss: mean squared error.  Optimiser: Adam on FP32 master weights (here FP64).

Plain numpy, FP64, one function per step, no fusion.  Parity: pinned by
central finite differences of the loss (gradients), the closed-form first Adam
step, the invariances of the features, and convergence on a known target.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
NIN = 6


def features(rl, ul, pl, rr, ur, pr, gamma):
    rl, ul, pl, rr, ur, pr = (np.asarray(a, dtype=np.float64) for a in (rl, ul, pl, rr, ur, pr))
    rho_ref = np.sqrt(rl * rr)
    p_ref = np.sqrt(pl * pr)
    c_ref = np.sqrt(gamma * p_ref / rho_ref)
    ubar = 0.5 * (ul + ur)
    x = np.stack([np.log(rl / rho_ref), (ul - ubar) / c_ref, np.log(pl / p_ref),
                  np.log(rr / rho_ref), (ur - ubar) / c_ref, np.log(pr / p_ref)], axis=1)
    return x, p_ref


def target(pstar, pl, pr):
    """y = ln(p* / sqrt(p_L p_R))."""
    return np.log(np.asarray(pstar, dtype=np.float64) / np.sqrt(np.asarray(pl) * np.asarray(pr)))


def init(seed=0):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0.0, np.sqrt(2.0 / NIN), (HIDDEN, NIN)),
        "b1": np.zeros(HIDDEN),
        "W2": rng.normal(0.0, np.sqrt(2.0 / HIDDEN), (HIDDEN, HIDDEN)),
        "b2": np.zeros(HIDDEN),
        "w3": rng.normal(0.0, np.sqrt(1.0 / HIDDEN), HIDDEN),
        "b3": np.zeros(1),
    }


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(P, x):
    """Returns (y [N], cache)."""
    z1 = x @ P["W1"].T + P["b1"]
    h1 = silu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = silu(z2)
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (x, z1, h1, z2, h2)


def mse(y, t):
    d = y - t
    return float(np.mean(d * d))


def backward(P, cache, y, t):
    """Gradients of the MSE loss with respect to every parameter."""
    x, z1, h1, z2, h2 = cache
    n = y.shape[0]
    dy = 2.0 * (y - t) / n
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dh2 = np.outer(dy, P["w3"])
    dz2 = dh2 * silu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * silu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_init(P):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in P.items()},
            "v": {k: np.zeros_like(v) for k, v in P.items()}}


def adam_step(P, g, S, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    S["t"] += 1
    t = S["t"]
    for k in P:
        S["m"][k] = beta1 * S["m"][k] + (1.0 - beta1) * g[k]
        S["v"][k] = beta2 * S["v"][k] + (1.0 - beta2) * g[k] * g[k]
        mhat = S["m"][k] / (1.0 - beta1 ** t)
        vhat = S["v"][k] / (1.0 - beta2 ** t)
        P[k] = P[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return P


def bf16(a):
    """Round float64 values to bfloat16 (round to nearest even) and back."""
    f = np.asarray(a, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(P, x):
    """Forward pass with the precisions of the tensor-core path: weights and
    layer inputs rounded to bfloat16, products accumulated in high precision."""
    z1 = bf16(x) @ bf16(P["W1"]).T + P["b1"]
    h1 = silu(z1)
    z2 = bf16(h1) @ bf16(P["W2"]).T + P["b2"]
    h2 = silu(z2)
    return h2 @ P["w3"] + P["b3"][0]


def guess(P, rl, ul, pl, rr, ur, pr, gamma):
    """Starting guess p0 = p_ref exp(y)."""
    x, p_ref = features(rl, ul, pl, rr, ur, pr, gamma)
    y, _ = forward(P, x)
    return p_ref * np.exp(y)

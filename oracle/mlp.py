"""Rank model: a small MLP that predicts per-level probe counts (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

The paper notes that the number of Hessian-vector products per level is C_l k
and that tuning the sampling to the structure of the Hessian pays (Section 3.3);
the learned part predicts, from level, box geometry and operator parameters,
the probe count that adaptive peeling would choose, so that peeling can start
there (adaptive growth remains the fallback and decides the error).

Model: x (F = 8 features) -> z1 = W1 x + b1 -> h1 = gelu(z1) -> z2 = W2 h1 + b2
-> h2 = gelu(z2) -> y = W3 h2 + b3, width 64, gelu in its tanh form
gelu(u) = u/2 (1 + tanh(c (u + 0.044715 u^3))), c = sqrt(2/pi).  Loss: mean
squared error.  Optimiser: Adam (Kingma and Ba 2015).  With bf16 = True the
weights used in the forward and backward passes are the master weights rounded
to bfloat16 (round to nearest even); arithmetic is FP64 here.

Parameter vector order: W1 (64 x F, row-major), b1, W2 (64 x 64, row-major),
b2, W3 (64), b3.
"""
from __future__ import annotations

import numpy as np

F = 8
H = 64
NPARAM = H * F + H + H * H + H + H + 1
C_GELU = float(np.sqrt(2.0 / np.pi))


def split(p: np.ndarray):
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def to_bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) through the float32 bit pattern."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(u):
    return 0.5 * u * (1.0 + np.tanh(C_GELU * (u + 0.044715 * u ** 3)))


def gelu_grad(u):
    t = np.tanh(C_GELU * (u + 0.044715 * u ** 3))
    return 0.5 * (1.0 + t) + 0.5 * u * (1.0 - t * t) * C_GELU * (1.0 + 3.0 * 0.044715 * u * u)


def effective(p: np.ndarray, bf16: bool) -> np.ndarray:
    return to_bf16(p) if bf16 else np.asarray(p, dtype=np.float64)


def forward(p, X, bf16=False):
    W1, b1, W2, b2, W3, b3 = split(effective(p, bf16))
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    return H2 @ W3 + b3[0], (Z1, H1, Z2, H2)


def loss_and_grad(p, X, t, bf16=False):
    """MSE loss and its gradient with respect to the (effective) parameters."""
    W1, b1, W2, b2, W3, b3 = split(effective(p, bf16))
    y, (Z1, H1, Z2, H2) = forward(p, X, bf16)
    B = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    gW3 = H2.T @ dy
    gb3 = np.array([dy.sum()])
    dZ2 = np.outer(dy, W3) * gelu_grad(Z2)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])
    return loss, g


def adam_step(p, m, v, g, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected first and second moments)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def level_features(tree, kappa_T: float, density: float, tol: float) -> np.ndarray:
    """Features of every level l = 0..L of a cluster tree (row l):
    l/L, log2(mean box size)/20, mean box diameter / root diameter, log10(kappa T)/4,
    sensor density, log10(tol)/10, log10(sqrt(kappa T) / mean box diameter)/2, log2(N)/20."""
    L = tree.L
    root = float(np.linalg.norm(tree.hi[0][0] - tree.lo[0][0]))
    root = root if root > 0 else 1.0
    out = np.zeros((L + 1, F))
    for l in range(L + 1):
        diam = float(np.mean(np.linalg.norm(tree.hi[l] - tree.lo[l], axis=1)))
        size = float(np.mean(tree.sizes[l]))
        out[l] = [l / max(L, 1), np.log2(size) / 20.0, diam / root, np.log10(kappa_T) / 4.0, density,
                  np.log10(tol) / 10.0, np.log10(np.sqrt(kappa_T) / max(diam, 1e-300)) / 2.0,
                  np.log2(tree.N) / 20.0]
    return out


def q_start_from_prediction(y: float, pad: int, q_max: int) -> int:
    """Probe count to start from: ceil(2^y) - 1 + pad, rounded up to a multiple of 8, in [8, q_max]."""
    q = int(np.ceil(2.0 ** y)) - 1 + pad
    q = (q + 7) // 8 * 8
    return int(min(max(q, 8), q_max))

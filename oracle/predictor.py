"""FP64 reference of the learned learning-signal predictor -- TEST
INFRASTRUCTURE ONLY (the CUDA library never imports it).

The predictor is not part of the paper.  It is a small MLP that maps the
network's per-step state to an estimate of the error signal E_k^t (Methods,
"Loss function": E_k = pi_k - pi*_k for softmax cross-entropy), so that the
learning signal L_j = sum_k B_jk E_k (Methods, "Gradients") can be formed
before a sample's target window opens.

State x^t (74 values per sample and step):
    x[0:K]      readout potentials y_k^t (Eq. leaky_integrator), K = 10
    x[K:K+64]   population rates r_g^t = G_beta of the group's mean spike
                count, r_g^t = beta r_g^{t-1} + (1 - beta) mean_{j: j mod 64
                = g} z_j^t (the exponential moving average of Eq. ema-rate,
                beta = exp(-dt / 20 ms)), in spikes per 1000 steps (x 1000,
                the paper's rate unit).
Network: 74 -> 256 -> 256 -> K, GELU(x) = x Phi(x) between layers (exact erf
form), trained with the mean squared error (1 / (2 R)) sum (Y - E)^2 over a
batch of R rows by Adam (Eq. adam1, Eq. adam2, Eq. adam).

The BF16 form rounds to BF16 (round to nearest even) at fixed points:
inputs, weights, hidden activations after GELU, and the backward deltas
that enter a matrix product; every product accumulates in FP32.  The
functions below give the FP64 definition of each step; `bf16` applies the
rounding where a test needs the BF16 operands themselves.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

N_IN_POP = 64
HIDDEN = 256


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as
    float32 (the BF16 value exactly)."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).reshape(a.shape)
    nan = np.isnan(a)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out


def gelu(x):
    """x Phi(x), Phi(x) = (1 + erf(x / sqrt 2)) / 2 written as erfc(-x / sqrt
    2) / 2 (no cancellation in the lower tail)."""
    x = np.asarray(x, np.float64)
    return 0.5 * x * erfc(-x / math.sqrt(2.0))


def gelu_grad(x):
    """Phi(x) + x phi(x)."""
    x = np.asarray(x, np.float64)
    return 0.5 * erfc(-x / math.sqrt(2.0)) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def init_params(n_in, n_out, seed=0, hidden=HIDDEN):
    """Weights N(0, 1/fan_in), zero biases (FP32 masters)."""
    rng = np.random.default_rng(seed)
    p = {}
    dims = [(n_in, hidden), (hidden, hidden), (hidden, n_out)]
    for i, (a, b) in enumerate(dims, 1):
        p[f"W{i}"] = (rng.standard_normal((a, b)) / math.sqrt(a)).astype(np.float32)
        p[f"b{i}"] = np.zeros(b, np.float32)
    return p


def forward(p, X):
    """FP64 forward pass; returns the output and the pre-activations."""
    X = np.asarray(X, np.float64)
    A1 = X @ p["W1"].astype(np.float64) + p["b1"]
    H1 = gelu(A1)
    A2 = H1 @ p["W2"].astype(np.float64) + p["b2"]
    H2 = gelu(A2)
    Y = H2 @ p["W3"].astype(np.float64) + p["b3"]
    return Y, dict(X=X, A1=A1, H1=H1, A2=A2, H2=H2)


def loss(Y, E):
    R = Y.shape[0]
    return 0.5 * float(((np.asarray(Y, np.float64) - E) ** 2).sum()) / R


def backward(p, cache, Y, E):
    """Gradients of `loss` w.r.t. every parameter (chain rule, FP64)."""
    R = Y.shape[0]
    dY = (np.asarray(Y, np.float64) - E) / R
    g = {"W3": cache["H2"].T @ dY, "b3": dY.sum(0)}
    dA2 = (dY @ p["W3"].astype(np.float64).T) * gelu_grad(cache["A2"])
    g["W2"] = cache["H1"].T @ dA2
    g["b2"] = dA2.sum(0)
    dA1 = (dA2 @ p["W2"].astype(np.float64).T) * gelu_grad(cache["A1"])
    g["W1"] = cache["X"].T @ dA1
    g["b1"] = dA1.sum(0)
    return g


def adam_step(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Eq. adam1, Eq. adam2, Eq. adam) in FP64; t counts
    from 1.  Returns the new (param, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def population_rates(raster, beta, groups=N_IN_POP):
    """r [B, T, groups]: r^t = beta r^{t-1} + (1 - beta) mean_{j mod groups
    = g} z_j^t, r^0 = 0 (Eq. ema-rate on the group-mean spike count)."""
    raster = np.asarray(raster, np.float64)
    B, T, N = raster.shape
    cnt = np.zeros((B, T, groups))
    size = np.zeros(groups)
    for g in range(groups):
        idx = np.arange(g, N, groups)
        size[g] = len(idx)
        if len(idx):
            cnt[:, :, g] = raster[:, :, idx].sum(axis=2)
    mean = cnt / np.maximum(size, 1.0)
    r = np.zeros((B, T, groups))
    prev = np.zeros((B, groups))
    for t in range(T):
        prev = beta * prev + (1.0 - beta) * mean[:, t]
        r[:, t] = prev
    return r


def softmax_error(y, onehot):
    """E = softmax(y) - pi* per row (Methods, "Loss function")."""
    y = np.asarray(y, np.float64)
    e = np.exp(y - y.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True) - onehot

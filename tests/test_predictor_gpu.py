"""Learned learning-signal predictor on the GPU vs the FP64 reference.

Each matrix product is checked on the GPU's own BF16 operands (read back
from the library) against FP64: FP32 accumulation of K products carries at
most K 2^-23 of the magnitude sum sum |a||b| (tensor-core accumulation,
truncation allowed), so |gpu - ref| <= (K + 2) 2^-23 (sum |a||b| + |bias|).
Element-wise BF16 roundings (GELU outputs, deltas) are checked within one
BF16 ulp (2^-8 relative) of the FP64 value of the same FP32 inputs; the
Adam step within FP32 rounding of the FP64 update.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import predictor as P

pytestmark = pytest.mark.gpu

U23 = 2.0 ** -23


def _gemm_check(gpu, A, B, bias, what):
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    ref = A @ B + (0.0 if bias is None else np.asarray(bias, np.float64))
    mag = np.abs(A) @ np.abs(B) + (0.0 if bias is None else np.abs(np.asarray(bias, np.float64)))
    tol = (A.shape[1] + 2) * U23 * mag + 1e-30
    err = np.abs(np.asarray(gpu, np.float64) - ref)
    bad = err > tol
    assert not bad.any(), f"{what}: {int(bad.sum())}/{bad.size} outside; worst {float((err / tol).max()):.3g}"
    return float((err / tol).max())


def _bf16_check(gpu, ref64, what, slack=None):
    ref64 = np.asarray(ref64, np.float64)
    tol = 2.0 ** -8 * np.abs(ref64) + (0.0 if slack is None else slack) + 1e-37
    err = np.abs(np.asarray(gpu, np.float64) - ref64)
    bad = err > tol
    assert not bad.any(), f"{what}: {int(bad.sum())}/{bad.size} outside one BF16 ulp"
    # most values are the exact BF16 rounding of the FP64 value
    exact = np.mean(np.asarray(gpu, np.float32) == P.bf16(ref64.astype(np.float32)))
    return exact


def _setup(R=300, seed=7, n_in=74, n_out=10):
    import paper_2511_21674_gb300 as ep
    p = P.init_params(n_in, n_out, seed=seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = (rng.standard_normal(p[k].shape) * 0.1).astype(np.float32)
    X = np.concatenate([rng.standard_normal((R, 10)) * 2.0, rng.uniform(0, 0.05, (R, n_in - 10))],
                       axis=1).astype(np.float32)
    E = (rng.standard_normal((R, n_out)) * 0.3).astype(np.float32)
    pred = ep.Predictor(n_in, n_out, params=ep.Predictor.pack(p), max_rows=512)
    return p, X, E, pred


def test_forward_layers_match_fp64_on_bf16_operands():
    p, X, E, pred = _setup()
    Y = pred.forward(X)
    Xb = pred.read("X")
    assert np.array_equal(Xb, P.bf16(X))
    Wb = {k: P.bf16(p[k]) for k in ("W1", "W2", "W3")}
    A1, H1, A2, H2, Yr = (pred.read(k) for k in ("A1", "H1", "A2", "H2", "Y"))
    assert np.array_equal(Yr, Y)
    _gemm_check(A1, Xb, Wb["W1"], p["b1"], "A1")
    ex1 = _bf16_check(H1, P.gelu(A1), "H1")
    _gemm_check(A2, H1, Wb["W2"], p["b2"], "A2")
    ex2 = _bf16_check(H2, P.gelu(A2), "H2")
    _gemm_check(Y, H2, Wb["W3"], p["b3"], "Y")
    assert ex1 > 0.99 and ex2 > 0.99
    pred.close()


def test_train_step_gradients_and_adam_match_fp64():
    p, X, E, pred = _setup(R=257, seed=11)
    flat0 = pred.read("params").astype(np.float64)
    lr = 1e-3
    loss = pred.train_step(X, E, lr)
    R = X.shape[0]
    Xb, A1, H1, A2, H2, Y = (pred.read(k) for k in ("X", "A1", "H1", "A2", "H2", "Y"))
    dY, dA2, dA1 = pred.read("dY"), pred.read("dA2"), pred.read("dA1")
    g = pred.unpack(pred.read("grads"))
    Wb = {k: P.bf16(p[k]) for k in ("W1", "W2", "W3")}
    # loss and output delta
    d = Y.astype(np.float64) - E
    lref = 0.5 * float((d * d).sum()) / R
    assert abs(loss - lref) <= 1e-5 * lref
    _bf16_check(dY, d / R, "dY", slack=2 * U23 * np.abs(Y) / R)
    # readout layer
    _gemm_check(g["W3"], H2.T, dY, None, "dW3")
    np.testing.assert_allclose(g["b3"], (d / R).sum(0), rtol=0, atol=(R + 2) * U23 * (np.abs(d) / R).sum(0).max())
    # hidden layers: deltas from the GPU's BF16 operands, GELU' at the GPU's pre-activations
    dH2 = dY.astype(np.float64) @ Wb["W3"].astype(np.float64).T
    mag2 = np.abs(dY) @ np.abs(Wb["W3"]).T
    _bf16_check(dA2, dH2 * P.gelu_grad(A2), "dA2",
                slack=(Wb["W3"].shape[1] + 2) * U23 * mag2 * np.abs(P.gelu_grad(A2)))
    _gemm_check(g["W2"], H1.T, dA2, None, "dW2")
    dH1 = dA2.astype(np.float64) @ Wb["W2"].astype(np.float64).T
    mag1 = np.abs(dA2) @ np.abs(Wb["W2"]).T
    _bf16_check(dA1, dH1 * P.gelu_grad(A1), "dA1",
                slack=(Wb["W2"].shape[1] + 2) * U23 * mag1 * np.abs(P.gelu_grad(A1)))
    _gemm_check(g["W1"], Xb.T, dA1, None, "dW1")
    # Adam's first step from the GPU's gradients
    gflat = pred.read("grads").astype(np.float64)
    w1, m1, v1 = P.adam_step(flat0, gflat, np.zeros_like(gflat), np.zeros_like(gflat), 1, lr)
    flat1 = pred.read("params").astype(np.float64)
    tol = 4 * U23 * (np.abs(flat0) + lr)
    err = np.abs(flat1 - w1)
    q = int(np.argmax(err / tol))
    assert err[q] <= tol[q], (f"Adam step: element {q} w0={flat0[q]:.9g} g={gflat[q]:.6g} "
                              f"gpu={flat1[q]:.9g} ref={w1[q]:.9g} ({int((err > tol).sum())} outside)")
    np.testing.assert_allclose(pred.read("m"), m1, rtol=1e-6, atol=1e-30)
    np.testing.assert_allclose(pred.read("v"), v1, rtol=1e-5, atol=1e-37)
    pred.close()


def test_training_fits_a_smooth_target():
    import paper_2511_21674_gb300 as ep
    rng = np.random.default_rng(3)
    n_in, n_out = 74, 10
    M = rng.standard_normal((n_in, n_out)) * 0.3
    X = rng.standard_normal((4096, n_in)).astype(np.float32)
    E = np.tanh(X @ M).astype(np.float32)
    pred = ep.Predictor(n_in, n_out, seed=5, max_rows=256)
    first = pred.train_step(X[:256], E[:256], 1e-3)
    for it in range(400):
        lo = (it * 256) % 4096
        last = pred.train_step(X[lo:lo + 256], E[lo:lo + 256], 1e-3)
    assert last < 0.1 * first, (first, last)
    pred.close()

"""Pins of the FP64 predictor reference (no GPU): library special cases,
finite differences and closed forms, so that a dropped term or a wrong
transpose in `oracle.predictor` fails here."""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import predictor as P


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32) * 10.0 ** rng.integers(-20, 20, 10000),
                        np.array([0.0, -0.0, 1.0, 3.0e38, -1e-40], np.float32)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(P.bf16(x), ref)
    # halfway cases: 1 + 2^-8 rounds down to 1 (even), 1 + 3 * 2^-8 up to 1 + 2^-6
    assert P.bf16(np.float32(1.0 + 2.0 ** -8)) == np.float32(1.0)
    assert P.bf16(np.float32(1.0 + 3 * 2.0 ** -8)) == np.float32(1.0 + 2.0 ** -6)


def test_gelu_is_x_times_normal_cdf_and_its_derivative():
    x = np.linspace(-8, 8, 2001)
    np.testing.assert_allclose(P.gelu(x), x * ndtr(x), rtol=1e-13, atol=1e-300)
    h = 1e-5
    fd = (P.gelu(x + h) - P.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(P.gelu_grad(x), fd, rtol=1e-8, atol=1e-9)


def _small(seed=3):
    p = P.init_params(5, 3, seed=seed, hidden=7)
    rng = np.random.default_rng(seed)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape).astype(np.float32) * 0.3
    X = rng.standard_normal((4, 5))
    E = rng.standard_normal((4, 3))
    return p, X, E


def test_backward_matches_central_differences():
    p, X, E = _small()
    Y, cache = P.forward(p, X)
    g = P.backward(p, cache, Y, E)
    h = 1e-6
    for k, v in p.items():
        fd = np.zeros(v.shape)
        for idx in np.ndindex(v.shape):
            q = {kk: vv.astype(np.float64).copy() for kk, vv in p.items()}
            q[k][idx] += h
            lp = P.loss(P.forward(q, X)[0], E)
            q[k][idx] -= 2 * h
            lm = P.loss(P.forward(q, X)[0], E)
            fd[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[k], fd, rtol=1e-6, atol=1e-9, err_msg=k)


def test_backward_matches_autograd():
    torch = pytest.importorskip("torch")
    p, X, E = _small(5)
    Y, cache = P.forward(p, X)
    g = P.backward(p, cache, Y, E)
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    x = torch.tensor(X)
    gl = torch.nn.functional.gelu
    a = gl(x @ t["W1"] + t["b1"])
    a = gl(a @ t["W2"] + t["b2"])
    y = a @ t["W3"] + t["b3"]
    loss = 0.5 * ((y - torch.tensor(E)) ** 2).sum() / X.shape[0]
    loss.backward()
    for k in p:
        np.testing.assert_allclose(g[k], t[k].grad.numpy(), rtol=1e-12, atol=1e-14, err_msg=k)


def test_adam_first_step_is_a_signed_step_of_size_lr():
    g = np.array([3.0, -0.5, 1e-3])
    w, m, v = P.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(w, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_population_rate_of_one_spike_is_a_geometric_tail():
    B, T, N = 1, 30, 130
    r = np.zeros((B, T, N), np.uint8)
    r[0, 4, 70] = 1                       # neuron 70 belongs to group 70 mod 64 = 6
    beta = math.exp(-1.0 / 20.0)
    pr = P.population_rates(r, beta)
    t = np.arange(T)
    size = len(range(6, N, 64))           # neurons 6, 70 (134 >= N)
    want = np.where(t >= 4, (1 - beta) * beta ** (t - 4) / size, 0.0)
    np.testing.assert_allclose(pr[0, :, 6], want, rtol=1e-13, atol=1e-300)
    assert np.all(np.delete(pr[0], 6, axis=1) == 0.0)


def test_softmax_error_rows_sum_to_zero():
    rng = np.random.default_rng(1)
    y = rng.standard_normal((50, 10)) * 5
    oh = np.eye(10)[rng.integers(0, 10, 50)]
    E = P.softmax_error(y, oh)
    np.testing.assert_allclose(E.sum(axis=1), 0.0, atol=1e-14)
    assert np.all(E[oh == 1] <= 0) and np.all(E[oh == 0] >= 0)

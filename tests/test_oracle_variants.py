"""Pins of the oracle's e-prop+ variants and constraints (CPU only).

* Adam (Eq. adam, Eq. eta-adam-fast, Eq. delta-w-adam-fast): one Adam step
  per update window on the window's batch-mean gradient equals
  torch.optim.Adam driven with the oracle's own plain gradients (the
  TensorFlow form with constant eps_hat is torch's form with
  eps = eps_hat / sqrt(1 - b2^k), an identity of the two algebraic forms);
* fixed weight signs: after one window the constrained weights equal the
  unconstrained ones wherever those kept their sign and are a zero of the
  initial sign elsewhere; no sign ever flips over several windows;
* ignore-and-fire (Methods, "Scaling"): every neuron fires exactly every
  `period` steps from a first spike in [1, period], whatever its input, the
  phases spread over the period, the schedule runs on across continuous
  calls, and the membrane and surrogate are still integrated;
* an unfiltered eligibility trace (kappa_e = 0) gives sum_t L^t e^t, the
  limit of the closed form of one arrival.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from workloads import configs as C

torch = pytest.importorskip("torch")


def _small(T=100, **kw):
    W = C.pattern_regression(T=T, n_rec=30, n_in=10, **kw)
    W["spec"].lr = 1e-3
    return W


def _oracle(W, w=None, w_out=None):
    s = W["spec"]
    return oracle.Oracle(s, W["ptr"], W["col"], W["w"] if w is None else w, W["delay"],
                         W["w_out"] if w_out is None else w_out, W["out_mask"], W["feedback"])


def _sim(o, W):
    s = W["spec"]
    return o.simulate(s.T, W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"])


@pytest.mark.parametrize("eps_hat", [1e-12, 1e-4])
def test_adam_per_window_equals_torch_adam(eps_hat):
    W = _small()
    s = W["spec"]
    s.optimizer, s.adam_eps = 1, eps_hat
    pv = oracle.params(s)                        # the constants as the oracle takes them
    b1, b2, eps_hat = pv["adam_b1"], pv["adam_b2"], pv["adam_eps"]
    o_adam = _oracle(W)
    w = torch.tensor(np.asarray(W["w"], np.float64), requires_grad=True)
    wo = torch.tensor(np.asarray(W["w_out"], np.float64), requires_grad=True)
    opt = torch.optim.Adam([w, wo], lr=pv["lr"], betas=(b1, b2), eps=0.0)
    for k in range(1, 5):
        _sim(o_adam, W)
        # the plain gradient at the current weights (SGD oracle, lr 0)
        s0 = C.Spec(**{**s.__dict__, "optimizer": 0, "lr": 0.0})
        W0 = dict(W, spec=s0)
        o = _oracle(W0, w.detach().numpy().astype(np.float64), wo.detach().numpy())
        _sim(o, W0)
        g, go = o.take_grads()
        assert np.abs(g).max() > 0
        w.grad = torch.tensor(g)
        wo.grad = torch.tensor(go)
        opt.param_groups[0]["eps"] = eps_hat / math.sqrt(1.0 - b2 ** k)
        opt.step()
        np.testing.assert_allclose(o_adam.w, w.detach().numpy(), rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(o_adam.w_out, wo.detach().numpy(), rtol=1e-11, atol=1e-14)
    # Adam moved the weights by about lr per step (its first step is a sign step)
    moved = np.abs(o_adam.w - np.asarray(W["w"], np.float64))
    assert np.median(moved[moved > 0]) > 0.5 * s.lr


def test_fixed_signs_stop_at_zero_and_never_flip():
    W = _small()
    s = W["spec"]
    s.lr = 2.0                                   # large: many weights would cross zero
    w0 = np.asarray(W["w"], np.float32)
    wo0 = np.asarray(W["w_out"], np.float32)
    free = _oracle(W)
    _sim(free, W)
    s.sign_mask = 7
    fixed = _oracle(W)
    _sim(fixed, W)
    for wu, wc, init in ((free.w, fixed.w, w0), (free.w_out, fixed.w_out, wo0)):
        init = init.reshape(wu.shape)
        keep = np.signbit(wu) == np.signbit(init)
        flipped = ~keep & (wu != 0)
        assert flipped.sum() > 10, "the test must push weights across zero"
        assert np.array_equal(wc[keep], wu[keep])
        assert np.all(wc[~keep] == 0.0)
        assert np.array_equal(np.signbit(wc), np.signbit(init))
    for _ in range(3):
        _sim(fixed, W)
        assert np.array_equal(np.signbit(fixed.w), np.signbit(w0))
        assert np.array_equal(np.signbit(fixed.w_out), np.signbit(wo0.reshape(fixed.w_out.shape)))


def test_only_the_selected_projections_keep_their_signs():
    W = _small()
    s = W["spec"]
    s.lr = 2.0
    nnz_in = int(W["ptr"][s.n_in])
    w0 = np.asarray(W["w"], np.float32)
    s.sign_mask = 2                              # recurrent only
    o = _oracle(W)
    _sim(o, W)
    assert np.array_equal(np.signbit(o.w[nnz_in:]), np.signbit(w0[nnz_in:]))
    assert np.any(np.signbit(o.w[:nnz_in]) != np.signbit(w0[:nnz_in]))


@pytest.mark.parametrize("period", [20, 7])
def test_ignore_and_fire_schedule(period):
    W = _small(T=200)
    s = W["spec"]
    s.if_period, s.if_seed = period, 99
    r = _sim(_oracle(W), W)
    z = r["raster"][0]                           # [T, N]
    for j in range(s.n_rec):
        steps = np.nonzero(z[:, j])[0] + 1
        assert 1 <= steps[0] <= period
        assert np.all(np.diff(steps) == period)
        assert steps[-1] + period > s.T
    first = np.argmax(z, axis=0)
    assert len(np.unique(first)) > min(period, s.n_rec) // 2
    # the membrane and the surrogate are still integrated from the inputs
    assert np.abs(r["margin"]).max() > 0
    # the schedule runs on across continuous calls
    W2 = _small(T=100)
    s2 = W2["spec"]
    s2.if_period, s2.if_seed, s2.continuous = period, 99, 1
    o = _oracle(W2)
    z1 = _sim(o, W2)["raster"][0]
    z2 = _sim(o, W2)["raster"][0]
    assert np.array_equal(np.concatenate([z1, z2]), z)


def test_unfiltered_eligibility_single_arrival():
    # one arrival at step a into a teacher-forced neuron with constant psi c
    # and learning signal l: with kappa_e = 0 the gradient is
    # sum_{t >= a} l c alpha^{t-a} = l c (1 - alpha^(T-a+1)) / (1 - alpha)
    alpha, c, l, a, T = 0.9, 0.4, 1.5, 3, 12
    st = np.zeros(3)
    g = 0.0
    for t in range(1, T + 1):
        g += oracle.eligibility_step(alpha, 0.0, 0.0, 0.0, c if t > 1 else 0.0, c, l,
                                     1.0 if t == a else 0.0, st)
    expect = l * c * (1 - alpha ** (T - a + 1)) / (1 - alpha)
    assert abs(g - expect) <= 1e-14 * abs(expect)

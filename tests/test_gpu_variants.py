"""e-prop+ variants, constraints, Adam and the scaling network on the GPU
against the FP64 oracle (GPU only).

The same two-oracle comparison as the plain method (`test_gpu_parity.py`):
oracle A teacher-forced with the GPU raster (decisions, readout, loss,
surrogate values, end-to-end gradients), oracle B forced with the raster and
the surrogate values (every gradient and weight element).  Cases:

* exponential surrogate (Eq. exponential-surrogate-gradient), fixed reset,
  temporal MSE (Eq. temporal-mse), unfiltered eligibility (kappa_e = 0);
* firing-rate regularisation (Eq. ema-rate, Eq. ema-gradient) in the
  single-window forms (one sample; a batch);
* fixed weight signs (Dale's law on the E/I network; all projections on
  the pattern task with a learning rate large enough to push weights to
  zero) in the dense window form and the batched form;
* sparse feedback with out-degree 100 and Dale's law on the E/I network;
* ignore-and-fire neurons with Poisson inputs, sparse readout in-degree and
  sparse feedback: the scaling experiment's network, scaled down;
* Adam (Eq. adam, Eq. eta-adam-fast, Eq. delta-w-adam-fast): each call's
  gradients against oracle B started from the GPU's weights, and each Adam
  step against torch.optim.Adam (FP64) driven by the GPU's own gradients;
  the evidence-accumulation task (batch 32, recall-window cross-entropy)
  with a per-sample oracle pool;
* generalized delays (Supplement "Generalized delays"): the readout delay
  d_out and the learning-signal delay d_ls, in the single-window forms.
"""
from __future__ import annotations

import copy
import math

import numpy as np
import pytest

import oracle
from tests import parity as P
from tests.test_gpu_parity import _gpu_net, _replica, run_parity, run_parity_pooled
from workloads import configs as C

pytestmark = pytest.mark.gpu


# ------------------------------------------------------------- e-prop+ variants


def test_exponential_surrogate():
    W = C.pattern_regression(T=300, surrogate=1)
    rep = run_parity(W, calls=2)
    assert rep["spikes"] > 300


def test_fixed_reset():
    W = C.pattern_regression(T=300, reset_mode=1, v_reset=0.1)
    rep = run_parity(W, calls=2)
    assert rep["spikes"] > 300


def test_temporal_mse_classification():
    W = C.event_classification(batch=4, T=150, len_lo=100, len_hi=150, n_rec=60, side=8,
                               events_per_300=3000.0, loss=2)
    rep = run_parity(W)
    assert rep["spikes"] > 100


@pytest.mark.parametrize("tk", [pytest.param(1, id="lazy"), pytest.param(3, id="dense")])
def test_unfiltered_eligibility(tk):
    W = _replica(True, 200, kappa_e=0.0)
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_kernel=tk))
    assert rep["events"] > 0


def test_rate_regularisation_single_sample():
    W = C.pattern_regression(T=400, c_reg=2.0, f_target=0.01, beta_reg=0.95)
    rep = run_parity(W, calls=2)
    assert rep["spikes"] > 300


def test_rate_regularisation_batch():
    W = C.event_classification(batch=4, T=150, len_lo=100, len_hi=150, n_rec=60, side=8,
                               events_per_300=3000.0, c_reg=2.0, f_target=0.02, beta_reg=0.9)
    rep = run_parity(W)
    assert rep["spikes"] > 100


def test_rate_regularisation_needs_single_windows():
    import paper_2511_21674_gb300 as ep
    W = _replica(True, 200, c_reg=1.0, beta_reg=0.9)
    with pytest.raises(ep.EpropError, match="rate regularisation"):
        _gpu_net(W)


# -------------------------------------------------------------- fixed signs


def _sign_check(net_w, w0):
    assert np.array_equal(np.signbit(net_w), np.signbit(np.asarray(w0, np.float32)))


def _near_zero(W, frac=0.25, scale=1e-7, key="w"):
    # a fraction of the weights start next to zero (sign kept), so that a
    # learning rate that leaves the dynamics within FP32 agreement still
    # pushes some of them across zero
    w = np.asarray(W[key], np.float32).copy()
    idx = np.arange(w.size)[np.arange(w.size) % int(round(1 / frac)) == 0]
    w.flat[idx] = np.where(np.signbit(w.flat[idx]), -scale, scale).astype(np.float32)
    W[key] = w
    return W


def test_fixed_signs_dense_window_form():
    W = C.pattern_regression(T=300, update_interval=100, continuous=1, sign_mask=7)
    _near_zero(_near_zero(W, scale=1e-10), scale=1e-10, key="w_out")
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_kernel=3))
    nnz_in = int(W["ptr"][W["spec"].n_in])
    for name, w0 in (("w_rec", W["w"][nnz_in:]), ("w_in", W["w"][:nnz_in]), ("w_out", W["w_out"])):
        w, _ = rep["res"][name]
        _sign_check(w, w0)
    zeros = sum(int(np.sum(rep["res"][k][0] == 0.0)) for k in ("w_rec", "w_in", "w_out"))
    assert zeros > 0, "some weights must reach zero"


def test_fixed_signs_batched_form():
    W = C.event_classification(batch=4, T=150, len_lo=100, len_hi=150, n_rec=60, side=8,
                               events_per_300=3000.0, sign_mask=7)
    _near_zero(W, scale=1e-8)
    rep = run_parity(W)
    w, _ = rep["res"]["w_in"]
    _sign_check(w, W["w"][:int(W["ptr"][W["spec"].n_in])])
    assert np.sum(w == 0.0) > 0


def test_dale_and_sparse_feedback_on_the_ei_network():
    # E/I replica of the large networks: the E/I sign of every recurrent
    # synapse is kept (Dale's law), each readout's feedback reaches 100
    # neurons only
    W = _replica(True, 200, fb_outdeg=100, dale=True)
    _near_zero(W, frac=0.1, scale=1e-9)
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_kernel=3))
    w, _ = rep["res"]["w_rec"]
    _sign_check(w, W["w"])
    assert rep["events"] > 0


# ---------------------------------------------------------- scaling network


def test_ignore_and_fire_scaling_network_replica():
    W = C.scaling_network(n_rec=3000, k_rec=300, n_in=100, k_in=10, n_out=4, k_out=200,
                          fb_outdeg=50, T=400, update_interval=100)
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_kernel=3))
    # the schedule: every neuron fires every 200 steps
    assert rep["spikes"] == 2 * 3000 * 400 // 200
    assert rep["mismatches"] == 0


# --------------------------------------------------------------------- Adam


def run_adam(W, calls, gpu_kw=None, pooled=False):
    """Adam on the GPU for `calls` single-window calls: each call's gradient
    against oracle B (forced raster and surrogate values) started from the
    GPU's weights, and each Adam step against torch.optim.Adam in FP64 fed
    with the GPU's own gradient."""
    import torch
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    assert s.optimizer == 1
    net = _gpu_net(W, **(gpu_kw or {}))
    nnz_in = int(W["ptr"][s.n_in]) if s.n_in else 0
    b1, b2 = float(np.float32(s.adam_b1)), float(np.float32(s.adam_b2))
    eps_hat = float(np.float32(s.adam_eps))
    lr = float(np.float32(s.lr))

    def read_all():
        w_in = net.weights(ep.PROJ_IN, with_grad=True) if s.n_in else (np.zeros(0), np.zeros(0))
        w_rec = net.weights(ep.PROJ_REC, with_grad=True)
        w_out = net.weights(ep.PROJ_OUT, with_grad=True)
        w = np.concatenate([w_in[0], w_rec[0]]).astype(np.float64)
        g = np.concatenate([w_in[1], w_rec[1]]).astype(np.float64)
        return w, g, w_out[0].astype(np.float64), w_out[1].astype(np.float64)

    w_prev, g_prev, wo_prev, go_prev = read_all()
    tw = torch.tensor(w_prev.copy(), requires_grad=True)
    two = torch.tensor(wo_prev.copy(), requires_grad=True)
    opt = torch.optim.Adam([tw, two], lr=lr, betas=(b1, b2), eps=0.0)
    # oracle B without learning (lr 0, SGD): the gradient at the GPU's weights
    s0 = copy.copy(s)
    s0.optimizer, s0.lr = 0, 0.0
    W0 = dict(W, spec=s0)
    orB = None if pooled else oracle.Oracle(s0, W["ptr"], W["col"], w_prev, W["delay"], wo_prev,
                                            W["out_mask"], W["feedback"])
    worst, cum = {}, {}
    for k in range(1, calls + 1):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
        _, _, raster = net.readout(raster=True)
        psi = net.surrogate()
        w_new, g_cum, wo_new, go_cum = read_all()
        g_gpu, go_gpu = g_cum - g_prev, go_cum - go_prev          # this call's batch-mean gradient
        if pooled:
            Wc = dict(W0, w=w_prev.astype(np.float32), w_out=wo_prev.astype(np.float32))
            outs = P.pooled_sample_oracles(Wc, raster, psi)
            gB = np.mean([o["gB"] for o in outs], axis=0)
            goB = np.mean([o["goB"] for o in outs], axis=0)
            mag = np.mean([o["magB"] + 0.1 * o["sensB"] + o["arrB"] for o in outs], axis=0)
            mago = np.mean([o["gomB"] + 0.1 * o["gosB"] for o in outs], axis=0)
        else:
            orB.w[:] = w_prev
            orB.w_out[:] = wo_prev
            rB = orB.simulate(s.T, W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"],
                              forced=raster, forced_psi=psi, record=True)
            gB, goB = orB.take_grads()
            m_, mo_ = orB.take_grad_magnitudes()
            se_, seo_ = orB.take_grad_sensitivities()
            single = not (s.continuous or s.update_interval > 0)
            arr = oracle.arrival_magnitude(s0, W["ptr"], W["col"], W["delay"], W["x_ptr"], W["x_ids"],
                                           W["lengths"], raster, rB["psi"], rB["L"]) if single else 0.0
            mag = m_ + 0.1 * se_ + arr
            mago = mo_ + 0.1 * seo_
        # the GPU keeps the cumulative gradient in FP32: compared as
        # cumulative sums (a difference of two FP32 sums would cancel)
        cum["g"] = cum.get("g", 0.0) + gB
        cum["go"] = cum.get("go", 0.0) + goB
        cum["m"] = cum.get("m", 0.0) + mag
        cum["mo"] = cum.get("mo", 0.0) + mago
        worst[f"g_{k}"] = P.assert_close(g_cum, cum["g"], f"calls 1..{k} synapse gradient", mag=cum["m"])
        worst[f"go_{k}"] = P.assert_close(go_cum, cum["go"], f"calls 1..{k} readout gradient", mag=cum["mo"])
        # the Adam step on the GPU's own gradient (torch, FP64); masked
        # readout weights take no step
        with torch.no_grad():
            tw.copy_(torch.tensor(w_prev))
            two.copy_(torch.tensor(wo_prev))
        tw.grad = torch.tensor(g_gpu)
        two.grad = torch.tensor(go_gpu)
        opt.param_groups[0]["eps"] = eps_hat / math.sqrt(1.0 - b2 ** k)
        opt.step()
        w_ref, wo_ref = tw.detach().numpy().copy(), two.detach().numpy().copy()
        if s.sign_mask:
            # fixed signs: a step that would cross zero stops at a zero of the
            # weight's own sign (bit 0 inputs, bit 1 recurrent, bit 2 readout)
            sel = np.zeros(w_ref.shape, bool)
            if s.sign_mask & 1:
                sel[:nnz_in] = True
            if s.sign_mask & 2:
                sel[nnz_in:] = True
            for ref, prev, on in ((w_ref, w_prev, sel), (wo_ref, wo_prev,
                                                         np.full(wo_ref.shape, bool(s.sign_mask & 4)))):
                flip = on & (np.signbit(ref) != np.signbit(prev))
                ref[flip] = np.where(np.signbit(prev[flip]), -0.0, 0.0)
        for name, a, ref, prev in (("w", w_new, w_ref, w_prev), ("w_out", wo_new, wo_ref, wo_prev)):
            dw = np.abs(ref - prev)
            tol = 1e-6 * np.abs(ref) + 1e-5 * dw + 1e-12
            ratio = float((np.abs(a - ref) / tol).max())
            worst[f"{name}_{k}"] = ratio
            assert ratio <= 1.0, f"call {k} {name}: Adam step off by {ratio:.3g} x tolerance"
        w_prev, g_prev, wo_prev, go_prev = w_new, g_cum, wo_new, go_cum
    net.close()
    P.report(dict(adam_worst=worst))
    print("adam:", {k: f"{v:.3g}" for k, v in worst.items()})
    return worst


def test_adam_batched_form():
    W = C.event_classification(batch=4, T=150, len_lo=100, len_hi=150, n_rec=60, side=8,
                               events_per_300=3000.0, optimizer=1, lr=2e-3)
    run_adam(W, calls=3)


def test_adam_dense_window_form_continuous():
    # one update window per call (T = U), state carried across calls
    W = _replica(True, 100, optimizer=1)
    W["spec"].lr = 1e-4
    run_adam(W, calls=3, gpu_kw=dict(trace_kernel=3))


def test_adam_with_fixed_signs():
    W = C.pattern_regression(T=200, optimizer=1, sign_mask=7)
    W["spec"].lr = 2e-2
    run_adam(W, calls=3)


def test_adam_rejects_lazy_catch_up():
    import paper_2511_21674_gb300 as ep
    W = _replica(True, 200, optimizer=1)
    with pytest.raises(ep.EpropError, match="Adam"):
        _gpu_net(W, trace_kernel=1)


def test_evidence_accumulation_with_adam_batch32():
    # the evidence-accumulation task as the paper trains it: mini-batch 32,
    # cross-entropy in the recall window, Adam; a shorter delay keeps the
    # oracle's time in bounds
    W = C.evidence_accumulation(batch=32, t_delay=300)
    run_adam(W, calls=2, pooled=True)


# ------------------------------------------------------- per-spike updates


@pytest.mark.parametrize("tk", [pytest.param(1, id="lazy"), pytest.param(3, id="dense")])
def test_weight_updates_with_every_spike(tk):
    # e-prop+ weight updates with every spike (Results, "Weight updates with
    # every spike"; Algorithm "Event-driven weight update"): with gradient
    # descent the weight a spike carries is w0 - eta * (the gradient of every
    # step before its emission), i.e. updates applied after every step
    # (update window of one step, continuous dynamics); the lazy form applies
    # them exactly at each presynaptic spike
    # one call of 80 steps: 80 updates of every weight (the FP32 weights of
    # the GPU and the FP64 weights of oracle A then still drive the same
    # membranes within the FP32 band)
    W = C.pattern_regression(T=80, update_interval=1, continuous=1)
    W["spec"].lr = 5e-4
    rep = run_parity(W, calls=1, gpu_kw=dict(trace_kernel=tk))
    assert rep["spikes"] > 50


# generalized delays (Supplement "Generalized delays"): the readout sees the
# recurrent spikes d_out steps late, the learning signal reaches the
# recurrent layer d_ls steps late (one update window per call)
@pytest.mark.parametrize("d_out,d_ls", [(2, 0), (1, 3)])
def test_generalized_delays_pattern_regression(d_out, d_ls):
    W = C.pattern_regression(T=300)
    W["spec"].d_out, W["spec"].d_ls = d_out, d_ls
    rep = run_parity(W, calls=2)
    assert rep["spikes"] > 300


def test_generalized_delays_batched_event_classification():
    W = C.event_classification(batch=4, T=150, len_lo=100, len_hi=150, n_rec=60, side=8,
                               events_per_300=3000.0)
    W["spec"].d_out, W["spec"].d_ls = 2, 2
    rep = run_parity(W)
    assert rep["spikes"] > 100


def test_generalized_delays_need_one_window_per_call():
    import paper_2511_21674_gb300 as ep
    W = _replica(True, 200)
    W["spec"].d_out = 1
    with pytest.raises(ep.EpropError, match="generalized delays"):
        _gpu_net(W)

"""The learned learning-signal predictor inside e-prop (GPU only).

* its per-step inputs (readout potentials, group rates) against their
  definition on the recorded readout and raster;
* e-prop driven by the predicted error signal against the FP64 oracle fed
  the same predictions (teacher-forced spikes and surrogate values);
* the gain: a predictor trained on the network's own (state, error) pairs
  brings the gradient of a sample whose target arrives only in its last 25
  steps closer to the gradient with the target known at every step than
  plain e-prop (which has no learning signal before the window); its
  predictions correlate with the true error on unseen samples (their
  squared error is reported: the class part of E is not observable from
  the state of an untrained network, so it need not beat predicting zero).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import predictor as P
from tests import parity as PT
from workloads import configs as C

pytestmark = pytest.mark.gpu


def _net(W, **kw):
    import paper_2511_21674_gb300 as ep
    kw.setdefault("launch_mode", 0)
    return ep.Network(W["spec"], W["ptr"], W["col"], W["w"], W["delay"], W["w_out"],
                      W["out_mask"], W["feedback"], **kw)


def _small(batch=4, sample_seed=None):
    return C.event_classification(batch=batch, T=120, len_lo=80, len_hi=120, n_rec=60, side=8,
                                  events_per_300=2000.0, sample_seed=sample_seed)


def test_predictor_inputs_follow_their_definition():
    import paper_2511_21674_gb300 as ep
    W = _small()
    s = W["spec"]
    net = _net(W, record_raster=1)
    pred = ep.Predictor(s.n_out + 64, s.n_out, seed=1, max_rows=64)
    net.attach_predictor(pred, mode=2)
    for _ in range(2):                        # the record buffer survives repeated calls
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
    y, _, raster = net.readout(raster=True)
    x = net.predictor_inputs()
    assert raster.sum() > 0
    np.testing.assert_array_equal(x[..., :s.n_out], y)
    r = 1000.0 * P.population_rates(raster, math.exp(-s.dt / 20.0))   # spikes per 1000 steps
    np.testing.assert_allclose(x[..., s.n_out:], r, rtol=5e-6, atol=1e-9)   # FP32 filter
    net.close()
    pred.close()


@pytest.mark.parametrize("update_interval", [0, 40])
def test_eprop_with_predicted_error_matches_oracle(update_interval):
    # the predictor's outputs stand in for E where the target window is
    # closed; the oracle takes the same outputs as its error signal there.
    # With update windows inside the call (40 steps, batch 4) the weights
    # step with the predicted signal before each sample's target window.
    import paper_2511_21674_gb300 as ep
    W = _small()
    s = W["spec"]
    s.update_interval = update_interval
    B, T, K = s.batch, s.T, s.n_out
    net = _net(W, record_raster=1, record_psi=1, record_grad=1)
    pred = ep.Predictor(K + 64, K, seed=3, max_rows=B * T)
    net.attach_predictor(pred, mode=3)
    net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], T)
    net.simulate(T)
    _, _, raster = net.readout(raster=True)
    psi = net.surrogate()
    x = net.predictor_inputs()
    E_hat = pred.forward(x.reshape(B * T, K + 64)).reshape(B, T, K)
    nnz_in = int(W["ptr"][s.n_in])
    _, g_in = net.weights(ep.PROJ_IN, with_grad=True)
    _, g_rec = net.weights(ep.PROJ_REC, with_grad=True)
    _, g_out = net.weights(ep.PROJ_OUT, with_grad=True)
    net.close()
    pred.close()
    o = oracle.Oracle(s, W["ptr"], W["col"], W["w"], W["delay"], W["w_out"], W["out_mask"], W["feedback"])
    r = o.simulate(T, W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"],
                   forced=raster, forced_psi=psi, record=True, E_override=E_hat)
    g, go = o.take_grads()
    m, mo = o.take_grad_magnitudes()
    se, seo = o.take_grad_sensitivities()
    tol = m + 0.1 * se
    if not update_interval:
        # one window per call: the kernels sum one table entry per arrival
        tol = tol + oracle.arrival_magnitude(s, W["ptr"], W["col"], W["delay"], W["x_ptr"], W["x_ids"],
                                             W["lengths"], raster, r["psi"], r["L"])
    assert np.abs(g).max() > 0
    PT.assert_close(g_in, g[:nnz_in], "g_in (predicted E)", mag=tol[:nnz_in])
    PT.assert_close(g_rec, g[nnz_in:], "g_rec (predicted E)", mag=tol[nnz_in:])
    PT.assert_close(g_out, go, "g_out (predicted E)", mag=mo + 0.1 * seo)


def _run_grads(W, samples, window_mode, pred=None):
    """Summed input+recurrent gradients over the given sample batches with
    frozen weights: window_mode 'full' (target at every step), 'plain' (last
    25 steps) or 'pred' (last 25 steps, predicted error before)."""
    import paper_2511_21674_gb300 as ep
    net = _net(W, record_grad=1)
    if window_mode == "pred":
        net.attach_predictor(pred, mode=1)
    for Ws in samples:
        win = np.ones_like(Ws["window"]) if window_mode == "full" else Ws["window"]
        net.set_inputs(Ws["x_ptr"], Ws["x_ids"], Ws["targets"], win, Ws["lengths"], W["spec"].T)
        net.simulate(W["spec"].T)
    g = np.concatenate([net.weights(ep.PROJ_IN, with_grad=True)[1],
                        net.weights(ep.PROJ_REC, with_grad=True)[1]])
    net.close()
    return g


def _cos(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


def test_trained_predictor_brings_the_gradient_closer_to_the_full_signal():
    import paper_2511_21674_gb300 as ep
    B = 16
    W = C.event_classification(batch=B)
    s = W["spec"]
    s.lr = 0.0                                  # frozen network: data and evaluation
    K, T = s.n_out, s.T
    # training pairs (x^t, E^t) with the target known at every step
    net = _net(W)
    pred = ep.Predictor(K + 64, K, seed=7, max_rows=256)
    net.attach_predictor(pred, mode=2)
    X, E = [], []
    for k in range(24):
        Ws = C.event_classification(batch=B, sample_seed=5000 + k)
        net.set_inputs(Ws["x_ptr"], Ws["x_ids"], Ws["targets"], np.ones_like(Ws["window"]),
                       Ws["lengths"], T)
        net.simulate(T)
        y, _ = net.readout()
        x = net.predictor_inputs()
        e = P.softmax_error(y, Ws["targets"])
        live = np.arange(T)[None, :] < Ws["lengths"][:, None]
        X.append(x[live])
        E.append(e[live])
    net.close()
    X = np.concatenate(X).astype(np.float32)
    E = np.concatenate(E).astype(np.float32)
    # input scale: unit spread per input over the training pairs
    pred.set_input_scale((1.0 / np.maximum(X.std(axis=0), 1e-3)).astype(np.float32))
    rng = np.random.default_rng(0)
    first = None
    for epoch in range(6):
        order = rng.permutation(len(X))
        for lo in range(0, len(X) - 255, 256):
            idx = order[lo:lo + 256]
            l = pred.train_step(X[idx], E[idx], 1e-3)
            first = l if first is None else first
    # held-out samples
    held = [C.event_classification(batch=B, sample_seed=9000 + k) for k in range(2)]
    mse_pred = mse_zero = 0.0
    dots = [0.0, 0.0, 0.0]
    net = _net(W)
    net.attach_predictor(pred, mode=2)
    for Ws in held:
        net.set_inputs(Ws["x_ptr"], Ws["x_ids"], Ws["targets"], np.ones_like(Ws["window"]),
                       Ws["lengths"], T)
        net.simulate(T)
        y, _ = net.readout()
        x = net.predictor_inputs()
        live = np.arange(T)[None, :] < Ws["lengths"][:, None]
        e = P.softmax_error(y, Ws["targets"])[live]
        xl = x[live]
        eh = np.concatenate([pred.forward(xl[lo:lo + 256]) for lo in range(0, len(xl), 256)])
        mse_pred += float(((eh - e) ** 2).sum())
        mse_zero += float((e ** 2).sum())
        dots[0] += float((eh * e).sum())
        dots[1] += float((eh * eh).sum())
        dots[2] += float((e * e).sum())
    net.close()
    g_full = _run_grads(W, held, "full")
    g_plain = _run_grads(W, held, "plain")
    g_pred = _run_grads(W, held, "pred", pred)
    c_plain, c_pred = _cos(g_plain, g_full), _cos(g_pred, g_full)
    corr = dots[0] / np.sqrt(dots[1] * dots[2])
    print(f"predictor: train loss {first:.4g} -> {l:.4g}; held-out cosine of predicted and "
          f"true error {corr:.3f}, MSE ratio to predicting zero {mse_pred / mse_zero:.3f}; "
          f"gradient cosine to the full-signal gradient: plain {c_plain:.3f}, with predictor "
          f"{c_pred:.3f}")
    pred.close()
    # the prediction points the right way on unseen samples, and the
    # gradient it drives is measurably closer to the full-signal gradient
    assert corr > 0.1
    assert c_pred > c_plain + 0.05


def _pairs(net, W, seeds, T):
    """(x^t, E^t) of every live step of the given sample batches, target
    known at every step (the network is frozen: lr 0)."""
    X, E = [], []
    for sd in seeds:
        Ws = C.event_classification(batch=W["spec"].batch, sample_seed=sd)
        net.set_inputs(Ws["x_ptr"], Ws["x_ids"], Ws["targets"], np.ones_like(Ws["window"]),
                       Ws["lengths"], T)
        net.simulate(T)
        y, _ = net.readout()
        x = net.predictor_inputs()
        live = np.arange(T)[None, :] < Ws["lengths"][:, None]
        X.append(x[live])
        E.append(P.softmax_error(y, Ws["targets"])[live])
    return np.concatenate(X).astype(np.float32), np.concatenate(E).astype(np.float32)


def _train_eprop(W, learner, lam, train_sets, epochs, eval_sets):
    """e-prop training over `epochs` passes of the given batches; with a
    learner, a copy of it whose output layer is scaled by lam is attached
    (mode 3: its estimate stands in for E outside the target window), and
    after every call the learner trains on the call's target-window steps
    (where the true E is known) and the copy is refreshed.  Returns the mean
    windowed loss and the accuracy on the held-out batches with frozen
    weights, and the training-loss curve."""
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    K = s.n_out
    net = _net(W, launch_mode=1)
    actor = None
    if learner is not None:
        actor = ep.Predictor(K + 64, K, seed=0, max_rows=4096)
        actor.set_input_scale(learner.input_scale)

        def refresh():
            p = learner.unpack(learner.read("params").copy())
            p["W3"], p["b3"] = p["W3"] * lam, p["b3"] * lam
            actor.set_params(learner.pack(p))
        refresh()
        net.attach_predictor(actor, mode=3)
    curve = []
    for _ in range(epochs):
        for Ws in train_sets:
            net.set_inputs(Ws["x_ptr"], Ws["x_ids"], Ws["targets"], Ws["window"], Ws["lengths"], s.T)
            net.simulate(s.T)
            y, loss = net.readout()
            curve.append(float(loss.mean()))
            if learner is not None:
                x = net.predictor_inputs()
                win = Ws["window"].astype(bool)
                e = P.softmax_error(y, Ws["targets"])
                for _ in range(2):
                    learner.train_step(x[win].astype(np.float32), e[win].astype(np.float32), 1e-3)
                refresh()
    w_in = net.weights(ep.PROJ_IN)
    w_rec = net.weights(ep.PROJ_REC)
    w_out = net.weights(ep.PROJ_OUT)
    net.close()
    if actor is not None:
        actor.close()
    # held-out loss and accuracy with the trained weights (lr 0)
    s2 = C.Spec(**{**s.__dict__, "lr": 0.0})
    W2 = dict(W, spec=s2, w=np.concatenate([w_in, w_rec]), w_out=w_out)
    net = _net(W2, launch_mode=1)
    losses, hits = [], []
    for Ws in eval_sets:
        net.set_inputs(Ws["x_ptr"], Ws["x_ids"], Ws["targets"], Ws["window"], Ws["lengths"], s.T)
        net.simulate(s.T)
        y, loss = net.readout()
        losses.append(loss)
        score = (y * Ws["window"][..., None]).sum(axis=1)          # readout summed over the window
        hits.append(np.argmax(score, axis=1) == Ws["classes"])
    net.close()
    return float(np.concatenate(losses).mean()), float(np.concatenate(hits).mean()), curve


def test_predictor_at_scale_final_loss_against_plain_eprop():
    # the stated experiment: the predictor trained on ~1e6 (state, E) pairs
    # that plain e-prop runs of the event-classification network generate,
    # then e-prop trained with and without it on the same batches and
    # judged by the held-out loss in the target window; the batch-256
    # inference time per step is reported
    import torch
    import paper_2511_21674_gb300 as ep
    W = C.event_classification(batch=64)
    s = W["spec"]
    K, T = s.n_out, s.T
    s0 = C.Spec(**{**s.__dict__, "lr": 0.0})
    net = _net(dict(W, spec=s0))
    pred = ep.Predictor(K + 64, K, seed=11, max_rows=4096)
    net.attach_predictor(pred, mode=2)
    X, E = _pairs(net, dict(W, spec=s0), range(20000, 20060), T)
    net.close()
    assert X.shape[0] >= 1_000_000, X.shape
    pred.set_input_scale((1.0 / np.maximum(X.std(axis=0), 1e-3)).astype(np.float32))
    rng = np.random.default_rng(1)
    first = last = None
    for epoch in range(3):
        order = rng.permutation(len(X))
        for lo in range(0, len(X) - 4095, 4096):
            idx = order[lo:lo + 4096]
            last = pred.train_step(X[idx], E[idx], 1e-3)
            first = last if first is None else first
    # batch-256 inference per step (device pointers, CUDA events)
    xd = torch.from_numpy(X[:256]).cuda()
    yd = torch.empty((256, K), dtype=torch.float32, device="cuda")
    lib = ep.load_library()
    for _ in range(10):
        lib.eprop_predictor_forward(pred.h, xd.data_ptr(), 256, yd.data_ptr(), 1)
    lib.eprop_predictor_sync(pred.h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(200):
        lib.eprop_predictor_forward(pred.h, xd.data_ptr(), 256, yd.data_ptr(), 1)
    e1.record()
    torch.cuda.synchronize()
    lib.eprop_predictor_sync(pred.h)
    us = 1000.0 * e0.elapsed_time(e1) / 200
    # e-prop with and without the predictor: Adam (lr 2e-3) on the same 8
    # batches for 6 epochs, judged on 2 held-out batches.  The predictor
    # keeps learning from each call's target window (the true E is known
    # there) and its estimate enters with weight 0.1 before the window (a
    # frozen predictor, or the full weight, made the network diverge: the
    # estimate of an untrained network's error is biased towards uniform
    # outputs, and outside the window it acts on 12 times as many steps)
    # the pre-trained parameters start the online learner (fresh Adam state)
    scale = (1.0 / np.maximum(X.std(axis=0), 1e-3)).astype(np.float32)
    learner = ep.Predictor(K + 64, K, seed=11, max_rows=4096, params=pred.read("params").copy())
    learner.set_input_scale(scale)
    learner.input_scale = scale
    pred.close()
    Wt = dict(W, spec=C.Spec(**{**s.__dict__, "optimizer": 1, "lr": 2e-3}))
    train = [C.event_classification(batch=64, sample_seed=30000 + k) for k in range(8)]
    held = [C.event_classification(batch=64, sample_seed=40000 + k) for k in range(2)]
    loss_plain, acc_plain, curve_plain = _train_eprop(Wt, None, 0.0, train, 6, held)
    params0 = learner.read("params").copy()
    loss_pred, acc_pred, curve_pred = _train_eprop(Wt, learner, 0.1, train, 6, held)
    # the same comparison with update windows of 50 steps inside each call
    # (seven weight steps per call; plain e-prop steps only in windows that
    # hold a target window, with the predictor in every window): reported
    Ww = dict(Wt, spec=C.Spec(**{**Wt["spec"].__dict__, "update_interval": 50}))
    loss_plain_w, acc_plain_w, _ = _train_eprop(Ww, None, 0.0, train, 6, held)
    learner.close()
    learner = ep.Predictor(K + 64, K, seed=11, max_rows=4096, params=params0)
    learner.set_input_scale(scale)
    learner.input_scale = scale
    loss_pred_w, acc_pred_w, _ = _train_eprop(Ww, learner, 0.1, train, 6, held)
    learner.close()
    chance = 25 * math.log(K)
    report = dict(pairs=int(X.shape[0]), predictor_train_loss=[first, last],
                  inference_us_per_step_batch256=us, chance_loss=chance,
                  heldout_loss_plain=loss_plain, heldout_loss_with_predictor=loss_pred,
                  heldout_accuracy_plain=acc_plain, heldout_accuracy_with_predictor=acc_pred,
                  train_loss_plain=curve_plain[::8], train_loss_with_predictor=curve_pred[::8],
                  windows50_heldout_loss_plain=loss_plain_w, windows50_heldout_loss_with_predictor=loss_pred_w,
                  windows50_heldout_accuracy_plain=acc_plain_w,
                  windows50_heldout_accuracy_with_predictor=acc_pred_w)
    PT.report(dict(predictor_scale=report))
    print("predictor at scale:", report)
    assert last < first
    assert loss_plain < 0.9 * chance, "plain e-prop must learn the task for the comparison to mean anything"
    # the gain: a lower held-out loss in the target window than plain e-prop
    # after the same number of updates
    assert loss_pred < loss_plain

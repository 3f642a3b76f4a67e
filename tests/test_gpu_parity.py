"""CUDA path vs FP64 oracle on the same seeded inputs (GPU only).

Each case runs the CUDA library through the C ABI, then the oracle on the
same arrays with its spikes teacher-forced to the GPU raster, and checks the
agreement rules of `tests/parity.py`: spike decisions bit-exact outside the
FP32 ambiguity band; readout, loss, weights and gradients within relative
1e-5 of the magnitude sum of their terms.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests import parity as P
from tests.helpers import raster_to_lists
from workloads import configs as C

pytestmark = pytest.mark.gpu


def _gpu_net(W, **kw):
    import paper_2511_21674_gb300 as ep
    kw.setdefault("record_grad", 1)
    kw.setdefault("record_raster", 1)
    kw.setdefault("launch_mode", 0)
    return ep.Network(W["spec"], W["ptr"], W["col"], W["w"], W["delay"], W["w_out"],
                      W["out_mask"], W["feedback"], **kw)


def _oracle(W):
    return oracle.Oracle(W["spec"], W["ptr"], W["col"], W["w"], W["delay"], W["w_out"],
                         W["out_mask"], W["feedback"])


def run_parity(W, calls=1, gpu_kw=None, inputs_per_call=None, check=True, grad_rtol=P.RTOL):
    """Runs `calls` simulate calls on both sides; returns a report dict."""
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    net = _gpu_net(W, **(gpu_kw or {}))
    orc = _oracle(W)
    rep = dict(ambiguous=0, mismatches=0, worst={})
    nnz_in = int(W["ptr"][s.n_in]) if s.n_in else 0
    nnz = int(W["ptr"][-1])
    g_or = np.zeros(nnz)
    g_mag = np.zeros(nnz)
    g_out_or = np.zeros((s.n_rec, s.n_out))
    g_out_mag = np.zeros((s.n_rec, s.n_out))
    w0 = np.abs(np.asarray(W["w"], np.float64))
    w_out0 = np.abs(np.asarray(W["w_out"], np.float64))
    for c in range(calls):
        inp = inputs_per_call[c] if inputs_per_call else W
        net.set_inputs(inp["x_ptr"], inp["x_ids"], inp["targets"], inp["window"], inp["lengths"], s.T)
        net.simulate(s.T)
        y, loss, raster = net.readout(raster=True)
        r = orc.simulate(s.T, inp["x_ptr"], inp["x_ids"], inp["targets"], inp["window"],
                         inp["lengths"], forced=raster)
        g, go = orc.take_grads()
        gm, gom = orc.take_grad_magnitudes()
        g_or += g
        g_mag += gm
        g_out_or += go
        g_out_mag += gom
        mm, amb = P.check_decisions(raster, r["margin"], s.v_th, s.t_ref, inp["lengths"])
        rep["mismatches"] += mm
        rep["ambiguous"] += amb
        rep.setdefault("spikes", 0)
        rep["spikes"] += int(raster.sum())
        if check:
            assert mm == 0, f"call {c}: {mm} spike decisions differ outside the ambiguity band"
            rep["worst"]["y"] = P.assert_close(y, r["y"], f"call {c} readout y", mag=r["y_abs"])
            rep["worst"]["loss"] = P.assert_close(loss, r["loss"], f"call {c} loss",
                                                  mag=_loss_mag(s, inp, r))
    net.sync()
    w_out, gw_out = net.weights(ep.PROJ_OUT, with_grad=True)
    w_rec, gw_rec = net.weights(ep.PROJ_REC, with_grad=True)
    rep["events"] = net.events()
    rec = slice(nnz_in, nnz)
    res = dict(w_rec=(w_rec, orc.w[rec], w0[rec] + s.lr * g_mag[rec]),
               g_rec=(gw_rec, g_or[rec], g_mag[rec]),
               w_out=(w_out, orc.w_out, w_out0 + s.lr * g_out_mag),
               g_out=(gw_out, g_out_or, g_out_mag))
    if s.n_in:
        w_in, gw_in = net.weights(ep.PROJ_IN, with_grad=True)
        inn = slice(0, nnz_in)
        res.update(w_in=(w_in, orc.w[inn], w0[inn] + s.lr * g_mag[inn]),
                   g_in=(gw_in, g_or[inn], g_mag[inn]))
    net.close()
    for k, (a, b, mag) in res.items():
        rep.setdefault("rel_l2", {})[k] = P.rel_l2(a, b)
        if check:
            rtol = grad_rtol if k.startswith("g") else P.RTOL
            rep["worst"][k] = P.assert_close(a, b, k, rtol=rtol, mag=mag)
    rep["res"] = {k: v[:2] for k, v in res.items()}
    return rep


def _loss_mag(s, inp, r):
    """loss + sum_t sum_k |E_k^t| |y|_abs,k^t per sample (first-order bound of
    the loss's sensitivity to the readout's rounding)."""
    y, yabs = r["y"], r["y_abs"]
    tg = np.asarray(inp["targets"], np.float64)
    win = np.asarray(inp["window"], np.float64)[..., None]
    if s.loss == 0:
        E = win * (y - tg)
    else:
        e = np.exp(y - y.max(axis=2, keepdims=True))
        E = win * (e / e.sum(axis=2, keepdims=True) - tg)
    return r["loss"] + (np.abs(E) * yabs).sum(axis=(1, 2))


def _pattern(**kw):
    return C.pattern_regression(**kw)


def test_pattern_regression_two_iterations():
    W = _pattern()
    rep = run_parity(W, calls=2)
    assert rep["spikes"] > 1000
    assert rep["ambiguous"] == 0


def test_pattern_regression_graph_mode_matches_eager():
    import paper_2511_21674_gb300 as ep
    W = _pattern(T=300)
    outs = []
    for mode in (0, 1):
        net = _gpu_net(W, launch_mode=mode)
        for _ in range(2):
            net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], 300)
            net.simulate(300)
        y, loss, r = net.readout(raster=True)
        outs.append((y, loss, r, net.weights(ep.PROJ_REC), net.weights(ep.PROJ_OUT)))
        net.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_gpu_runs_are_bitwise_deterministic():
    import paper_2511_21674_gb300 as ep
    W = C.sparse_balanced(n_rec=3000, k_in=300, T=200)
    outs = []
    for _ in range(2):
        net = _gpu_net(W)
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], 200)
        net.simulate(200)
        y, loss, r = net.readout(raster=True)
        outs.append((y, r, net.weights(ep.PROJ_REC, with_grad=True)[1]))
        net.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_event_classification_alif_batch_uneven_lengths():
    W = C.event_classification(batch=4)
    rep = run_parity(W)
    assert rep["spikes"] > 100


def test_sparse_balanced_scaled_replica_fp32():
    # same in-degree structure as the 1e5-neuron network, 4000 neurons
    W = C.sparse_balanced(n_rec=4000, k_in=1000, T=400, n_coupled=500)
    rep = run_parity(W)
    assert rep["events"] > 0


def test_million_sparse_scaled_replica_continuous_windows():
    # continuous dynamics, update window of 100 steps, two calls of 200 steps:
    # exercises the lazy catch-up of synapses across skipped windows
    W = C.million_sparse(n_rec=4000, k_in=1000, T=200, n_out=10)
    rep = run_parity(W, calls=2)
    assert rep["events"] > 0


def test_alif_continuous_short_windows():
    W = C.event_classification(batch=1, T=240, len_lo=240, len_hi=240, n_rec=60,
                               side=8, events_per_300=400.0)
    s = W["spec"]
    s.update_interval, s.continuous = 40, 1
    s.loss = 0
    rng = np.random.default_rng(0)
    W["targets"] = rng.normal(size=W["targets"].shape).astype(np.float32)
    W["window"][:] = 1
    run_parity(W, calls=2)


def test_delays_and_refractory_small_dense():
    rng = np.random.default_rng(9)
    W = C.sparse_balanced(n_rec=300, k_in=120, T=300, n_coupled=300, n_out=3, J=0.05)
    W["spec"].t_ref = 3
    W["spec"].max_delay = 5
    run_parity(W)


def test_forced_raster_on_gpu_matches_oracle_free_run():
    import torch
    import paper_2511_21674_gb300 as ep
    W = _pattern(T=400)
    s = W["spec"]
    orc = _oracle(W)
    r = orc.simulate(s.T, W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"])
    g_or, go_or = orc.take_grads()
    net = _gpu_net(W)
    net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
    forced = torch.from_numpy(r["raster"]).cuda()
    net.simulate(s.T, forced=forced)
    _, _, raster = net.readout(raster=True)
    assert np.array_equal(raster, r["raster"])
    w_rec, g_rec = net.weights(ep.PROJ_REC, with_grad=True)
    nnz_in = int(W["ptr"][s.n_in])
    gm, gom = orc.take_grad_magnitudes()
    P.assert_close(g_rec, g_or[nnz_in:], "forced recurrent gradient", mag=gm[nnz_in:])
    P.assert_close(net.weights(ep.PROJ_OUT, with_grad=True)[1], go_or, "forced readout gradient",
                   mag=gom)
    net.close()


def test_no_input_spikes_and_silent_network():
    W = _pattern(T=100)
    W["x_ptr"] = np.zeros_like(W["x_ptr"])
    W["x_ids"] = np.zeros(0, np.int32)
    rep = run_parity(W)
    assert rep["spikes"] == 0
    for k, (a, b) in rep["res"].items():
        if k.startswith("g_") and k != "g_out":
            assert np.all(a == 0)


def test_bf16_traces_report_error():
    # form (1): traces stored in BF16, FP32 accumulation; reported, not gated
    W = C.million_sparse(n_rec=4000, k_in=1000, T=200, n_out=10)
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_dtype=1), check=False)
    print("bf16 traces: rel_l2", rep["rel_l2"], "decision mismatches", rep["mismatches"])
    assert rep["rel_l2"]["g_rec"] < 5e-2

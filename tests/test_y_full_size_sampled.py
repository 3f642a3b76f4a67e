"""Parity at the full benchmark size on sampled synapses (GPU only).

The million-neuron workload (1e6 LIF neurons, in-degree 1000, 1e9 synapses,
delays 1..5, update window 100, continuous dynamics) runs in the launch
configuration the benchmark times (dense window form, one captured graph
per call, default launch shapes), with the recording switches on.  The
whole-network oracle cannot run at this size, so 256 synapses drawn at
random are checked one by one: `oracle.sampled_gradients` recomputes each
one's gradient in FP64 from the run's own history (its source's spikes, its
target's surrogate values, the readout), i.e. oracle B of the small parity
tests applied to a sample.  FP32 traces are held to the parity tolerance of
`tests/parity.py` (1e-5 of the magnitude sum of the terms plus 0.1 of the
sensitivity to the error signal) over two calls of 200 steps (four update
windows, state carried across the calls); BF16 traces, the benchmark's
storage, are held to 1e-2 relative L2 over the sample, the bound the small
BF16 test uses.  This file sorts before the no-allocation test and after
the others, so that a failure here stops a -x run late.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from tests import parity as P

pytestmark = pytest.mark.gpu

SAMPLE = 256
CALLS = 2
T_CALL = 200


def _run(trace_dtype):
    import torch
    import paper_2511_21674_gb300 as ep
    from workloads import gpu_build as G
    W = G.million_sparse_torch(T=T_CALL)
    s = W["spec"]
    T, K = s.T, s.n_out
    ptr, col, dly = W["ptr"], W["col"], W["delay"]
    nnz = int(col.shape[0])
    rng = np.random.default_rng(2468)
    q = np.sort(rng.choice(nnz, SAMPLE, replace=False))
    qt = torch.from_numpy(q).to(ptr.device)
    j = col[qt].long()
    i = torch.searchsorted(ptr, qt, right=True) - 1          # source row of each synapse
    sample = dict(i=i.cpu().numpy(), j=j.cpu().numpy(), d=dly[qt].long().cpu().numpy(),
                  w0=W["w"][qt].double().cpu().numpy(),
                  fb=W["feedback"][j].double().cpu().numpy())
    w_out0 = W["w_out"].cpu().numpy()
    net = ep.Network(s, ptr, col, W["w"], dly, W["w_out"], None, W["feedback"], launch_mode=1,
                     trace_dtype=trace_dtype, record_grad=1, record_raster=1, record_psi=1)
    del W["ptr"], W["col"], W["w"], W["delay"], W["w_out"], W["feedback"], ptr, col, dly
    torch.cuda.empty_cache()
    spk, psi, ys, ya_in = [], [], [], []
    for _ in range(CALLS):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], T)
        net.simulate(T)
        y, _, r = net.readout(raster=True)
        ps = net.surrogate()
        spk.append(r[0][:, sample["i"]])           # recurrent sources: n_in = 0
        psi.append(ps[0][:, sample["j"]])
        ys.append(y[0])
        ya_in.append(r[0])
        del ps
    wd = torch.empty(nnz, dtype=torch.float32, device="cuda")
    gd = torch.empty(nnz, dtype=torch.float32, device="cuda")
    net._check(net.lib.eprop_read_weights_grads(net.h, ep.PROJ_REC, wd.data_ptr(), gd.data_ptr(), 1))
    w_gpu = wd[qt].double().cpu().numpy()
    g_gpu = gd[qt].double().cpu().numpy()
    events = net.events()
    net.close()
    del wd, gd
    torch.cuda.empty_cache()
    raster = np.concatenate(ya_in, axis=0)
    kappa = math.exp(-s.dt / s.tau_out)
    y_abs = oracle.readout_magnitude(raster, w_out0, kappa)
    tg = np.concatenate([np.asarray(W["targets"], np.float64).reshape(T, K)] * CALLS, axis=0)
    win = np.concatenate([np.asarray(W["window"]).reshape(T)] * CALLS, axis=0)
    G_ref, mag, sens = oracle.sampled_gradients(
        s, np.concatenate(spk, axis=0).T, sample["d"], np.concatenate(psi, axis=0).T,
        np.concatenate(ys, axis=0), tg, win, sample["fb"], y_abs)
    return s, sample, events, g_gpu, w_gpu, G_ref, mag, sens


def test_full_size_sampled_gradients_fp32_traces():
    s, sample, events, g, w, G_ref, mag, sens = _run(trace_dtype=0)
    assert events > 5e8                               # ~5 Hz over 200 steps at 1e9 synapses
    assert np.count_nonzero(G_ref) > SAMPLE // 2
    tol = mag + 0.1 * sens
    P.assert_close(g, G_ref, "sampled recurrent gradients (FP32 traces)", mag=tol)
    P.assert_close(w, sample["w0"] - s.lr * G_ref, "sampled recurrent weights (FP32 traces)",
                   mag=np.abs(sample["w0"]) + s.lr * tol)


def test_full_size_sampled_gradients_bf16_traces():
    _, _, _, g, _, G_ref, _, _ = _run(trace_dtype=1)
    err = P.rel_l2(g, G_ref)
    print(f"BF16 traces, full size: relative L2 over {SAMPLE} sampled gradients {err:.3g}")
    assert err < 1e-2

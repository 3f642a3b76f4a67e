"""Band-major learning state (trace_kernel 4) on the GPU.

The band form stores the synapse records by target band and keeps a band's
window coefficients in shared memory; its arithmetic per synapse is that of
the source-major dense window pass (trace_kernel 3) and its delivery sums
the same int64 fixed-point arrivals, so the two forms must give the same
bits: spikes, readout, loss, every weight and gradient (read back in the
creation order).  Networks here span several bands (more than 12288 LIF or
4608 ALIF neurons).  The band form's parity with the FP64 oracle runs in
the parity suites (the trace_kernel parametrisations of
tests/test_gpu_parity.py) and once here on a multi-band network.
"""
from __future__ import annotations

import numpy as np
import pytest

from tests.test_gpu_parity import _gpu_net, run_parity
from workloads import configs as C

pytestmark = pytest.mark.gpu


def _multiband(n_rec=30_000, k_in=100, T=200, **over):
    # in-degree x weight as in the 1000-in-degree workload (~5 Hz)
    return C.million_sparse(n_rec=n_rec, k_in=k_in, J=0.1, n_out=10, T=T, lr=1e-5, **over)


def _run(W, calls, **kw):
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    net = _gpu_net(W, **kw)
    out = []
    for _ in range(calls):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
        out.append(net.readout(raster=True))
    net.sync()
    res = dict(calls=out, events=net.events(), out=net.weights(ep.PROJ_OUT, with_grad=True),
               rec=net.weights(ep.PROJ_REC, with_grad=True))
    if s.n_in:
        res["inp"] = net.weights(ep.PROJ_IN, with_grad=True)
    net.close()
    return res


def _assert_same_bits(a, b):
    assert a["events"] == b["events"]
    for c, (x, y) in enumerate(zip(a["calls"], b["calls"])):
        for k, (u, v) in enumerate(zip(x, y)):
            assert np.array_equal(np.asarray(u), np.asarray(v)), f"call {c}, readout item {k} differs"
    for key in ("out", "rec", "inp"):
        if key not in a:
            continue
        for name, u, v in zip(("w", "grad"), a[key], b[key]):
            u, v = np.asarray(u), np.asarray(v)
            bad = np.flatnonzero(u.view(np.uint32) != v.view(np.uint32))
            assert bad.size == 0, (f"{key} {name}: {bad.size} of {u.size} differ, first {bad[:5]}, "
                                   f"max |diff| {np.abs(u - v).max():.3g}")


@pytest.mark.parametrize("dtype", [0, 1, 2], ids=["fp32", "bf16", "fp16"])
def test_band_form_matches_source_major_bits(dtype):
    W = _multiband()
    a = _run(W, 3, trace_kernel=3, trace_dtype=dtype)
    b = _run(W, 3, trace_kernel=4, trace_dtype=dtype)
    assert a["events"] > 0
    _assert_same_bits(a, b)


def test_band_form_rows_in_any_order():
    # synapses of every row shuffled: the band records keep each row's
    # creation order and the read-back returns that order
    W = _multiband()
    ptr = W["ptr"]
    rng = np.random.default_rng(7)
    perm = np.arange(int(ptr[-1]))
    for r in range(len(ptr) - 1):
        seg = perm[ptr[r]:ptr[r + 1]]
        rng.shuffle(seg)
    for k in ("col", "w", "delay"):
        W[k] = np.ascontiguousarray(np.asarray(W[k])[perm])
    _assert_same_bits(_run(W, 2, trace_kernel=3), _run(W, 2, trace_kernel=4))


def test_band_form_sparse_rows_past_the_staged_records():
    # out-degree 5 over 4 bands: a tile of 1024 records spans ~800 source
    # rows, more than the 128 row records staged per tile
    W = C.million_sparse(n_rec=40_000, k_in=5, J=0.4, n_out=10, T=200, lr=1e-5)
    a = _run(W, 2, trace_kernel=3)
    assert a["events"] > 0
    _assert_same_bits(a, _run(W, 2, trace_kernel=4))


def test_band_form_alif_several_bands():
    W = _multiband(n_rec=12_000, k_in=100, neuron_model=1, beta_a=0.05, tau_a=200.0)
    a = _run(W, 2, trace_kernel=3)
    assert a["events"] > 0
    _assert_same_bits(a, _run(W, 2, trace_kernel=4))


def test_band_form_with_inputs_and_ignore_and_fire():
    # the scaling network's structure (Poisson inputs, ignore-and-fire, sparse
    # readout and feedback) over two bands
    W = C.scaling_network(n_rec=15_000, k_rec=100, n_in=100, k_in=10, n_out=4, k_out=200,
                          fb_outdeg=50, T=400, update_interval=100)
    _assert_same_bits(_run(W, 2, trace_kernel=3), _run(W, 2, trace_kernel=4))


def test_band_form_parity_with_the_oracle_multiband():
    # a small learning rate keeps the weights near their initial values (at
    # lr 1e-5 this network's weights grow a hundredfold within one call, and
    # their FP32 rounding moves membranes outside the decision band)
    W = _multiband(n_rec=30_000, k_in=100, T=200)
    W["spec"].lr = 1e-7
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_kernel=4))
    assert rep["events"] > 0
    assert rep["rows_2plus"] > 0


def test_band_form_restrictions():
    import paper_2511_21674_gb300 as ep
    W = _multiband(n_rec=20_000, T=200)
    W["spec"].optimizer = 1
    with pytest.raises(ep.EpropError, match="trace_kernel 4"):
        _gpu_net(W, trace_kernel=4)

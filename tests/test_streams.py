"""Readout work on a second stream (GPU only).

Without a predictor the per-step readout kernels and the window's readout
weight update run on a second stream, forked from the main stream after each
neuron update and joined back at window ends; a predictor attached in
record-only mode keeps every kernel on the main stream without changing any
arithmetic.  Both schedules must give the same bits, eager and captured.
"""
from __future__ import annotations

import numpy as np
import pytest

from workloads import configs as C

pytestmark = pytest.mark.gpu


def _run(W, serial, launch_mode, calls=3):
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    net = ep.Network(W["spec"], W["ptr"], W["col"], W["w"], W["delay"], W["w_out"],
                     W["out_mask"], W["feedback"], record_grad=1, record_raster=1,
                     launch_mode=launch_mode)
    pred = None
    if serial:
        pred = ep.Predictor(s.n_out + 64, s.n_out, seed=1, max_rows=s.batch)
        net.attach_predictor(pred, mode=2)
    for _ in range(calls):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
    y, loss, r = net.readout(raster=True)
    out = (y, loss, r, *net.weights(ep.PROJ_REC, with_grad=True), *net.weights(ep.PROJ_OUT, with_grad=True))
    net.close()
    if pred is not None:
        pred.close()
    return out


@pytest.mark.parametrize("launch_mode", [0, 1])
def test_forked_readout_matches_the_single_stream_schedule(launch_mode):
    # continuous dynamics, update window 100 inside calls of 200 steps: the
    # readout stream trails the neuron updates within each window
    W = C.million_sparse(n_rec=4000, k_in=400, J=0.025, n_out=10, T=200, drive_rate=1.25, lr=1e-5)
    a = _run(W, serial=False, launch_mode=launch_mode)
    b = _run(W, serial=True, launch_mode=launch_mode)
    assert a[2].sum() > 0
    for x, y in zip(a, b):
        assert np.array_equal(x, y)

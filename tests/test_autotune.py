"""Autotuner of the launch shapes (GPU only): it must leave the network
state exactly as it found it and apply the shape it reports; results do not
depend on the CTAs per SM (exact fixed-point delivery, per-synapse traces),
so a tuned network matches an untuned one bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

from workloads import configs as C

pytestmark = pytest.mark.gpu


def _net(W, **kw):
    import paper_2511_21674_gb300 as ep
    kw.setdefault("record_grad", 1)
    kw.setdefault("record_raster", 1)
    return ep.Network(W["spec"], W["ptr"], W["col"], W["w"], W["delay"], W["w_out"],
                      W["out_mask"], W["feedback"], **kw)


def _calls(net, W, n):
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    for _ in range(n):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
    y, loss, r = net.readout(raster=True)
    return (y, loss, r, net.weights(ep.PROJ_REC, with_grad=True)[1], net.weights(ep.PROJ_OUT))


def test_autotune_before_the_first_call_applies_its_choice_and_keeps_the_state():
    W = C.million_sparse(n_rec=3000, k_in=300, J=0.033, n_out=5, T=200, drive_rate=1.25, lr=1e-5)
    s = W["spec"]
    a = _net(W)
    a.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
    res = a.autotune()
    assert res["trace_kernel"] in (1, 3) and 1 <= res["blocks_per_sm"] <= 4
    assert len(res["candidates"]) == 8 and all(ms > 0 for _, _, ms in res["candidates"])
    out_a = _calls(a, W, 2)
    b = _net(W, trace_kernel=res["trace_kernel"], blocks_per_sm=res["blocks_per_sm"])
    out_b = _calls(b, W, 2)
    for x, y in zip(out_a, out_b):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def test_autotune_of_the_batched_form_midway_keeps_the_state():
    W = C.event_classification(batch=8, T=200, len_lo=150, len_hi=200, n_rec=100, side=16,
                               events_per_300=3000.0)
    a, b = _net(W, launch_mode=1), _net(W, launch_mode=1)
    _calls(a, W, 1)
    _calls(b, W, 1)
    res = a.autotune()
    assert len(res["candidates"]) == 4        # the trace form is fixed once state exists
    out_a, out_b = _calls(a, W, 2), _calls(b, W, 2)
    for x, y in zip(out_a, out_b):
        assert np.array_equal(x, y)
    a.close()
    b.close()

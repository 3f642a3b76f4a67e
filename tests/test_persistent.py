"""Form (2): the persistent step loop (launch_mode 2) (GPU only).

Every step of a call runs in one cooperative kernel with grid barriers
between the neuron phase and the delivery phase, captured in the call's
CUDA graph.  Its arithmetic is that of the per-step kernels, so its results
must be bit-identical to the graph of per-step launches (launch_mode 1),
which the parity tests check against the FP64 oracle; one batched case is
also checked against the oracle directly.
"""
from __future__ import annotations

import numpy as np
import pytest

from tests.test_gpu_parity import _gpu_net, run_parity
from workloads import configs as C

pytestmark = pytest.mark.gpu


def _outputs(W, mode, calls=2):
    import paper_2511_21674_gb300 as ep
    s = W["spec"]
    net = _gpu_net(W, launch_mode=mode)
    for _ in range(calls):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
    y, loss, r = net.readout(raster=True)
    out = [y, loss, r, net.surrogate(), *net.weights(ep.PROJ_REC, with_grad=True),
           *net.weights(ep.PROJ_OUT, with_grad=True), net.events()]
    if s.n_in:
        out += list(net.weights(ep.PROJ_IN, with_grad=True))
    net.close()
    return out


@pytest.mark.parametrize("case", ["batch64", "single_sample"])
def test_persistent_loop_is_bitwise_the_graph_of_launches(case):
    if case == "batch64":
        W = C.event_classification(batch=64)
    else:
        W = C.pattern_regression(T=400)
    a = _outputs(W, 1)
    b = _outputs(W, 2)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_persistent_loop_against_the_oracle():
    W = C.event_classification(batch=4, T=150, len_lo=100, len_hi=150, n_rec=60, side=8,
                               events_per_300=3000.0)
    rep = run_parity(W, gpu_kw=dict(launch_mode=2))
    assert rep["spikes"] > 100


def test_persistent_loop_rejects_carried_state():
    import paper_2511_21674_gb300 as ep
    W = C.pattern_regression(T=200, update_interval=100, continuous=1)
    with pytest.raises(ep.EpropError, match="launch_mode 2"):
        _gpu_net(W, launch_mode=2)

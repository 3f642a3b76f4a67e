"""Update windows inside a call with a mini-batch (GPU only).

With batch > 1 and update_interval > 0 every synapse carries one
eligibility state per sample and the shared weight takes one step with the
batch mean at every window end (Eq. accumulated-gradients, Eq.
gradient-descent): online updates before a sample's target window, in the
batched form.  The FP64 oracle runs the same batch time-driven with the same
window ends; oracle A is teacher-forced with the GPU raster, oracle B also
with its surrogate values (the parity rules of tests/test_gpu_parity.py).
"""
from __future__ import annotations

import pytest

from tests.test_gpu_parity import _gpu_net, _replica, run_parity
from workloads import configs as C

pytestmark = pytest.mark.gpu


def test_alif_event_classification_batch_with_update_windows():
    # 4 ALIF samples of uneven length (200-300 steps), windows of 100 steps:
    # samples end inside the last window; CE on each sample's last 25 steps
    W = C.event_classification(batch=4, T=300, len_lo=200, len_hi=300, n_rec=60, side=8,
                               events_per_300=3000.0, update_interval=100)
    rep = run_parity(W, calls=2)
    assert rep["spikes"] > 100
    assert rep["rows_2plus"] > 0


def test_lif_sparse_replica_batch_with_update_windows():
    # the million-neuron replica with 3 samples (each its own Poisson
    # drive), windows of 100 steps inside calls of 300 steps, every call
    # from zero state
    W = _replica(True, 300, batch=3)
    W["spec"].continuous = 0
    rep = run_parity(W, calls=2)
    assert rep["events"] > 0
    assert rep["rows_3plus"] > 0


def test_batch_with_update_windows_and_16bit_traces():
    # BF16 traces per sample: reported against the oracle (relative L2)
    from tests import parity as P
    W = _replica(True, 200, batch=2)
    W["spec"].continuous = 0
    rep = run_parity(W, calls=2, gpu_kw=dict(trace_dtype=1), check=False)
    gw, ref = rep["res"]["g_rec"]
    assert P.rel_l2(gw, ref) < 1e-2


def test_batch_restrictions():
    import paper_2511_21674_gb300 as ep
    W = _replica(False, 200, batch=2, update_interval=100)
    W["spec"].continuous = 1
    with pytest.raises(ep.EpropError, match="continuous = 0"):
        _gpu_net(W)
    W["spec"].continuous = 0
    with pytest.raises(ep.EpropError, match="lazy"):
        _gpu_net(W, trace_kernel=1)

"""Raster readout through the library's fixed device scratch (GPU only).

eprop_readout_raster_static serves callers that cannot allocate device
memory when they read a raster (a monitor beside a simulation that holds
the device's memory, a loop that must not trigger an allocation's implicit
synchronisation).  It must return the same raster as eprop_readout (which
allocates its scratch on first use), on consecutive calls; called first on
a fresh network it must leave the device's free memory unchanged; it
rejects a raster larger than its scratch.  Collected last so that it also
runs after every other GPU test in the session.
"""
from __future__ import annotations

import numpy as np
import pytest

from workloads import configs as C

pytestmark = pytest.mark.gpu


def _net(W, **kw):
    import paper_2511_21674_gb300 as ep
    return ep.Network(W["spec"], W["ptr"], W["col"], W["w"], W["delay"], W["w_out"],
                      W["out_mask"], W["feedback"], record_raster=1, launch_mode=0, **kw)


def test_static_raster_matches_allocating_readout_on_consecutive_calls():
    W = C.event_classification(batch=3, T=120, len_lo=80, len_hi=120, n_rec=60, side=8,
                               events_per_300=2000.0)
    s = W["spec"]
    net = _net(W)
    spikes = 0
    for _ in range(2):
        net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
        net.simulate(s.T)
        _, _, r_alloc = net.readout(raster=True)
        r_static = net.raster_static()
        assert r_static.shape == r_alloc.shape
        assert np.array_equal(r_static, r_alloc)
        spikes += int(r_alloc.sum())
    net.close()
    assert spikes > 0


def test_static_raster_allocates_nothing_on_a_fresh_network():
    # a network that has never read a raster: eprop_readout would allocate
    # its scratch now; the static variant must not change the free memory
    import torch
    W = C.event_classification(batch=2, T=100, len_lo=100, len_hi=100, n_rec=50, side=8,
                               events_per_300=2000.0)
    s = W["spec"]
    net = _net(W)
    net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], s.T)
    net.simulate(s.T)
    net.sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    r_static = net.raster_static()
    r_again = net.raster_static()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    _, _, r_alloc = net.readout(raster=True)
    net.close()
    assert np.array_equal(r_static, r_alloc)
    assert np.array_equal(r_again, r_alloc)
    assert r_alloc.sum() > 0


def test_static_raster_rejects_more_than_its_scratch():
    import paper_2511_21674_gb300 as ep
    from paper_2511_21674_gb300 import EpropError
    limit = 16 * 1024 * 1024
    n_rec, T = 20000, 1000                     # 2e7 bytes > 16 MiB
    assert n_rec * T > limit
    W = C.million_sparse(n_rec=n_rec, k_in=5, n_out=2, T=T)
    net = _net(W)
    net.set_inputs(W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], T)
    with pytest.raises(EpropError, match="EPROP_STATIC_RASTER_BYTES"):
        net.raster_static()
    net.close()

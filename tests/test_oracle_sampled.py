"""Pins of the oracle's sampled-synapse gradients (CPU only).

`oracle.sampled_gradients` computes the gradient of chosen synapses from a
given postsynaptic history (source spikes, surrogate values, readout); the
full-size parity test relies on it where the whole-network simulation
cannot run.  Here it is pinned against the whole-network FP64 simulation of
small networks on every synapse: the same gradient, magnitude sum and
sensitivity sum over several update windows and two continuous calls, for
LIF with MSE and delays 1..5 and for ALIF with softmax cross-entropy, input
sources and a closed target window.  Its learning signal and readout
magnitude are pinned against the ones the simulation records.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from workloads import configs as C


def _runs(W, calls):
    s = W["spec"]
    o = oracle.Oracle(s, W["ptr"], W["col"], W["w"], W["delay"], W["w_out"], W["out_mask"], W["feedback"])
    rs = [o.simulate(s.T, W["x_ptr"], W["x_ids"], W["targets"], W["window"], W["lengths"], record=True)
          for _ in range(calls)]
    g, _ = o.take_grads()
    m, _ = o.take_grad_magnitudes()
    se, _ = o.take_grad_sensitivities()
    return rs, g, m, se


def _source_spikes(W, rs):
    """[T_total, n_src] spikes of every source over the concatenated calls."""
    s = W["spec"]
    T = s.T
    out = []
    for r in rs:
        x = np.zeros((T, s.n_in), np.uint8)
        for t in range(T):
            ids = W["x_ids"][W["x_ptr"][t]:W["x_ptr"][t + 1]]
            x[t, ids] = 1
        out.append(np.concatenate([x, r["raster"][0]], axis=1))
    return np.concatenate(out, axis=0)


def _check_all_synapses(W, calls):
    s = W["spec"]
    rs, g, m, se = _runs(W, calls)
    ptr = np.asarray(W["ptr"])
    col = np.asarray(W["col"])
    nnz = int(ptr[-1])
    src_of = np.repeat(np.arange(ptr.shape[0] - 1), np.diff(ptr))
    spk = _source_spikes(W, rs)
    psi = np.concatenate([r["psi"][0] for r in rs], axis=0)
    y = np.concatenate([r["y"][0] for r in rs], axis=0)
    y_abs = np.concatenate([r["y_abs"][0] for r in rs], axis=0)
    tg = np.concatenate([np.asarray(W["targets"], np.float64).reshape(s.T, s.n_out)] * calls, axis=0)
    win = np.concatenate([np.asarray(W["window"]).reshape(s.T)] * calls, axis=0)
    fb = np.asarray(W["feedback"], np.float64)
    # the learning signal the sampled form builds equals the recorded one
    E, _ = oracle.error_signal(s, y, tg, win, y_abs)
    L_rec = np.concatenate([r["L"][0] for r in rs], axis=0)
    np.testing.assert_allclose(E @ fb.T, L_rec, rtol=1e-12, atol=1e-14 * np.abs(L_rec).max())
    G, mag, sens = oracle.sampled_gradients(s, spk[:, src_of].T, np.asarray(W["delay"]),
                                            psi[:, col].T, y, tg, win, fb[col], y_abs)
    assert nnz == G.shape[0] and np.abs(g).max() > 0
    np.testing.assert_allclose(G, g, rtol=0, atol=1e-12 * (m.max() + 1e-300))
    np.testing.assert_allclose(mag, m, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(sens, se, rtol=1e-12, atol=1e-300)
    return rs


def test_lif_mse_delays_continuous_windows_every_synapse():
    W = C.million_sparse(n_rec=300, k_in=30, J=0.1, n_out=5, T=200, drive_rate=1.25, lr=1e-4)
    rs = _check_all_synapses(W, calls=2)
    assert sum(int(r["raster"].sum()) for r in rs) > 100
    assert W["spec"].update_interval == 100 and W["spec"].continuous == 1


def test_alif_cross_entropy_inputs_and_target_window_every_synapse():
    W = C.event_classification(batch=1, T=240, len_lo=240, len_hi=240, n_rec=60, side=6,
                               events_per_300=800.0)
    s = W["spec"]
    s.update_interval, s.continuous = 40, 1
    s.feedback = 1
    rng = np.random.default_rng(11)
    W["feedback"] = (rng.standard_normal((s.n_rec, s.n_out)) / math.sqrt(s.n_out)).astype(np.float32)
    W["window"] = np.asarray(W["window"]).copy()
    W["window"][:, :120] = 0            # error signal only in the second half
    rs = _check_all_synapses(W, calls=2)
    assert sum(int(r["raster"].sum()) for r in rs) > 50


def test_readout_magnitude_matches_the_simulation():
    W = C.million_sparse(n_rec=300, k_in=30, J=0.1, n_out=5, T=200, drive_rate=1.25, lr=0.0)
    s = W["spec"]
    rs, _, _, _ = _runs(W, 1)
    ya = oracle.readout_magnitude(rs[0]["raster"][0], W["w_out"], math.exp(-s.dt / s.tau_out))
    np.testing.assert_allclose(ya, rs[0]["y_abs"][0], rtol=1e-12, atol=1e-300)

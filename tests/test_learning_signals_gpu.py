"""The window's learning-signal product L = B E on the tensor cores (GPU only).

eprop_learning_signals forms L[b][u][j] = sum_k B[j][k] E[b][u][k]
(Eq. final-gradient) with TF32 operands split into hi + lo parts and FP32
accumulation.  Compared element by element with the FP64 product of the
same FP32 inputs: |L_gpu - L_ref| <= RTOL * sum_k |B_jk E_k| with RTOL =
1e-5, the parity tolerance of every accumulated FP32 quantity (the FP32
rounding of a K-term sum is bounded relative to the sum of the terms'
magnitudes).  The worst ratio is also reported against 1e-6 (the level of
an FP32 FMA loop).  Shapes cover ragged tiles: neurons not a multiple of
the 128-row tile, window lengths not a multiple of 16 and above the 256
columns of one pass, K not a multiple of the 8-element K-step nor of the
32-element chunk, K = 1, K of seven chunks, several samples, and one window
of one sample over many tiles (the warp-specialised form of U, K <= 128).
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-5

SHAPES = [
    # (n_rec, U, n_out, batch)
    (1000, 100, 100, 1),       # million-neuron workload's window, scaled down
    (300, 37, 10, 3),          # event classification's readouts, ragged U
    (130, 300, 1, 2),          # pattern regression: K = 1, two passes of columns
    (129, 16, 33, 1),          # two K chunks, last one with one element
    (5000, 257, 64, 1),        # 257 steps: a pass of 256 and one of 1
    (257, 512, 8, 1),          # exactly two full passes
    (300, 50, 200, 1),         # K = 200: seven K-chunks
    (4000, 100, 100, 3),       # several samples over many tiles
    # one window of one sample (the warp-specialised form): several tiles
    # per CTA (stage and accumulator reuse), full U and K, tiny shapes
    (100_000, 100, 100, 1),
    (2000, 128, 128, 1),
    (300, 5, 7, 1),
]


def _run(n_rec, U, K, B, seed):
    import torch
    import paper_2511_21674_gb300 as ep
    rng = np.random.default_rng(seed)
    fb = rng.normal(size=(n_rec, K)).astype(np.float32)
    E = rng.normal(size=(B, U, K)).astype(np.float32)
    # a few exact zeros and wide magnitudes, as error signals outside a
    # target window and feedback rows of unconnected neurons have
    E[:, ::7, :] = 0.0
    fb[::11, :] *= 1e-3
    L = ep.learning_signals(torch.from_numpy(fb).cuda(), torch.from_numpy(E).cuda()).cpu().numpy()
    f64, e64 = fb.astype(np.float64), E.astype(np.float64)
    ref = np.einsum("jk,buk->buj", f64, e64)
    mag = np.einsum("jk,buk->buj", np.abs(f64), np.abs(e64))
    return L, ref, mag


@pytest.mark.parametrize("shape", SHAPES, ids=[f"N{a}_U{b}_K{c}_B{d}" for a, b, c, d in SHAPES])
def test_learning_signals_match_fp64(shape):
    n_rec, U, K, B = shape
    L, ref, mag = _run(n_rec, U, K, B, seed=sum(shape))
    assert L.shape == (B, U, n_rec)
    err = np.abs(L.astype(np.float64) - ref)
    ratio = float((err / (RTOL * mag + 1e-30)).max())
    print(f"L = B E {shape}: worst |err| / (1e-5 sum|B||E|) = {ratio:.3g}")
    assert ratio <= 1.0
    # exact zeros stay zero (rows of E that are zero)
    assert np.all(L[:, ::7, :] == 0.0)


def test_learning_signals_reject_host_pointers():
    import ctypes
    import paper_2511_21674_gb300 as ep
    lib = ep.load_library()
    a = np.zeros(16, np.float32)
    st = lib.eprop_learning_signals(a.ctypes.data, a.ctypes.data, a.ctypes.data, 4, 2, 2, 1, None)
    assert st == 1
    assert b"device pointers" in lib.eprop_last_error(None)
    del ctypes

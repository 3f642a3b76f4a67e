"""GPU-vs-oracle comparison helpers for the parity tests.

Agreement rules (written out here and in each test):
* spike rasters: the oracle is teacher-forced with the GPU raster; every GPU
  spike decision must equal the oracle's FP64 decision (v - v_th > 0 and not
  refractory) except where |v - v_th| <= DELTA_V * (1 + |v|), a bound on the
  FP32 rounding of the membrane recursion; such ambiguous steps are counted;
* every accumulated quantity q = sum_i x_i is compared with a relative
  tolerance of RTOL = 1e-5 taken on the condition of the sum,
  |gpu - oracle| <= RTOL * sum_i |x_i|  (>= RTOL * |q|),
  because the FP32 rounding error of a sum is bounded relative to the sum
  of the magnitudes of its terms, not to its possibly cancelled value.  The
  oracle reports these magnitude sums: sum_t |g^t| per gradient element,
  the |W_out|-filtered |y| per readout step; a weight after updates is
  compared on |w_0| + lr * sum |g^t|; a loss on loss + sum |E| |y|_abs.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-5
FLOOR = 1e-3
DELTA_V = 1e-5


def refractory_mask(raster, t_ref):
    """[B, T, N] True where the neuron is refractory at that step."""
    B, T, N = raster.shape
    ref = np.zeros_like(raster, dtype=bool)
    for k in range(1, t_ref + 1):
        ref[:, k:, :] |= raster[:, :-k, :].astype(bool)
    return ref


def check_decisions(raster_gpu, margin_or, v_th_or, t_ref, lengths):
    """Returns (mismatches outside the ambiguity band, ambiguous count)."""
    ref = refractory_mask(raster_gpu, t_ref)
    decide = (margin_or > 0.0) & ~ref
    B, T, N = raster_gpu.shape
    active = np.arange(T)[None, :, None] < np.asarray(lengths)[:, None, None]
    v = margin_or + v_th_or
    amb = np.abs(margin_or) <= DELTA_V * (1.0 + np.abs(v))
    diff = (decide != raster_gpu.astype(bool)) & active
    return int((diff & ~amb).sum()), int((amb & active & ~ref).sum())


def assert_close(gpu, ref, what, rtol=RTOL, floor=FLOOR, mag=None):
    """|gpu - ref| <= rtol * mag element-wise (mag = magnitude sum of the
    terms of each element, >= |ref|); without mag, a relative tolerance with
    a floor of `floor` times the largest |ref|."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    if ref.size == 0:
        return 0.0
    if mag is not None:
        mag = np.asarray(mag, dtype=np.float64).ravel()
        tol = rtol * np.maximum(mag, np.abs(ref)) + 1e-30
    else:
        scale = np.abs(ref).max()
        tol = rtol * np.maximum(np.abs(ref), floor * scale) + 1e-30
    err = np.abs(gpu - ref)
    bad = err > tol
    worst = float((err / tol).max())
    if bad.any():
        idx = np.nonzero(bad)[0][:5]
        raise AssertionError(f"{what}: {int(bad.sum())}/{ref.size} elements outside tolerance; "
                             f"worst err/tol={worst:.3g}; first {idx.tolist()} gpu={gpu[idx]} ref={ref[idx]}")
    return worst


def rel_l2(gpu, ref):
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(gpu - ref) / den) if den > 0 else float(np.linalg.norm(gpu))

"""GPU-vs-oracle comparison helpers for the parity tests.

Agreement rules (written out here and in each test):
* spike rasters: the oracle is teacher-forced with the GPU raster; every GPU
  spike decision must equal the oracle's FP64 decision (v - v_th > 0 and not
  refractory) except where |v - v_th| <= DELTA_V * (1 + |v|), a bound on the
  FP32 rounding of the membrane recursion; such ambiguous steps are counted;
  DELTA_V = 2e-6 is the same membrane bound the surrogate check below uses
  (the compensated FP32 membrane stays within 2e-6 (1 + |v - v_th|) of the
  FP64 one: the surrogate check, Lipschitz in the membrane, passes with it);
* surrogate values: |psi_gpu - psi_oracle| <= gamma beta_sg 2e-6 (1 + |v -
  v_th|), the FP32 Lipschitz bound of psi in the membrane;
* every accumulated quantity q = sum_i x_i is compared with a relative
  tolerance of RTOL = 1e-5 taken on the condition of the sum,
  |gpu - oracle| <= RTOL * sum_i |x_i|  (>= RTOL * |q|),
  because the FP32 rounding error of a sum is bounded relative to the sum
  of the magnitudes of its terms, not to its possibly cancelled value.  The
  oracle reports these magnitude sums: sum_t |g^t| per gradient element,
  the |W_out|-filtered |y| per readout step; a weight after updates is
  compared on |w_0| + lr * sum |g^t|; a loss on loss + sum |E| |y|_abs.
  In single-window calls the magnitude sum also counts the per-arrival terms
  the event-driven sum is formed from (oracle.arrival_magnitude).
  Gradients additionally carry 0.1 x their sensitivity to a relative
  perturbation of the error signal (sum_t Lsens^t |ebar^t|, i.e. an FP32
  error of 1e-6 relative on y and y*), for steps where y - y* cancels.
"""
from __future__ import annotations

import json
import os

import numpy as np

RTOL = 1e-5
FLOOR = 1e-3
DELTA_V = 2e-6


def refractory_mask(raster, t_ref):
    """[B, T, N] True where the neuron is refractory at that step."""
    B, T, N = raster.shape
    ref = np.zeros_like(raster, dtype=bool)
    for k in range(1, t_ref + 1):
        ref[:, k:, :] |= raster[:, :-k, :].astype(bool)
    return ref


def check_decisions(raster_gpu, margin_or, v_th_or, t_ref, lengths, prev_raster=None):
    """Returns (mismatches outside the ambiguity band, ambiguous count).
    prev_raster: the previous call's raster when dynamics are continuous
    (a spike at its end keeps the neuron refractory into this call)."""
    if prev_raster is not None and t_ref > 0:
        full = np.concatenate([prev_raster[:, -t_ref:], raster_gpu], axis=1)
        ref = refractory_mask(full, t_ref)[:, t_ref:]
    else:
        ref = refractory_mask(raster_gpu, t_ref)
    decide = (margin_or > 0.0) & ~ref
    B, T, N = raster_gpu.shape
    active = np.arange(T)[None, :, None] < np.asarray(lengths)[:, None, None]
    v = margin_or + v_th_or
    amb = np.abs(margin_or) <= DELTA_V * (1.0 + np.abs(v))
    diff = (decide != raster_gpu.astype(bool)) & active
    return int((diff & ~amb).sum()), int((amb & active & ~ref).sum())


def psi_error(psi_gpu, r_or, spec):
    """max over elements of |psi_gpu - psi_oracle| / bound, where bound =
    gamma beta_sg 2e-6 (1 + |v - v_th|) + 1e-9: the surrogate is Lipschitz in
    the membrane with constant gamma beta_sg, and the GPU's compensated FP32
    membrane differs from the FP64 one by a few FP32 roundings of |v - v_th|
    (values above 1 mean outside the bound).  r_or needs record=True."""
    m = r_or["margin"]
    bound = spec.gamma * spec.beta_sg * 2e-6 * (1.0 + np.abs(m)) + 1e-9
    err = np.abs(psi_gpu.astype(np.float64) - r_or["psi"]) / bound
    return float(err.max()) if err.size else 0.0


def loss_magnitude(s, W, r):
    """loss + sum_t sum_k |E_k^t| |y|_abs,k^t per sample (first-order bound of
    the loss's sensitivity to the readout's rounding)."""
    y, yabs = r["y"], r["y_abs"]
    tg = np.asarray(W["targets"], np.float64)
    win = np.asarray(W["window"], np.float64)[..., None]
    if s.loss == 0:
        E = win * (y - tg)
    elif s.loss == 2:
        E = win * (2.0 / y.shape[2]) * (y - tg)
    else:
        e = np.exp(y - y.max(axis=2, keepdims=True))
        E = win * (e / e.sum(axis=2, keepdims=True) - tg)
    return r["loss"] + (np.abs(E) * yabs).sum(axis=(1, 2))


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


def survey_ratio(gpu, ref, rtol=RTOL, floor=FLOOR):
    """Worst |gpu - ref| / (rtol * max(|ref|, floor * max|ref|)) over the
    elements: the plain relative rule (1e-5 relative with a floor at 1e-3
    of the largest element), reported beside the magnitude-sum gate."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    if ref.size == 0:
        return 0.0
    tol = rtol * np.maximum(np.abs(ref), floor * np.abs(ref).max()) + 1e-30
    return float((np.abs(gpu - ref) / tol).max())


def gate_ratio(gpu, ref, mag, rtol=RTOL):
    """Worst |gpu - ref| / (rtol * max(mag, |ref|)) (<= 1 passes)."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    if ref.size == 0:
        return 0.0
    mag = np.asarray(mag, dtype=np.float64).ravel()
    tol = rtol * np.maximum(mag, np.abs(ref)) + 1e-30
    return float((np.abs(gpu - ref) / tol).max())


def report(rep: dict):
    """Appends the report of one parity case as a JSON line to the file
    named by EPROP_PARITY_REPORT (if set), tagged with the running test."""
    path = os.environ.get("EPROP_PARITY_REPORT")
    if not path:
        return
    keep = {k: v for k, v in rep.items() if k != "res"}
    keep["test"] = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    with open(path, "a") as f:
        f.write(json.dumps(keep, default=float) + "\n")


# ------------------------------------------------------------------
# per-sample oracle runs (a batch split over worker processes)


def sample_slice(W, b):
    """The one-sample workload of sample b of a batched workload (same
    network, the sample's inputs, targets, window and length)."""
    import copy
    s = copy.copy(W["spec"])
    B, T = s.batch, s.T
    s.batch = 1
    p0, p1 = int(W["x_ptr"][b * T]), int(W["x_ptr"][(b + 1) * T])
    Wb = {k: W[k] for k in ("ptr", "col", "w", "delay", "w_out", "out_mask", "feedback")}
    Wb.update(spec=s, x_ptr=np.asarray(W["x_ptr"][b * T:(b + 1) * T + 1]) - p0,
              x_ids=np.asarray(W["x_ids"][p0:p1]),
              targets=np.asarray(W["targets"][b:b + 1]), window=np.asarray(W["window"][b:b + 1]),
              lengths=np.asarray(W["lengths"][b:b + 1]))
    return Wb


def sample_oracle_job(job):
    """Oracles A (teacher-forced spikes) and B (spikes and surrogate values)
    of one sample of a single-window batched call; returns everything the
    parity check aggregates over the batch."""
    import oracle
    oracle.set_threads(1)                 # one thread per worker process
    Wb, raster, psi = job
    s = Wb["spec"]
    mk = lambda: oracle.Oracle(s, Wb["ptr"], Wb["col"], Wb["w"], Wb["delay"], Wb["w_out"],
                               Wb["out_mask"], Wb["feedback"])
    orA, orB = mk(), mk()
    args = (s.T, Wb["x_ptr"], Wb["x_ids"], Wb["targets"], Wb["window"], Wb["lengths"])
    rA = orA.simulate(*args, forced=raster, record=True)
    rB = orB.simulate(*args, forced=raster, forced_psi=psi, record=True)
    out = {}
    out["gA"], out["goA"] = orA.take_grads()
    out["gB"], out["goB"] = orB.take_grads()
    out["magB"], out["gomB"] = orB.take_grad_magnitudes()
    out["sensB"], out["gosB"] = orB.take_grad_sensitivities()
    out["arrB"] = oracle.arrival_magnitude(s, Wb["ptr"], Wb["col"], Wb["delay"], Wb["x_ptr"],
                                           Wb["x_ids"], Wb["lengths"], raster, rB["psi"], rB["L"])
    out["wB"], out["woB"] = orB.w, orB.w_out
    out["mm"], out["amb"] = check_decisions(raster, rA["margin"], s.v_th, s.t_ref, Wb["lengths"])
    out["psi_err"] = psi_error(psi, rA, s)
    out["yA"], out["y_absA"], out["lossA"] = rA["y"], rA["y_abs"], rA["loss"]
    out["loss_magA"] = loss_magnitude(s, Wb, rA)
    return out


def pooled_sample_oracles(W, raster, psi, processes=None):
    """sample_oracle_job for every sample of the batch, in a pool of worker
    processes started with 'spawn' (safe beside an initialised CUDA
    context)."""
    import multiprocessing as mp
    B = W["spec"].batch
    jobs = [(sample_slice(W, b), raster[b:b + 1], psi[b:b + 1]) for b in range(B)]
    n = processes or min(B, max(1, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(sample_oracle_job, jobs)

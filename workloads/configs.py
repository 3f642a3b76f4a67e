"""Seeded synthetic workloads shaped like the paper's tasks.

Every array is drawn from counter-based hashes (`hashrng`) of the seed and
the element's indices, so a workload can be regenerated on any host (numpy)
or directly on a GPU (torch) with identical integer structure.

Workloads (steps of 1 ms):

* ``pattern_regression`` -- pattern generation (Methods, "Pattern
  generation"): 20 frozen Poisson inputs at 50 Hz, 100 LIF neurons with
  all-to-all recurrence (no autapses), one leaky readout, target = sum of four
  sinusoids, T = 1000, symmetric feedback.
* ``event_classification`` -- a stand-in for N-MNIST (Methods,
  "Neuromorphic MNIST"): 2 x 34 x 34 input channels driven by class-specific
  Gaussian blobs whose centre follows three 100-step saccade legs of a
  triangle, 200 ALIF neurons, 10 % recurrent connectivity, 10 readouts,
  softmax cross-entropy in each sample's last 25 steps, batch of samples of
  uneven length.
* ``sparse_balanced`` / ``million_sparse`` -- the scaling-type networks
  (Methods, "Scaling"): LIF neurons with fixed in-degree drawn without
  autapses or multapses, 80 % excitatory / 20 % inhibitory sources, integer
  delays 1..5, external Poisson drive, random feedback, regression targets.

* ``evidence_accumulation`` -- the cue task (Methods, "Evidence
  accumulation"): left/right cue populations, a recall population and
  background noise, label = the side with more cues, softmax cross-entropy
  in the recall window (the learning window), ALIF neurons for memory.
* ``scaling_network`` -- the scaling experiment's network (Methods,
  "Scaling"): ignore-and-fire neurons at 5 Hz with random phases, Poisson
  inputs, input in-degree 100, recurrent in-degree 10,000 (no autapses or
  multapses), 10 readouts with in-degree 1000, feedback out-degree 100.

Options shared by the sparse networks: ``fb_outdeg`` (each readout's
feedback reaches only that many recurrent neurons) and ``dale`` (the
excitatory / inhibitory sign of every recurrent synapse is kept through
learning).

The module holds the inputs' structure only; none of the learning method's
arithmetic lives here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from . import hashrng as H

# stream tags that keep the hash streams of different arrays apart
_TAG_PRE, _TAG_DELAY, _TAG_W1, _TAG_W2, _TAG_WO1, _TAG_WO2 = 11, 12, 13, 14, 15, 16
_TAG_B1, _TAG_B2, _TAG_X, _TAG_TGT, _TAG_BERN, _TAG_WIN = 17, 18, 19, 20, 21, 22
_TAG_CLS, _TAG_LEN, _TAG_DRV = 23, 24, 25
_TAG_FB, _TAG_OUT, _TAG_IN, _TAG_CUE, _TAG_IF = 26, 27, 28, 29, 30


@dataclasses.dataclass
class Spec:
    """Parameters of one network + learning set-up (plain numbers only)."""
    name: str
    n_in: int
    n_rec: int
    n_out: int
    batch: int = 1
    T: int = 1000                  # steps per simulate call
    neuron_model: int = 0          # 0 LIF, 1 ALIF
    dt: float = 1.0
    tau_m: float = 20.0
    tau_a: float = 200.0
    beta_a: float = 0.0
    v_th: float = 0.6
    t_ref: int = 2
    tau_out: float = 20.0
    kappa_e: Optional[float] = None  # None: kappa (readout decay)
    gamma: float = 0.3 / 0.6       # surrogate height  (gamma_orig / v_th)
    beta_sg: float = 1.0 / 0.6     # surrogate slope   (1 / v_th)
    loss: int = 0                  # 0 MSE, 1 softmax cross-entropy
    feedback: int = 0              # 0 symmetric B = W_out^T, 1 fixed random
    update_interval: int = 0       # U; 0 means "once per simulate call"
    continuous: int = 0            # 1: no state reset between calls
    lr: float = 1e-3
    max_delay: int = 1
    drive_weight: float = 0.0      # external Poisson drive weight (0: none)
    drive_rate: float = 0.0        # mean drive events per neuron and step
    drive_seed: int = 0
    seed: int = 1234
    # e-prop+ variants and constraints (defaults: the plain method)
    surrogate: int = 0             # 0 piecewise linear, 1 exponential
    reset_mode: int = 0            # 0 soft (subtract v_th), 1 fixed value v_reset
    v_reset: float = 0.0
    c_reg: float = 0.0             # firing-rate regularisation coefficient (0: off)
    f_target: float = 0.0          # target rate in spikes per step
    beta_reg: float = 0.0          # EMA constant of the rate filter
    sign_mask: int = 0             # fixed weight signs: 1 input, 2 recurrent, 4 readout
    optimizer: int = 0             # 0 SGD, 1 Adam
    adam_b1: float = 0.9
    adam_b2: float = 0.999
    adam_eps: float = 1e-7         # TensorFlow's constant eps_hat
    if_period: int = 0             # ignore-and-fire period in steps (0: off)
    if_seed: int = 0
    # generalized delays (Supplement "Generalized delays"): recurrent to
    # readout (d_out) and learning signal back to the recurrent layer (d_ls)
    d_out: int = 0
    d_ls: int = 0

    @property
    def alpha(self) -> float:
        return math.exp(-self.dt / self.tau_m)

    @property
    def kappa(self) -> float:
        return math.exp(-self.dt / self.tau_out)

    def drive_thresholds(self) -> np.ndarray:
        """Inversion table of the Poisson drive as uint32 thresholds.

        count = #{m : u32 >= thr[m]} where thr[m] = floor(2^32 * CDF(m)).
        """
        if self.drive_weight == 0.0 or self.drive_rate <= 0.0:
            return np.zeros(0, dtype=np.uint32)
        lam = self.drive_rate
        thr = []
        p = math.exp(-lam)
        cdf = p
        m = 0
        while cdf < 1.0 - 1e-12 and m < 63:
            thr.append(min(int(math.floor(cdf * 4294967296.0)), 4294967295))
            m += 1
            p *= lam / m
            cdf += p
        return np.asarray(thr, dtype=np.uint32)


def _normal(seed, tag, a, b):
    h1 = H.key3_np(seed ^ (tag * 0x1000193), a, b)
    h2 = H.key3_np(seed ^ ((tag + 97) * 0x1000193), a, b)
    return H.normal_np(h1, h2)


def _uniform(seed, tag, a, b):
    return H.uniform_np(H.key3_np(seed ^ (tag * 0x1000193), a, b))


def _u64(seed, tag, a, b):
    return H.key3_np(seed ^ (tag * 0x1000193), a, b)


# ---------------------------------------------------------------------------
# connectivity


def fixed_indegree_pairs(n_pre: int, n_post: int, k: int, seed: int,
                         same_population: bool):
    """(pre, post) pairs with in-degree exactly k, no multapses.

    For each target j and stratum m < k, the source offset is drawn uniformly
    inside stratum m of [1, n_pre - 1] (stratified uniform sampling), which
    makes the k sources of a target distinct by construction; for a
    recurrent population the offset is added to j modulo n, so no source
    equals its target (no autapses).
    """
    span = n_pre - 1 if same_population else n_pre
    base = 1 if same_population else 0
    if k > span:
        raise ValueError("in-degree larger than the number of sources")
    s = span // k
    j = np.repeat(np.arange(n_post, dtype=np.uint64), k)
    m = np.tile(np.arange(k, dtype=np.uint64), n_post)
    off = base + m.astype(np.int64) * s + (
        _u64(seed, _TAG_PRE, j, m) % np.uint64(s)).astype(np.int64)
    if same_population:
        pre = (j.astype(np.int64) + off) % n_pre
    else:
        pre = off
    return pre.astype(np.int64), j.astype(np.int64), m.astype(np.int64)


def bernoulli_pairs(n_pre: int, n_post: int, p: float, seed: int,
                    same_population: bool):
    pre = np.repeat(np.arange(n_pre, dtype=np.uint64), n_post)
    post = np.tile(np.arange(n_post, dtype=np.uint64), n_pre)
    keep = _uniform(seed, _TAG_BERN, pre, post) < p
    if same_population:
        keep &= pre != post
    return pre[keep].astype(np.int64), post[keep].astype(np.int64)


def to_csr(pre_src: np.ndarray, post: np.ndarray, w: np.ndarray,
           delay: np.ndarray, n_src: int):
    """Sort synapses by source (stable, then by target) into CSR arrays."""
    order = np.lexsort((post, pre_src))
    pre_s = pre_src[order]
    counts = np.bincount(pre_s, minlength=n_src)
    ptr = np.zeros(n_src + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    return (ptr, post[order].astype(np.int32), w[order].astype(np.float32),
            delay[order].astype(np.uint8))


# ---------------------------------------------------------------------------
# targets and inputs


def sinusoid_targets(seed: int, T: int, n_out: int, batch: int) -> np.ndarray:
    """Sum of four sinusoids, periods U[100, 1000] ms, amplitudes U[0.5, 2],
    phases U[0, 2 pi] (Methods, "Pattern generation"), one per readout."""
    t = np.arange(1, T + 1, dtype=np.float64)
    out = np.zeros((batch, T, n_out), dtype=np.float64)
    for b in range(batch):
        for k in range(n_out):
            for q in range(4):
                idx = np.uint64((b * 1000003 + k) * 4 + q)
                per = 100.0 + 900.0 * _uniform(seed, _TAG_TGT, idx, 0)
                amp = 0.5 + 1.5 * _uniform(seed, _TAG_TGT, idx, 1)
                ph = 2.0 * np.pi * _uniform(seed, _TAG_TGT, idx, 2)
                out[b, :, k] += amp * np.sin(2.0 * np.pi * t / per + ph)
    # scale so that the summed target has unit-order magnitude
    return (out / 4.0).astype(np.float32)


def step_lists(raster: np.ndarray):
    """Raster [B][T][n] (bool) -> (ptr [B*T+1] int64, ids int32)."""
    B, T, n = raster.shape
    flat = raster.reshape(B * T, n)
    counts = flat.sum(axis=1)
    ptr = np.zeros(B * T + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    ids = np.nonzero(flat)[1].astype(np.int32)
    return ptr, ids


# ---------------------------------------------------------------------------
# workloads


def _weights(seed, tag, pre, post, std):
    return (std * _normal(seed, tag, pre.astype(np.uint64),
                          post.astype(np.uint64))).astype(np.float32)


def pattern_regression(seed: int = 1234, T: int = 1000, n_in: int = 20,
                       n_rec: int = 100, n_out: int = 1, rate_hz: float = 50.0,
                       **over) -> dict:
    # learning rate 1e-3 on the loss averaged over the T steps of a sample,
    # i.e. 1e-3 / T on the summed loss of Eq. mean-squared-error
    spec = Spec(name="pattern_regression", n_in=n_in, n_rec=n_rec,
                n_out=n_out, T=T, lr=1e-3 / T, max_delay=1, seed=seed)
    for key, val in over.items():
        setattr(spec, key, val)
    # input -> recurrent: all-to-all, delay 1
    pre_i = np.repeat(np.arange(n_in), n_rec)
    post_i = np.tile(np.arange(n_rec), n_in)
    w_i = _weights(seed, _TAG_W1, pre_i, post_i, 1.0 / math.sqrt(n_in))
    # recurrent: all-to-all without autapses, delay 1
    pre_r, post_r, _ = fixed_indegree_pairs(n_rec, n_rec, n_rec - 1, seed, True)
    w_r = _weights(seed, _TAG_W2, pre_r, post_r, 1.0 / math.sqrt(n_rec))
    src = np.concatenate([pre_i, pre_r + n_in])
    post = np.concatenate([post_i, post_r])
    w = np.concatenate([w_i, w_r])
    d = np.ones(src.shape[0], dtype=np.uint8)
    ptr, col, wv, dv = to_csr(src, post, w, d, n_in + n_rec)
    j = np.arange(n_rec)
    w_out = np.stack([_weights(seed, _TAG_WO1, j, np.full(n_rec, k),
                               1.0 / math.sqrt(n_rec)) for k in range(n_out)],
                     axis=1)
    # frozen Poisson input raster
    B = spec.batch
    ii = np.arange(n_in, dtype=np.uint64)[None, None, :]
    tt = np.arange(1, T + 1, dtype=np.uint64)[None, :, None]
    bb = np.arange(B, dtype=np.uint64)[:, None, None]
    raster = _uniform(seed, _TAG_X, ii + np.uint64(n_in) * bb, tt) < rate_hz * spec.dt / 1000.0
    x_ptr, x_ids = step_lists(raster)
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.ascontiguousarray(w_out, dtype=np.float32),
                out_mask=np.ones(n_rec, dtype=np.uint8), feedback=None,
                x_ptr=x_ptr, x_ids=x_ids,
                targets=sinusoid_targets(seed, T, n_out, B),
                window=np.ones((B, T), dtype=np.uint8),
                lengths=np.full(B, T, dtype=np.int32))


def event_classification(seed: int = 1235, batch: int = 64, T: int = 350,
                         len_lo: int = 250, len_hi: int = 350, side: int = 34,
                         n_rec: int = 200, n_out: int = 10, p_rec: float = 0.1,
                         events_per_300: float = 4000.0, w_in_scale: float = 3.0,
                         sample_seed: int | None = None, **over) -> dict:
    # seed fixes the network and the class rate maps; sample_seed (default:
    # seed) draws the samples (classes, lengths, events) of the batch
    ss = seed if sample_seed is None else sample_seed
    n_in = 2 * side * side
    spec = Spec(name="event_classification", n_in=n_in, n_rec=n_rec,
                n_out=n_out, batch=batch, T=T, neuron_model=1, tau_a=200.0,
                beta_a=1.7, loss=1, lr=5e-3, max_delay=1, seed=seed)
    for key, val in over.items():
        setattr(spec, key, val)
    pre_i = np.repeat(np.arange(n_in), n_rec)
    post_i = np.tile(np.arange(n_rec), n_in)
    w_i = _weights(seed, _TAG_W1, pre_i, post_i, w_in_scale / math.sqrt(n_in))
    pre_r, post_r = bernoulli_pairs(n_rec, n_rec, p_rec, seed, True)
    w_r = _weights(seed, _TAG_W2, pre_r, post_r, 1.0 / math.sqrt(p_rec * n_rec))
    src = np.concatenate([pre_i, pre_r + n_in])
    post = np.concatenate([post_i, post_r])
    w = np.concatenate([w_i, w_r])
    d = np.ones(src.shape[0], dtype=np.uint8)
    ptr, col, wv, dv = to_csr(src, post, w, d, n_in + n_rec)
    j = np.arange(n_rec)
    w_out = np.stack([_weights(seed, _TAG_WO1, j, np.full(n_rec, k),
                               1.0 / math.sqrt(n_rec)) for k in range(n_out)],
                     axis=1)
    # per-sample class, length and event raster
    bidx = np.arange(batch, dtype=np.uint64)
    cls = (_u64(ss, _TAG_CLS, bidx, 0) % np.uint64(n_out)).astype(np.int64)
    lengths = (len_lo + (_u64(ss, _TAG_LEN, bidx, 0) %
                         np.uint64(len_hi - len_lo + 1)).astype(np.int64)).astype(np.int32)
    kk = np.arange(n_out, dtype=np.uint64)
    centre = side * (0.25 + 0.5 * np.stack([_uniform(seed, _TAG_CLS, kk, 1),
                                            _uniform(seed, _TAG_CLS, kk, 2)], 1))
    sigma = 2.5 + 2.0 * _uniform(seed, _TAG_CLS, kk, 3)
    # triangle of three 100-step saccade legs: upper left -> lower middle ->
    # upper right -> upper left (Methods, "Neuromorphic MNIST")
    corners = np.array([[-2.0, -2.0], [0.0, 2.0], [2.0, -2.0], [-2.0, -2.0]])
    t = np.arange(1, T + 1)
    leg = np.minimum((t - 1) // 100, 2)
    frac = ((t - 1) % 100) / 100.0
    shift = corners[leg] + (corners[leg + 1] - corners[leg]) * frac[:, None]
    xs = np.arange(side)
    gx, gy = np.meshgrid(xs, xs, indexing="ij")
    raster = np.zeros((batch, T, n_in), dtype=bool)
    for b in range(batch):
        c = cls[b]
        cx = centre[c, 0] + shift[:, 0]
        cy = centre[c, 1] + shift[:, 1]
        dist2 = ((gx[None] - cx[:, None, None]) ** 2 +
                 (gy[None] - cy[:, None, None]) ** 2)
        rate_on = np.exp(-dist2 / (2.0 * sigma[c] ** 2))
        # OFF polarity: ring around the blob
        rate_off = np.exp(-(np.sqrt(dist2) - 2.0 * sigma[c]) ** 2 / (2.0 * sigma[c] ** 2))
        rates = np.concatenate([rate_on.reshape(T, -1), rate_off.reshape(T, -1)], 1)
        rates *= (events_per_300 / 300.0) / rates.sum(axis=1, keepdims=True)
        u = _uniform(ss, _TAG_X, np.uint64(b) * np.uint64(n_in) +
                     np.arange(n_in, dtype=np.uint64)[None, :],
                     np.arange(1, T + 1, dtype=np.uint64)[:, None])
        rb = u < np.minimum(rates, 1.0)
        rb[lengths[b]:] = False
        raster[b] = rb
    x_ptr, x_ids = step_lists(raster)
    targets = np.zeros((batch, T, n_out), dtype=np.float32)
    targets[np.arange(batch), :, cls] = 1.0
    window = np.zeros((batch, T), dtype=np.uint8)
    for b in range(batch):
        window[b, lengths[b] - 25:lengths[b]] = 1
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.ascontiguousarray(w_out, dtype=np.float32),
                out_mask=np.ones(n_rec, dtype=np.uint8), feedback=None,
                x_ptr=x_ptr, x_ids=x_ids, targets=targets, window=window,
                lengths=lengths, classes=cls)


def sparse_feedback(seed: int, n_rec: int, n_out: int, outdeg: int, std: float = 1.0) -> np.ndarray:
    """B [n_rec, n_out] with exactly `outdeg` nonzero N(0, std^2) entries per
    readout k: target m of readout k is drawn uniformly inside stratum m of
    the neurons (distinct targets by construction)."""
    if outdeg > n_rec:
        raise ValueError("feedback out-degree larger than the population")
    fb = np.zeros((n_rec, n_out), dtype=np.float32)
    s = n_rec // outdeg
    m = np.arange(outdeg, dtype=np.uint64)
    for k in range(n_out):
        kk = np.full(outdeg, k, dtype=np.uint64)
        j = m.astype(np.int64) * s + (_u64(seed, _TAG_FB, kk, m) % np.uint64(s)).astype(np.int64)
        fb[j, k] = (std * _normal(seed, _TAG_B2, j.astype(np.uint64), kk)).astype(np.float32)
    return fb


def _ei_network_np(spec: Spec, k_in: int, J: float, g: float, seed: int):
    n = spec.n_rec
    pre, post, m = fixed_indegree_pairs(n, n, k_in, seed, True)
    w = np.where(pre < int(0.8 * n), J, -g * J).astype(np.float32)
    d = (1 + (_u64(seed, _TAG_DELAY, post.astype(np.uint64), m.astype(np.uint64))
              % np.uint64(spec.max_delay))).astype(np.uint8)
    return to_csr(pre, post, w, d, n)


def sparse_balanced(seed: int = 1236, n_rec: int = 100_000, k_in: int = 1000,
                    T: int = 2000, n_out: int = 1, n_coupled: int = 500,
                    J: float = 0.01, g: float = 5.0,
                    drive_weight: float = 0.04, drive_rate: float = 1.2,
                    name: str = "sparse_balanced", fb_outdeg: Optional[int] = None,
                    dale: bool = False, **over) -> dict:
    """E/I network with fixed in-degree and delays 1..5, numpy build."""
    # lr 1e-6 keeps the firing rate near its configured value while the
    # weights learn (1e-4 drives the network into a high-rate state)
    spec = Spec(name=name, n_in=0, n_rec=n_rec, n_out=n_out, T=T,
                feedback=1, lr=1e-6, max_delay=5, drive_weight=drive_weight,
                drive_rate=drive_rate, drive_seed=seed * 7919 + 17, seed=seed)
    for key, val in over.items():
        setattr(spec, key, val)
    ptr, col, wv, dv = _ei_network_np(spec, k_in, J, g, seed)
    j = np.arange(n_rec)
    mask = np.zeros(n_rec, dtype=np.uint8)
    mask[:n_coupled] = 1
    w_out = np.stack([_weights(seed, _TAG_WO1, j, np.full(n_rec, k),
                               1.0 / math.sqrt(n_coupled)) for k in range(n_out)],
                     axis=1) * mask[:, None]
    fb = np.stack([_weights(seed, _TAG_B1, j, np.full(n_rec, k), 1.0)
                   for k in range(n_out)], axis=1)
    if fb_outdeg is not None:
        fb = sparse_feedback(seed, n_rec, n_out, fb_outdeg)
    if dale:
        spec.sign_mask |= 2
    B = spec.batch
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.ascontiguousarray(w_out, dtype=np.float32),
                out_mask=mask, feedback=np.ascontiguousarray(fb, dtype=np.float32),
                x_ptr=np.zeros(B * T + 1, dtype=np.int64),
                x_ids=np.zeros(0, dtype=np.int32),
                targets=sinusoid_targets(seed, T, n_out, B),
                window=np.ones((B, T), dtype=np.uint8),
                lengths=np.full(B, T, dtype=np.int32))


def million_sparse_spec(n_rec: int = 1_000_000, T: int = 1000, n_out: int = 100,
                        seed: int = 1237, **over) -> Spec:
    # drive 0.03 x Poisson(0.85) per step: ~5 Hz at 1e6 neurons, in-degree 1000
    spec = Spec(name="million_sparse", n_in=0, n_rec=n_rec, n_out=n_out, T=T,
                feedback=1, update_interval=100, continuous=1, lr=1e-6,
                max_delay=5, drive_weight=0.03, drive_rate=0.85,
                drive_seed=seed * 7919 + 17, seed=seed)
    for key, val in over.items():
        setattr(spec, key, val)
    return spec


def million_sparse(seed: int = 1237, n_rec: int = 1_000_000, k_in: int = 1000,
                   T: int = 1000, n_out: int = 100, J: float = 0.01,
                   g: float = 5.0, fb_outdeg: Optional[int] = None, dale: bool = False,
                   **over) -> dict:
    """Million-neuron workload built with numpy (use for scaled replicas).

    The full-size instance is built on the GPU by
    `million_sparse_torch`, which produces the same integer structure.
    """
    spec = million_sparse_spec(n_rec=n_rec, T=T, n_out=n_out, seed=seed, **over)
    ptr, col, wv, dv = _ei_network_np(spec, k_in, J, g, seed)
    j = np.arange(n_rec)
    w_out = np.stack([_weights(seed, _TAG_WO1, j, np.full(n_rec, k),
                               1.0 / math.sqrt(n_rec)) for k in range(n_out)],
                     axis=1)
    fb = np.stack([_weights(seed, _TAG_B1, j, np.full(n_rec, k), 1.0 / math.sqrt(n_out))
                   for k in range(n_out)], axis=1)
    if fb_outdeg is not None:
        fb = sparse_feedback(seed, n_rec, n_out, fb_outdeg)
    if dale:
        spec.sign_mask |= 2
    B = spec.batch
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.ascontiguousarray(w_out, dtype=np.float32),
                out_mask=np.ones(n_rec, dtype=np.uint8),
                feedback=np.ascontiguousarray(fb, dtype=np.float32),
                x_ptr=np.zeros(B * T + 1, dtype=np.int64),
                x_ids=np.zeros(0, dtype=np.int32),
                targets=sinusoid_targets(seed, T, n_out, B),
                window=np.ones((B, T), dtype=np.uint8),
                lengths=np.full(B, T, dtype=np.int32))


# ---------------------------------------------------------------------------
# evidence accumulation (Methods, "Evidence accumulation")


def evidence_accumulation(seed: int = 1240, batch: int = 32, n_cues: int = 7,
                          t_cue: int = 100, t_gap: int = 50, t_delay: int = 1000,
                          t_recall: int = 150, pop: int = 10, n_rec: int = 100,
                          rate_cue_hz: float = 40.0, rate_bg_hz: float = 10.0,
                          sample_seed: Optional[int] = None, **over) -> dict:
    """The cue task: input populations (pop channels each) 0 left cues,
    1 right cues, 2 recall cue, 3 background noise.  Each of n_cues cue slots
    shows one side's population at rate_cue for t_cue steps, then t_gap
    silent steps; after t_delay steps of background only, the recall
    population fires for t_recall steps.  The label is the side with more
    cues; the softmax cross-entropy is applied in the recall steps only (the
    learning window).  ALIF neurons (tau_a 2000 ms) keep the evidence; fully
    connected recurrence without autapses; two readouts; Adam."""
    ss = seed if sample_seed is None else sample_seed
    n_in = 4 * pop
    T = n_cues * (t_cue + t_gap) + t_delay + t_recall
    spec = Spec(name="evidence_accumulation", n_in=n_in, n_rec=n_rec, n_out=2,
                batch=batch, T=T, neuron_model=1, tau_a=2000.0, beta_a=1.7,
                loss=1, lr=5e-3, optimizer=1, max_delay=1, seed=seed)
    for key, val in over.items():
        setattr(spec, key, val)
    pre_i = np.repeat(np.arange(n_in), n_rec)
    post_i = np.tile(np.arange(n_rec), n_in)
    w_i = _weights(seed, _TAG_W1, pre_i, post_i, 1.0 / math.sqrt(n_in))
    pre_r, post_r, _ = fixed_indegree_pairs(n_rec, n_rec, n_rec - 1, seed, True)
    w_r = _weights(seed, _TAG_W2, pre_r, post_r, 1.0 / math.sqrt(n_rec))
    src = np.concatenate([pre_i, pre_r + n_in])
    post = np.concatenate([post_i, post_r])
    w = np.concatenate([w_i, w_r])
    d = np.ones(src.shape[0], dtype=np.uint8)
    ptr, col, wv, dv = to_csr(src, post, w, d, n_in + n_rec)
    j = np.arange(n_rec)
    w_out = np.stack([_weights(seed, _TAG_WO1, j, np.full(n_rec, k), 1.0 / math.sqrt(n_rec))
                      for k in range(2)], axis=1)
    # cue sides per sample and slot; label = majority side (n_cues is odd)
    bb = np.arange(batch, dtype=np.uint64)
    sides = np.stack([(_u64(ss, _TAG_CUE, bb, np.uint64(c)) & np.uint64(1)).astype(np.int64)
                      for c in range(n_cues)], axis=1)                 # [batch, n_cues]
    label = (sides.sum(axis=1) * 2 > n_cues).astype(np.int64)          # 1: right wins
    rate = np.zeros((batch, T, n_in))
    rate[:, :, 3 * pop:] = rate_bg_hz
    for c in range(n_cues):
        t0 = c * (t_cue + t_gap)
        for b in range(batch):
            p0 = sides[b, c] * pop
            rate[b, t0:t0 + t_cue, p0:p0 + pop] = rate_cue_hz
    t_rec0 = T - t_recall
    rate[:, t_rec0:, 2 * pop:3 * pop] = rate_cue_hz
    u = _uniform(ss, _TAG_X, bb[:, None, None] * np.uint64(n_in) + np.arange(n_in, dtype=np.uint64)[None, None, :],
                 np.arange(1, T + 1, dtype=np.uint64)[None, :, None])
    raster = u < rate * spec.dt / 1000.0
    x_ptr, x_ids = step_lists(raster)
    targets = np.zeros((batch, T, 2), dtype=np.float32)
    targets[np.arange(batch), :, label] = 1.0
    window = np.zeros((batch, T), dtype=np.uint8)
    window[:, t_rec0:] = 1
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.ascontiguousarray(w_out, dtype=np.float32),
                out_mask=np.ones(n_rec, dtype=np.uint8), feedback=None,
                x_ptr=x_ptr, x_ids=x_ids, targets=targets, window=window,
                lengths=np.full(batch, T, dtype=np.int32), labels=label)


# ---------------------------------------------------------------------------
# the scaling experiment's network (Methods, "Scaling")


def scaling_spec(n_rec: int = 128_000, n_in: int = 1000, n_out: int = 10, T: int = 20_000,
                 update_interval: int = 1000, rate_hz: float = 5.0, seed: int = 1241, **over) -> Spec:
    period = int(round(1000.0 / rate_hz))
    spec = Spec(name="scaling", n_in=n_in, n_rec=n_rec, n_out=n_out, T=T, feedback=1,
                update_interval=update_interval, continuous=1, lr=1e-6, max_delay=5,
                if_period=period, if_seed=seed * 7919 + 29, seed=seed)
    for key, val in over.items():
        setattr(spec, key, val)
    return spec


def poisson_inputs(seed: int, n_in: int, T: int, rate_hz: float, batch: int = 1):
    """Poisson spike generators (frozen): (x_ptr, x_ids)."""
    ii = np.arange(n_in, dtype=np.uint64)[None, None, :]
    tt = np.arange(1, T + 1, dtype=np.uint64)[None, :, None]
    bb = np.arange(batch, dtype=np.uint64)[:, None, None]
    raster = _uniform(seed, _TAG_IN, ii + np.uint64(n_in) * bb, tt) < rate_hz / 1000.0
    return step_lists(raster)


def readout_indegree_mask(seed: int, n_rec: int, n_out: int, k_out: int) -> np.ndarray:
    """[n_rec, n_out] mask with exactly k_out recurrent sources per readout
    (stratified draw, distinct sources)."""
    mask = np.zeros((n_rec, n_out), dtype=np.uint8)
    s = n_rec // k_out
    m = np.arange(k_out, dtype=np.uint64)
    for k in range(n_out):
        kk = np.full(k_out, k, dtype=np.uint64)
        j = m.astype(np.int64) * s + (_u64(seed, _TAG_OUT, kk, m) % np.uint64(s)).astype(np.int64)
        mask[j, k] = 1
    return mask


def scaling_network(seed: int = 1241, n_rec: int = 128_000, k_rec: int = 10_000, n_in: int = 1000,
                    k_in: int = 100, n_out: int = 10, k_out: int = 1000, fb_outdeg: int = 100,
                    T: int = 20_000, update_interval: int = 1000, rate_hz: float = 5.0,
                    J: float = 0.001, g: float = 5.0, dale: bool = False, **over) -> dict:
    """numpy build of the scaling network (use scaled-down sizes here; the
    full network is built on the GPU by `gpu_build.scaling_torch`): inputs
    first in the CSR, recurrent E/I weights +J / -gJ (80/20 by source),
    input weights +J."""
    spec = scaling_spec(n_rec=n_rec, n_in=n_in, n_out=n_out, T=T,
                        update_interval=update_interval, rate_hz=rate_hz, seed=seed, **over)
    # input synapses: k_in distinct inputs per recurrent neuron
    pre_i, post_i, _ = fixed_indegree_pairs(n_in, n_rec, k_in, seed ^ 0x5151, False)
    w_i = np.full(pre_i.shape[0], J, dtype=np.float32)
    pre_r, post_r, m = fixed_indegree_pairs(n_rec, n_rec, k_rec, seed, True)
    w_r = np.where(pre_r < int(0.8 * n_rec), J, -g * J).astype(np.float32)
    d_r = (1 + (_u64(seed, _TAG_DELAY, post_r.astype(np.uint64), m.astype(np.uint64))
                % np.uint64(spec.max_delay))).astype(np.uint8)
    d_i = np.ones(pre_i.shape[0], dtype=np.uint8)
    src = np.concatenate([pre_i, pre_r + n_in])
    post = np.concatenate([post_i, post_r])
    ptr, col, wv, dv = to_csr(src, post, np.concatenate([w_i, w_r]), np.concatenate([d_i, d_r]),
                              n_in + n_rec)
    mask = readout_indegree_mask(seed, n_rec, n_out, k_out)
    j = np.arange(n_rec)
    w_out = np.stack([_weights(seed, _TAG_WO1, j, np.full(n_rec, k), 1.0 / math.sqrt(k_out))
                      for k in range(n_out)], axis=1) * mask
    fb = sparse_feedback(seed, n_rec, n_out, fb_outdeg)
    if dale:
        spec.sign_mask |= 2
    x_ptr, x_ids = poisson_inputs(seed, n_in, T, rate_hz)
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.ascontiguousarray(w_out, dtype=np.float32), out_mask=mask,
                feedback=fb, x_ptr=x_ptr, x_ids=x_ids,
                targets=sinusoid_targets(seed, T, n_out, 1),
                window=np.ones((1, T), dtype=np.uint8), lengths=np.full(1, T, dtype=np.int32))

"""FP64 CPU oracle of e-prop -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The CUDA library never calls it and it
never calls the CUDA library; the two share no code.  The only thing they
share is the seeded input generators of the `workloads` package.

Contents
--------
* ``Oracle``: ctypes wrapper around the plain C time-driven simulation in
  ``eprop_oracle.c`` (Methods: neuron models, loss functions, gradients,
  optimisation; Algorithm 1 "Time-driven gradient computation").
* ``eligibility_step``: the oracle's per-synapse recursion (Eq. eligibility-
  vector-substituted, Eq. filtered-eligibility-trace), exported for pins.
* ``event_driven_gradients``: the event-driven restatement (Algorithm 5,
  "Optimized event-driven weight update"): each synapse is visited only at
  the arrivals of its presynaptic spikes and integrates its trace over the
  left-open interval since the previous arrival; used to check that the
  event-driven and the time-driven organisations give the same gradient.
* ``sampled_gradients``: the gradient of a sample of synapses over a run
  whose postsynaptic history (spikes, surrogate values, readout) is given,
  with ``error_signal`` and ``readout_magnitude``: the oracle side of the
  sampled parity check at sizes the full simulation cannot reach.
* ``build()``: compiles the C oracle with gcc into ``oracle/_lib``.

Parity status per function: all functions are pinned by the CPU tests in
``tests/test_oracle_*.py`` (closed forms, autograd BPTT special case, hand
sums, reductions, event/time-driven invariant).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "libeprop_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain -O2, no fast-math, OpenMP over the
    per-synapse loop) and return the path.  The thread count follows
    OMP_NUM_THREADS (the tests run it with one thread unless set)."""
    src = os.path.join(_HERE, "eprop_oracle.c")
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", src,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Cfg(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_rec", ctypes.c_int32),
                ("n_out", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("neuron_model", ctypes.c_int32), ("t_ref", ctypes.c_int32),
                ("loss", ctypes.c_int32), ("feedback", ctypes.c_int32),
                ("update_interval", ctypes.c_int32), ("continuous", ctypes.c_int32),
                ("max_delay", ctypes.c_int32), ("n_drive_thr", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("rho", ctypes.c_double),
                ("kappa", ctypes.c_double), ("kappa_e", ctypes.c_double),
                ("beta_a", ctypes.c_double), ("v_th", ctypes.c_double),
                ("gamma", ctypes.c_double), ("beta_sg", ctypes.c_double),
                ("lr", ctypes.c_double), ("drive_weight", ctypes.c_double),
                ("drive_seed", ctypes.c_uint64),
                ("drive_thr", ctypes.c_void_p),
                ("surrogate", ctypes.c_int32), ("reset_mode", ctypes.c_int32),
                ("v_reset", ctypes.c_double), ("c_reg", ctypes.c_double),
                ("f_target", ctypes.c_double), ("beta_reg", ctypes.c_double),
                ("sign_mask", ctypes.c_int32), ("optimizer", ctypes.c_int32),
                ("adam_b1", ctypes.c_double), ("adam_b2", ctypes.c_double),
                ("adam_eps", ctypes.c_double), ("if_period", ctypes.c_int32),
                ("if_seed", ctypes.c_uint64), ("d_out", ctypes.c_int32), ("d_ls", ctypes.c_int32)]


class _State(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("nnz", ctypes.c_int64)] + [
        (name, ctypes.c_void_p) for name in (
            "ptr", "col", "delay", "w", "w_out", "out_mask", "fb", "v", "a",
            "psi_prev", "ref", "z_prev", "ring", "src_hist", "zbar", "epsa",
            "ebar", "g", "y", "zk", "g_out", "grad_acc", "grad_out_acc",
            "counters", "g_abs", "g_out_abs", "grad_abs_acc", "grad_out_abs_acc",
            "y_abs", "g_lsens", "g_out_lsens", "grad_lsens_acc", "grad_out_lsens_acc",
            "rate", "ebar_reg", "w_neg", "w_out_neg", "adam_m", "adam_v", "adam_m_out", "adam_v_out",
            "z_hist", "ebar_hist", "L_hist", "Ls_hist")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_simulate.restype = ctypes.c_int
            lib.oracle_simulate.argtypes = [ctypes.POINTER(_Cfg), ctypes.POINTER(_State),
                                            ctypes.c_int32] + [ctypes.c_void_p] * 15
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_eligibility_step.restype = ctypes.c_double
            lib.oracle_eligibility_step.argtypes = [ctypes.c_double] * 8 + [ctypes.c_void_p] * 3
            lib.oracle_synapse_sample.restype = None
            lib.oracle_synapse_sample.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int64, ctypes.c_int32] + \
                [ctypes.c_void_p] * 7
            lib.oracle_arrival_contrib.restype = None
            lib.oracle_arrival_contrib.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int32, ctypes.c_int32,
                                                                           ctypes.c_int64] + [ctypes.c_void_p] * 3
            _lib = lib
    return _lib


def _f32(x) -> float:
    return float(np.float32(x))


def params(spec) -> dict:
    """The model constants of a spec as the oracle uses them: every
    coefficient the library takes as an FP32 field and uses as it is (the
    adaptation strength, threshold, surrogate constants, learning rate,
    drive weight, filter constant kappa_e when given, reset value,
    regularisation and Adam constants) is taken at its FP32 value, so both
    evaluate the method for the same numbers; the decay factors alpha =
    exp(-dt / tau_m), rho = exp(-dt / tau_a), kappa = exp(-dt / tau_out) are
    formed in FP64 from the spec's time constants (the workloads use time
    constants that FP32 holds exactly)."""
    dt, tau_m, tau_a, tau_out = spec.dt, spec.tau_m, spec.tau_a, spec.tau_out
    kappa = math.exp(-dt / tau_out)
    return dict(alpha=math.exp(-dt / tau_m), rho=math.exp(-dt / tau_a), kappa=kappa,
                kappa_e=kappa if spec.kappa_e is None or spec.kappa_e < 0 else _f32(spec.kappa_e),
                beta_a=_f32(spec.beta_a) if spec.neuron_model == 1 else 0.0,
                v_th=_f32(spec.v_th), gamma=_f32(spec.gamma), beta_sg=_f32(spec.beta_sg),
                lr=_f32(spec.lr), drive_weight=_f32(spec.drive_weight), v_reset=_f32(spec.v_reset),
                c_reg=_f32(spec.c_reg), f_target=_f32(spec.f_target), beta_reg=_f32(spec.beta_reg),
                adam_b1=_f32(spec.adam_b1), adam_b2=_f32(spec.adam_b2), adam_eps=_f32(spec.adam_eps))


def set_threads(n: int) -> int:
    """Host threads of the oracle's per-synapse loop (results do not depend
    on it); returns the count in effect."""
    return int(_load().oracle_set_threads(int(n)))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def eligibility_step(alpha, rho, beta_a, kappa_e, psi_prev, psi, L, arrive,
                     state: np.ndarray) -> float:
    """One step of the oracle's synapse recursion; state = [zbar, eps_a, ebar]
    (float64, updated in place).  Returns g^t = L^t ebar^t."""
    lib = _load()
    st = state
    assert st.dtype == np.float64 and st.shape == (3,)
    base = st.ctypes.data
    return lib.oracle_eligibility_step(alpha, rho, beta_a, kappa_e, psi_prev,
                                       psi, L, arrive, base, base + 8, base + 16)


def arrival_contrib(spec, psi, L, U=None):
    """Q[a-1, j]: gradient contribution of one unit presynaptic arrival at
    step a into neuron j, summed to the end of a's update window (width U,
    default T), from the recorded surrogate values psi and learning signals
    L ([T, N] of one sample) -- the per-event term of the event-driven update
    (Sec. "From time-driven to event-driven e-prop")."""
    lib = _load()
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    T, N = psi.shape
    Q = np.zeros((T, N))
    p = params(spec)
    lib.oracle_arrival_contrib(p["alpha"], p["rho"], p["beta_a"], p["kappa_e"], T, U or T, N, _p(psi),
                               _p(L), _p(Q))
    return Q


def error_signal(spec, y, targets, window, y_abs):
    """Error signal E [T, K] of one sample and its sensitivity Esens [T, K]
    from a readout y and its magnitude y_abs ([T, K]), as the C oracle forms
    them: MSE E_k = win (y_k - y*_k) (Eq. mean-squared-error), temporal MSE
    E_k = win (2 / K)(y_k - y*_k) (Eq. temporal-mse), softmax CE
    E_k = win (pi_k - pi*_k) (Eq. softmax, Eq. cross-entropy-loss);
    Esens = win (y_abs + |y*|) for MSE and win (pi (y_abs + sum_l pi_l
    y_abs_l) + pi + |pi*|) for CE."""
    y = np.asarray(y, np.float64)
    tg = np.asarray(targets, np.float64)
    win = np.asarray(window, np.float64)[:, None]
    ya = np.asarray(y_abs, np.float64)
    if spec.loss == 0:
        return win * (y - tg), win * (ya + np.abs(tg))
    if spec.loss == 2:          # temporal MSE (Eq. temporal-mse)
        c = 2.0 / y.shape[1]
        return win * c * (y - tg), win * c * (ya + np.abs(tg))
    e = np.exp(y - y.max(axis=1, keepdims=True))
    pi = e / e.sum(axis=1, keepdims=True)
    pya = (pi * ya).sum(axis=1, keepdims=True)
    return win * (pi - tg), win * (pi * (ya + pya) + pi + np.abs(tg))


def readout_magnitude(raster, w_out, kappa):
    """y_abs [T, K] = kappa-filtered sum over the spiking neurons of |W_out|
    (raster [T, N] of one sample; the magnitude companion of the leaky
    readout, Eq. leaky_integrator, for the parity tolerance)."""
    raster = np.asarray(raster)
    wa = np.abs(np.asarray(w_out, np.float64))
    T, K = raster.shape[0], wa.shape[1]
    out = np.zeros((T, K))
    acc = np.zeros(K)
    for t in range(T):
        idx = np.nonzero(raster[t])[0]
        acc = kappa * acc + (wa[idx].sum(axis=0) if idx.size else 0.0)
        out[t] = acc
    return out


def sampled_gradients(spec, src_spikes, delay, psi, y, targets, window, fb_rows, y_abs):
    """Gradients of a sample of synapses over a run whose postsynaptic
    history is given (teacher forcing), batch of one, fixed feedback B.

    src_spikes [S, T]: spike of each synapse's source at emission steps 1..T
    delay      [S]   : the synapse's delay d (arrival at emission + d)
    psi        [S, T]: surrogate psi_j^t of each synapse's target
    y, targets [T, K], window [T], y_abs [T, K]: readout, target, target
               window and readout magnitude of the run
    fb_rows    [S, K]: B_jk of each synapse's target j
    Returns (G, mag, sens) [S]: sum_t L_j^t ebar^t over the run with
    L_j = sum_k B_jk E_k (Eq. final-gradient) and the recursion of
    `eligibility_step` (Eq. eligibility-vector-substituted, Eq. filtered-
    eligibility-trace), sum_t |g^t| and sum_t Lsens_j^t |ebar^t|."""
    lib = _load()
    src = np.asarray(src_spikes, np.uint8)
    S, T = src.shape
    d = np.asarray(delay, np.int64).reshape(S)
    E, Es = error_signal(spec, y, targets, window, y_abs)
    fb = np.asarray(fb_rows, np.float64)
    L = np.ascontiguousarray(fb @ E.T)
    Ls = np.ascontiguousarray(np.abs(fb) @ Es.T)
    arrive = np.zeros((S, T), np.uint8)
    for s in range(S):
        if d[s] < T:
            arrive[s, d[s]:] = src[s, :T - d[s]]
    psi = np.ascontiguousarray(psi, np.float64)
    assert psi.shape == (S, T)
    p = params(spec)
    G, mag, sens = np.zeros(S), np.zeros(S), np.zeros(S)
    lib.oracle_synapse_sample(p["alpha"], p["rho"], p["beta_a"], p["kappa_e"], S, T, _p(arrive), _p(psi),
                              _p(L), _p(Ls), _p(G), _p(mag), _p(sens))
    return G, mag, sens


def arrival_magnitude(spec, ptr, col, delay, x_ptr, x_ids, lengths, raster, psi, L):
    """Per synapse (CSR order), the batch mean over samples of sum_a |Q_j(a)|
    over the synapse's arrivals a = s + d <= length (single update window):
    the condition of the event-driven gradient sum."""
    B, T, N = raster.shape
    n_in = spec.n_in
    out = np.zeros(len(col))
    ptr = np.asarray(ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    delay = np.asarray(delay, dtype=np.int64)
    d_out, d_ls = int(getattr(spec, "d_out", 0)), int(getattr(spec, "d_ls", 0))
    for b in range(B):
        ln = int(lengths[b])
        Lb = L[b]
        if d_out or d_ls:
            # generalized delays: step t pairs with the learning signal of
            # t + d_out, delivered only when formed by the sample's end - d_ls
            Lb = np.zeros_like(L[b])
            m = max(0, min(T - d_out, ln - d_ls - d_out))
            Lb[:m] = L[b][d_out:d_out + m]
        Qa = np.abs(arrival_contrib(spec, psi[b], Lb))
        src = np.zeros((ln, n_in + N), dtype=bool)
        for t in range(ln):
            src[t, x_ids[x_ptr[b * T + t]:x_ptr[b * T + t + 1]]] = True
        src[:, n_in:] = raster[b, :ln].astype(bool)
        for i in range(n_in + N):
            steps = np.nonzero(src[:, i])[0] + 1
            if steps.size == 0:
                continue
            q = np.arange(ptr[i], ptr[i + 1])
            for s in steps:
                a = s + delay[q]
                ok = a <= ln
                out[q[ok]] += Qa[a[ok] - 1, col[q[ok]]]
    return out / B


class Oracle:
    """Time-driven FP64 e-prop on one network (state persists across calls).

    Arguments are the plain arrays produced by the `workloads` generators:
    a spec (`workloads.configs.Spec`) and the CSR synapse arrays by source.
    """

    def __init__(self, spec, ptr, col, w, delay, w_out, out_mask, feedback=None):
        self.spec = spec
        B, N, K = spec.batch, spec.n_rec, spec.n_out
        D1 = spec.max_delay + 1
        self.n_src = spec.n_in + N
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.delay = np.ascontiguousarray(delay, dtype=np.uint8)
        self.w = np.array(w, dtype=np.float64)
        self.nnz = int(self.ptr[-1])
        assert self.ptr.shape[0] == self.n_src + 1 and self.col.shape[0] == self.nnz
        if self.nnz:
            assert int(self.delay.min()) >= 1 and int(self.delay.max()) <= spec.max_delay
        self.w_out = np.array(w_out, dtype=np.float64).reshape(N, K)
        # per-weight readout mask [N, K]; a per-neuron mask [N] applies to the row
        om = np.ones(N, np.uint8) if out_mask is None else np.asarray(out_mask, dtype=np.uint8)
        if om.ndim == 1:
            om = np.repeat(om[:, None], K, axis=1)
        self.out_mask = np.ascontiguousarray(om.reshape(N, K))
        self.fb = None if feedback is None else np.array(feedback, dtype=np.float64).reshape(N, K)
        if spec.feedback and self.fb is None:
            raise ValueError("random feedback needs a feedback matrix")
        self.thr = np.ascontiguousarray(spec.drive_thresholds(), dtype=np.uint32)
        z = np.zeros
        self.v, self.a, self.psi_prev = z((B, N)), z((B, N)), z((B, N))
        self.ref = z((B, N), np.int32)
        self.z_prev = z((B, N), np.uint8)
        self.ring = z((B, D1, N))
        self.src_hist = z((B, D1, self.n_src), np.uint8)
        self.zbar, self.epsa, self.ebar = z((B, self.nnz)), z((B, self.nnz)), z((B, self.nnz))
        self.g = z(self.nnz)
        self.y, self.zk = z((B, K)), z((B, N))
        self.g_out = z((N, K))
        self.grad_acc = z(self.nnz)
        self.grad_out_acc = z((N, K))
        self.counters = z(3, np.int64)   # absolute step, step since reset, Adam steps
        self.g_abs = z(self.nnz)
        self.g_out_abs = z((N, K))
        self.grad_abs_acc = z(self.nnz)
        self.grad_out_abs_acc = z((N, K))
        self.y_abs = z((B, K))
        self.g_lsens = z(self.nnz)
        self.g_out_lsens = z((N, K))
        self.grad_lsens_acc = z(self.nnz)
        self.grad_out_lsens_acc = z((N, K))
        self.rate = z((B, N))
        self.ebar_reg = z((B, self.nnz))
        # fixed signs: the sign bit of each initial weight (float32 values as given)
        self.w_neg = np.ascontiguousarray(np.signbit(np.asarray(w, np.float32)), dtype=np.uint8)
        self.w_out_neg = np.ascontiguousarray(np.signbit(np.asarray(w_out, np.float32)).reshape(N, K),
                                              dtype=np.uint8)
        self.adam_m, self.adam_v = z(self.nnz), z(self.nnz)
        self.adam_m_out, self.adam_v_out = z((N, K)), z((N, K))
        # generalized delays: rings of the last d_out + 1 spike vectors, the
        # last d_out + d_ls + 1 traces of every synapse and d_ls + 1 signals
        d_out, d_ls = int(getattr(spec, "d_out", 0)), int(getattr(spec, "d_ls", 0))
        self.z_hist = z((B, d_out + 1, N), np.uint8)
        self.ebar_hist = z((B, self.nnz, d_out + d_ls + 1))
        self.L_hist, self.Ls_hist = z((B, d_ls + 1, N)), z((B, d_ls + 1, N))

    def _cfg(self, T):
        s = self.spec
        p = params(s)
        return _Cfg(n_in=s.n_in, n_rec=s.n_rec, n_out=s.n_out, batch=s.batch,
                    neuron_model=s.neuron_model, t_ref=s.t_ref, loss=s.loss,
                    feedback=s.feedback, update_interval=s.update_interval,
                    continuous=s.continuous, max_delay=s.max_delay,
                    n_drive_thr=int(self.thr.shape[0]),
                    alpha=p["alpha"], rho=p["rho"], kappa=p["kappa"], kappa_e=p["kappa_e"],
                    beta_a=p["beta_a"], v_th=p["v_th"], gamma=p["gamma"], beta_sg=p["beta_sg"],
                    lr=p["lr"], drive_weight=p["drive_weight"], drive_seed=s.drive_seed,
                    drive_thr=_p(self.thr) if self.thr.shape[0] else None,
                    surrogate=s.surrogate, reset_mode=s.reset_mode, v_reset=p["v_reset"],
                    c_reg=p["c_reg"], f_target=p["f_target"], beta_reg=p["beta_reg"],
                    sign_mask=s.sign_mask, optimizer=s.optimizer, adam_b1=p["adam_b1"],
                    adam_b2=p["adam_b2"], adam_eps=p["adam_eps"], if_period=s.if_period,
                    if_seed=s.if_seed, d_out=int(getattr(s, "d_out", 0)), d_ls=int(getattr(s, "d_ls", 0)))

    def _state(self):
        st = _State(n_src=self.n_src, nnz=self.nnz)
        for name in ("ptr", "col", "delay", "w", "w_out", "out_mask", "v", "a",
                     "psi_prev", "ref", "z_prev", "ring", "src_hist", "zbar",
                     "epsa", "ebar", "g", "y", "zk", "g_out", "grad_acc",
                     "grad_out_acc", "counters", "g_abs", "g_out_abs", "grad_abs_acc",
                     "grad_out_abs_acc", "y_abs", "g_lsens", "g_out_lsens", "grad_lsens_acc",
                     "grad_out_lsens_acc", "rate", "ebar_reg", "w_neg", "w_out_neg", "adam_m",
                     "adam_v", "adam_m_out", "adam_v_out", "z_hist", "ebar_hist", "L_hist", "Ls_hist"):
            setattr(st, name, _p(getattr(self, name)))
        st.fb = _p(self.fb)
        return st

    def simulate(self, T, x_ptr, x_ids, targets, window=None, lengths=None,
                 forced=None, record=False, forced_psi=None, E_override=None):
        """Run T steps; returns a dict with y [B,T,K], loss [B], raster
        [B,T,N] (uint8), margin [B,T,N] (v - v_th) and, if record, psi and L.
        forced / forced_psi teacher-force the spikes / the surrogate values;
        E_override [B,T,K] replaces the error signal where window = 0."""
        s = self.spec
        B, N, K = s.batch, s.n_rec, s.n_out
        if s.update_interval and T % s.update_interval:
            raise ValueError("T must be a multiple of the update interval")
        x_ptr = np.ascontiguousarray(x_ptr, dtype=np.int64)
        x_ids = np.ascontiguousarray(x_ids, dtype=np.int32)
        assert x_ptr.shape[0] == B * T + 1
        tg = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(B, T, K))
        win = None if window is None else np.ascontiguousarray(window, dtype=np.uint8).reshape(B, T)
        lens = np.full(B, T, np.int32) if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
        fz = None if forced is None else np.ascontiguousarray(forced, dtype=np.uint8).reshape(B, T, N)
        fpsi = None if forced_psi is None else np.ascontiguousarray(forced_psi, dtype=np.float64).reshape(B, T, N)
        eov = None if E_override is None else np.ascontiguousarray(E_override, dtype=np.float64).reshape(B, T, K)
        out = dict(y=np.zeros((B, T, K)), loss=np.zeros(B),
                   raster=np.zeros((B, T, N), np.uint8), margin=np.zeros((B, T, N)),
                   y_abs=np.zeros((B, T, K)))
        if record:
            out["psi"] = np.zeros((B, T, N))
            out["L"] = np.zeros((B, T, N))
        cfg = self._cfg(T)
        st = self._state()
        rc = _load().oracle_simulate(ctypes.byref(cfg), ctypes.byref(st), T,
                                     _p(x_ptr), _p(x_ids), _p(tg), _p(win), _p(lens),
                                     _p(fz), _p(out["y"]), _p(out["loss"]),
                                     _p(out["raster"]), _p(out["margin"]),
                                     _p(out.get("psi")), _p(out.get("L")), _p(out["y_abs"]),
                                     _p(fpsi), _p(eov))
        if rc:
            raise MemoryError("oracle_simulate failed")
        return out

    def take_grads(self):
        """Summed batch-mean gradients applied since the last call (input and
        recurrent synapses in CSR order, and W_out [N, K]); resets them."""
        g, go = self.grad_acc.copy(), self.grad_out_acc.copy()
        self.grad_acc[:] = 0.0
        self.grad_out_acc[:] = 0.0
        return g, go

    def take_grad_magnitudes(self):
        """Sums of |g^t| matching `take_grads` (the condition of each
        accumulated gradient, for the parity tolerance); resets them."""
        g, go = self.grad_abs_acc.copy(), self.grad_out_abs_acc.copy()
        self.grad_abs_acc[:] = 0.0
        self.grad_out_abs_acc[:] = 0.0
        return g, go

    def take_grad_sensitivities(self):
        """sum_t Lsens^t |ebar^t| (and sum_t Esens_k^t zbar_kappa,j^t for W_out)
        matching `take_grads`: the gradients' first-order sensitivity to a
        relative perturbation of the error signals; resets them."""
        g, go = self.grad_lsens_acc.copy(), self.grad_out_lsens_acc.copy()
        self.grad_lsens_acc[:] = 0.0
        self.grad_out_lsens_acc[:] = 0.0
        return g, go


def event_driven_gradients(spec, ptr, col, delay, src_raster, psi, L, T_len=None):
    """Event-driven restatement of the recurrent/input gradient of one sample.

    Follows Algorithm 5 ("Optimized event-driven weight update"): a synapse
    stores the times of its arriving presynaptic spikes; at each arrival
    (and once more at the end of the sample) it integrates its eligibility
    state over the left-open interval (t_prev, t] from the postsynaptic
    history psi^t, L^t and adds sum L^t F_kappa(e^t) to its gradient.

    src_raster : [T, n_src] source spikes (emission steps 1..T)
    psi, L     : [T, N] postsynaptic history of the sample
    returns    : gradient per synapse (CSR order), sum over the sample
    """
    import math
    T = psi.shape[0] if T_len is None else T_len
    p = params(spec)
    alpha, rho, kappa_e, beta_a = p["alpha"], p["rho"], p["kappa_e"], p["beta_a"]
    n_src = ptr.shape[0] - 1
    grads = np.zeros(int(ptr[-1]))
    for i in range(n_src):
        spikes = np.nonzero(src_raster[:T, i])[0] + 1      # emission steps
        for q in range(int(ptr[i]), int(ptr[i + 1])):
            j, d = int(col[q]), int(delay[q])
            arrivals = [int(s) + d for s in spikes if int(s) + d <= T]
            if not arrivals:
                continue
            zbar = epsa = ebar = 0.0
            g = 0.0
            t_prev = arrivals[0] - 1        # everything before is zero
            times = set(arrivals)
            for t_evt in arrivals[1:] + [T]:
                # left-open interval (t_prev, t_evt]
                for t in range(t_prev + 1, t_evt + 1):
                    pp = psi[t - 2, j] if t >= 2 else 0.0
                    p = psi[t - 1, j]
                    epsa_new = pp * zbar + (rho - pp * beta_a) * epsa
                    zbar = alpha * zbar + (1.0 if t in times else 0.0)
                    epsa = epsa_new
                    ebar = kappa_e * ebar + p * (zbar - beta_a * epsa)
                    g += L[t - 1, j] * ebar
                t_prev = t_evt
            grads[q] = g
    return grads

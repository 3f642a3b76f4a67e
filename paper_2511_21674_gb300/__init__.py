"""GB300 event-driven e-prop: thin Python binding of the C ABI (libeprop.so).

Only argument marshalling lives here; every step of the simulation and of
the learning rule runs in the CUDA kernels of ``libeprop.so``.  PyTorch is
used for device memory and streams only.  The binding fails loudly when the
library is missing: there is no CPU fallback.

Typical use::

    import paper_2511_21674_gb300 as ep
    net = ep.Network(spec, ptr, col, w, delay, w_out, out_mask, feedback)
    net.set_inputs(x_ptr, x_ids, targets, window, lengths, T)
    net.simulate(T)
    w = net.weights(ep.PROJ_REC)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libeprop.so")

PROJ_IN, PROJ_REC, PROJ_OUT = 0, 1, 2
ABI_VERSION = 2
MAX_DRIVE_THR = 64

_STATUS = {0: "EPROP_OK", 1: "EPROP_EINVAL", 2: "EPROP_ENOMEM", 3: "EPROP_ECUDA",
           4: "EPROP_ETIMEOUT", 5: "EPROP_ESTATE"}


class EpropError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "abi_version", "n_in", "n_rec", "n_out", "batch", "neuron_model", "t_ref", "loss",
        "feedback", "update_interval", "continuous", "max_delay", "trace_dtype",
        "record_grad", "record_raster", "record_psi", "n_drive_thr", "launch_mode", "trace_kernel",
        "blocks_per_sm", "profile")] + [
        (n, ctypes.c_float) for n in (
            "dt", "tau_m", "tau_a", "beta_a", "v_th", "tau_out", "kappa_e", "gamma",
            "beta_sg", "lr", "drive_weight")] + [
        ("drive_seed", ctypes.c_uint64),
        ("drive_thr", ctypes.c_uint32 * MAX_DRIVE_THR),
        ("surrogate", ctypes.c_int32), ("reset_mode", ctypes.c_int32), ("v_reset", ctypes.c_float),
        ("c_reg", ctypes.c_float), ("f_target", ctypes.c_float), ("beta_reg", ctypes.c_float),
        ("sign_mask", ctypes.c_int32), ("optimizer", ctypes.c_int32),
        ("adam_b1", ctypes.c_float), ("adam_b2", ctypes.c_float), ("adam_eps", ctypes.c_float),
        ("if_period", ctypes.c_int32), ("if_seed", ctypes.c_uint64),
        ("d_out", ctypes.c_int32), ("d_ls", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("events", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("trace_launches", ctypes.c_int64), ("windows", ctypes.c_int64),
                ("trace_ms", ctypes.c_double)]


class Synapses(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("target", ctypes.c_void_p),
                ("weight", ctypes.c_void_p), ("delay", ctypes.c_void_p)]


class TuneResult(ctypes.Structure):
    _fields_ = [("trace_kernel", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("n_candidates", ctypes.c_int32),
                ("cand_trace_kernel", ctypes.c_int32 * 16), ("cand_blocks_per_sm", ctypes.c_int32 * 16),
                ("cand_ms", ctypes.c_double * 16)]


_lib = None

EXPORTS = ("eprop_create_network", "eprop_set_inputs_targets", "eprop_simulate",
           "eprop_read_weights_grads", "eprop_readout", "eprop_readout_raster_static",
           "eprop_read_surrogate",
           "eprop_get_stats", "eprop_sync",
           "eprop_destroy", "eprop_last_error",
           "eprop_predictor_create", "eprop_predictor_num_params", "eprop_predictor_forward",
           "eprop_predictor_train_step", "eprop_predictor_read", "eprop_predictor_set_params",
           "eprop_predictor_sync", "eprop_predictor_destroy", "eprop_predictor_last_error",
           "eprop_attach_predictor", "eprop_read_predictor_inputs", "eprop_autotune",
           "eprop_predictor_set_input_scale", "eprop_learning_signals")


def load_library(path: str = LIB_PATH):
    """Loads libeprop.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_2511_21674_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.eprop_create_network.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(Synapses), vp, vp, vp,
                                         i32, vp, ctypes.POINTER(vp)]
    lib.eprop_set_inputs_targets.argtypes = [vp, vp, vp, i64, vp, vp, vp, i32, i32]
    lib.eprop_simulate.argtypes = [vp, i32, vp]
    lib.eprop_read_weights_grads.argtypes = [vp, i32, vp, vp, i32]
    lib.eprop_readout.argtypes = [vp, vp, vp, vp, i32]
    lib.eprop_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.eprop_read_surrogate.argtypes = [vp, vp, i32]
    lib.eprop_readout_raster_static.argtypes = [vp, vp, i32]
    lib.eprop_sync.argtypes = [vp]
    lib.eprop_destroy.argtypes = [vp]
    lib.eprop_destroy.restype = None
    lib.eprop_last_error.argtypes = [vp]
    lib.eprop_last_error.restype = ctypes.c_char_p
    u64, f32 = ctypes.c_uint64, ctypes.c_float
    lib.eprop_predictor_create.argtypes = [i32, i32, i32, i32, vp, u64, vp, ctypes.POINTER(vp)]
    lib.eprop_predictor_num_params.argtypes = [vp]
    lib.eprop_predictor_forward.argtypes = [vp, vp, i32, vp, i32]
    lib.eprop_predictor_train_step.argtypes = [vp, vp, vp, i32, f32, vp, i32]
    lib.eprop_predictor_read.argtypes = [vp, i32, vp, i64]
    lib.eprop_predictor_set_params.argtypes = [vp, vp]
    lib.eprop_predictor_sync.argtypes = [vp]
    lib.eprop_predictor_destroy.argtypes = [vp]
    lib.eprop_predictor_last_error.argtypes = [vp]
    lib.eprop_predictor_last_error.restype = ctypes.c_char_p
    lib.eprop_attach_predictor.argtypes = [vp, vp, i32]
    lib.eprop_autotune.argtypes = [vp, ctypes.POINTER(TuneResult)]
    lib.eprop_predictor_set_input_scale.argtypes = [vp, vp]
    lib.eprop_read_predictor_inputs.argtypes = [vp, vp, i32]
    lib.eprop_learning_signals.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp]
    void_ret = ("eprop_destroy", "eprop_last_error", "eprop_predictor_destroy", "eprop_predictor_last_error")
    for name in EXPORTS:
        if name not in void_ret:
            getattr(lib, name).restype = ctypes.c_int
    lib.eprop_predictor_num_params.restype = i64
    _lib = lib
    return lib


def learning_signals(feedback, E, stream=None):
    """L [batch, U, n_rec] = sum_k feedback[j, k] E[b, u, k] on the tensor
    cores (eprop_learning_signals); feedback [n_rec, n_out] and E [batch, U,
    n_out] are CUDA float32 tensors."""
    import torch
    lib = load_library()
    if not (feedback.is_cuda and E.is_cuda):
        raise ValueError("feedback and E must be CUDA tensors")
    feedback = feedback.contiguous().float()
    E = E.contiguous().float()
    n_rec, n_out = feedback.shape
    batch, U, k2 = E.shape
    if k2 != n_out:
        raise ValueError("E's last dimension must equal feedback's second")
    L = torch.empty((batch, U, n_rec), dtype=torch.float32, device=E.device)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.eprop_learning_signals(feedback.data_ptr(), E.data_ptr(), L.data_ptr(), n_rec, U, n_out,
                                    batch, stream)
    if st != 0:
        raise EpropError(st, lib.eprop_last_error(None).decode())
    return L


def make_config(spec, launch_mode: int = 1, trace_dtype: int = 0, record_grad: int = 1,
                record_raster: int = 0, trace_kernel: int = 0, blocks_per_sm: int = 0,
                profile: int = 0, record_psi: int = 0) -> Config:
    """C configuration from a `workloads.configs.Spec`-like object."""
    c = Config()
    c.abi_version = ABI_VERSION
    c.n_in, c.n_rec, c.n_out, c.batch = spec.n_in, spec.n_rec, spec.n_out, spec.batch
    c.neuron_model, c.t_ref, c.loss, c.feedback = spec.neuron_model, spec.t_ref, spec.loss, spec.feedback
    c.update_interval, c.continuous, c.max_delay = spec.update_interval, spec.continuous, spec.max_delay
    c.trace_dtype, c.record_grad, c.record_raster = trace_dtype, record_grad, record_raster
    c.record_psi = record_psi
    c.launch_mode = launch_mode
    c.trace_kernel, c.blocks_per_sm, c.profile = trace_kernel, blocks_per_sm, profile
    c.dt, c.tau_m, c.tau_a = spec.dt, spec.tau_m, spec.tau_a
    c.beta_a = spec.beta_a if spec.neuron_model == 1 else 0.0
    c.v_th, c.tau_out = spec.v_th, spec.tau_out
    c.kappa_e = -1.0 if spec.kappa_e is None else spec.kappa_e
    c.gamma, c.beta_sg, c.lr = spec.gamma, spec.beta_sg, spec.lr
    c.drive_weight = spec.drive_weight
    c.drive_seed = spec.drive_seed
    thr = spec.drive_thresholds()
    c.n_drive_thr = int(thr.shape[0]) if spec.drive_weight != 0.0 else 0
    for m in range(int(thr.shape[0])):
        c.drive_thr[m] = int(thr[m])
    c.surrogate, c.reset_mode, c.v_reset = spec.surrogate, spec.reset_mode, spec.v_reset
    c.c_reg, c.f_target, c.beta_reg = spec.c_reg, spec.f_target, spec.beta_reg
    c.sign_mask, c.optimizer = spec.sign_mask, spec.optimizer
    c.adam_b1, c.adam_b2, c.adam_eps = spec.adam_b1, spec.adam_b2, spec.adam_eps
    c.if_period, c.if_seed = spec.if_period, spec.if_seed
    c.d_out, c.d_ls = int(getattr(spec, "d_out", 0)), int(getattr(spec, "d_ls", 0))
    return c


def _ptr(a):
    """(address, is_device) of a numpy array or torch tensor (or None)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, False
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), a.is_cuda
    raise TypeError(f"unsupported array type {type(a)}")


def _same_place(arrs):
    places = {dev for _, dev in (_ptr(a) for a in arrs if a is not None)}
    if len(places) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return bool(places.pop()) if places else False


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Network:
    """One network on the current CUDA device (owned by libeprop).

    Arrays may be numpy (host) or CUDA torch tensors (device); all arrays of
    one call must live on the same side.
    """

    def __init__(self, spec, ptr, col, w, delay, w_out, out_mask=None, feedback=None,
                 stream=None, **cfg_kw):
        self.lib = load_library()
        self.spec = spec
        self.cfg = make_config(spec, **cfg_kw)
        host = isinstance(ptr, np.ndarray)
        if host:
            ptr, col = _np(ptr, np.int64), _np(col, np.int32)
            w, delay = _np(w, np.float32), _np(delay, np.uint8)
            w_out = _np(w_out, np.float32)
            if out_mask is not None:
                # a per-neuron mask [n_rec] applies to every readout of the neuron
                out_mask = _np(out_mask, np.uint8)
                if out_mask.ndim == 1:
                    out_mask = np.ascontiguousarray(np.repeat(out_mask[:, None], spec.n_out, axis=1))
            feedback = None if feedback is None else _np(feedback, np.float32)
        self._keep = (ptr, col, w, delay, w_out, out_mask, feedback)
        is_dev = _same_place([ptr, col, w, delay, w_out, out_mask, feedback])
        syn = Synapses(n_src=spec.n_in + spec.n_rec, nnz=int(col.shape[0]),
                       row_ptr=_ptr(ptr)[0], target=_ptr(col)[0], weight=_ptr(w)[0],
                       delay=_ptr(delay)[0])
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        out = ctypes.c_void_p()
        st = self.lib.eprop_create_network(ctypes.byref(self.cfg), ctypes.byref(syn),
                                           _ptr(w_out)[0], _ptr(out_mask)[0], _ptr(feedback)[0],
                                           int(is_dev), stream, ctypes.byref(out))
        if st != 0:
            raise EpropError(st, self.lib.eprop_last_error(None).decode())
        self.h = out
        self._keep = None
        self.nnz = int(col.shape[0])
        self.nnz_in = int(ptr[spec.n_in]) if spec.n_in else 0
        self.T = None

    def _check(self, st):
        if st != 0:
            raise EpropError(st, self.lib.eprop_last_error(self.h).decode())

    def set_inputs(self, x_ptr, x_ids, targets, window=None, lengths=None, T=None):
        s = self.spec
        T = s.T if T is None else T
        if isinstance(x_ptr, np.ndarray):
            x_ptr, x_ids = _np(x_ptr, np.int64), _np(x_ids, np.int32)
            targets = _np(targets, np.float32)
            window = None if window is None else _np(window, np.uint8)
            lengths = None if lengths is None else _np(lengths, np.int32)
        is_dev = _same_place([x_ptr, x_ids, targets, window, lengths])
        self._check(self.lib.eprop_set_inputs_targets(
            self.h, _ptr(x_ptr)[0], _ptr(x_ids)[0], int(x_ids.shape[0]), _ptr(targets)[0],
            _ptr(window)[0], _ptr(lengths)[0], int(T), int(is_dev)))
        self.T = T

    def simulate(self, T=None, forced=None):
        T = self.T if T is None else T
        fp = None
        if forced is not None:
            addr, dev = _ptr(forced)
            if not dev:
                raise ValueError("forced raster must be a CUDA tensor")
            fp = addr
        self._check(self.lib.eprop_simulate(self.h, int(T), fp))

    def sync(self):
        self._check(self.lib.eprop_sync(self.h))

    def weights(self, proj, with_grad=False):
        s = self.spec
        if proj == PROJ_OUT:
            n = s.n_rec * s.n_out
        elif proj == PROJ_IN:
            n = self.nnz_in
        else:
            n = self.nnz - self.nnz_in
        w = np.zeros(n, np.float32)
        g = np.zeros(n, np.float32) if with_grad else None
        self._check(self.lib.eprop_read_weights_grads(self.h, proj, w.ctypes.data,
                                                      None if g is None else g.ctypes.data, 0))
        if proj == PROJ_OUT:
            w = w.reshape(s.n_rec, s.n_out)
            g = None if g is None else g.reshape(s.n_rec, s.n_out)
        return (w, g) if with_grad else w

    def readout(self, raster=False):
        s = self.spec
        T = self.T
        y = np.zeros((s.batch, T, s.n_out), np.float32)
        loss = np.zeros(s.batch, np.float32)
        r = np.zeros((s.batch, T, s.n_rec), np.uint8) if raster else None
        self._check(self.lib.eprop_readout(self.h, y.ctypes.data, loss.ctypes.data,
                                           None if r is None else r.ctypes.data, 0))
        return (y, loss, r) if raster else (y, loss)

    def raster_static(self):
        """Raster [batch, T, n_rec] of the last call through the library's
        fixed device scratch (no device allocation; needs record_raster=1)."""
        s = self.spec
        r = np.zeros((s.batch, self.T, s.n_rec), np.uint8)
        self._check(self.lib.eprop_readout_raster_static(self.h, r.ctypes.data, 0))
        return r

    def autotune(self) -> dict:
        """Times the candidate launch shapes on the current inputs, keeps the
        fastest and leaves the network state as it was (eprop_autotune)."""
        r = TuneResult()
        self._check(self.lib.eprop_autotune(self.h, ctypes.byref(r)))
        cands = [(r.cand_trace_kernel[q], r.cand_blocks_per_sm[q], r.cand_ms[q]) for q in range(r.n_candidates)]
        return dict(trace_kernel=r.trace_kernel, blocks_per_sm=r.blocks_per_sm, candidates=cands)

    def attach_predictor(self, pred, mode: int = 1):
        """mode 0 detach; bit 0 predicted E outside the target window; bit 1
        record the predictor inputs of every step."""
        self._pred = pred if mode else None
        self._check(self.lib.eprop_attach_predictor(self.h, pred.h if pred is not None else None, mode))

    def predictor_inputs(self):
        """x [batch, T, n_out + 64] of the last call (attached with bit 1)."""
        s = self.spec
        x = np.zeros((s.batch, self.T, s.n_out + 64), np.float32)
        self._check(self.lib.eprop_read_predictor_inputs(self.h, x.ctypes.data, 0))
        return x

    def surrogate(self):
        """psi [batch, T, n_rec] of the last call (needs record_psi=1)."""
        s = self.spec
        psi = np.zeros((s.batch, self.T, s.n_rec), np.float32)
        self._check(self.lib.eprop_read_surrogate(self.h, psi.ctypes.data, 0))
        return psi

    def stats(self) -> dict:
        st = Stats()
        self._check(self.lib.eprop_get_stats(self.h, ctypes.byref(st)))
        return dict(events=st.events, kernel_launches=st.kernel_launches,
                    trace_launches=st.trace_launches, windows=st.windows, trace_ms=st.trace_ms)

    def events(self) -> int:
        return int(self.stats()["events"])

    def close(self):
        if getattr(self, "h", None):
            self.lib.eprop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ predictor

PRED_BUFFERS = dict(params=0, grads=1, A1=2, H1=3, A2=4, H2=5, Y=6, dY=7, dA2=8, dA1=9,
                    m=10, v=11, X=12)


class Predictor:
    """Learned learning-signal predictor (BF16 MLP on the GPU); see
    include/eprop_predictor.h.  Arrays are host numpy float32."""

    def __init__(self, n_in: int, n_out: int, hidden: int = 256, max_rows: int = 4096,
                 params=None, seed: int = 0, stream=None):
        self.lib = load_library()
        self.n_in, self.n_out, self.hidden, self.max_rows = n_in, n_out, hidden, max_rows
        ptr = None
        if params is not None:
            params = np.ascontiguousarray(params, np.float32)
            ptr = params.ctypes.data
        st = None if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        rc = self.lib.eprop_predictor_create(n_in, hidden, n_out, max_rows, ptr, seed, st, ctypes.byref(h))
        if rc != 0:
            raise EpropError(rc, self.lib.eprop_predictor_last_error(None).decode())
        self.h = h
        self.n_params = int(self.lib.eprop_predictor_num_params(self.h))
        self.rows = 0

    def _check(self, rc):
        if rc != 0:
            raise EpropError(rc, self.lib.eprop_predictor_last_error(self.h).decode())

    @staticmethod
    def pack(p: dict) -> np.ndarray:
        return np.concatenate([np.asarray(p[k], np.float32).ravel()
                               for k in ("W1", "b1", "W2", "b2", "W3", "b3")])

    def unpack(self, flat) -> dict:
        dims = [(self.n_in, self.hidden), (self.hidden, self.hidden), (self.hidden, self.n_out)]
        out, o = {}, 0
        for i, (a, b) in enumerate(dims, 1):
            out[f"W{i}"] = np.asarray(flat[o:o + a * b]).reshape(a, b)
            o += a * b
            out[f"b{i}"] = np.asarray(flat[o:o + b])
            o += b
        return out

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float32)
        y = np.zeros((x.shape[0], self.n_out), np.float32)
        self._check(self.lib.eprop_predictor_forward(self.h, x.ctypes.data, x.shape[0], y.ctypes.data, 0))
        self.rows = x.shape[0]
        return y

    def train_step(self, x, e, lr: float) -> float:
        x = np.ascontiguousarray(x, np.float32)
        e = np.ascontiguousarray(e, np.float32)
        loss = np.zeros(1, np.float32)
        self._check(self.lib.eprop_predictor_train_step(self.h, x.ctypes.data, e.ctypes.data, x.shape[0],
                                                        lr, loss.ctypes.data, 0))
        self.rows = x.shape[0]
        return float(loss[0])

    def read(self, name: str) -> np.ndarray:
        which = PRED_BUFFERS[name]
        R, H, K, I = self.rows, self.hidden, self.n_out, self.n_in
        size = {0: self.n_params, 1: self.n_params, 10: self.n_params, 11: self.n_params,
                6: R * K, 7: R * K, 12: R * I}.get(which, R * H)
        out = np.zeros(size, np.float32)
        self._check(self.lib.eprop_predictor_read(self.h, which, out.ctypes.data, size))
        if which in (0, 1, 10, 11):
            return out
        cols = {6: K, 7: K, 12: I}.get(which, H)
        return out.reshape(R, cols)

    def set_input_scale(self, scale):
        scale = np.ascontiguousarray(scale, np.float32)
        assert scale.shape == (self.n_in,)
        self._check(self.lib.eprop_predictor_set_input_scale(self.h, scale.ctypes.data))

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        self._check(self.lib.eprop_predictor_set_params(self.h, flat.ctypes.data))

    def close(self):
        if getattr(self, "h", None):
            self.lib.eprop_predictor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

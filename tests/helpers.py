"""Small shared helpers for tests (no method arithmetic)."""
from __future__ import annotations

import math

import numpy as np

from workloads import configs as C


def tiny_net(n_in, n_rec, n_out, pairs_in, pairs_rec, w_in, w_rec, d_in, d_rec,
             w_out, spec_kw, feedback=None):
    """CSR arrays for an explicit list of synapses.

    pairs_in: list of (input i, target j); pairs_rec: list of (source i, target j)
    """
    src = [i for i, _ in pairs_in] + [n_in + i for i, _ in pairs_rec]
    post = [j for _, j in pairs_in] + [j for _, j in pairs_rec]
    w = list(w_in) + list(w_rec)
    d = list(d_in) + list(d_rec)
    ptr, col, wv, dv = C.to_csr(np.asarray(src, np.int64), np.asarray(post, np.int64),
                                np.asarray(w, np.float32), np.asarray(d, np.uint8),
                                n_in + n_rec)
    spec = C.Spec(name="tiny", n_in=n_in, n_rec=n_rec, n_out=n_out, **spec_kw)
    return dict(spec=spec, ptr=ptr, col=col, w=wv, delay=dv,
                w_out=np.asarray(w_out, np.float32).reshape(n_rec, n_out),
                out_mask=np.ones(n_rec, np.uint8), feedback=feedback)


def raster_to_lists(raster):
    return C.step_lists(np.asarray(raster, dtype=bool))


def tau_for(decay: float) -> float:
    """Time constant (dt = 1) whose decay factor exp(-1/tau) equals decay."""
    return -1.0 / math.log(decay)

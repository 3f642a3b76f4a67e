"""Builds the fixed-in-degree E/I networks directly on a GPU with torch.

Produces the same integer structure (sources, targets, delays, E/I signs)
as `configs._ei_network_np` from the same counter hashes, in chunks so that a
billion-synapse network fits comfortably in device memory.  Holds no
arithmetic of the learning method.
"""
from __future__ import annotations

import math

import numpy as np

from . import configs as C
from . import hashrng as H


def _u64_t(seed, tag, a, b):
    return H.key3_torch(seed ^ (tag * 0x1000193), a, b)


def ei_network_torch(n: int, k_in: int, max_delay: int, J: float, g: float, seed: int,
                     device="cuda", chunk_targets: int = 100_000):
    """CSR by source on `device`: (row_ptr int64 [n+1], col int32, w f32, delay u8)."""
    import torch
    span = n - 1
    s = span // k_in
    if k_in > span:
        raise ValueError("in-degree larger than the number of sources")
    keys, dels = [], []
    m = torch.arange(k_in, device=device, dtype=torch.int64)
    for j0 in range(0, n, chunk_targets):
        j1 = min(n, j0 + chunk_targets)
        j = torch.arange(j0, j1, device=device, dtype=torch.int64).repeat_interleave(k_in)
        mm = m.repeat(j1 - j0)
        h = _u64_t(seed, C._TAG_PRE, j, mm)
        # unsigned modulo of the 64-bit hash: split into high/low 32-bit halves
        hi = (h >> 32) & 0xFFFFFFFF
        lo = h & 0xFFFFFFFF
        r = ((hi % s) * ((1 << 32) % s) + lo % s) % s
        off = 1 + mm * s + r
        pre = (j + off) % n
        keys.append(pre * n + j)
        hd = _u64_t(seed, C._TAG_DELAY, j, mm)
        hi = (hd >> 32) & 0xFFFFFFFF
        lo = hd & 0xFFFFFFFF
        dels.append((1 + ((hi % max_delay) * ((1 << 32) % max_delay) + lo % max_delay) % max_delay)
                    .to(torch.uint8))
        del j, mm, h, hi, lo, r, off, pre, hd
    key = torch.cat(keys)
    del keys
    dly = torch.cat(dels)
    del dels
    key, order = torch.sort(key)
    dly = dly[order]
    del order
    pre = key // n
    col = (key - pre * n).to(torch.int32)
    del key
    counts = torch.bincount(pre, minlength=n)
    ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    ptr[1:] = torch.cumsum(counts, 0)
    w = torch.where(pre < int(0.8 * n), torch.tensor(J, device=device),
                    torch.tensor(-g * J, device=device)).to(torch.float32)
    del pre
    return ptr, col, w, dly


def dense_normal_torch(seed: int, tag: int, n_rows: int, n_cols: int, std: float, device="cuda"):
    """[n_rows, n_cols] N(0, std^2) from the workload hash (float32)."""
    import torch
    out = torch.empty((n_rows, n_cols), dtype=torch.float32, device=device)
    rows = torch.arange(n_rows, device=device, dtype=torch.int64)
    for k in range(n_cols):
        kk = torch.full_like(rows, k)
        h1 = H.key3_torch(seed ^ (tag * 0x1000193), rows, kk)
        h2 = H.key3_torch(seed ^ ((tag + 97) * 0x1000193), rows, kk)
        out[:, k] = (std * H.normal_torch(h1, h2)).to(torch.float32)
    return out


def million_sparse_torch(seed: int = 1237, n_rec: int = 1_000_000, k_in: int = 1000,
                         T: int = 1000, n_out: int = 100, J: float = 0.01, g: float = 5.0,
                         device="cuda", **over) -> dict:
    """The million-neuron workload with its network built on the GPU."""
    spec = C.million_sparse_spec(n_rec=n_rec, T=T, n_out=n_out, seed=seed, **over)
    ptr, col, w, dly = ei_network_torch(n_rec, k_in, spec.max_delay, J, g, seed, device)
    w_out = dense_normal_torch(seed, C._TAG_WO1, n_rec, n_out, 1.0 / math.sqrt(n_rec), device)
    fb = dense_normal_torch(seed, C._TAG_B1, n_rec, n_out, 1.0 / math.sqrt(n_out), device)
    B = spec.batch
    return dict(spec=spec, ptr=ptr, col=col, w=w, delay=dly, w_out=w_out,
                out_mask=None, feedback=fb,
                x_ptr=np.zeros(B * T + 1, dtype=np.int64), x_ids=np.zeros(0, dtype=np.int32),
                targets=C.sinusoid_targets(seed, T, n_out, B),
                window=np.ones((B, T), dtype=np.uint8),
                lengths=np.full(B, T, dtype=np.int32))

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
    m = torch.arange(k_in, device=device, dtype=torch.int64)

    def chunk(j0, j1):
        """(pre, target, delay) of the synapses onto targets j0..j1-1, by target."""
        j = torch.arange(j0, j1, device=device, dtype=torch.int64).repeat_interleave(k_in)
        mm = m.repeat(j1 - j0)
        h = _u64_t(seed, C._TAG_PRE, j, mm)
        # unsigned modulo of the 64-bit hash: split into high/low 32-bit halves
        hi = (h >> 32) & 0xFFFFFFFF
        lo = h & 0xFFFFFFFF
        r = ((hi % s) * ((1 << 32) % s) + lo % s) % s
        pre = (j + 1 + mm * s + r) % n
        hd = _u64_t(seed, C._TAG_DELAY, j, mm)
        hi = (hd >> 32) & 0xFFFFFFFF
        lo = hd & 0xFFFFFFFF
        d = (1 + ((hi % max_delay) * ((1 << 32) % max_delay) + lo % max_delay) % max_delay).to(torch.uint8)
        return pre, j, d

    if n * k_in >= (1 << 31) - 1:
        # too many synapses for one sort: counting placement by source, chunk
        # by chunk in ascending target order, gives the same CSR (targets of
        # a row ascending, as the sorted build)
        counts = torch.zeros(n, dtype=torch.int64, device=device)
        for j0 in range(0, n, chunk_targets):
            pre, _, _ = chunk(j0, min(n, j0 + chunk_targets))
            counts += torch.bincount(pre, minlength=n)
        ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
        ptr[1:] = torch.cumsum(counts, 0)
        nnz = int(ptr[-1])
        col = torch.empty(nnz, dtype=torch.int32, device=device)
        dly = torch.empty(nnz, dtype=torch.uint8, device=device)
        w = torch.empty(nnz, dtype=torch.float32, device=device)
        fill = ptr[:-1].clone()
        for j0 in range(0, n, chunk_targets):
            pre, j, d = chunk(j0, min(n, j0 + chunk_targets))
            pre_s, order = torch.sort(pre, stable=True)     # targets stay ascending within a source
            grp, cnt = torch.unique_consecutive(pre_s, return_counts=True)
            first = torch.cumsum(cnt, 0) - cnt
            rank = torch.arange(pre_s.numel(), device=device) - torch.repeat_interleave(first, cnt)
            pos = fill[pre_s] + rank
            col[pos] = j[order].to(torch.int32)
            dly[pos] = d[order]
            w[pos] = torch.where(pre_s < int(0.8 * n), torch.tensor(J, device=device),
                                 torch.tensor(-g * J, device=device)).to(torch.float32)
            fill[grp] += cnt
            del pre, j, d, pre_s, order, grp, cnt, first, rank, pos
        return ptr, col, w, dly
    keys, dels = [], []
    for j0 in range(0, n, chunk_targets):
        pre, j, d = chunk(j0, min(n, j0 + chunk_targets))
        keys.append(pre * n + j)
        dels.append(d)
        del pre, j, d
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


def scaling_torch(seed: int = 1241, n_rec: int = 128_000, k_rec: int = 10_000, n_in: int = 1000,
                  k_in: int = 100, n_out: int = 10, k_out: int = 1000, fb_outdeg: int = 100,
                  T: int = 20_000, update_interval: int = 1000, rate_hz: float = 5.0,
                  J: float = 0.001, g: float = 5.0, device="cuda", **over) -> dict:
    """The scaling experiment's network (`configs.scaling_network`) with its
    recurrent synapses built on the GPU: the same integer structure, weights
    and inputs as the numpy build."""
    import torch
    spec = C.scaling_spec(n_rec=n_rec, n_in=n_in, n_out=n_out, T=T, update_interval=update_interval,
                          rate_hz=rate_hz, seed=seed, **over)
    pre_i, post_i, _ = C.fixed_indegree_pairs(n_in, n_rec, k_in, seed ^ 0x5151, False)
    w_i = np.full(pre_i.shape[0], J, dtype=np.float32)
    ptr_i, col_i, wv_i, dv_i = C.to_csr(pre_i, post_i, w_i, np.ones(pre_i.shape[0], np.uint8), n_in)
    del pre_i, post_i, w_i
    ptr_r, col_r, w_r, d_r = ei_network_torch(n_rec, k_rec, spec.max_delay, J, g, seed, device,
                                              chunk_targets=max(1, 10_000_000 // k_rec))
    nnz_in = int(ptr_i[-1])
    ptr = torch.cat([torch.from_numpy(ptr_i).to(device), ptr_r[1:] + nnz_in])
    col = torch.cat([torch.from_numpy(col_i).to(device), col_r])
    del col_r
    w = torch.cat([torch.from_numpy(wv_i).to(device), w_r])
    del w_r
    dly = torch.cat([torch.from_numpy(dv_i).to(device), d_r])
    del d_r
    mask = C.readout_indegree_mask(seed, n_rec, n_out, k_out)
    j = np.arange(n_rec)
    w_out = np.stack([C._weights(seed, C._TAG_WO1, j, np.full(n_rec, k), 1.0 / math.sqrt(k_out))
                      for k in range(n_out)], axis=1) * mask
    fb = C.sparse_feedback(seed, n_rec, n_out, fb_outdeg)
    x_ptr, x_ids = C.poisson_inputs(seed, n_in, T, rate_hz)
    return dict(spec=spec, ptr=ptr, col=col, w=w, delay=dly,
                w_out=torch.from_numpy(np.ascontiguousarray(w_out, dtype=np.float32)).to(device),
                out_mask=torch.from_numpy(mask).to(device),
                feedback=torch.from_numpy(fb).to(device), x_ptr=x_ptr, x_ids=x_ids,
                targets=C.sinusoid_targets(seed, T, n_out, 1),
                window=np.ones((1, T), dtype=np.uint8), lengths=np.full(1, T, dtype=np.int32))

"""Counter-based hashing used to draw every synthetic input.

The mixer is the SplitMix64 output function (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; constants as in
Vigna's public-domain splitmix64.c).  It is applied to integer counters
(seed, neuron, step, ...) so that any element of any array can be
regenerated independently, on the CPU with numpy or on a GPU with torch,
with bit-identical results.

This module holds no arithmetic of the learning method.
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1


def mix_int(x: int) -> int:
    """SplitMix64 output function on a Python int (reference, scalar)."""
    z = (x + GOLDEN) & MASK64
    z = ((z ^ (z >> 30)) * M1) & MASK64
    z = ((z ^ (z >> 27)) * M2) & MASK64
    return z ^ (z >> 31)


def mix_np(x: np.ndarray) -> np.ndarray:
    """Vectorised SplitMix64 output function on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))


def _to_signed(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def mix_torch(x):
    """SplitMix64 on torch int64 tensors (two's-complement wraparound).

    torch has no uint64 arithmetic, so logical right shifts are emulated by
    an arithmetic shift followed by a mask; multiplication wraps modulo 2^64
    exactly as the unsigned product does.
    """
    import torch

    def lsr(v, k):
        return (v >> k) & ((1 << (64 - k)) - 1)

    z = x + _to_signed(GOLDEN)
    z = (z ^ lsr(z, 30)) * _to_signed(M1)
    z = (z ^ lsr(z, 27)) * _to_signed(M2)
    return z ^ lsr(z, 31)


def key3_np(seed: int, a, b) -> np.ndarray:
    """hash(seed, a, b) for broadcastable integer arrays a, b (numpy)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    return mix_np(mix_np(np.uint64(seed) ^ a) ^ b)


def key3_torch(seed: int, a, b):
    return mix_torch(mix_torch(a ^ _to_signed(seed & MASK64)) ^ b)


def uniform_np(h: np.ndarray) -> np.ndarray:
    """53-bit uniform in [0, 1) from a uint64 hash."""
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_torch(h):
    import torch
    return ((h >> 11) & ((1 << 53) - 1)).to(torch.float64) * (1.0 / (1 << 53))


def normal_np(h1: np.ndarray, h2: np.ndarray) -> np.ndarray:
    """Standard normal by the Box-Muller transform of two hashes."""
    u1 = 1.0 - uniform_np(h1)          # (0, 1]
    u2 = uniform_np(h2)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def normal_torch(h1, h2):
    import torch
    u1 = 1.0 - uniform_torch(h1)
    u2 = uniform_torch(h2)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * torch.pi * u2)


def drive_hash_int(seed: int, sample: int, t_abs: int, j: int) -> int:
    """Key of the external drive count of neuron j at absolute step t_abs.

    hash = mix(mix(mix(seed ^ j) ^ t_abs) ^ sample); the count is the number
    of thresholds of the drive table that the upper 32 bits reach.  Both the
    CUDA library and the oracle re-implement this key from this definition.
    """
    return mix_int(mix_int(mix_int((seed ^ j) & MASK64) ^ t_abs) ^ sample)

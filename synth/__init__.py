"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle legs.

This module holds none of the method's arithmetic: it only draws bit patterns.
The generator is SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw ``i`` of stream ``(seed, stream)`` is the SplitMix64 output
function applied to ``key + (i + 1) * GAMMA`` where ``key`` mixes the seed and
the stream id.

Value recipe (per element of a ``1/E/M`` format; one 64-bit draw ``r``):

* sign = bit 0 of ``r`` (uniform);
* fraction = bits 1..M of ``r`` (uniform);
* exponent field: with ``h = r >> 32`` and ``t = h % 100``: ``t == 0`` -> 0
  (zero or subnormal), ``t == 1`` -> all ones (Inf or NaN), otherwise uniform
  over the normal range ``1 .. 2^E - 2`` via ``1 + (h // 100) % (2^E - 2)``.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_A, SEED_B, SEED_C = 1602, 4716, 1604716
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int = 0) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.array([(seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03) & (2 ** 64 - 1)],
                     dtype=np.uint64)
        return _mix(k)[0]


def splitmix64(seed: int, n: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """``n`` 64-bit draws of stream ``(seed, stream)`` starting at counter ``start``."""
    key = stream_key(seed, stream)
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for lo in range(0, n, _CHUNK):
            hi = min(n, lo + _CHUNK)
            i = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            out[lo:hi] = _mix(key + i * GAMMA)
    return out


def container_dtype(B: int):
    """Standard-representation container for a B-bit pattern."""
    return np.uint8 if B <= 8 else (np.uint16 if B <= 16 else np.uint32)


def splitmix64_at(seed: int, idx, stream: int = 0) -> np.ndarray:
    """Draws at arbitrary counters: element k is draw ``idx[k]`` of the stream."""
    key = stream_key(seed, stream)
    i = np.asarray(idx, dtype=np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        return _mix(key + i * GAMMA)


def _fp_from_draws(E: int, M: int, r: np.ndarray) -> np.ndarray:
    emax = (1 << E) - 1
    s = r & np.uint64(1)
    f = (r >> np.uint64(1)) & np.uint64((1 << M) - 1)
    h = r >> np.uint64(32)
    t = h % np.uint64(100)
    e = np.uint64(1) + (h // np.uint64(100)) % np.uint64(emax - 1)
    e = np.where(t == 0, np.uint64(0), np.where(t == 1, np.uint64(emax), e))
    return (s << np.uint64(E + M)) | (e << np.uint64(M)) | f


def fp_values(E: int, M: int, n: int, seed: int, stream: int = 0, start: int = 0,
              dtype=None) -> np.ndarray:
    """``n`` B-bit patterns of format 1/E/M with the recipe in the module doc."""
    B = 1 + E + M
    dtype = dtype or container_dtype(B)
    out = np.empty(n, dtype=dtype)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        r = splitmix64(seed, hi - lo, stream, start + lo)
        out[lo:hi] = _fp_from_draws(E, M, r).astype(dtype)
    return out


def fp_values_at(E: int, M: int, idx, seed: int, stream: int = 0) -> np.ndarray:
    """The values ``fp_values`` gives at the element indices ``idx`` (uint32)."""
    return _fp_from_draws(E, M, splitmix64_at(seed, idx, stream)).astype(np.uint32)


def uniform_bits(B: int, n: int, seed: int, stream: int = 0, dtype=None) -> np.ndarray:
    """``n`` uniformly random B-bit patterns (every encoding equally likely)."""
    dtype = dtype or container_dtype(B)
    r = splitmix64(seed, n, stream)
    return (r & np.uint64((1 << B) - 1)).astype(dtype)


def all_pairs(B: int):
    """Every ordered pair of B-bit patterns: a = i >> B, b = i & (2^B - 1)."""
    i = np.arange(1 << (2 * B), dtype=np.uint64)
    dt = container_dtype(B)
    return (i >> np.uint64(B)).astype(dt), (i & np.uint64((1 << B) - 1)).astype(dt)


def log_uniform_lengths(n: int, lo: int, hi: int, seed: int, stream: int = 0) -> np.ndarray:
    """``n`` integers floor(exp(U[ln lo, ln hi])) from the seeded stream."""
    r = splitmix64(seed, n, stream)
    u = (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    v = np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
    return np.clip(v, lo, hi)


def uniform01(n: int, seed: int, stream: int = 0) -> np.ndarray:
    r = splitmix64(seed, n, stream)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

"""Seeded synthetic inputs for the join path.

This module only draws numbers: key columns, payload columns and the
band-join (a, k) columns.  It holds none of the join arithmetic, so the
CUDA path, the CPU oracle, the tests and the benchmark can all take their
inputs from it without sharing any part of the method.

Every draw is counter based: value i of stream (seed, stream_id) is the
SplitMix64 output for counter i (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written with torch int64
operations.  The same call therefore gives the same integers on the CPU and
on a CUDA device, in any order and at any size.

Workload shapes (the paper's own data, TPC-H and its "keys divided by a
positive integer" variant of Sec. 5.1.3, is not available; these synthetic
stand-ins follow its structure):

* uniform int32 keys in [lo, hi)                    -> ``uniform_keys``
* Zipf(theta) ranks over a domain of D keys,
  mapped to keys by a fixed bijection                 -> ``zipf_keys``
* the "divide the key by a positive integer" transform
  that raises the tuples per key (Sec. 5.1.3)         -> ``divide_keys``
* independent uniform (a, k) columns for band joins  -> ``band_columns``
* payload = row id                                     -> ``row_ids``
"""
from __future__ import annotations

import math

import torch

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB


def _s64(x: int) -> int:
    """Reinterpret an unsigned 64-bit constant as a signed int64."""
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def _srl(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of an int64 tensor (torch shifts arithmetically)."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def _fmix(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output mixer (a bijection on 64-bit words)."""
    z = (z ^ _srl(z, 30)) * _s64(_MIX1)
    z = (z ^ _srl(z, 27)) * _s64(_MIX2)
    return z ^ _srl(z, 31)


def _fmix_int(z: int) -> int:
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _MIX1) & _MASK64
    z = ((z ^ (z >> 27)) * _MIX2) & _MASK64
    return z ^ (z >> 31)


def stream_seed(seed: int, stream: int) -> int:
    """64-bit state for sub-stream ``stream`` of ``seed`` (e.g. R = 0, S = 1)."""
    return _fmix_int(_fmix_int(seed * 0x100000001B3 + 0x51ED27) ^ (stream * _GAMMA))


def raw_u64(n: int, seed: int, stream: int = 0, device="cpu",
            offset: int = 0) -> torch.Tensor:
    """SplitMix64 words ``offset .. offset+n-1`` of a stream, as int64 bit patterns."""
    base = stream_seed(seed, stream)
    i = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    return _fmix(i * _s64(_GAMMA) + _s64(base))


def uniform_int(n, lo, hi, seed, stream=0, device="cpu", dtype=torch.int32):
    """n integers uniform in [lo, hi) (modulo draw from 63 random bits)."""
    if hi <= lo:
        raise ValueError("empty range")
    span = hi - lo
    if span > (1 << 62):
        raise ValueError("range too wide")
    u = _srl(raw_u64(n, seed, stream, device), 1)
    return (lo + (u % span)).to(dtype)


def uniform_float(n, seed, stream=0, device="cpu") -> torch.Tensor:
    """n doubles uniform in [0, 1) with 53 random bits each."""
    u = _srl(raw_u64(n, seed, stream, device), 11)
    return u.to(torch.float64) * (1.0 / (1 << 53))


def row_ids(n, device="cpu") -> torch.Tensor:
    """Payload column equal to the row index (int32)."""
    return torch.arange(n, dtype=torch.int32, device=device)


def uniform_keys(n, lo, hi, seed, stream=0, device="cpu", dtype=torch.int32):
    """Join keys uniform in [lo, hi)."""
    return uniform_int(n, lo, hi, seed, stream, device, dtype)


def zipf_cdf(theta: float, domain: int, device="cpu") -> torch.Tensor:
    """Cumulative distribution of Zipf(theta) over ranks 1..domain (float64)."""
    k = torch.arange(1, domain + 1, dtype=torch.float64, device=device)
    w = k.pow(-float(theta)) if theta != 0 else torch.ones_like(k)
    c = torch.cumsum(w, 0)
    c /= c[-1].clone()
    return c


def zipf_ranks(n, theta, domain, seed, stream=0, device="cpu", cdf=None):
    """n zero-based ranks drawn from Zipf(theta) over ``domain`` ranks.

    Exact inverse-CDF sampling: rank = #{k : cdf[k] <= u} for u ~ U[0,1).
    theta = 0 is the uniform distribution and skips the table.
    """
    if theta == 0:
        return uniform_int(n, 0, domain, seed, stream, device, torch.int64)
    if cdf is None:
        cdf = zipf_cdf(theta, domain, device)
    out = torch.empty(n, dtype=torch.int64, device=device)
    step = 1 << 26
    for o in range(0, n, step):
        m = min(step, n - o)
        u = _srl(raw_u64(m, seed, stream, device, offset=o), 11).to(torch.float64) * (1.0 / (1 << 53))
        r = torch.searchsorted(cdf, u, right=True)
        out[o:o + m] = r.clamp_(max=domain - 1)
    return out


def rank_to_key32(rank: torch.Tensor, domain_bits: int, seed: int) -> torch.Tensor:
    """Bijection of [0, 2^domain_bits): key = (rank * 0x9E3779B1 + c) mod 2^bits.

    The multiplier is odd, so the map is a permutation of the domain; it
    scatters the popular ranks across the key space.
    """
    c = stream_seed(seed, 7) & ((1 << domain_bits) - 1)
    m = (1 << domain_bits) - 1
    return ((rank * 0x9E3779B1 + c) & m).to(torch.int32)


def rank_to_key64(rank: torch.Tensor, seed: int) -> torch.Tensor:
    """Bijection of 64-bit words: key = SplitMix64-mix(rank xor c), as int64."""
    c = _s64(stream_seed(seed, 9))
    return _fmix(rank ^ c)


def zipf_keys(n, theta, domain_bits, seed, stream=0, device="cpu",
              dtype=torch.int32, cdf=None):
    """Zipf(theta) keys over 2^domain_bits ranks mapped by a fixed bijection."""
    domain = 1 << domain_bits
    r = zipf_ranks(n, theta, domain, seed, stream, device, cdf)
    if dtype == torch.int32:
        return rank_to_key32(r, domain_bits, seed)
    return rank_to_key64(r, seed)


def divide_keys(keys: torch.Tensor, divisor: int) -> torch.Tensor:
    """Sec. 5.1.3's synthetic transform: integer-divide every key by ``divisor``."""
    return torch.div(keys, divisor, rounding_mode="floor").to(keys.dtype)


def band_columns(n, domain_bits, seed, stream=0, device="cpu"):
    """Independent uniform int32 columns (a, k) in [0, 2^domain_bits)."""
    a = uniform_int(n, 0, 1 << domain_bits, seed, 2 * stream + 100, device)
    k = uniform_int(n, 0, 1 << domain_bits, seed, 2 * stream + 101, device)
    return a, k


def log_uniform_int(n, lo, hi, seed, stream=0, device="cpu") -> torch.Tensor:
    """n integers log-uniform in [lo, hi] (for mixed instance sizes)."""
    u = uniform_float(n, seed, stream, device)
    v = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return v.floor().clamp_(lo, hi).to(torch.int64)

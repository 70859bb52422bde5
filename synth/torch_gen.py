"""The generators of ``synth`` written with torch tensor ops, for device-side
generation of the large workloads (2^27 .. 2^30 keys).

Same counter-based SplitMix64 stream and the same recipes as the numpy
versions; the integer recipes (uniform, sorted, reverse, distinct16, zipf,
dup64, uniform64) produce bit-identical arrays, which
``tests/test_synth.py`` checks on the CPU.  ``lognormal3`` goes through
float64 log/cos/exp, whose last bit may differ between libraries, so callers
that compare against the oracle hand the oracle the very array generated here.
Like the numpy module, nothing here sorts, merges or partitions.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import (DIST_DISTINCT16, DIST_DUP64, DIST_LOGNORMAL3, DIST_SORTED, DIST_UNIFORM, DIST_ZIPF,
               _LN_MU, _LN_SIGMA, _LN_W, _zipf_cdf, stream_seed)

_CHUNK = 1 << 25


def _s64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


_GAMMA = _s64(0x9E3779B97F4A7C15)
_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)


def _srl(x, k: int):
    """Logical right shift of int64 words holding uint64 bits."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed: int, start: int, count: int, device) -> torch.Tensor:
    """x_i for i in [start, start + count) as int64 tensors holding uint64 bits."""
    ctr = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = ctr * _GAMMA + _s64(seed)
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def _unit_double(x):
    return _srl(x, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def _fill(n: int, device, dtype, fn):
    out = torch.empty(n, dtype=dtype, device=device)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        out[c0:c1] = fn(c0, c1 - c0)
    return out


def _low32(x):
    return (x & 0xFFFFFFFF).to(torch.uint32)


def uniform_u32(n: int, seed: int, device="cuda") -> torch.Tensor:
    ss = stream_seed(seed, DIST_UNIFORM)
    return _fill(n, device, torch.uint32, lambda c0, c: _low32(splitmix64(ss, c0, c, device)))


def sorted_u32(n: int, seed: int, device="cuda") -> torch.Tensor:
    if n == 0:
        return torch.empty(0, dtype=torch.uint32, device=device)
    span = max(1, (1 << 32) // n)
    ss = stream_seed(seed, DIST_SORTED)
    out = torch.empty(n, dtype=torch.uint32, device=device)
    acc = 0
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        x = splitmix64(ss, c0, c1 - c0, device)
        # unsigned remainder of the 64-bit word by (span + 1) < 2^31
        m = span + 1
        hi = _srl(x, 32)
        lo = x & 0xFFFFFFFF
        gaps = ((hi % m) * ((1 << 32) % m) + lo % m) % m
        run = torch.cumsum(gaps, 0) + acc
        acc = int(run[-1].item())
        out[c0:c1] = torch.clamp(run, max=0xFFFFFFFF).to(torch.uint32)
    return out


def reverse_u32(n: int, seed: int, device="cuda") -> torch.Tensor:
    return torch.flip(sorted_u32(n, seed, device).view(torch.int32), [0]).contiguous().view(torch.uint32)


def distinct16_u32(n: int, seed: int, device="cuda") -> torch.Tensor:
    ss = stream_seed(seed, DIST_DISTINCT16)
    table = _low32(splitmix64(ss ^ 0x5A5A5A5A5A5A5A5A, 0, 16, device)).to(torch.int64)
    return _fill(n, device, torch.uint32,
                 lambda c0, c: table[splitmix64(ss, c0, c, device) & 15].to(torch.uint32))


def _fmix32(h):
    """MurmurHash3's 32-bit finaliser on int64 words holding uint32 values."""
    h = h ^ (h >> 16)
    h = (h * 0x85EBCA6B) & 0xFFFFFFFF
    h = h ^ (h >> 13)
    h = (h * 0xC2B2AE35) & 0xFFFFFFFF
    return h ^ (h >> 16)


def zipf_u32(n: int, seed: int, s: float = 1.1, ranks: int = 1 << 20, device="cuda") -> torch.Tensor:
    cdf = torch.from_numpy(_zipf_cdf(ranks, s)).to(device)
    ss = stream_seed(seed, DIST_ZIPF)

    def chunk(c0, c):
        u = _unit_double(splitmix64(ss, c0, c, device))
        r = torch.clamp(torch.searchsorted(cdf, u, right=True), max=ranks - 1) + 1
        return _fmix32(r).to(torch.uint32)
    return _fill(n, device, torch.uint32, chunk)


def lognormal3_u32(n: int, seed: int, device="cuda") -> torch.Tensor:
    ss = stream_seed(seed, DIST_LOGNORMAL3)
    cw = torch.tensor(np.cumsum(_LN_W), dtype=torch.float64, device=device)
    mu = torch.tensor(_LN_MU, dtype=torch.float64, device=device)
    sg = torch.tensor(_LN_SIGMA, dtype=torch.float64, device=device)

    def chunk(c0, c):
        x = splitmix64(ss, 3 * c0, 3 * c, device).view(-1, 3)
        comp = torch.clamp(torch.searchsorted(cw, _unit_double(x[:, 0]).contiguous(), right=True), 0, 2)
        u1 = 1.0 - _unit_double(x[:, 1])
        u2 = _unit_double(x[:, 2])
        g = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        z = mu[comp] + sg[comp] * g
        v = torch.floor(torch.exp(torch.clamp(z, max=23.0)))
        return torch.clamp(v, max=4294967295.0).to(torch.int64).to(torch.uint32)
    return _fill(n, device, torch.uint32, chunk)


def u32_distribution(name: str, n: int, seed: int, device="cuda") -> torch.Tensor:
    fn = {"uniform": uniform_u32, "sorted": sorted_u32, "reverse": reverse_u32,
          "distinct16": distinct16_u32, "zipf": zipf_u32, "lognormal3": lognormal3_u32}[name]
    return fn(n, seed, device=device)


def uniform_u64(n: int, seed: int, device="cuda") -> torch.Tensor:
    ss = stream_seed(seed, DIST_UNIFORM) ^ 0xA5A5A5A5A5A5A5A5
    return _fill(n, device, torch.int64, lambda c0, c: splitmix64(ss, c0, c, device)).view(torch.uint64)


def dup_u64(n: int, seed: int, distinct: int = 1 << 20, device="cuda"):
    """(keys uint64, values uint32 = original index); distinct must be a power of two."""
    assert distinct & (distinct - 1) == 0, "device path takes power-of-two dictionaries"
    ss = stream_seed(seed, DIST_DUP64)
    table = splitmix64(ss ^ 0x3C3C3C3C3C3C3C3C, 0, distinct, device)
    keys = _fill(n, device, torch.int64,
                 lambda c0, c: table[splitmix64(ss, c0, c, device) & (distinct - 1)]).view(torch.uint64)
    vals = torch.arange(n, dtype=torch.int64, device=device).to(torch.uint32)
    return keys, vals

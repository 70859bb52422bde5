"""Seeded synthetic inputs for the sort workloads.

This module only draws numbers: it holds none of the sorting method's
arithmetic (no comparison, merge or partition).  Both the CPU oracle tests and
the GPU path take their inputs from here, so the two sides see the same bytes.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used counter-style,

    x_i = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15)   (mod 2^64)

so any element can be regenerated from (seed, i) alone.  ``mix64`` is a
bijection of 64-bit words, hence distinct counters give distinct outputs; the
duplicate-heavy dictionaries below rely on that.

Workload recipes (the paper's own inputs are ``np.random.randint(n, size=n)``
integers, Section "MPI Merge Sort", Dividing array into subarrays):

* ``uniform_u32``     low 32 bits of x_i.
* ``sorted_u32``      nondecreasing by construction: running sum of gaps drawn
                      uniform in [0, floor(2^32 / n)].
* ``reverse_u32``     ``sorted_u32`` read backwards.
* ``distinct16_u32``  D[x_i mod 16], D = 16 seeded 32-bit words.
* ``zipf_u32``        rank r in [1, 2^20] with P(r) ~ r^-s (s = 1.1) by
                      inverse-CDF lookup, key = fmix32(r) (a bijective 32-bit
                      finaliser, so frequent keys are spread over the range).
* ``dup_u64``         D[x_i mod 2^20], D = 2^20 distinct 64-bit words; the
                      value of element i is i, so stability is checkable.
* ``lognormal3_u32``  mixture of three lognormals (weights 0.5/0.3/0.2,
                      ln-space mu 14/18/21, sigma 1.0/0.5/0.3), key =
                      min(floor(e^z), 2^32 - 1).
* ``segment_lengths`` L = max(1, min(65536, floor(exp(u * ln 65537)))).
* ``poisson_requests`` exponential gaps, sizes log-uniform in [2^10, 2^24].
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 24

# Stream ids: a workload seed s and a distribution index k give the stream
# seed s * 16 + k, so the five 2^28 distributions never share a stream.
DIST_UNIFORM, DIST_SORTED, DIST_REVERSE, DIST_DISTINCT16, DIST_ZIPF = 0, 1, 2, 3, 4
DIST_DUP64, DIST_LOGNORMAL3, DIST_SEGLENS, DIST_REQUESTS = 5, 6, 7, 8
DIST_NAMES = ("uniform", "sorted", "reverse", "distinct16", "zipf")


def stream_seed(seed: int, dist: int) -> int:
    return (int(seed) * 16 + int(dist)) & 0xFFFFFFFFFFFFFFFF


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """x_i for i in [start, start + count) as uint64."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for c0 in range(0, count, _CHUNK):
            c1 = min(count, c0 + _CHUNK)
            ctr = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
            out[c0:c1] = _mix64(s + ctr * GAMMA)
    return out


def unit_double(x: np.ndarray) -> np.ndarray:
    """Top 53 bits of x as a double in [0, 1)."""
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def fmix32(h: np.ndarray) -> np.ndarray:
    """MurmurHash3's 32-bit finaliser (bijective on uint32)."""
    h = h.astype(np.uint32)
    with np.errstate(over="ignore"):
        h ^= h >> np.uint32(16)
        h *= np.uint32(0x85EBCA6B)
        h ^= h >> np.uint32(13)
        h *= np.uint32(0xC2B2AE35)
        h ^= h >> np.uint32(16)
    return h


def uniform_u32(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    ss = stream_seed(seed, DIST_UNIFORM)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        out[c0:c1] = splitmix64(ss, c0, c1 - c0).astype(np.uint32)
    return out


def sorted_u32(n: int, seed: int) -> np.ndarray:
    if n == 0:
        return np.empty(0, dtype=np.uint32)
    span = max(1, (1 << 32) // n)
    ss = stream_seed(seed, DIST_SORTED)
    out = np.empty(n, dtype=np.uint32)
    acc = np.uint64(0)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        gaps = splitmix64(ss, c0, c1 - c0) % np.uint64(span + 1)
        run = np.cumsum(gaps, dtype=np.uint64) + acc
        acc = run[-1]
        out[c0:c1] = np.minimum(run, np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return out


def reverse_u32(n: int, seed: int) -> np.ndarray:
    return np.ascontiguousarray(sorted_u32(n, seed)[::-1])


def distinct16_u32(n: int, seed: int) -> np.ndarray:
    ss = stream_seed(seed, DIST_DISTINCT16)
    table = splitmix64(ss ^ 0x5A5A5A5A5A5A5A5A, 0, 16).astype(np.uint32)
    out = np.empty(n, dtype=np.uint32)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        out[c0:c1] = table[(splitmix64(ss, c0, c1 - c0) & np.uint64(15)).astype(np.int64)]
    return out


_ZIPF_CACHE: dict = {}


def _zipf_cdf(ranks: int, s: float) -> np.ndarray:
    key = (ranks, s)
    if key not in _ZIPF_CACHE:
        w = np.arange(1, ranks + 1, dtype=np.float64) ** (-s)
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        _ZIPF_CACHE[key] = cdf
    return _ZIPF_CACHE[key]


def zipf_u32(n: int, seed: int, s: float = 1.1, ranks: int = 1 << 20) -> np.ndarray:
    cdf = _zipf_cdf(ranks, s)
    ss = stream_seed(seed, DIST_ZIPF)
    out = np.empty(n, dtype=np.uint32)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        u = unit_double(splitmix64(ss, c0, c1 - c0))
        r = np.minimum(np.searchsorted(cdf, u, side="right"), ranks - 1) + 1
        out[c0:c1] = fmix32(r.astype(np.uint32))
    return out


def u32_distribution(name: str, n: int, seed: int) -> np.ndarray:
    fn = {"uniform": uniform_u32, "sorted": sorted_u32, "reverse": reverse_u32,
          "distinct16": distinct16_u32, "zipf": zipf_u32,
          "lognormal3": lognormal3_u32}[name]
    return fn(n, seed)


def uniform_u64(n: int, seed: int) -> np.ndarray:
    return splitmix64(stream_seed(seed, DIST_UNIFORM) ^ 0xA5A5A5A5A5A5A5A5, 0, n)


def dup_u64(n: int, seed: int, distinct: int = 1 << 20):
    """(keys uint64, values uint32 = original index)."""
    ss = stream_seed(seed, DIST_DUP64)
    table = splitmix64(ss ^ 0x3C3C3C3C3C3C3C3C, 0, distinct)
    keys = np.empty(n, dtype=np.uint64)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        keys[c0:c1] = table[(splitmix64(ss, c0, c1 - c0) % np.uint64(distinct)).astype(np.int64)]
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


_LN_W = (0.5, 0.3, 0.2)
_LN_MU = (14.0, 18.0, 21.0)
_LN_SIGMA = (1.0, 0.5, 0.3)


def lognormal3_u32(n: int, seed: int) -> np.ndarray:
    ss = stream_seed(seed, DIST_LOGNORMAL3)
    out = np.empty(n, dtype=np.uint32)
    cw = np.cumsum(_LN_W)
    mu = np.asarray(_LN_MU)
    sg = np.asarray(_LN_SIGMA)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        x = splitmix64(ss, 3 * c0, 3 * (c1 - c0)).reshape(-1, 3)
        comp = np.searchsorted(cw, unit_double(x[:, 0]), side="right").clip(0, 2)
        u1 = 1.0 - unit_double(x[:, 1])          # (0, 1]
        u2 = unit_double(x[:, 2])
        g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        z = mu[comp] + sg[comp] * g
        v = np.floor(np.exp(np.minimum(z, 23.0)))
        out[c0:c1] = np.minimum(v, 4294967295.0).astype(np.uint32)
    return out


def segment_lengths(nseg: int, seed: int, max_len: int = 65536) -> np.ndarray:
    u = unit_double(splitmix64(stream_seed(seed, DIST_SEGLENS), 0, nseg))
    L = np.floor(np.exp(u * math.log(max_len + 1)))
    return np.clip(L, 1, max_len).astype(np.int64)


def segment_offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    np.cumsum(lengths, out=off[1:])
    return off


def poisson_requests(count: int, seed: int, rate_per_s: float,
                     lo: int = 1 << 10, hi: int = 1 << 24):
    """(arrival times in s, sizes) for a Poisson stream of sort requests."""
    x = splitmix64(stream_seed(seed, DIST_REQUESTS), 0, 2 * count).reshape(-1, 2)
    gaps = -np.log(1.0 - unit_double(x[:, 0])) / rate_per_s
    t = np.cumsum(gaps)
    sizes = np.exp(math.log(lo) + unit_double(x[:, 1]) * (math.log(hi) - math.log(lo)))
    sizes = np.clip(np.floor(sizes), lo, hi).astype(np.int64)
    return t, sizes

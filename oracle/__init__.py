"""CPU oracle for the merge sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The GPU library (``paper_2211_16479_gb300``)
never imports it and shares no code with it.

``msort_oracle.c`` holds the plain top-down merge sort of Section "Sequential
Merge Sort" (Fig. 2, split fixed to ``right = array[mid:]``), the two-way merge
that takes from the left run on ties, the co-rank by running that merge, the
multiprocessing/merge-tree variant (Figs. 6-7 and 16-17) and the segmented
sort.  ``mlp.py`` holds the fp64 reference of the small CDF network used by
the learned partitioner.  This module compiles the C file with gcc and wraps
it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msort_oracle.c")
_LOCK = threading.Lock()
_LIBS: dict = {}


def lib_path(mutant: int = 0, outdir: str | None = None) -> str:
    outdir = outdir or os.path.join(_HERE, "_build")
    return os.path.join(outdir, f"liboracle_m{mutant}.so")


def build(mutant: int = 0, outdir: str | None = None, force: bool = False) -> str:
    """Compile the oracle (optionally with a planted mistake) and return the .so path."""
    path = lib_path(mutant, outdir)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-Wall", "-fPIC", "-shared", "-pthread",
               f"-DORACLE_MUTANT={int(mutant)}", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return path


_P = ctypes.c_void_p
_SZ = ctypes.c_size_t


def _bind(lib):
    for suf in _SUFFIXES.values():
        f = getattr(lib, f"oracle_sort_{suf}")
        f.argtypes, f.restype = [_P, _P, _SZ], ctypes.c_int
        f = getattr(lib, f"oracle_par_sort_{suf}")
        f.argtypes, f.restype = [_P, _P, _SZ, ctypes.c_int], ctypes.c_int
        f = getattr(lib, f"oracle_merge_{suf}")
        f.argtypes, f.restype = [_P, _P, _SZ, _P, _P, _SZ, _P, _P], None
        f = getattr(lib, f"oracle_corank_{suf}")
        f.argtypes, f.restype = [_P, _SZ, _P, _SZ, _SZ], ctypes.c_int64
        f = getattr(lib, f"oracle_segmented_sort_{suf}")
        f.argtypes, f.restype = [_P, _P, _P, _SZ], ctypes.c_int
    lib.oracle_mutant_id.restype = ctypes.c_int
    return lib


def load(mutant: int = 0, outdir: str | None = None):
    key = (mutant, outdir)
    with _LOCK:
        if key not in _LIBS:
            _LIBS[key] = _bind(ctypes.CDLL(build(mutant, outdir)))
        return _LIBS[key]


# Key dtypes and the oracle's order for each: unsigned and signed integers
# by value, floating point by IEEE 754 totalOrder on the bit patterns.
_SUFFIXES = {np.dtype(np.uint32): "u32", np.dtype(np.uint64): "u64", np.dtype(np.int32): "i32",
             np.dtype(np.int64): "i64", np.dtype(np.float32): "f32", np.dtype(np.float64): "f64"}


def _suffix(keys: np.ndarray) -> str:
    try:
        return _SUFFIXES[keys.dtype]
    except KeyError:
        raise TypeError(f"oracle keys must be 32/64-bit unsigned, signed or float, got {keys.dtype}") from None


def _ptr(a):
    return None if a is None else a.ctypes.data


def sort(keys: np.ndarray, vals: np.ndarray | None = None, lib=None):
    """Stable sort; returns new (keys, vals) arrays (vals None for keys only)."""
    lib = lib or load()
    k = np.ascontiguousarray(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    if v is not None and len(v) != len(k):
        raise ValueError("keys and vals differ in length")
    rc = getattr(lib, f"oracle_sort_{_suffix(k)}")(_ptr(k), _ptr(v), len(k))
    if rc:
        raise MemoryError("oracle sort could not allocate its temporary")
    return k, v


def par_sort(keys: np.ndarray, vals: np.ndarray | None = None, workers: int = 1, lib=None):
    lib = lib or load()
    k = np.ascontiguousarray(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    rc = getattr(lib, f"oracle_par_sort_{_suffix(k)}")(_ptr(k), _ptr(v), len(k), int(workers))
    if rc:
        raise MemoryError("oracle parallel sort could not allocate")
    return k, v


def sort_inplace(keys: np.ndarray, vals: np.ndarray | None = None, workers: int = 1, lib=None):
    """Sort contiguous arrays in place (used to time the oracle without copies)."""
    lib = lib or load()
    assert keys.flags.c_contiguous and (vals is None or vals.flags.c_contiguous)
    if workers > 1:
        rc = getattr(lib, f"oracle_par_sort_{_suffix(keys)}")(_ptr(keys), _ptr(vals), len(keys), int(workers))
    else:
        rc = getattr(lib, f"oracle_sort_{_suffix(keys)}")(_ptr(keys), _ptr(vals), len(keys))
    if rc:
        raise MemoryError("oracle sort could not allocate")


def merge(ak, bk, av=None, bv=None, lib=None):
    lib = lib or load()
    ak = np.ascontiguousarray(ak)
    bk = np.ascontiguousarray(bk, dtype=ak.dtype)
    ok = np.empty(len(ak) + len(bk), dtype=ak.dtype)
    ov = None
    if av is not None:
        av = np.ascontiguousarray(av, dtype=np.uint32)
        bv = np.ascontiguousarray(bv, dtype=np.uint32)
        ov = np.empty(len(ok), dtype=np.uint32)
    getattr(lib, f"oracle_merge_{_suffix(ak)}")(_ptr(ak), _ptr(av), len(ak), _ptr(bk), _ptr(bv),
                                                 len(bk), _ptr(ok), _ptr(ov))
    return ok, ov


def corank(a, b, d: int, lib=None) -> int:
    """Number of elements of A among the first d outputs of merge(A, B)."""
    lib = lib or load()
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b, dtype=a.dtype)
    r = getattr(lib, f"oracle_corank_{_suffix(a)}")(_ptr(a), len(a), _ptr(b), len(b), int(d))
    if r < 0:
        raise ValueError("diagonal beyond |A| + |B|")
    return int(r)


def split_points(keys, positions, split_keys, split_pos):
    """For each splitter (split_keys[t], split_pos[t]): how many elements
    come before it when elements are ordered by (key, global position), a
    total order.  Written as the plain count over the (unsorted) elements,
    the partition step of the one-exchange form of Section "MPI Merge Sort"'s
    scatter-sort-merge (each rank keeps the slice between two splitters).
    Unsigned or signed integer keys."""
    keys = np.asarray(keys)
    positions = np.asarray(positions, dtype=np.uint64)
    out = np.empty(len(split_keys), dtype=np.uint64)
    for t, (sk, sp) in enumerate(zip(np.asarray(split_keys, dtype=keys.dtype),
                                     np.asarray(split_pos, dtype=np.uint64))):
        out[t] = np.count_nonzero((keys < sk) | ((keys == sk) & (positions < sp)))
    return out


def segmented_sort(keys, offsets, vals=None, lib=None):
    lib = lib or load()
    k = np.ascontiguousarray(keys).copy()
    v = None if vals is None else np.ascontiguousarray(vals, dtype=np.uint32).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = getattr(lib, f"oracle_segmented_sort_{_suffix(k)}")(_ptr(k), _ptr(v), _ptr(off), len(off) - 1)
    if rc:
        raise ValueError(f"oracle segmented sort failed ({rc})")
    return k, v

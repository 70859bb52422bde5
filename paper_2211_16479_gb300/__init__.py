"""Python binding of libmsort (stable GPU merge sort for GB300 / sm_103a).

Every function here marshals arguments and calls the C ABI declared in
``include/msort.h`` under the same name; all sorting runs in the library's
CUDA kernels.  Tensors supply device pointers, ``torch.cuda`` supplies the
current stream; there is no CPU code path.  If ``libmsort.so`` has not been
built, importing the library raises ``ImportError`` instead of falling back.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmsort.so")

MSORT_OK, MSORT_ERR_INVALID_ARG, MSORT_ERR_UNSUPPORTED, MSORT_ERR_OOM = 0, 1, 2, 3
MSORT_ERR_CUDA, MSORT_ERR_TIMEOUT, MSORT_ERR_BUSY = 4, 5, 6
MSORT_U32, MSORT_U64, MSORT_I32, MSORT_I64, MSORT_F32, MSORT_F64 = 0, 1, 2, 3, 4, 5
MSORT_KERNEL_TILE, MSORT_KERNEL_PARTITION, MSORT_KERNEL_MERGE = 0, 1, 2
MSORT_KERNEL_SEGMENTED, MSORT_KERNEL_MLP, MSORT_KERNEL_SINGLE = 3, 4, 5
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "BUSY"}


class MsortError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"msort {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class msort_options(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("merge_block", ctypes.c_int), ("partition_mode", ctypes.c_int),
                ("learned_passes", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("merge_ways", ctypes.c_int), ("single_launch", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


_P, _SZ, _I, _ST = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int
_OPT = ctypes.POINTER(msort_options)


class msort_server_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("queued", ctypes.c_uint64), ("inflight", ctypes.c_uint64),
                ("max_inflight", ctypes.c_uint64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("keys_per_s", ctypes.c_double),
                ("arena_high_water", ctypes.c_uint64), ("budget", ctypes.c_uint64)]

_SIGS = {
    "msort_ctx_create": ([_I, _SZ, ctypes.POINTER(_P)], _ST),
    "msort_ctx_destroy": ([_P], _ST),
    "msort_last_error": ([_P], ctypes.c_char_p),
    "msort_ctx_sync": ([_P, _P], _ST),
    "msort_scratch_bytes": ([_SZ, _I, _I, _OPT], _SZ),
    "msort_plan_info": ([_SZ, _I, _I, _OPT, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)], _ST),
    "msort_plan_passes": ([_SZ, _I, _I, _OPT, ctypes.POINTER(_I), ctypes.POINTER(_I)], _ST),
    "msort_sort": ([_P, _P, _SZ, _I, _OPT, _P], _ST),
    "msort_sort_pairs": ([_P, _P, _P, _SZ, _I, _OPT, _P], _ST),
    "msort_sort_copy": ([_P, _P, _P, _P, _P, _SZ, _I, _OPT, _P], _ST),
    "msort_sort_host": ([_P, _P, _P, _P, _P, _SZ, _I, _OPT, _P], _ST),
    "msort_sort_host_async": ([_P, _P, _P, _P, _P, _SZ, _I, _OPT, _P], _ST),
    "msort_merge": ([_P, _P, _P, _SZ, _P, _P, _SZ, _P, _P, _I, _P], _ST),
    "msort_merge_runs": ([_P, _P, _P, _P, _SZ, _P, _P, _I, _P], _ST),
    "msort_external_plan": ([_P, _SZ, _I, _SZ, _SZ, _P, _SZ], _SZ),
    "msort_split_points": ([_P, _P, _P, _SZ, ctypes.c_uint64, _P, _P, _SZ, _P, _I, _P], _ST),
    "msort_segmented_sort": ([_P, _P, _P, _P, _SZ, _SZ, _I, _OPT, _P], _ST),
    "msort_sort_noalloc": ([_P, _P, _P, _P, _SZ, _I, _P], _ST),
    "msort_noalloc_max_keys": ([_I, _I], _SZ),
    "msort_noalloc_sync": ([_P], _ST),
    "msort_selftest_wait_timeout": ([_P, ctypes.c_longlong, _P], _ST),
    "msort_selftest_grid_timeout": ([_P, _P, _SZ, ctypes.c_longlong, _P], _ST),
    "msort_tune": ([_P, ctypes.c_char_p, _I], _ST),
    "msort_tune_load": ([_P, ctypes.c_char_p], _ST),
    "msort_tune_clear": ([_P], _ST),
    "msort_mlp_grad": ([_P, _P, _SZ, _P, _P, _P], _ST),
    "msort_mlp_train": ([_P, _P, _SZ, _P, _I, _I, ctypes.c_float, _P], _ST),
    "msort_learned_model": ([_P, _P, _P], _ST),
    "msort_learned_set_model": ([_P, _P, ctypes.c_float], _ST),
    "msort_ctx_partition_stats": ([_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)], _ST),
    "msort_partition_splits": ([_P, _P, _SZ, _SZ, _SZ, _I, _P, _I, _P], _ST),
    "msort_server_create": ([_I, _SZ, _I, ctypes.POINTER(_P)], _ST),
    "msort_server_submit": ([_P, _P, _P, _SZ, _I, ctypes.POINTER(ctypes.c_uint64)], _ST),
    "msort_server_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)], _ST),
    "msort_server_wait": ([_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], _ST),
    "msort_server_get_stats": ([_P, ctypes.POINTER(msort_server_stats)], _ST),
    "msort_server_reset_stats": ([_P], _ST),
    "msort_server_destroy": ([_P], _ST),
    "msort_ctx_set_profiling": ([_P, _I], _ST),
    "msort_ctx_kernel_times": ([_P, _I, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)], _ST),
    "msort_ctx_launch_count": ([_P], ctypes.c_ulonglong),
    "msort_ctx_kernel_log": ([_P, _I, _P, _SZ, ctypes.POINTER(ctypes.c_uint64)], _ST),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libmsort.so (raises ImportError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_2211_16479_gb300._build.build() first")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.argtypes, fn.restype = args, res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors passed to msort must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy array (host)
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


_KEY_TYPES = {"uint32": MSORT_U32, "uint64": MSORT_U64, "int32": MSORT_I32, "int64": MSORT_I64,
              "float32": MSORT_F32, "float64": MSORT_F64}


def _key_type(x, key_type):
    """Key type from the dtype: unsigned, signed (two's complement order) or
    floating point (IEEE totalOrder); key_type overrides it."""
    if key_type is not None:
        return int(key_type)
    name = str(getattr(x, "dtype", "")).replace("torch.", "")
    if name in _KEY_TYPES:
        return _KEY_TYPES[name]
    raise TypeError(f"key dtype {name!r} is not a 32/64-bit integer or float; pass key_type explicitly")


def _numel(x, n):
    if n is not None:
        return int(n)
    if hasattr(x, "numel"):
        return int(x.numel())
    if hasattr(x, "size") and not callable(x.size):
        return int(x.size)
    raise ValueError("n is required for raw pointers")


def _stream(stream, like=None):
    if stream is None:
        import torch
        dev = like.device if like is not None and hasattr(like, "device") and like.device.type == "cuda" else None
        return torch.cuda.current_stream(dev).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(options):
    if options is None:
        return None
    if isinstance(options, msort_options):
        return ctypes.byref(options)
    o = msort_options()
    for k, v in dict(options).items():
        setattr(o, k, int(v))
    return ctypes.byref(o)


def _check(ctx, status):
    if status != MSORT_OK:
        msg = load_library().msort_last_error(ctx)
        raise MsortError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C ABI, same names
# ---------------------------------------------------------------------------
def msort_ctx_create(device: int = 0, scratch_budget_bytes: int = 0):
    out = ctypes.c_void_p()
    _check(None, load_library().msort_ctx_create(int(device), int(scratch_budget_bytes), ctypes.byref(out)))
    return out


def msort_ctx_destroy(ctx) -> None:
    _check(ctx, load_library().msort_ctx_destroy(ctx))


def msort_last_error(ctx) -> str:
    r = load_library().msort_last_error(ctx)
    return r.decode() if r else ""


def msort_ctx_sync(ctx, stream=None) -> None:
    _check(ctx, load_library().msort_ctx_sync(ctx, _stream(stream)))


def msort_scratch_bytes(n: int, key_type: int, with_vals: bool, options=None) -> int:
    return int(load_library().msort_scratch_bytes(int(n), int(key_type), int(bool(with_vals)), _opts(options)))


def msort_plan_passes(n: int, key_type: int, with_vals: bool, options=None):
    """(ways, memory_passes): merge rounds per pass over memory (2 or 4) and
    the number of merge passes over memory the plan makes."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(None, load_library().msort_plan_passes(int(n), int(key_type), int(bool(with_vals)), _opts(options),
                                                  ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def msort_plan_info(n: int, key_type: int, with_vals: bool, options=None):
    """(tile, merge_block, passes) of the plan a sort of n elements uses."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(None, load_library().msort_plan_info(int(n), int(key_type), int(bool(with_vals)), _opts(options),
                                                ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def msort_sort(ctx, keys, n=None, key_type=None, options=None, stream=None) -> None:
    _check(ctx, load_library().msort_sort(ctx, _ptr(keys), _numel(keys, n), _key_type(keys, key_type),
                                          _opts(options), _stream(stream, keys)))


def msort_sort_pairs(ctx, keys, vals, n=None, key_type=None, options=None, stream=None) -> None:
    _check(ctx, load_library().msort_sort_pairs(ctx, _ptr(keys), _ptr(vals), _numel(keys, n),
                                                _key_type(keys, key_type), _opts(options), _stream(stream, keys)))


def msort_sort_copy(ctx, keys_in, keys_out, vals_in=None, vals_out=None, n=None, key_type=None,
                    options=None, stream=None) -> None:
    _check(ctx, load_library().msort_sort_copy(ctx, _ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                               _numel(keys_in, n), _key_type(keys_in, key_type), _opts(options),
                                               _stream(stream, keys_in)))


def msort_segmented_sort(ctx, keys, offsets, vals=None, nseg=None, n=None, key_type=None, options=None,
                         stream=None) -> None:
    """Sort every segment [offsets[i], offsets[i+1]) of keys (and vals) in
    place; offsets is a device uint64/int64 tensor of nseg + 1 entries."""
    nseg = int(offsets.numel()) - 1 if nseg is None else int(nseg)
    _check(ctx, load_library().msort_segmented_sort(ctx, _ptr(keys), _ptr(vals), _ptr(offsets), nseg,
                                                    _numel(keys, n), _key_type(keys, key_type), _opts(options),
                                                    _stream(stream, keys)))


def msort_merge(ctx, a, b, out, va=None, vb=None, vout=None, key_type=None, stream=None) -> None:
    """out = stable merge of sorted a and b (ties from a first)."""
    _check(ctx, load_library().msort_merge(ctx, _ptr(a), _ptr(va), _numel(a, None), _ptr(b), _ptr(vb),
                                           _numel(b, None), _ptr(out), _ptr(vout), _key_type(a, key_type),
                                           _stream(stream, out)))


def msort_merge_runs(ctx, keys, offsets, out, vals=None, out_vals=None, key_type=None, stream=None) -> None:
    """out = stable merge of the sorted runs keys[offsets[i]:offsets[i+1]]
    laid end to end (ties in run order); offsets: host sequence of
    nruns + 1 counts starting at 0."""
    import numpy as np
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    _check(ctx, load_library().msort_merge_runs(ctx, _ptr(keys), _ptr(vals), offs.ctypes.data, max(len(offs) - 1, 0),
                                                _ptr(out), _ptr(out_vals), _key_type(keys, key_type),
                                                _stream(stream, out)))


def msort_split_points(ctx, keys, idx, offset: int, split_keys, split_pos, cuts, key_type=None,
                       stream=None) -> None:
    """cuts[t] = number of elements of the sorted chunk (keys, local indices
    idx, global position offset + idx) ordered before the splitter
    (split_keys[t], split_pos[t]) in (key, position) order; all device
    tensors, cuts and split_pos 64-bit."""
    _check(ctx, load_library().msort_split_points(ctx, _ptr(keys), _ptr(idx), _numel(keys, None), int(offset),
                                                  _ptr(split_keys), _ptr(split_pos), _numel(split_keys, None),
                                                  _ptr(cuts), _key_type(keys, key_type), _stream(stream, keys)))


def msort_external_plan(runs, chunk: int, block_max: int):
    """Blocks of the out-of-core sort for sorted runs of `chunk` keys laid
    end to end in the host array `runs` (uint32 or uint64): returns the
    (blocks + 1) x runs array of cut positions (see include/msort.h)."""
    import numpy as np
    runs = np.ascontiguousarray(runs)
    kt = _key_type(runs, None)
    lib = load_library()
    nb = lib.msort_external_plan(runs.ctypes.data, runs.size, kt, chunk, block_max, None, 0)
    if nb == 0:
        raise ValueError("invalid arguments to msort_external_plan")
    nruns = -(-runs.size // chunk)
    cuts = np.zeros((nb + 1) * nruns, dtype=np.uint64)
    lib.msort_external_plan(runs.ctypes.data, runs.size, kt, chunk, block_max, cuts.ctypes.data, cuts.size)
    return cuts.reshape(nb + 1, nruns)


def msort_sort_host(ctx, keys, vals=None, out_keys=None, out_vals=None, n=None, key_type=None,
                    options=None, stream=None) -> None:
    """Sort host buffers (numpy arrays or CPU tensors; pinned is fastest).
    The result goes to out_keys/out_vals, or back into keys/vals."""
    if out_keys is None:
        out_keys, out_vals = keys, vals
    _check(ctx, load_library().msort_sort_host(ctx, _ptr(keys), _ptr(vals), _ptr(out_keys), _ptr(out_vals),
                                               _numel(keys, n), _key_type(keys, key_type), _opts(options),
                                               _stream(stream)))


def msort_sort_host_async(ctx, keys, vals=None, out_keys=None, out_vals=None, n=None, key_type=None,
                          options=None, stream=None) -> None:
    """Enqueue a host-buffer sort and return; the result is in out_keys
    (out_vals) once `stream` completes (torch stream .synchronize() or
    msort_ctx_sync).  Keep the host buffers alive and the input unchanged
    until then."""
    if out_keys is None:
        out_keys, out_vals = keys, vals
    _check(ctx, load_library().msort_sort_host_async(ctx, _ptr(keys), _ptr(vals), _ptr(out_keys), _ptr(out_vals),
                                                     _numel(keys, n), _key_type(keys, key_type), _opts(options),
                                                     _stream(stream)))


def msort_sort_noalloc(keys_in, keys_out, vals_in=None, vals_out=None, n=None, key_type=None,
                       stream=None) -> None:
    """Stable sort without any device allocation (scratch is a fixed array
    inside the library; see msort_sort_noalloc in include/msort.h).  Calls
    that overlap on the GPU race on that array: keep them on one stream."""
    _check(None, load_library().msort_sort_noalloc(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                                   _numel(keys_in, n), _key_type(keys_in, key_type),
                                                   _stream(stream, keys_in)))


def msort_noalloc_sync(stream=None) -> None:
    """Wait for `stream` and raise if the last msort_sort_noalloc call's
    kernels recorded an error (a bounded wait that gave up)."""
    _check(None, load_library().msort_noalloc_sync(_stream(stream)))


def msort_noalloc_max_keys(key_type: int, with_vals: bool) -> int:
    return int(load_library().msort_noalloc_max_keys(int(key_type), int(bool(with_vals))))


def msort_selftest_wait_timeout(ctx, limit_cycles: int = 100000, stream=None) -> None:
    """Enqueue the bounded-wait self-test: one merge block that gives up its
    wait after limit_cycles; the next msort_ctx_sync raises TIMEOUT."""
    _check(ctx, load_library().msort_selftest_wait_timeout(ctx, int(limit_cycles), _stream(stream)))


def msort_selftest_grid_timeout(ctx, keys, limit_cycles: int = 100000, n=None, stream=None) -> None:
    """Enqueue the grid-barrier self-test of the single-launch sort on the
    uint32 device tensor `keys` (left unordered); the next msort_ctx_sync
    raises TIMEOUT."""
    _check(ctx, load_library().msort_selftest_grid_timeout(ctx, _ptr(keys), _numel(keys, n), int(limit_cycles),
                                                           _stream(stream, keys)))


def msort_tune(ctx, cache_path=None, quick: bool = False) -> None:
    _check(ctx, load_library().msort_tune(ctx, cache_path.encode() if cache_path else None, int(bool(quick))))


def msort_tune_load(ctx, cache_path: str) -> None:
    _check(ctx, load_library().msort_tune_load(ctx, cache_path.encode()))


def msort_tune_clear(ctx) -> None:
    _check(ctx, load_library().msort_tune_clear(ctx))


def msort_mlp_grad(ctx, x, params, grad, m=None, stream=None) -> None:
    _check(ctx, load_library().msort_mlp_grad(ctx, _ptr(x), _numel(x, m), _ptr(params), _ptr(grad),
                                              _stream(stream, x)))


def msort_mlp_train(ctx, x, params, steps: int, lr: float = 1e-3, knot_init: bool = False, m=None,
                    stream=None) -> None:
    _check(ctx, load_library().msort_mlp_train(ctx, _ptr(x), _numel(x, m), _ptr(params), int(bool(knot_init)),
                                               int(steps), float(lr), _stream(stream, x)))


def msort_learned_model(ctx):
    """(97 parameters as a list, max sample error) of the last trained model."""
    p = (ctypes.c_float * 97)()
    e = ctypes.c_float()
    _check(ctx, load_library().msort_learned_model(ctx, p, ctypes.byref(e)))
    return list(p), float(e.value)


def msort_learned_set_model(ctx, params, err: float = 0.0) -> None:
    """Install a fixed model (sequence of 97 floats) for partition_mode 1, or
    None to go back to training per sort."""
    if params is None:
        _check(ctx, load_library().msort_learned_set_model(ctx, None, 0.0))
        return
    arr = (ctypes.c_float * 97)(*[float(v) for v in params])
    _check(ctx, load_library().msort_learned_set_model(ctx, arr, float(err)))


def msort_partition_splits(ctx, keys, run_length: int, block: int, mode: int, splits, key_type=None,
                           stream=None) -> None:
    """splits[c] = co-rank of output block c of the pairwise merge of the
    sorted runs of run_length keys in `keys` (mode 0 exact, 1 learned, 2
    ratio guess, 3 counted exact); splits: int64/uint64 device tensor of
    ceil(n / block) entries."""
    _check(ctx, load_library().msort_partition_splits(ctx, _ptr(keys), _numel(keys, None), int(run_length),
                                                      int(block), int(mode), _ptr(splits), _key_type(keys, key_type),
                                                      _stream(stream, keys)))


def msort_ctx_partition_stats(ctx):
    """(probes, searches) counted by guided partitions while profiling."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, load_library().msort_ctx_partition_stats(ctx, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def msort_ctx_set_profiling(ctx, on) -> None:
    """on: 0 off, 1 (or True) CUDA events around every launch, 2 events and
    probe counting in guided partitions."""
    _check(ctx, load_library().msort_ctx_set_profiling(ctx, int(on)))


def msort_ctx_kernel_times(ctx, kind: int):
    """(launches, total milliseconds) of the kernels of `kind` logged since the last call."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(ctx, load_library().msort_ctx_kernel_times(ctx, int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def msort_ctx_kernel_log(ctx, kind: int, cap: int = 4096):
    """Device milliseconds of each logged launch of `kind`, in launch order
    (at most cap of them); clears that log."""
    buf = (ctypes.c_double * max(int(cap), 1))()
    n = ctypes.c_uint64()
    _check(ctx, load_library().msort_ctx_kernel_log(ctx, int(kind), buf, int(cap), ctypes.byref(n)))
    return [float(buf[i]) for i in range(min(int(n.value), int(cap)))]


def msort_ctx_launch_count(ctx) -> int:
    return int(load_library().msort_ctx_launch_count(ctx))


def msort_server_create(device: int = 0, mem_budget_bytes: int = 8 << 30, max_slots: int = 8):
    out = ctypes.c_void_p()
    _check(None, load_library().msort_server_create(int(device), int(mem_budget_bytes), int(max_slots),
                                                    ctypes.byref(out)))
    return out


def msort_server_submit(server, keys, vals=None, n=None, key_type=None) -> int:
    rid = ctypes.c_uint64()
    _check(None, load_library().msort_server_submit(server, _ptr(keys), _ptr(vals), _numel(keys, n),
                                                    _key_type(keys, key_type), ctypes.byref(rid)))
    return int(rid.value)


def msort_server_poll(server, req_id: int):
    """(done, latency_ms)."""
    done = ctypes.c_int()
    lat = ctypes.c_double()
    _check(None, load_library().msort_server_poll(server, int(req_id), ctypes.byref(done), ctypes.byref(lat)))
    return bool(done.value), float(lat.value)


def msort_server_wait(server, req_id: int, timeout_ms: float = 60000.0) -> float:
    lat = ctypes.c_double()
    _check(None, load_library().msort_server_wait(server, int(req_id), float(timeout_ms), ctypes.byref(lat)))
    return float(lat.value)


def msort_server_get_stats(server) -> dict:
    st = msort_server_stats()
    _check(None, load_library().msort_server_get_stats(server, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in st._fields_}


def msort_server_reset_stats(server) -> None:
    _check(None, load_library().msort_server_reset_stats(server))


def msort_server_destroy(server) -> None:
    _check(None, load_library().msort_server_destroy(server))


class Server:
    """Owns a msort serving loop; usable as a context manager."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 8 << 30, max_slots: int = 8):
        self.handle = msort_server_create(device, mem_budget_bytes, max_slots)

    def submit(self, keys, vals=None) -> int:
        return msort_server_submit(self.handle, keys, vals)

    def wait(self, req_id: int, timeout_ms: float = 60000.0) -> float:
        return msort_server_wait(self.handle, req_id, timeout_ms)

    def stats(self) -> dict:
        return msort_server_get_stats(self.handle)

    def close(self):
        if self.handle is not None and self.handle.value:
            msort_server_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Context:
    """Owns a msort context; usable as a context manager."""

    def __init__(self, device: int = 0, scratch_budget_bytes: int = 0):
        self.handle = msort_ctx_create(device, scratch_budget_bytes)

    def close(self):
        if self.handle is not None and self.handle.value:
            msort_ctx_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Benchmark: stable GPU merge sort of 2^28 uint32 keys under five distributions.

One step = one out-of-place sort of each of the five 2^28-key arrays
(uniform, already sorted, reverse sorted, 16 distinct values, Zipf(1.1) over
2^20 ranks), keys only: the tile sort plus R = ceil(log2(2^28 / T)) rounds of
the merge tree, one pairwise merge pass per round (--merge-ways 4 merges two
rounds per pass instead), all in the library's kernels.  value = keys sorted per second (Gkeys/s) over
the timed steps, inputs resident in HBM.  Each input is 1 GiB, larger than
the 126 MB L2, so no L2 flush is needed between steps.

Printed as one JSON line on rank 0.  Also reported:
  e2e           the same sorts through the host-buffer API: pinned host keys
                in, host keys out, every copy inside the timed region; a
                step enqueues the five sorts with msort_sort_host_async; the
                timed region (the same number of steps as the value) ends
                when the last step's results are in host memory
                (sync_call_value: msort_sort_host, one sort at a time); both
                are the median of --e2e-reps repetitions, all reported,
                since the host link is shared with the machine's other work;
  roofline      the merge pass (the dominant kernel; one read and one write
                of every key per launch) against measured HBM copy
                bandwidth, its duration from CUDA events on its stream,
                taken in a second timed region of K steps with an event pair
                around every launch (value comes from the first region,
                without those events, the sorts replayed from CUDA graphs);
  cpu_baseline  the CPU oracle (chunked merge sort with a pairwise merge tree
                on every host core) on a bounded sample of the same inputs;
  clocks        nvidia-smi samples taken during the timed region;
  chosen_vs_plain  the forms the method was extended with, each against the
                plain sort on identical inputs in interleaved repetitions, with
                identical output checked on the device: the learned partition
                (2^30 lognormal-mixture keys; the model-free ratio start as the
                ablation), the batched segmented sort (50,000 arrays) and the
                continuous-batching server (2,000 requests; p50/p99);
  small_config  the 2^20-key configuration (L2-resident): the single
                cooperative launch against the multi-launch plan;
  pairs_config  the key-value configuration: a stable sort of 2^27 (uint64
                key, uint32 original index) pairs with heavy duplicates, its
                stability checked on the device.

--impl reference times the CPU oracle itself on the same metric (there is no
GPU reference implementation of this method).
Multi-GPU (torchrun): every rank sorts its own copy of the workload
(replicas; the sort has no cross-GPU exchange), value = all ranks' keys /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 28
DISTS = ("uniform", "sorted", "reverse", "distinct16", "zipf")
METRIC = "Gkeys/s sorted (stable merge sort, 2^28 uint32 keys x 5 distributions)"
UNIT = "Gkeys/s"
NOMINAL_HBM_GBS = 8000.0


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("paper_2211_16479_gb300/csrc/sort_kernels.cuh", "paper_2211_16479_gb300/csrc/merge4.cuh")


def _code_only(src: str) -> str:
    """C++ source with comments and whitespace removed."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "".join(src.split())


def _kernel_source_hash(read=None):
    """16 hex digits of sha256 over the sort kernels' code (comments and
    whitespace removed): a comment edit keeps recorded counters valid, a
    code edit invalidates them.  read(rel) -> text overrides the files."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, rel)) as f:
                text = f.read()
        else:
            text = read(rel)
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel="k_merge4_pass"):
    """dram bytes per merge-pass launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_u32_2p28.txt")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("kernel_source_sha256_16") != _kernel_source_hash():
            return None
        return float(fields["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir: str | None = None):
        import tempfile
        self.proc = None
        self.path = os.path.join(out_dir or tempfile.gettempdir(), f"msort_clocks_gpu{gpu_index}_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx = max(mx, float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _multiset_hash(t):
    """Order-independent hash of a device key array: the sum of a 64-bit
    mix of every key (wrapping), computed on the device."""
    import torch
    x = t.to(torch.int64) if t.dtype in (torch.uint32, torch.int32) else t.view(torch.int64)
    x = x * -4658895280553007687 ^ (x >> 29 & 0x7FFFFFFFF)  # 0xBF58476D1CE4E5B9 as int64
    x = x * -7723592293110705685  # 0x94D049BB133111EB as int64
    return int(x.sum().item())


def cpu_oracle_rate(sample_keys, seconds_target=12.0):
    """Time the oracle's chunked merge sort on all host cores; returns
    (Gkeys/s, cores, description)."""
    import numpy as np

    import oracle
    cores = len(os.sched_getaffinity(0))
    lib = oracle.load()
    total_keys, total_t, reps = 0, 0.0, 0
    while total_t < seconds_target or reps < 1:
        for a in sample_keys:
            work = np.array(a, copy=True)
            t0 = time.perf_counter()
            oracle.sort_inplace(work, None, workers=cores, lib=lib)
            total_t += time.perf_counter() - t0
            total_keys += len(a)
        reps += 1
        if reps >= 400:
            break
    return total_keys / total_t / 1e9, cores, reps


def cpu_context_rates(sample_keys):
    """Context for the CPU baseline on the same sample (one pass each): the
    oracle's merge sort on one core (the paper's sequential merge sort) and
    numpy's stable sort (a library routine; a radix sort for integers)."""
    import numpy as np

    import oracle
    lib = oracle.load()
    n = sum(len(a) for a in sample_keys)
    t0 = time.perf_counter()
    for a in sample_keys:
        work = np.array(a, copy=True)
        oracle.sort_inplace(work, None, workers=1, lib=lib)
    t1 = time.perf_counter()
    for a in sample_keys:
        np.sort(a, kind="stable")
    t2 = time.perf_counter()
    return {"oracle_one_core_gkeys": n / (t1 - t0) / 1e9, "numpy_stable_sort_gkeys": n / (t2 - t1) / 1e9}


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import synth
    m = 1 << 22
    samples = [synth.u32_distribution(d, m, 1) for d in DISTS]
    cores = len(os.sched_getaffinity(0))
    import oracle
    lib = oracle.load()
    for _ in range(args.warmup):  # untimed warm-up steps
        for a in samples:
            oracle.sort_inplace(np.array(a, copy=True), None, workers=cores, lib=lib)
    t_total, keys = 0.0, 0
    for _ in range(args.steps):
        for a in samples:
            w = np.array(a, copy=True)
            t0 = time.perf_counter()
            oracle.sort_inplace(w, None, workers=cores, lib=lib)
            t_total += time.perf_counter() - t0
            keys += m
    v = keys / t_total / 1e9
    sample = f"first 2^22 keys of each of the 5 distributions (1/64 of the 2^28 arrays), per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded SplitMix64 recipes)",
            "config": {"workload": "2^28 uint32 keys x 5 distributions, keys only, stable sort (sampled)",
                       "n": N, "distributions": list(DISTS)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen

    rank, world, local = _dist_env()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    opts = {"tile": args.tile, "merge_block": args.merge_block, "merge_ways": args.merge_ways,
            "use_graph": args.graph}  # graph replay is skipped while launches are profiled
    T, W, passes = ms.msort_plan_info(n, ms.MSORT_U32, False, opts)
    ways, mem_passes = ms.msort_plan_passes(n, ms.MSORT_U32, False, opts)
    merge_kernel = "k_merge4_pass" if ways == 4 else "k_merge_pass"

    inputs = [torch_gen.u32_distribution(d, n, 1, device=dev) for d in DISTS]
    out = torch.empty_like(inputs[0])
    torch.cuda.synchronize()
    ctx = ms.Context(local)
    h = ctx.handle
    stream = torch.cuda.current_stream(dev)

    def step():
        for a in inputs:
            ms.msort_sort_copy(h, a, out, options=opts, stream=stream)

    def barrier():
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    # correctness guard on the last warm-up output: sorted, and the same
    # multiset of keys as its input
    last = out.to(torch.int64)
    assert bool((last[1:] >= last[:-1]).all()), "output not sorted"
    assert _multiset_hash(out) == _multiset_hash(inputs[-1]), "output is not a permutation of the input"
    del last

    def timed(profiled):
        # K steps bracketed by a barrier and a device synchronisation, CUDA
        # events on the launching stream
        ms.msort_ctx_set_profiling(h, profiled)
        launches0 = ms.msort_ctx_launch_count(h)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
        kt = {k: ms.msort_ctx_kernel_times(h, k) for k in
              (ms.MSORT_KERNEL_TILE, ms.MSORT_KERNEL_PARTITION, ms.MSORT_KERNEL_MERGE)} if profiled else None
        ms.msort_ctx_set_profiling(h, False)
        return e0.elapsed_time(e1), ms.msort_ctx_launch_count(h) - launches0, kt

    # Timed region 1 (the value): the sorts alone, replayed from CUDA graphs
    # unless --graph 0.  Timed region 2 (the roofline): the same steps with
    # a CUDA event pair around every launch, which adds host work between
    # launches (the kernels themselves are unchanged).
    sampler = ClockSampler(local)
    sampler.start()
    elapsed_ms, launches, _ = timed(False)
    clocks = sampler.stop()
    prof_ms, _, kt = timed(True)

    # per-distribution rates (single timed sort each, profiling off)
    per_dist = {}
    for d, a in zip(DISTS, inputs):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(3):
            ms.msort_sort_copy(h, a, out, options=opts, stream=stream)
        s1.record(stream)
        s1.synchronize()
        per_dist[d] = round(3 * n / (s0.elapsed_time(s1) * 1e-3) / 1e9, 3)

    torch_sort = _torch_sort_gkeys(inputs[0], 3) if not args.no_torch_sort else None

    from paper_2211_16479_gb300 import dist as msdist
    t_max = msdist.max_over_ranks(elapsed_ms, device=dev)
    keys_total = args.steps * len(DISTS) * n * world
    value = keys_total / (t_max * 1e-3) / 1e9

    # roofline of the dominant kernel (merge pass)
    peak, peak_kind = _peaks()
    m_launches, m_ms = kt[ms.MSORT_KERNEL_MERGE]
    t_launches, t_ms = kt[ms.MSORT_KERNEL_TILE]
    p_launches, p_ms = kt[ms.MSORT_KERNEL_PARTITION]
    bytes_per_merge = 2 * n * 4
    merge_avg_s = (m_ms / max(1, m_launches)) * 1e-3
    achieved = bytes_per_merge / merge_avg_s / 1e9
    alg_bytes_sort = 2 * n * 4 * (1 + mem_passes)

    # end to end through the host-buffer API
    e2e = None
    if not args.no_e2e:
        h_in = [a.cpu().pin_memory() for a in inputs]
        h_out = torch.empty(n, dtype=torch.uint32).pin_memory()
        h_outs = [torch.empty(n, dtype=torch.uint32).pin_memory() for _ in range(2)]
        # one untimed pass over every host buffer: the first transfer out of
        # a newly pinned buffer costs extra (device page-table setup)
        for i, a in enumerate(h_in):
            ms.msort_sort_host(h, a, out_keys=h_outs[i & 1], options=opts, stream=stream)
        barrier()
        # a step: the five sorts through the asynchronous host API (one
        # sort's device-to-host copy overlaps the next ones' host-to-device
        # copies and sorts); every step's copies run inside the timed region,
        # which ends when the last result is in host memory
        # The host link is shared with the machine's other tenants, so the
        # measurement is repeated and the median reported with every sample.
        def e2e_async():
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                for i, a in enumerate(h_in):
                    ms.msort_sort_host_async(h, a, out_keys=h_outs[i & 1], options=opts, stream=stream)
            stream.synchronize()
            barrier()
            te = msdist.max_over_ranks(time.perf_counter() - t0, device=dev)
            return args.e2e_steps * len(DISTS) * n * world / te / 1e9

        def e2e_sync():  # the synchronous call, one sort at a time, for comparison
            t1 = time.perf_counter()
            for a in h_in:
                ms.msort_sort_host(h, a, out_keys=h_outs[0], options=opts, stream=stream)
            barrier()
            ts = msdist.max_over_ranks(time.perf_counter() - t1, device=dev)
            return len(DISTS) * n * world / ts / 1e9

        av = [e2e_async() for _ in range(args.e2e_reps)]
        sv = [e2e_sync() for _ in range(args.e2e_reps)]
        e2e = {"value": float(np.median(av)), "unit": UNIT,
               "h2d_bytes_per_step": len(DISTS) * n * 4, "d2h_bytes_per_step": len(DISTS) * n * 4,
               "steps": args.e2e_steps, "repetitions": args.e2e_reps, "samples": [round(x, 3) for x in av],
               "api": "msort_sort_host_async x5 per step, stream sync after the last step; median of the repetitions",
               "sync_call_value": float(np.median(sv)), "sync_call_samples": [round(x, 3) for x in sv]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sample = [a[: 1 << 22].cpu().numpy() for a in inputs]
        v, cores, reps = cpu_oracle_rate(sample, seconds_target=args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first 2^22 keys of each of the 5 inputs, {reps} rounds, chunked oracle "
                         f"merge sort + pairwise merge tree on {cores} threads",
               "context": cpu_context_rates(sample)}

    # the chosen forms against the plain sort (rank 0, after the collectives)
    chosen = small = pairs = None
    if rank == 0 and not args.no_chosen:
        if not args.no_e2e:
            del h_in, h_out, h_outs
        chosen = chosen_vs_plain(args, h, dev, stream)
        small = form_small(h, dev, stream, 500)
        pairs = form_pairs(h, dev, stream, 5)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded SplitMix64 recipes, generated on the device)",
            "config": {"workload": "2^28 uint32 keys x 5 distributions (uniform, sorted, reverse, 16 distinct, "
                                   "Zipf 1.1 over 2^20 ranks), keys only, stable out-of-place sort",
                       "n": n, "distributions": list(DISTS), "tile": T, "merge_rounds": passes,
                       "merge_ways": ways, "memory_passes": mem_passes,
                       "l2": "inputs are 1 GiB each (> 126 MB L2); no flush between steps",
                       "graph_replay": bool(args.graph),
                       "timed_regions": "value: K steps without per-launch events; roofline and "
                                        "kernel_ms_per_step: K more steps with a CUDA event pair per launch",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "kernel": merge_kernel + "<u32>",
                         "traffic": _ncu_traffic(merge_kernel) if n == N else None, "algorithmic_bytes_per_launch": bytes_per_merge,
                         "launches": m_launches, "avg_ms": m_ms / max(1, m_launches)},
            "whole_sort_roofline": {"algorithmic_bytes": alg_bytes_sort,
                                    "frac_of_measured_hbm": alg_bytes_sort * len(DISTS) * args.steps /
                                    (t_max * 1e-3) / 1e9 / peak,
                                    "frac_of_8tbs": alg_bytes_sort * len(DISTS) * args.steps /
                                    (t_max * 1e-3) / 1e9 / NOMINAL_HBM_GBS},
            "kernel_ms_per_step": {"tile_sort": t_ms / args.steps, "partition": p_ms / args.steps,
                                   "merge": m_ms / args.steps},
            "profiled_ms_per_step": prof_ms / args.steps,
            "per_distribution_gkeys": per_dist,
            "torch_sort_stable_gkeys_uniform": torch_sort,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "chosen_vs_plain": chosen,
            "small_config": small,
            "pairs_config": pairs,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        tdist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Additional workloads (one JSON line each; the default run is the 2^28 sort)
# ---------------------------------------------------------------------------
def _events_ms(fn, reps, stream=None):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _base_line(metric, value, unit, args, ms_per_step, config, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic (seeded SplitMix64 recipes, generated on the device)",
            "config": config}
    line.update(extra)
    return line


def _torch_sort_gkeys(a_u32, reps):
    """torch.sort(stable=True) on the same keys, for context: the uint32 keys
    are viewed as int32 with the sign bit flipped (same order)."""
    import torch
    k = a_u32.view(torch.int32) ^ torch.iinfo(torch.int32).min
    torch.sort(k, stable=True)
    torch.cuda.synchronize()
    t = _events_ms(lambda: torch.sort(k, stable=True), reps)
    return a_u32.numel() / t / 1e6


def form_small(h, dev, stream, reps):
    """The small configuration: one stable sort of 2^20 uniform uint32 keys
    (4 MiB, L2-resident, so launch cost and dependent latency dominate).
    The default plan at this size is the single cooperative launch; the
    multi-launch plan (tile sort, then a partition and a merge launch per
    round) is timed beside it, both replayed from CUDA graphs and both
    launched directly, with torch.sort(stable=True) as context."""
    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen
    n = 1 << 20
    a = torch_gen.u32_distribution("uniform", n, 1, device=dev)
    outs = {}
    exp = torch.sort(a.to(torch.int64)).values.to(torch.uint32)
    res = {}
    arms = {"single_graph": {"use_graph": 1}, "single_launch": {},
            "multi_graph": {"use_graph": 1, "single_launch": -1}, "multi_launch": {"single_launch": -1}}
    for name, o in arms.items():
        outs[name] = torch.empty_like(a)
        step = (lambda o=o, out=outs[name]: ms.msort_sort_copy(h, a, out, options=o, stream=stream))
        for _ in range(5):
            step()
        torch.cuda.synchronize()
        assert bool((outs[name] == exp).all()), f"small sort mismatch ({name})"
        res[name] = _events_ms(step, reps, stream)
    T, W, P = ms.msort_plan_info(n, ms.MSORT_U32, False)
    peak, kind = _peaks()
    alg = 2 * n * 4 * (1 + P)
    best = res["single_graph"]
    return {"workload": "2^20 uniform uint32 keys, keys only, stable out-of-place sort", "n": n,
            "tile": T, "merge_rounds": P, "repetitions": reps,
            "us_per_sort": {k: v * 1e3 for k, v in res.items()},
            "gkeys_per_s": n / best / 1e6,
            "speedup_vs_multi_launch_graph": res["multi_graph"] / best,
            "identical_output": True,
            "roofline": {"bound": "latency (L2-resident)", "algorithmic_bytes": alg,
                         "achieved_gbs": alg / (best * 1e-3) / 1e9, "frac_of_hbm_peak_nominal":
                         alg / (best * 1e-3) / 1e9 / peak, "peak": peak, "peak_kind": kind,
                         "note": "the 4 MiB array stays in the 126 MB L2: the HBM roofline is nominal here"},
            "torch_sort_stable_gkeys": _torch_sort_gkeys(a, reps)}


def run_small(args):
    import torch

    import paper_2211_16479_gb300 as ms
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = ms.Context(0)
    f = form_small(ctx.handle, dev, stream, max(args.steps, 10) * 50)
    line = _base_line("Gkeys/s sorted (stable merge sort, 2^20 uint32 keys)", f["gkeys_per_s"], "Gkeys/s", args,
                      f["us_per_sort"]["single_graph"] * 1e-3,
                      {"workload": f["workload"] + ", single cooperative launch replayed from a CUDA graph",
                       "n": f["n"], "tile": f["tile"], "merge_rounds": f["merge_rounds"]},
                      dtype="u32", detail=f)
    print(json.dumps(line), flush=True)
    ctx.close()


def run_float(args):
    """2^28 float32 keys uniform in [-1, 1) (both signs): the same sort with
    the order-preserving key transform folded into the tile sort's load and
    the last merge round's store, timed beside 2^28 uint32 keys."""
    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen
    n = 1 << 28
    bits = torch_gen.uniform_u32(n, 1, device="cuda")
    top24 = (bits.view(torch.int32) >> 8) & 0xFFFFFF  # the top 24 bits of each word
    keys = (top24.to(torch.float32) * (2.0 ** -23) - 1.0).contiguous()
    out = torch.empty_like(keys)
    u_out = torch.empty_like(bits)
    ctx = ms.Context(0)
    h = ctx.handle
    o = {"use_graph": args.graph}
    res = {}
    for name, src, dst in (("float32", keys, out), ("uint32", bits, u_out)):
        step = lambda: ms.msort_sort_copy(h, src, dst, options=o)
        for _ in range(args.warmup):
            step()
        res[name] = _events_ms(step, args.steps)
    torch.cuda.synchronize()
    assert bool((out[1:] >= out[:-1]).all()), "float output not sorted"
    line = _base_line("Gkeys/s sorted (stable merge sort, 2^28 float32 keys, IEEE totalOrder)", n / res["float32"] / 1e6,
                      "Gkeys/s", args, res["float32"],
                      {"workload": "2^28 float32 keys uniform in [-1, 1), keys only, stable out-of-place sort",
                       "n": n, "graph_replay": bool(args.graph)},
                      dtype="f32 (sorted as u32 after an order-preserving transform)",
                      uint32_same_size_gkeys=n / res["uint32"] / 1e6,
                      float_over_uint32=res["uint32"] / res["float32"])
    print(json.dumps(line), flush=True)
    ctx.close()


def run_external(args):
    """Out-of-core: 2^30 uint32 keys (4 GiB) in pinned host memory sorted by a
    context whose device budget is 1 GiB (sorted runs of budget-sized
    chunks, then a blockwise merge through the device); every copy is
    inside the timed region."""
    import time

    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen
    n = 1 << 30
    budget = 1 << 30
    h_in = torch_gen.uniform_u32(n, 1, device="cuda").cpu().pin_memory()
    h_out = torch.empty(n, dtype=torch.uint32).pin_memory()
    ctx = ms.Context(0, scratch_budget_bytes=budget)
    h = ctx.handle
    ms.msort_sort_host(h, h_in, out_keys=h_out)  # warm-up (buffers, first copies)
    k = h_out[:: 1 << 16].to(torch.int64)
    assert bool((k[1:] >= k[:-1]).all()), "external output not sorted"
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        ms.msort_sort_host(h, h_in, out_keys=h_out)
        times.append(time.perf_counter() - t0)
    t = min(times)
    line = _base_line("Gkeys/s sorted out of core (2^30 uint32 keys in host memory, 1 GiB device budget)",
                      n / t / 1e9, "Gkeys/s", args, t * 1e3,
                      {"workload": "2^30 uniform uint32 keys in pinned host memory, device budget 1 GiB "
                                   "(the array is 4x the budget)", "n": n, "budget_bytes": budget},
                      dtype="u32", h2d_bytes=2 * n * 4, d2h_bytes=2 * n * 4,
                      note="two host round trips: sorted runs, then the blockwise merge")
    print(json.dumps(line), flush=True)
    ctx.close()


def form_pairs(h, dev, stream, reps):
    """The key-value configuration: a stable sort of 2^27 (uint64 key,
    uint32 value) pairs, keys drawn from 2^20 distinct values (heavy
    duplicates), values = original index, so the output is the stable sort
    exactly when the keys ascend and equal keys keep increasing values; that
    is checked on the device.  reps timed repetitions (CUDA events each),
    then one profiled sort for the kernel split."""
    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen
    n = 1 << 27
    keys, vals = torch_gen.dup_u64(n, 1, device=dev)
    ok, ov = torch.empty_like(keys), torch.empty_like(vals)
    step = lambda: ms.msort_sort_copy(h, keys, ok, vals, ov, stream=stream)
    for _ in range(3):
        step()
    ms.msort_ctx_sync(h, stream)
    k64 = ok.view(torch.int64) ^ torch.iinfo(torch.int64).min  # unsigned order as signed
    v64 = ov.to(torch.int64)
    same = k64[1:] == k64[:-1]
    stable = bool((k64[1:] >= k64[:-1]).all()) and bool((v64[1:][same] > v64[:-1][same]).all())
    del k64, v64, same
    t = [_events_ms(step, 1, stream) for _ in range(reps)]
    ms.msort_ctx_set_profiling(h, True)
    step()
    kern = {name: ms.msort_ctx_kernel_times(h, k)[1] for name, k in
            (("tile_sort", ms.MSORT_KERNEL_TILE), ("partition", ms.MSORT_KERNEL_PARTITION),
             ("merge", ms.MSORT_KERNEL_MERGE))}
    ms.msort_ctx_set_profiling(h, False)
    T, W, P = ms.msort_plan_info(n, ms.MSORT_U64, True)
    alg = 2 * n * 12 * (1 + P)
    med = statistics.median(t)
    peak, kind = _peaks()
    del keys, vals, ok, ov
    torch.cuda.empty_cache()
    return {"workload": "2^27 (uint64 key, uint32 original index) pairs, keys from 2^20 distinct values, "
                        "stable out-of-place sort",
            "n": n, "tile": T, "merge_block_outputs": W, "merge_passes": P, "repetitions": reps,
            "ms": _spread(t), "gpairs_per_s": n / med / 1e6, "stable_and_sorted": stable,
            "kernel_ms_per_sort": kern,
            "merge_pass_gbs": 2 * n * 12 * P / (kern["merge"] * 1e-3) / 1e9,
            "roofline": {"bound": "hbm", "algorithmic_bytes": alg,
                         "frac_of_peak": alg / (med * 1e-3) / 1e9 / peak, "peak": peak, "peak_kind": kind}}


def run_pairs(args):
    """Stable key-value sort of 2^27 pairs: uint64 keys from 2^20 distinct
    values, uint32 values = original index."""
    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen
    n = 1 << 27
    keys, vals = torch_gen.dup_u64(n, 1, device="cuda")
    ok, ov = torch.empty_like(keys), torch.empty_like(vals)
    ctx = ms.Context(0)
    h = ctx.handle
    step = lambda: ms.msort_sort_copy(h, keys, ok, vals, ov)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # stability guard: equal keys keep increasing original indices
    k64 = ok.view(torch.int64) ^ torch.iinfo(torch.int64).min
    v64 = ov.to(torch.int64)
    same = k64[1:] == k64[:-1]
    assert bool((k64[1:] >= k64[:-1]).all()) and bool((v64[1:][same] > v64[:-1][same]).all())
    t = _events_ms(step, args.steps)
    ms.msort_ctx_set_profiling(h, True)
    step()
    kern = {name: ms.msort_ctx_kernel_times(h, k)[1] for name, k in
            (("tile_sort", ms.MSORT_KERNEL_TILE), ("partition", ms.MSORT_KERNEL_PARTITION),
             ("merge", ms.MSORT_KERNEL_MERGE))}
    ms.msort_ctx_set_profiling(h, False)
    T, W, P = ms.msort_plan_info(n, ms.MSORT_U64, True)
    alg = 2 * n * 12 * (1 + P)
    peak, kind = _peaks()
    line = _base_line("Gpairs/s sorted (stable, 2^27 uint64 keys + uint32 values)", n / t / 1e6, "Gpairs/s", args, t,
                      {"workload": "2^27 (uint64 key, uint32 original index) pairs, keys from 2^20 distinct values",
                       "n": n, "tile": T, "merge_block_outputs": W, "merge_passes": P},
                      dtype="u64+u32", kernel_ms_per_sort=kern,
                      merge_pass_gbs=2 * n * 12 * P / (kern["merge"] * 1e-3) / 1e9,
                      whole_sort_roofline={"algorithmic_bytes": alg,
                                           "frac_of_measured_hbm": alg / (t * 1e-3) / 1e9 / peak,
                                           "frac_of_8tbs": alg / (t * 1e-3) / 1e9 / NOMINAL_HBM_GBS})
    print(json.dumps(line), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# The chosen forms against the plain sort (learned partition, batched
# segmented sort, continuous-batching server): each times its two arms in
# interleaved repetitions (A, B, A, B, ...) on identical inputs and checks on
# the device that both arms give identical output.
# ---------------------------------------------------------------------------
def _spread(xs):
    xs = [float(x) for x in xs]
    return {"min": min(xs), "median": statistics.median(xs), "max": max(xs), "samples": [round(x, 4) for x in xs]}


def _interleaved(arms, reps, stream):
    """arms: {name: (prepare, run)}; prepare() is untimed, run() is timed by
    CUDA events on `stream`.  Returns {name: [ms per repetition]}."""
    import torch
    out = {k: [] for k in arms}
    for _ in range(reps):
        for name, (prep, run) in arms.items():
            if prep is not None:
                prep()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            out[name].append(e0.elapsed_time(e1))
    return out


def _sort_bytes(n, tile, key_bytes=4):
    """Algorithmic bytes of one sort: a read and a write of every key per
    pass, tile sort plus ceil(log2(n / tile)) merge passes."""
    passes = 0
    L = tile
    while L < n:
        L *= 2
        passes += 1
    return 2 * n * key_bytes * (1 + passes)


def form_learned(h, dev, stream, reps, log2n, warmup):
    """2^log2n uint32 keys of the lognormal mixture: the exact merge-path
    partition (the plain sort) against the learned partition in its default
    mode (the passes whose runs hold >= 2^22 keys), with the model-free
    length-ratio start as the ablation arm."""
    import torch

    import paper_2211_16479_gb300 as ms
    from synth import torch_gen
    n = 1 << log2n
    src = torch_gen.lognormal3_u32(n, 1, device=dev)
    modes = {"exact": {}, "learned": {"partition_mode": 1}, "ratio_guess": {"partition_mode": 2}}
    outs = {k: torch.empty_like(src) for k in modes}

    def sorter(k):
        return lambda: ms.msort_sort_copy(h, src, outs[k], options=modes[k], stream=stream)
    for _ in range(warmup):
        for k in modes:
            sorter(k)()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    t = _interleaved({k: (None, sorter(k)) for k in modes}, reps, stream)
    clocks = sampler.stop()
    identical = {k: bool(torch.equal(outs[k].view(torch.int32), outs["exact"].view(torch.int32))) for k in modes}
    del outs["ratio_guess"]
    # partition time per pass (event pairs only, no probe counting)
    per_pass, probes = {}, {}
    for k in modes:
        ms.msort_ctx_set_profiling(h, 1)
        ms.msort_sort_copy(h, src, outs["exact"], options=modes[k], stream=stream)
        per_pass[k] = [round(x * 1e3, 2) for x in ms.msort_ctx_kernel_log(h, ms.MSORT_KERNEL_PARTITION)]
        ms.msort_ctx_set_profiling(h, 0)
    # probes per search (level 2 counts them; not timed)
    for name, o in (("exact", {"partition_mode": 3, "learned_passes": 64}),
                    ("learned", {"partition_mode": 1, "learned_passes": 64}),
                    ("ratio_guess", {"partition_mode": 2, "learned_passes": 64})):
        ms.msort_ctx_set_profiling(h, 2)
        ms.msort_sort_copy(h, src, outs["exact"], options=o, stream=stream)
        pr, se = ms.msort_ctx_partition_stats(h)
        ms.msort_ctx_set_profiling(h, 0)
        probes[name] = pr / se if se else None
    _, err = ms.msort_learned_model(h)
    T, _, P = ms.msort_plan_info(n, ms.MSORT_U32, False)
    first_guided = next((i for i in range(P) if (T << i) >= (1 << 22)), P)
    med = {k: statistics.median(v) for k, v in t.items()}
    peak, kind = _peaks()
    alg = _sort_bytes(n, T)
    return {"workload": f"2^{log2n} uint32 keys, lognormal mixture (0.5/0.3/0.2; ln-space mu 14/18/21; "
                        f"sigma 1/0.5/0.3), keys only, out of place",
            "n": n, "repetitions": reps, "order": "interleaved exact, learned, ratio_guess per repetition",
            "plain_arm": "exact merge-path partition (partition_mode 0)",
            "chosen_arm": "learned partition, default mode (partition_mode 1: guided search on the passes whose runs "
                          f"hold >= 2^22 keys, passes {first_guided}..{P - 1} of {P})",
            "ms": {k: _spread(v) for k, v in t.items()},
            "speedup": med["exact"] / med["learned"],
            "speedup_vs_ratio_guess": med["ratio_guess"] / med["learned"],
            "identical_output": identical["learned"] and identical["ratio_guess"],
            "partition_us_per_pass": per_pass,
            "partition_us_guided_passes": {k: round(sum(v[first_guided:]), 1) for k, v in per_pass.items()},
            "probes_per_search_all_passes": probes,
            "model_max_sample_error": err,
            "roofline": {"bound": "hbm", "algorithmic_bytes": alg,
                         "frac_of_peak": {k: alg / (m * 1e-3) / 1e9 / peak for k, m in med.items()},
                         "peak": peak, "peak_kind": kind},
            "clocks": clocks}


def form_segmented(h, dev, stream, reps, warmup):
    """50,000 uint32 arrays with lengths log-uniform in [1, 65536]: the
    batched segmented sort (one persistent launch per length bucket, CUDA
    graph replay) against the plain sort giving the same result (one stable
    sort of the 64-bit keys (segment index << 32 | key))."""
    import numpy as np
    import torch

    import paper_2211_16479_gb300 as ms
    import synth
    from synth import torch_gen
    lens = synth.segment_lengths(50000, 1)
    off = synth.segment_offsets(lens)
    n = int(off[-1])
    src = torch_gen.uniform_u32(n, 1, device=dev)
    work = torch.empty_like(src)
    doff = torch.from_numpy(off.astype(np.int64)).to(dev)
    seg_id = torch.repeat_interleave(torch.arange(len(lens), device=dev, dtype=torch.int64),
                                     torch.from_numpy(lens).to(dev))
    comp = ((seg_id << 32) | src.to(torch.int64)).view(torch.uint64)
    del seg_id
    pout = torch.empty_like(comp)
    opt = {"use_graph": 1}
    arms = {"plain": (None, lambda: ms.msort_sort_copy(h, comp, pout, options=opt, stream=stream)),
            "segmented": (lambda: work.copy_(src),
                          lambda: ms.msort_segmented_sort(h, work, doff, options=opt, stream=stream))}
    for _ in range(warmup):
        for prep, run in arms.values():
            if prep:
                prep()
            run()
    ms.msort_ctx_sync(h, stream)
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    t = _interleaved(arms, reps, stream)
    clocks = sampler.stop()
    ms.msort_ctx_sync(h, stream)
    same = bool(torch.equal((pout.view(torch.int64) & 0xFFFFFFFF).to(torch.int32), work.view(torch.int32)))
    med = {k: statistics.median(v) for k, v in t.items()}
    # algorithmic bytes: on-chip segments (<= 16896 keys) move once; longer
    # ones add ceil(log2(len / 16896)) merge passes
    seg_bytes = sum(_sort_bytes(int(L), 16896) for L in lens if L > 1)
    T64, _, _ = ms.msort_plan_info(n, ms.MSORT_U64, False)
    plain_bytes = _sort_bytes(n, T64, 8)
    peak, kind = _peaks()
    return {"workload": "50,000 uint32 arrays, lengths log-uniform in [1, 65536], uniform keys, in place",
            "n": n, "segments": 50000, "repetitions": reps, "order": "interleaved plain, segmented",
            "plain_arm": "one stable plain sort of the 64-bit keys (segment << 32 | key), CUDA-graph replay",
            "chosen_arm": "msort_segmented_sort, CUDA-graph replay",
            "ms": {k: _spread(v) for k, v in t.items()},
            "gkeys_per_s": {k: n / m / 1e6 for k, m in med.items()},
            "speedup": med["plain"] / med["segmented"],
            "identical_output": same,
            "roofline": {"bound": "hbm", "algorithmic_bytes": {"segmented": seg_bytes, "plain": plain_bytes},
                         "frac_of_peak": {"segmented": seg_bytes / (med["segmented"] * 1e-3) / 1e9 / peak,
                                          "plain": plain_bytes / (med["plain"] * 1e-3) / 1e9 / peak},
                         "peak": peak, "peak_kind": kind},
            "clocks": clocks}


# Concurrent requests of the serving form's chosen arm: at saturation 16
# slots finished the 2,000-request stream in 86 ms against 91 ms for 8 (24:
# 85.7), with the same p99 under Poisson arrivals at 0.9 load.
SERVING_SLOTS = 16
SERVING_ARM = f"continuous_{SERVING_SLOTS}_slots"


def form_serving(dev, reps, count, rho, sweep=(0.3, 0.6)):
    """Sort requests with sizes log-uniform in [2^10, 2^24] (uniform uint32
    keys, 8 GB device budget): continuous batching (SERVING_SLOTS slots) against the
    same requests served one at a time in arrival order (1 slot, the plain
    sort per request), at saturation (all submitted at once) and under
    Poisson arrivals at `rho` x the one-slot service rate; then p50/p99 of
    both arms at the lighter loads in `sweep`."""
    import numpy as np
    import torch

    import paper_2211_16479_gb300 as ms
    import synth
    from synth import torch_gen
    _, sizes = synth.poisson_requests(count, 1, rate_per_s=1.0)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    total = int(offs[-1])
    pristine = torch_gen.uniform_u32(total, 7, device=dev)
    buf = torch.empty_like(pristine)
    sort_bytes = sum(_sort_bytes(int(x), 16896) for x in sizes)

    def run(slots, rate):
        buf.copy_(pristine)
        torch.cuda.synchronize()
        t_arr = synth.poisson_requests(count, 1, rate_per_s=rate)[0] if rate else None
        with ms.Server(dev.index or 0, mem_budget_bytes=8 << 30, max_slots=slots) as srv:
            ids = []
            t0 = time.perf_counter()
            for i in range(count):
                if rate:
                    while time.perf_counter() - t0 < t_arr[i]:
                        pass
                ids.append(srv.submit(buf[int(offs[i]):int(offs[i + 1])]))
            for rid in ids:
                srv.wait(rid, 600000.0)
            wall = time.perf_counter() - t0
            st = srv.stats()
        return {"wall_ms": wall * 1e3, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                "gkeys_per_s": total / wall / 1e9, "max_inflight": st["max_inflight"],
                "arena_high_water_gb": st["arena_high_water"] / 1e9}

    run(1, 0.0)  # warm-up: the servers' first launches and buffers
    ref = None
    run(1, 0.0)
    ref = buf.clone()
    run(SERVING_SLOTS, 0.0)
    same = bool(torch.equal(buf.view(torch.int32), ref.view(torch.int32)))
    del ref
    mu = run(1, 0.0)["gkeys_per_s"] * 1e9 / float(np.mean(sizes))  # one-slot service rate, requests/s
    rate = rho * mu
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    res = {"saturation": {"fifo_1_slot": [], SERVING_ARM: []},
           "poisson": {"fifo_1_slot": [], SERVING_ARM: []}}
    for _ in range(reps):
        res["saturation"]["fifo_1_slot"].append(run(1, 0.0))
        res["saturation"][SERVING_ARM].append(run(SERVING_SLOTS, 0.0))
        res["poisson"]["fifo_1_slot"].append(run(1, rate))
        res["poisson"][SERVING_ARM].append(run(SERVING_SLOTS, rate))
    lighter = {f"{x:g}": {"fifo_1_slot": [], SERVING_ARM: []} for x in sweep}
    for _ in range(reps):
        for x in sweep:
            lighter[f"{x:g}"]["fifo_1_slot"].append(run(1, x * mu))
            lighter[f"{x:g}"][SERVING_ARM].append(run(SERVING_SLOTS, x * mu))
    clocks = sampler.stop()

    def summary(runs):
        return {k: _spread([r[k] for r in runs]) for k in ("wall_ms", "p50_ms", "p99_ms", "gkeys_per_s")} | \
            {"max_inflight": max(r["max_inflight"] for r in runs),
             "arena_high_water_gb": max(r["arena_high_water_gb"] for r in runs)}
    out = {ph: {arm: summary(v) for arm, v in d.items()} for ph, d in res.items()}
    load_sweep = {x: {arm: {"p50_ms": statistics.median(r["p50_ms"] for r in v),
                            "p99_ms": statistics.median(r["p99_ms"] for r in v),
                            "p99_spread": _spread([r["p99_ms"] for r in v])}
                      for arm, v in d.items()} for x, d in lighter.items()}
    sat_f = statistics.median(r["wall_ms"] for r in res["saturation"]["fifo_1_slot"])
    sat_c = statistics.median(r["wall_ms"] for r in res["saturation"][SERVING_ARM])
    p99_f = statistics.median(r["p99_ms"] for r in res["poisson"]["fifo_1_slot"])
    p99_c = statistics.median(r["p99_ms"] for r in res["poisson"][SERVING_ARM])
    p50_c = statistics.median(r["p50_ms"] for r in res["poisson"][SERVING_ARM])
    peak, kind = _peaks()
    return {"workload": f"{count} uint32 sort requests, sizes log-uniform in [2^10, 2^24], uniform keys, in place, "
                        "8 GB device budget", "requests": count, "keys": total,
            "repetitions": reps,
            "order": f"interleaved per repetition: saturation 1 slot, {SERVING_SLOTS} slots; Poisson 1, {SERVING_SLOTS}",
            "plain_arm": "fifo_1_slot: the same requests sorted one at a time in arrival order",
            "chosen_arm": f"{SERVING_ARM}: up to {SERVING_SLOTS} requests on the GPU at once, admitted as slots and "
                          "memory free",
            "poisson_rate_per_s": rate, "offered_load": rho,
            "saturation": out["saturation"], "poisson": out["poisson"],
            "poisson_lighter_loads": load_sweep,
            "speedup": sat_f / sat_c,
            "speedup_meaning": f"saturation wall time, one slot / {SERVING_SLOTS} slots",
            "p50_ms": p50_c, "p99_ms": p99_c, "p99_fifo_ms": p99_f,
            "identical_output": same,
            "roofline": {"bound": "hbm", "algorithmic_bytes": sort_bytes,
                         "frac_of_peak_saturation": {"fifo_1_slot": sort_bytes / (sat_f * 1e-3) / 1e9 / peak,
                                                     SERVING_ARM: sort_bytes / (sat_c * 1e-3) / 1e9 / peak},
                         "peak": peak, "peak_kind": kind},
            "clocks": clocks}


def chosen_vs_plain(args, h, dev, stream):
    import torch
    r = {}
    r["learned"] = form_learned(h, dev, stream, args.chosen_reps, args.learned_log2n, 2)
    torch.cuda.empty_cache()
    r["segmented"] = form_segmented(h, dev, stream, args.chosen_reps, 2)
    torch.cuda.empty_cache()
    r["serving"] = form_serving(dev, args.chosen_reps, args.serving_requests, 0.9)
    torch.cuda.empty_cache()
    return r


def _form_line(name, f, args):
    med = {k: v["median"] for k, v in f["ms"].items()} if "ms" in f else None
    if name == "serving":
        c = f["saturation"][SERVING_ARM]["gkeys_per_s"]["median"]
        return _base_line("Gkeys/s served (continuous batching of sort requests, saturation)", c, "Gkeys/s", args,
                          f["saturation"][SERVING_ARM]["wall_ms"]["median"],
                          {"workload": f["workload"], "requests": f["requests"], "keys": f["keys"]},
                          dtype="u32", detail=f)
    chosen = "learned" if name == "learned" else "segmented"
    return _base_line(f"Gkeys/s sorted ({name} form vs plain sort)", f["n"] / med[chosen] / 1e6, "Gkeys/s", args,
                      med[chosen], {"workload": f["workload"], "n": f["n"]}, dtype="u32", detail=f)


def run_form(args):
    import torch

    import paper_2211_16479_gb300 as ms
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = ms.Context(0)
    h = ctx.handle
    reps = max(args.chosen_reps, 5)
    if args.workload == "learned":
        f = form_learned(h, dev, stream, reps, args.learned_log2n, args.warmup)
    elif args.workload == "segmented":
        f = form_segmented(h, dev, stream, reps, args.warmup)
    else:
        f = form_serving(dev, reps, args.serving_requests, 0.9)
    print(json.dumps(_form_line(args.workload, f, args)), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--merge-block", type=int, default=0)
    ap.add_argument("--merge-ways", type=int, default=0, help="0 = plan default, 2 = pairwise passes, 4 = four-way")
    ap.add_argument("--no-torch-sort", action="store_true", help="skip the torch.sort(stable=True) context figure")
    ap.add_argument("--graph", type=int, default=1, help="1 = replay each sort from a captured CUDA graph")
    ap.add_argument("--e2e-steps", type=int, default=None, help="steps of the end-to-end measurement (default: --steps)")
    ap.add_argument("--e2e-reps", type=int, default=5, help="repetitions of the end-to-end measurement (median)")
    ap.add_argument("--learned-log2n", type=int, default=30, help="size of the learned-partition workload (log2)")
    ap.add_argument("--chosen-reps", type=int, default=5, help="interleaved repetitions per chosen-vs-plain arm")
    ap.add_argument("--serving-requests", type=int, default=2000, help="requests per serving run")
    ap.add_argument("--no-chosen", action="store_true", help="skip the chosen-vs-plain comparisons")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="sort",
                    choices=["sort", "small", "float", "external", "pairs", "segmented", "learned", "serving"])
    args = ap.parse_args()
    if args.e2e_steps is None:
        args.e2e_steps = args.steps
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "sort":
        fn = {"small": run_small, "float": run_float, "external": run_external, "pairs": run_pairs,
              "segmented": run_form, "learned": run_form, "serving": run_form}
        fn[args.workload](args)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

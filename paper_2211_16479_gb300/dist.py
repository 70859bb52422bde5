"""Multi-GPU forms of the sort over torch.distributed (one process per GPU).

``tree_merge_sort`` is the paper's message-passing merge sort (Section "MPI
Merge Sort": scatter, local sort, then the merge tree of Figs. 16-17): every
rank sorts its chunk, then in rounds the upper half of the still-active
ranks sends its run to a partner in the lower half, which merges, until
rank 0 holds the whole sorted array.  The paper needs a power-of-two rank
count; here the split is ceil(active / 2), so any count works.  On GPU
ranks the local sort and every merge are this library's kernels
(``msort_sort`` / ``msort_merge``) and the runs travel by NCCL send/recv;
the functions are injectable so that the rank schedule itself can be
exercised on CPU ranks (gloo).

``sample_sort`` is the one-exchange form of the same method for many GPUs:
every rank sorts its chunk, regular samples of all chunks choose p - 1
splitters, one all-to-all exchange moves every element to the rank that owns
its key range, and each rank merges the p sorted pieces it received with the
pairwise merge tree.  Splitters are (key, global position) pairs, so ranks
split even runs of equal keys and the result is exactly the stable sort of
the gathered array (rank r holds the r-th slice), with balanced slices
whatever the duplicates.

``max_over_ranks`` / ``sum_over_ranks`` are the reductions the benchmark
uses to report whole-job throughput from independent replicas.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as tdist


def max_over_ranks(value: float, device=None) -> float:
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.SUM)
    return float(t.item())


def merge_schedule(world: int):
    """Rounds of the merge tree: a list of [(receiver, sender), ...] per round."""
    rounds = []
    active = world
    while active > 1:
        split = (active + 1) // 2
        rounds.append([(r - split, r) for r in range(split, active)])
        active = split
    return rounds


def _gpu_sort(ctx):
    import paper_2211_16479_gb300 as ms

    def sort(t):
        ms.msort_sort(ctx, t)
        return t
    return sort


def _gpu_merge(ctx):
    import paper_2211_16479_gb300 as ms

    def merge(a, b):
        out = torch.empty(a.numel() + b.numel(), dtype=a.dtype, device=a.device)
        ms.msort_merge(ctx, a, b, out)
        return out
    return merge


def tree_merge_sort(local: torch.Tensor, ctx=None, local_sort=None, merge=None):
    """Sort the concatenation of every rank's ``local`` chunk (rank order).

    Returns the fully sorted tensor on rank 0 and None elsewhere.  Equal
    keys keep rank order then position order (the merges take the lower
    rank's run first), so the result is the stable sort of the gathered
    array.  ``local_sort(t) -> t`` and ``merge(a, b) -> c`` default to the
    library's GPU kernels through ``ctx``.
    """
    if local_sort is None or merge is None:
        if ctx is None:
            raise ValueError("a msort context is needed for the GPU local sort and merges")
        local_sort = local_sort or _gpu_sort(ctx)
        merge = merge or _gpu_merge(ctx)
    rank, world = tdist.get_rank(), tdist.get_world_size()
    run = local_sort(local.contiguous())
    for pairs in merge_schedule(world):
        for recv, send in pairs:
            if rank == send:
                n = torch.tensor([run.numel()], dtype=torch.int64, device=run.device)
                tdist.send(n, dst=recv)
                if run.numel():
                    tdist.send(run, dst=recv)
                run = None
            elif rank == recv:
                n = torch.zeros(1, dtype=torch.int64, device=run.device)
                tdist.recv(n, src=send)
                other = torch.empty(int(n.item()), dtype=run.dtype, device=run.device)
                if other.numel():
                    tdist.recv(other, src=send)
                run = merge(run, other)
        if run is None:
            break
    return run if rank == 0 else None


# ---------------------------------------------------------------------------
# Sample sort
# ---------------------------------------------------------------------------
def _wire(t: torch.Tensor) -> torch.Tensor:
    """Keys or values for the collectives at their own width, bit-preserving:
    a signed view of the same size (int32 or int64)."""
    return t.view(torch.int64) if t.element_size() == 8 else t.view(torch.int32)


def _gather(t: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """t[idx] through a signed view of the same width."""
    return _wire(t)[idx].view(t.dtype)


def _gpu_sort_pairs(ctx):
    import paper_2211_16479_gb300 as ms

    def sort(k, v):
        k, v = k.contiguous().clone(), v.contiguous().clone()
        if k.numel():
            ms.msort_sort_pairs(ctx, k, v)
        return k, v
    return sort


def _gpu_merge_pairs(ctx):
    import paper_2211_16479_gb300 as ms

    def merge(a, va, b, vb):
        out = torch.empty(a.numel() + b.numel(), dtype=a.dtype, device=a.device)
        vout = None if va is None else torch.empty(out.numel(), dtype=va.dtype, device=va.device)
        if out.numel():
            ms.msort_merge(ctx, a, b, out, va, vb, vout)
        return out, vout
    return merge


def _gpu_merge_runs(ctx):
    import paper_2211_16479_gb300 as ms

    def merge_runs(k, v, offsets):
        out = torch.empty_like(k)
        vout = None if v is None else torch.empty_like(v)
        if k.numel():
            ms.msort_merge_runs(ctx, k, offsets, out, vals=v, out_vals=vout)
        return out, vout
    return merge_runs


def _gpu_split_points(ctx):
    import paper_2211_16479_gb300 as ms

    def split_points(keys, idx, offset, split_keys, split_pos):
        cuts = torch.zeros(split_keys.numel(), dtype=torch.int64, device=keys.device)
        if split_keys.numel():
            ms.msort_split_points(ctx, keys, idx, offset, split_keys, split_pos, cuts)
        return cuts
    return split_points


def _merge_runs_by_pairs(merge):
    """merge_runs(k, v, offsets) from a stable two-way merge(a, va, b, vb):
    the pairwise tree over the runs laid end to end (ties in run order)."""
    def merge_runs(k, v, offsets):
        offs = [int(x) for x in offsets]
        pieces = [(k[a:b], None if v is None else v[a:b]) for a, b in zip(offs, offs[1:])]
        if not pieces:
            return k, v
        while len(pieces) > 1:
            pieces = [merge(*pieces[i], *pieces[i + 1]) if i + 1 < len(pieces) else pieces[i]
                      for i in range(0, len(pieces), 2)]
        return pieces[0]
    return merge_runs


def sample_sort(local: torch.Tensor, vals: torch.Tensor | None = None, ctx=None, local_sort=None, merge=None,
                oversample: int = 16, merge_runs=None, split_points=None):
    """Stable sort of the concatenation (in rank order) of every rank's
    ``local`` chunk (and ``vals`` alongside).  Returns this rank's slice
    (keys, vals): the slices, concatenated in rank order, are the sorted
    array.  Steps, all on the device for GPU ranks (only per-rank counts,
    O(p) numbers, reach the host):

    1. ``local_sort(k, v) -> (k, v)``: stable sort of the chunk by key,
       carrying the local index 0..n-1 as the uint32 value;
    2. ``oversample * p`` regular samples of the sorted chunk, (key, global
       position), are all-gathered at the keys' own width; the p sample
       runs, each sorted by (key, position) and in rank = position order,
       are merged by ``merge_runs``; every (m / p)-th becomes a splitter;
    3. ``split_points(keys, idx, offset, split_keys, split_pos) -> cuts``:
       elements of the sorted chunk ordered before each splitter;
    4. one all-to-all exchange of counts, keys and values (at their own
       width);
    5. ``merge_runs(k, v, offsets) -> (k, v)``: stable merge of the p
       received pieces laid end to end in source-rank order.

    ``merge_runs`` may be replaced by a two-way ``merge(a, va, b, vb)``
    (stable, ties from a), applied as a pairwise tree.  All default to the
    library's kernels through ``ctx`` (msort_sort_pairs, msort_merge_runs,
    msort_split_points).  Chunks hold fewer than 2^31 elements."""
    if merge_runs is None and merge is not None:
        merge_runs = _merge_runs_by_pairs(merge)
    if local_sort is None or merge_runs is None or split_points is None:
        if ctx is None:
            raise ValueError("a msort context is needed for the GPU local sort, merges and cuts")
        local_sort = local_sort or _gpu_sort_pairs(ctx)
        merge_runs = merge_runs or _gpu_merge_runs(ctx)
        split_points = split_points or _gpu_split_points(ctx)
    rank, world = tdist.get_rank(), tdist.get_world_size()
    dev = local.device
    # the collectives run on the device for NCCL, on the host for gloo
    comm = dev if tdist.get_backend() == "nccl" else torch.device("cpu")
    n = local.numel()
    sizes = [torch.zeros(1, dtype=torch.int64, device=comm) for _ in range(world)]
    tdist.all_gather(sizes, torch.tensor([n], dtype=torch.int64, device=comm))
    sizes = [int(x) for x in sizes]
    offset = sum(sizes[:rank])

    # 1. local stable sort; the local index rides along as the value
    idx = torch.arange(n, dtype=torch.int32, device=dev).view(torch.uint32)
    sk, si = local_sort(local.contiguous(), idx)
    si_long = si.view(torch.int32).to(torch.int64)
    sv = None if vals is None else _gather(vals.contiguous(), si_long)

    # 2. regular samples (key, global position) -> sorted by the library's
    # merge of the p sample runs -> p - 1 splitters
    s = max(1, oversample * world)
    smp_k = torch.zeros(s, dtype=_wire(sk).dtype, device=dev)
    smp_p = torch.zeros(s, dtype=torch.int64, device=dev)
    if n:
        pick = torch.div((torch.arange(s, dtype=torch.int64, device=dev) * 2 + 1) * n, 2 * s, rounding_mode="floor")
        smp_k = _wire(sk)[pick]
        smp_p = si_long[pick] + offset
    all_k = [torch.zeros(s, dtype=smp_k.dtype, device=comm) for _ in range(world)]
    all_p = [torch.zeros(s, dtype=torch.int64, device=comm) for _ in range(world)]
    tdist.all_gather(all_k, smp_k.to(comm))
    tdist.all_gather(all_p, smp_p.to(comm))
    counts = [s if sizes[r] else 0 for r in range(world)]
    gk = torch.cat([all_k[r][:counts[r]] for r in range(world)]).to(dev).view(sk.dtype)
    gp = torch.cat([all_p[r][:counts[r]] for r in range(world)]).to(dev)
    m = gk.numel()
    run_offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    order = torch.arange(m, dtype=torch.int32, device=dev).view(torch.uint32)
    mk, mo = merge_runs(gk, order, run_offsets)
    at = torch.tensor([(j * m) // world for j in range(1, world)], dtype=torch.int64, device=dev)
    if m:
        spl_k = _gather(mk, at)
        spl_p = gp[mo.view(torch.int32).to(torch.int64)[at]]
        cuts = split_points(sk, si, offset, spl_k, spl_p)
        cuts = [int(x) for x in cuts.tolist()]
    else:
        cuts = [0] * (world - 1)
    bounds = [0] + cuts + [n]
    send = torch.tensor([bounds[r + 1] - bounds[r] for r in range(world)], dtype=torch.int64, device=comm)

    # 3. one exchange: counts, then keys (and values) at their own width
    recv = torch.zeros(world, dtype=torch.int64, device=comm)
    tdist.all_to_all_single(recv, send)
    send_l, recv_l = send.tolist(), recv.tolist()
    total = int(sum(recv_l))

    def exchange(t):
        w = _wire(t).to(comm)
        got = torch.zeros(total, dtype=w.dtype, device=comm)
        tdist.all_to_all_single(got, w, output_split_sizes=recv_l, input_split_sizes=send_l)
        return got.to(dev).view(t.dtype)
    got_k = exchange(sk)
    got_v = None if vals is None else exchange(sv)

    # 4. the p sorted pieces, end to end in source-rank order: one stable merge
    return merge_runs(got_k, got_v, np.concatenate([[0], np.cumsum(recv_l)]).astype(np.uint64))

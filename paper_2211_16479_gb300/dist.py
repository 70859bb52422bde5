"""Multi-GPU forms of the sort over torch.distributed (one process per GPU).

``tree_merge_sort`` is the paper's message-passing merge sort (Section "MPI
Merge Sort": scatter, local sort, then the merge tree of Fig. 13): every
rank sorts its chunk, then in rounds the upper half of the still-active
ranks sends its run to a partner in the lower half, which merges, until
rank 0 holds the whole sorted array.  The paper needs a power-of-two rank
count; here the split is ceil(active / 2), so any count works.  On GPU
ranks the local sort and every merge are this library's kernels
(``msort_sort`` / ``msort_merge``) and the runs travel by NCCL send/recv;
the functions are injectable so that the rank schedule itself can be
exercised on CPU ranks (gloo).

``max_over_ranks`` / ``sum_over_ranks`` are the reductions the benchmark
uses to report whole-job throughput from independent replicas.
"""
from __future__ import annotations

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

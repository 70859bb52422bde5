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
def _to_wire(t: torch.Tensor) -> torch.Tensor:
    """Keys or values as int64 for the collectives, bit-preserving: 64-bit
    types by a view, 32-bit ones through their int32 view (torch has few
    kernels for unsigned types)."""
    return t.view(torch.int64) if t.element_size() == 8 else t.view(torch.int32).to(torch.int64)


def _from_wire(t: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    return t.view(like.dtype) if like.element_size() == 8 else t.to(torch.int32).view(like.dtype)


def _gather(t: torch.Tensor, idx: torch.Tensor) -> torch.Tensor:
    """t[idx] through a signed view of the same width."""
    signed = torch.int64 if t.element_size() == 8 else torch.int32
    return t.view(signed)[idx].view(t.dtype)


def _np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


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


def _split_points(keys: np.ndarray, gpos: np.ndarray, sk: np.ndarray, sg: np.ndarray) -> np.ndarray:
    """For each splitter (sk[t], sg[t]), the number of local elements ordered
    before it: keys below sk[t], plus those equal to it whose global position
    is below sg[t] (within equal keys the global positions increase)."""
    lo = np.searchsorted(keys, sk, side="left")
    hi = np.searchsorted(keys, sk, side="right")
    out = np.empty(len(sk), dtype=np.int64)
    for t in range(len(sk)):
        out[t] = lo[t] + np.searchsorted(gpos[lo[t]:hi[t]], sg[t], side="left")
    return out


def sample_sort(local: torch.Tensor, vals: torch.Tensor | None = None, ctx=None, local_sort=None, merge=None,
                oversample: int = 16, merge_runs=None):
    """Stable sort of the concatenation (in rank order) of every rank's
    ``local`` chunk (and ``vals`` alongside).  Returns this rank's slice
    (keys, vals): the slices, concatenated in rank order, are the sorted
    array.  ``local_sort(k, v) -> (k, v)`` sorts by key, stably, carrying
    uint32 values.  The p received pieces are merged either by
    ``merge_runs(k, v, offsets) -> (k, v)``, the stable merge of sorted runs
    laid end to end, or, when only ``merge(a, va, b, vb) -> (c, vc)`` (the
    stable merge of two, ties from a) is given, by a pairwise tree of it.
    Both default to the library's GPU kernels through ``ctx``
    (``msort_merge_runs``: every round of the tree in one launch pair).
    Chunks must hold fewer than 2^31 elements."""
    if local_sort is None or (merge is None and merge_runs is None):
        if ctx is None:
            raise ValueError("a msort context is needed for the GPU local sort and merges")
        local_sort = local_sort or _gpu_sort_pairs(ctx)
        if merge is None and merge_runs is None:
            merge_runs = _gpu_merge_runs(ctx)
    rank, world = tdist.get_rank(), tdist.get_world_size()
    dev = local.device
    # the collectives run on the device for NCCL, on the host for gloo
    comm = dev if tdist.get_backend() == "nccl" else torch.device("cpu")
    n = local.numel()
    sizes = [torch.zeros(1, dtype=torch.int64, device=comm) for _ in range(world)]
    tdist.all_gather(sizes, torch.tensor([n], dtype=torch.int64, device=comm))
    offset = int(sum(int(x) for x in sizes[:rank]))

    # 1. local stable sort; the local index rides along as the value
    idx = torch.arange(n, dtype=torch.int32, device=dev).view(torch.uint32)
    sk_local, si = local_sort(local.contiguous(), idx)
    si64 = si.view(torch.int32).to(torch.int64)
    sv_local = None if vals is None else _gather(vals.contiguous(), si64)
    keys_np = _np(sk_local)
    gpos_np = _np(si64) + offset  # global input position of every sorted element

    # 2. regular samples (s per rank) -> p - 1 splitters, as (key, position)
    s = max(1, oversample * world)
    smp_k = torch.zeros(s, dtype=torch.int64)
    smp_g = torch.full((s,), -1, dtype=torch.int64)
    if n:
        pick = (np.arange(s, dtype=np.int64) * 2 + 1) * n // (2 * s)
        smp_k[:] = _to_wire(torch.from_numpy(np.ascontiguousarray(keys_np[pick])))
        smp_g[:] = torch.from_numpy(gpos_np[pick])
    all_k = [torch.zeros(s, dtype=torch.int64, device=comm) for _ in range(world)]
    all_g = [torch.zeros(s, dtype=torch.int64, device=comm) for _ in range(world)]
    tdist.all_gather(all_k, smp_k.to(comm))
    tdist.all_gather(all_g, smp_g.to(comm))
    gk = _np(_from_wire(torch.cat(all_k).cpu(), local.cpu()))
    gg = _np(torch.cat(all_g).cpu())
    keep = gg >= 0
    gk, gg = gk[keep], gg[keep]
    order = np.lexsort((gg, gk))  # by key, then by global position
    gk, gg = gk[order], gg[order]
    m = len(gk)
    at = (np.arange(1, world) * m) // world
    cuts = _split_points(keys_np, gpos_np, gk[at], gg[at]) if m else np.zeros(world - 1, dtype=np.int64)
    bounds = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    send = torch.from_numpy(np.diff(bounds)).to(comm)

    # 3. one exchange: counts, then keys (and values)
    recv = torch.zeros(world, dtype=torch.int64, device=comm)
    tdist.all_to_all_single(recv, send)
    send_l, recv_l = send.tolist(), recv.tolist()
    total = int(sum(recv_l))

    def exchange(t):
        wire = _to_wire(t).to(comm) if n else torch.zeros(0, dtype=torch.int64, device=comm)
        got = torch.zeros(total, dtype=torch.int64, device=comm)
        tdist.all_to_all_single(got, wire, output_split_sizes=recv_l, input_split_sizes=send_l)
        return got
    got_k = exchange(sk_local)
    got_v = None if vals is None else exchange(sv_local)

    # 4. p sorted pieces in source-rank order: the pairwise merge tree
    if merge_runs is not None:
        k = _from_wire(got_k, local).to(dev)
        v = None if vals is None else _from_wire(got_v, vals).to(dev)
        return merge_runs(k, v, np.concatenate([[0], np.cumsum(recv_l)]).astype(np.uint64))
    pieces, o = [], 0
    for c in recv_l:
        k = _from_wire(got_k[o:o + c], local).to(dev)
        v = None if vals is None else _from_wire(got_v[o:o + c], vals).to(dev)
        pieces.append((k, v))
        o += c
    while len(pieces) > 1:
        pieces = [merge(*pieces[i], *pieces[i + 1]) if i + 1 < len(pieces) else pieces[i]
                  for i in range(0, len(pieces), 2)]
    return pieces[0]

"""The multi-rank paths on CPU ranks (gloo, world sizes 2-4).

* the paper's merge tree (Section "MPI Merge Sort", Figs. 16-17) through
  ``dist.tree_merge_sort``: rank schedule, run exchange and merge order give
  the stable sort of the gathered array (local sort and merge are the CPU
  oracle here; on GPU ranks they are the library's kernels);
* a rank that dies before sending makes its receiver fail with an error
  within the process-group timeout instead of hanging;
* the benchmark's whole-job reductions (max time, summed work) over ranks.
"""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2211_16479_gb300 import dist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=30):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world,
                             timeout=datetime.timedelta(seconds=timeout_s))


def _oracle_sort(t):
    k, _ = oracle.sort(t.numpy())
    return torch.from_numpy(k)


def _oracle_merge(a, b):
    k, _ = oracle.merge(a.numpy(), b.numpy())
    return torch.from_numpy(k)


def _tree_worker(rank, world, port, n, q):
    _init(rank, world, port)
    try:
        keys = synth.uniform_u64(n, 3) % np.uint64(1000)   # duplicates across ranks
        size = -(-n // world)                               # ceil(n / p) chunks, ragged last
        local = torch.from_numpy(keys[rank * size:(rank + 1) * size].copy())
        out = dist.tree_merge_sort(local, local_sort=_oracle_sort, merge=_oracle_merge)
        if rank == 0:
            exp, _ = oracle.sort(keys)
            q.put(bool(np.array_equal(out.numpy(), exp)))
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_tree_merge_sort_cpu_ranks(world):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tree_worker, args=(r, world, port, 10007, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True


def test_schedule_matches_paper_for_powers_of_two():
    # the process tree of Fig. 16 with 8 ranks: 4..7 -> 0..3, then 2,3 -> 0,1, then 1 -> 0
    assert dist.merge_schedule(8) == [[(0, 4), (1, 5), (2, 6), (3, 7)], [(0, 2), (1, 3)], [(0, 1)]]
    assert dist.merge_schedule(1) == []


def _dead_worker(rank, world, port, q):
    _init(rank, world, port, timeout_s=5)
    if rank == 1:
        os._exit(3)   # dies before its send: the receiver must not hang
    try:
        dist.tree_merge_sort(torch.arange(10, dtype=torch.int64), local_sort=lambda t: t,
                             merge=lambda a, b: torch.cat([a, b]))
        q.put("finished")
    except Exception as e:  # noqa: BLE001 - any error is the expected outcome
        q.put("error:" + type(e).__name__)


def test_dead_rank_gives_error_not_hang():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung waiting for a dead peer"
    assert q.get(timeout=5).startswith("error:")


def _reduce_worker(rank, world, port, q):
    _init(rank, world, port)
    try:
        t = dist.max_over_ranks(10.0 + rank)
        s = dist.sum_over_ranks(100)
        if rank == 0:
            q.put((t, s))
    finally:
        tdist.destroy_process_group()


def test_whole_job_reductions():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reduce_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    assert q.get(timeout=5) == (11.0, 200.0)


# --- sample sort: one all-to-all exchange (the multi-GPU design) -------------
def _oracle_sort_pairs(k, v):
    kk, vv = oracle.sort(k.numpy(), v.numpy())
    return torch.from_numpy(kk), torch.from_numpy(vv)


def _oracle_merge_pairs(a, va, b, vb):
    k, v = oracle.merge(a.numpy(), b.numpy(), None if va is None else va.numpy(),
                        None if vb is None else vb.numpy())
    return torch.from_numpy(k), (None if v is None else torch.from_numpy(v))


def _oracle_merge_runs(k, v, offsets):
    # the pairwise tree of oracle merges over the runs laid end to end
    offs = [int(x) for x in offsets]
    pieces = [(k[a:b].numpy(), None if v is None else v[a:b].numpy()) for a, b in zip(offs, offs[1:])]
    while len(pieces) > 1:
        pieces = [oracle.merge(pieces[i][0], pieces[i + 1][0], pieces[i][1], pieces[i + 1][1])
                  if i + 1 < len(pieces) else pieces[i] for i in range(0, len(pieces), 2)]
    mk, mv = pieces[0]
    return torch.from_numpy(mk), (None if mv is None else torch.from_numpy(mv))


def _oracle_split_points(keys, idx, offset, split_keys, split_pos):
    pos = idx.numpy().astype(np.uint64) + np.uint64(offset)
    return torch.from_numpy(oracle.split_points(keys.numpy(), pos, split_keys.numpy(), split_pos.numpy())
                            .astype(np.int64))


def _sample_keys(kind, n):
    if kind == "uniform":
        return synth.uniform_u64(n, 5)
    if kind == "dup16":
        return synth.uniform_u64(n, 6) % np.uint64(16)
    return np.full(n, 7, dtype=np.uint64)  # all equal


def _sample_worker(rank, world, port, n, kind, q, runs=False):
    _init(rank, world, port)
    try:
        keys = _sample_keys(kind, n)
        vals = np.arange(n, dtype=np.uint32)
        # uneven chunks, one of them empty when world > 2
        cuts = [0] + sorted({(n * (r * r + 1)) // (world * world + 1) for r in range(1, world)}) + [n]
        if world > 2:
            cuts[1] = cuts[0]  # rank 0 holds nothing
        lk = torch.from_numpy(keys[cuts[rank]:cuts[rank + 1]].copy())
        lv = torch.from_numpy(vals[cuts[rank]:cuts[rank + 1]].copy())
        if runs:
            k, v = dist.sample_sort(lk, lv, local_sort=_oracle_sort_pairs, merge_runs=_oracle_merge_runs,
                                    split_points=_oracle_split_points)
        else:
            k, v = dist.sample_sort(lk, lv, local_sort=_oracle_sort_pairs, merge=_oracle_merge_pairs,
                                    split_points=_oracle_split_points)
        parts = [None] * world
        tdist.all_gather_object(parts, (k.numpy(), v.numpy()))
        if rank == 0:
            gk = np.concatenate([p[0] for p in parts])
            gv = np.concatenate([p[1] for p in parts])
            ek, ev = oracle.sort(keys, vals)
            sizes = [len(p[0]) for p in parts]
            balanced = max(sizes) <= 1.5 * n / world + 64
            q.put((bool(np.array_equal(gk, ek) and np.array_equal(gv, ev)), balanced, sizes))
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["uniform", "dup16", "equal"])
def test_sample_sort_cpu_ranks(world, kind):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sample_worker, args=(r, world, port, 20011, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    same, balanced, sizes = q.get(timeout=5)
    assert same, sizes
    assert balanced, sizes  # (key, position) splitters split runs of equal keys too


@pytest.mark.parametrize("world", [2, 3])
def test_sample_sort_cpu_ranks_merge_runs(world):
    # the received pieces merged by one merge_runs call (the GPU default)
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sample_worker, args=(r, world, port, 20011, "dup16", q, True))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    same, balanced, sizes = q.get(timeout=5)
    assert same and balanced, sizes

"""GPU parity of msort_merge (one round of the merge tree), of
msort_merge_runs (every round over runs of unequal length laid end to end)
and of the distributed sorts on one GPU rank."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import need_gpu, to_dev, to_host, torch

ms = pytest.importorskip("paper_2211_16479_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = ms.Context(0)
    yield c.handle
    c.close()


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("na,nb", [(0, 0), (0, 5), (7, 0), (1, 1), (4351, 4353), (8448, 1), (100000, 37),
                                   (1 << 20, (1 << 19) + 3)])
def test_merge_two_runs(ctx, kt, pairs, na, nb):
    if kt == "u32":
        a = np.sort(synth.uniform_u32(na, 1) % np.uint32(500))
        b = np.sort(synth.uniform_u32(nb, 2) % np.uint32(500))
    else:
        a = np.sort(synth.dup_u64(na, 1, distinct=300)[0])
        b = np.sort(synth.dup_u64(nb, 2, distinct=300)[0])
    va = np.arange(na, dtype=np.uint32) if pairs else None
    vb = np.arange(na, na + nb, dtype=np.uint32) if pairs else None
    da, db = to_dev(a), to_dev(b)
    out = torch.empty(na + nb, dtype=da.dtype, device="cuda")
    dva = to_dev(va) if pairs else None
    dvb = to_dev(vb) if pairs else None
    vout = torch.empty(na + nb, dtype=torch.uint32, device="cuda") if pairs else None
    ms.msort_merge(ctx, da, db, out, va=dva, vb=dvb, vout=vout)
    ek, ev = oracle.merge(a, b, va, vb)
    assert np.array_equal(to_host(out), ek)
    if pairs:
        assert np.array_equal(to_host(vout), ev)


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("shift", [(1, 2), (3, 1), (2, 3)])
@pytest.mark.parametrize("na,nb", [(1, 2), (37, 5), (4351, 4353), (100003, 77777)])
def test_merge_unaligned_outputs(ctx, kt, pairs, shift, na, nb):
    """Outputs (and inputs) that start 1 to 3 elements into their buffers:
    each merge block stages its outputs shifted by the destination's offset
    within 16 bytes and bulk-stores the aligned middle; the head and tail
    go by plain stores."""
    ks, vs = shift
    if kt == "u32":
        a = np.sort(synth.uniform_u32(na, 3) % np.uint32(700))
        b = np.sort(synth.uniform_u32(nb, 4) % np.uint32(700))
    else:
        a = np.sort(synth.dup_u64(na, 3, distinct=400)[0])
        b = np.sort(synth.dup_u64(nb, 4, distinct=400)[0])
    va = np.arange(na, dtype=np.uint32) if pairs else None
    vb = np.arange(na, na + nb, dtype=np.uint32) if pairs else None
    da = to_dev(np.concatenate([a[:1].repeat(ks), a]))[ks:]
    db = to_dev(np.concatenate([b[:1].repeat(vs), b]))[vs:]
    big = torch.zeros(na + nb + 8, dtype=da.dtype, device="cuda")
    out = big[ks:ks + na + nb]
    dva = to_dev(np.concatenate([np.zeros(vs, np.uint32), va]))[vs:] if pairs else None
    dvb = to_dev(np.concatenate([np.zeros(ks, np.uint32), vb]))[ks:] if pairs else None
    vbig = torch.zeros(na + nb + 8, dtype=torch.uint32, device="cuda") if pairs else None
    vout = vbig[vs:vs + na + nb] if pairs else None
    ms.msort_merge(ctx, da, db, out, va=dva, vb=dvb, vout=vout)
    ek, ev = oracle.merge(a, b, va, vb)
    got = to_host(big)
    assert np.array_equal(got[ks:ks + na + nb], ek)
    assert not got[:ks].any() and not got[ks + na + nb:].any()  # nothing written outside the view
    if pairs:
        gv = to_host(vbig)
        assert np.array_equal(gv[vs:vs + na + nb], ev)
        assert not gv[:vs].any() and not gv[vs + na + nb:].any()


def _run_lengths(seed, count, hi):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, hi, size=count)
    lens[::5] = 0  # empty runs
    return [int(x) for x in lens]


RUN_LENGTHS = [[0], [5], [0, 0, 3], [8448, 1], [4351, 0, 4353, 17], [1, 1, 1, 1, 1, 1, 1],
               _run_lengths(1, 33, 30000), _run_lengths(2, 65, 20000), _run_lengths(3, 130, 9000),
               [1 << 19, 3, (1 << 19) + 5, 8447, 100000, 0, 77777]]


@pytest.mark.parametrize("kt", ["u32", "u64"])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("lens", RUN_LENGTHS, ids=[f"runs{len(x)}_{sum(x)}" for x in RUN_LENGTHS])
def test_merge_runs(ctx, kt, pairs, lens):
    runs = []
    for i, ln in enumerate(lens):
        if kt == "u32":
            runs.append(np.sort(synth.uniform_u32(ln, 10 + i) % np.uint32(700)))
        else:
            runs.append(np.sort(synth.dup_u64(ln, 10 + i, distinct=700)[0]))
    keys = np.concatenate(runs) if runs else np.zeros(0, dtype=np.uint32)
    n = keys.size
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    # the stable merge of sorted runs in run order is the stable sort of
    # their concatenation
    ek, ev = oracle.sort(keys, vals)
    dk = to_dev(keys)
    out = torch.empty_like(dk)
    dv = to_dev(vals) if pairs else None
    vout = torch.empty_like(dv) if pairs else None
    ms.msort_merge_runs(ctx, dk, offsets, out, vals=dv, out_vals=vout)
    if n:
        assert np.array_equal(to_host(out), ek)
        assert np.array_equal(to_host(dk), keys)  # input untouched
        if pairs:
            assert np.array_equal(to_host(vout), ev)


def test_merge_runs_rejects(ctx):
    k = to_dev(np.arange(100, dtype=np.uint32))
    out = torch.empty_like(k)
    for offs, o, status in (([0, 60, 50, 100], out, ms.MSORT_ERR_INVALID_ARG),  # decreasing
                            ([5, 100], out, ms.MSORT_ERR_INVALID_ARG),  # not starting at 0
                            ([0, 50, 100], k, ms.MSORT_ERR_INVALID_ARG)):  # output overlaps input
        with pytest.raises(ms.MsortError) as e:
            ms.msort_merge_runs(ctx, k, offs, o)
        assert e.value.status == status
    f = to_dev(np.arange(100, dtype=np.float32))
    with pytest.raises(ms.MsortError) as e:
        ms.msort_merge_runs(ctx, f, [0, 50, 100], torch.empty_like(f))
    assert e.value.status == ms.MSORT_ERR_UNSUPPORTED
    ms.msort_ctx_sync(ctx)


def test_tree_merge_sort_single_gpu_rank(ctx):
    import datetime
    import os
    import socket

    import torch.distributed as tdist

    from paper_2211_16479_gb300 import dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("nccl", rank=0, world_size=1, timeout=datetime.timedelta(seconds=60))
    try:
        keys = synth.uniform_u32(300001, 4)
        out = dist.tree_merge_sort(to_dev(keys), ctx=ctx)
        assert np.array_equal(to_host(out), oracle.sort(keys)[0])
    finally:
        tdist.destroy_process_group()


def test_sample_sort_gpu_pieces_and_single_rank(ctx):
    """The sample sort's GPU building blocks (local pair sort carrying the
    local index, stable merge with values) against the oracle, and one
    single-rank NCCL run through the device collectives."""
    import datetime
    import os
    import socket

    import torch.distributed as tdist

    from paper_2211_16479_gb300 import dist
    n = 300007
    keys = synth.uniform_u64(n, 11) % np.uint64(5000)
    vals = np.arange(n, dtype=np.uint32)
    k, v = dist._gpu_sort_pairs(ctx)(to_dev(keys), to_dev(vals))
    ek, ev = oracle.sort(keys, vals)
    assert np.array_equal(to_host(k), ek) and np.array_equal(to_host(v), ev)
    a, b = ek[: n // 3], ek[n // 3:]
    va, vb = ev[: n // 3], ev[n // 3:]
    m, mv = dist._gpu_merge_pairs(ctx)(to_dev(a), to_dev(va), to_dev(b), to_dev(vb))
    em, emv = oracle.merge(a, b, va, vb)
    assert np.array_equal(to_host(m), em) and np.array_equal(to_host(mv), emv)
    # the pieces a rank receives, merged in one call
    cuts = [0, n // 7, n // 7, n // 2, n - 5, n]
    pk = np.concatenate([np.sort(keys[c0:c1]) for c0, c1 in zip(cuts, cuts[1:])])
    pv = np.arange(n, dtype=np.uint32)
    rk, rv = dist._gpu_merge_runs(ctx)(to_dev(pk), to_dev(pv), np.array(cuts, dtype=np.uint64))
    ek2, ev2 = oracle.sort(pk, pv)
    assert np.array_equal(to_host(rk), ek2) and np.array_equal(to_host(rv), ev2)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    tdist.init_process_group("nccl", rank=0, world_size=1, timeout=datetime.timedelta(seconds=60))
    try:
        sk, sv = dist.sample_sort(to_dev(keys), to_dev(vals), ctx=ctx)
        assert np.array_equal(to_host(sk), ek) and np.array_equal(to_host(sv), ev)
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_split_points_match_oracle(ctx, dtype):
    """msort_split_points: cuts of a stably sorted chunk at (key, global
    position) splitters, against the oracle's plain count; splitters equal to
    elements, between positions, below and above every key, and all-equal
    chunks."""
    rng = np.random.default_rng(17)
    for n, hi in ((0, 10), (1, 3), (1000, 4), (300007, 5000), (65536, 1)):
        keys = rng.integers(0, hi, size=n).astype(dtype)
        idx = np.arange(n, dtype=np.uint32)
        sk, si = oracle.sort(keys, idx)
        offset = 123456789012
        pos = si.astype(np.uint64) + np.uint64(offset)
        m = 257
        pick = rng.integers(0, max(n, 1), size=m)
        spl_k = np.concatenate([sk[pick] if n else np.zeros(m, dtype), [0, np.iinfo(dtype).max]]).astype(dtype)
        spl_p = np.concatenate([pos[pick] + rng.integers(0, 2, size=m).astype(np.uint64) if n
                                else np.zeros(m, np.uint64), [0, 1 << 62]]).astype(np.uint64)
        cuts = torch.zeros(len(spl_k), dtype=torch.int64, device="cuda")
        ms.msort_split_points(ctx, to_dev(sk), to_dev(si), offset, to_dev(spl_k), to_dev(spl_p), cuts)
        exp = oracle.split_points(keys, np.arange(n, dtype=np.uint64) + np.uint64(offset), spl_k, spl_p)
        assert np.array_equal(to_host(cuts).astype(np.uint64), exp), n

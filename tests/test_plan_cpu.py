"""Host-side plan logic of the plain sort (no GPU needed): tile, merge rounds,
and how the rounds map to passes over memory (pairwise or four-way)."""
import pytest

ms = pytest.importorskip("paper_2211_16479_gb300")


def _rounds(n, tile):
    r, L = 0, tile
    while L < n:
        r, L = r + 1, 2 * L
    return r


MULTI = {"single_launch": -1}  # the multi-launch plan (tile sort + a partition and a merge per round)


@pytest.mark.parametrize("n", [1, 16896, 16897, 2 * 16896 + 1, 4 * 16896 + 1, 1 << 20, 1 << 28, (1 << 28) + 1])
def test_pass_mapping(n):
    T, W, rounds = ms.msort_plan_info(n, ms.MSORT_U32, False, MULTI)
    assert T == 16896 and rounds == _rounds(n, T)
    ways, mem = ms.msort_plan_passes(n, ms.MSORT_U32, False, MULTI)
    assert ways == 2 and mem == rounds  # default: one merge round per pass
    if n > 1 << 22:  # beyond the single launch the default is this plan
        assert ms.msort_plan_info(n, ms.MSORT_U32, False) == (T, W, rounds)
    ways, mem = ms.msort_plan_passes(n, ms.MSORT_U32, False, {"merge_ways": 4})
    if rounds >= 2:
        assert ways == 4 and mem == rounds // 2 + rounds % 2
    else:
        assert ways == 2 and mem == rounds


def test_pairs_and_guided_partition_stay_pairwise():
    n = 1 << 24
    for kt in (ms.MSORT_U32, ms.MSORT_U64):
        ways, mem = ms.msort_plan_passes(n, kt, True)
        assert ways == 2 and mem == ms.msort_plan_info(n, kt, True)[2]
    ways, mem = ms.msort_plan_passes(n, ms.MSORT_U32, False, {"partition_mode": 1})
    assert ways == 2
    ways, mem = ms.msort_plan_passes(n, ms.MSORT_U32, False, {"merge_ways": 2})
    assert ways == 2 and mem == ms.msort_plan_info(n, ms.MSORT_U32, False)[2]


def test_invalid_merge_ways():
    n = 1 << 20
    with pytest.raises(ms.MsortError):
        ms.msort_plan_passes(n, ms.MSORT_U32, False, {"merge_ways": 3})
    with pytest.raises(ms.MsortError):
        ms.msort_plan_passes(n, ms.MSORT_U32, True, {"merge_ways": 4})
    with pytest.raises(ms.MsortError):
        ms.msort_plan_passes(n, ms.MSORT_U64, False, {"merge_ways": 4, "partition_mode": 2})
    assert ms.msort_scratch_bytes(n, ms.MSORT_U32, True, {"merge_ways": 4}) == 0


@pytest.mark.parametrize("kt,ks", [(ms.MSORT_U32, 4), (ms.MSORT_U64, 8)])
def test_four_way_scratch_is_small(kt, ks):
    # the four-way grid adds a few bytes per G keys on top of the ping-pong buffer
    n = 1 << 26
    s4 = ms.msort_scratch_bytes(n, kt, False, {"merge_ways": 4})
    s2 = ms.msort_scratch_bytes(n, kt, False)
    assert s2 >= n * ks and s4 > s2
    assert s4 - s2 < 0.05 * n * ks


@pytest.mark.parametrize("kt,width", [(ms.MSORT_I32, ms.MSORT_U32), (ms.MSORT_F32, ms.MSORT_U32),
                                      (ms.MSORT_I64, ms.MSORT_U64), (ms.MSORT_F64, ms.MSORT_U64)])
def test_transformed_keys_plan_like_unsigned_and_refuse_other_passes(kt, width):
    # signed and float keys sort as unsigned keys of their width after the
    # order-preserving transform, so their plans match; four-way passes and
    # the learned partition do not take transformed keys and are refused
    n = (1 << 20) + 3
    assert ms.msort_plan_info(n, kt, False) == ms.msort_plan_info(n, width, False)
    assert ms.msort_scratch_bytes(n, kt, True) == ms.msort_scratch_bytes(n, width, True)
    for opts in ({"merge_ways": 4}, {"partition_mode": 1}):
        assert ms.msort_scratch_bytes(n, kt, False, opts) == 0
        with pytest.raises(ms.MsortError) as e:
            ms.msort_plan_passes(n, kt, False, opts)
        assert e.value.status == ms.MSORT_ERR_INVALID_ARG


@pytest.mark.parametrize("n,tile", [(1, 4352), (1 << 16, 4352), (1 << 19, 4352), ((1 << 19) + 1, 8704),
                                    (1 << 20, 8704), ((1 << 20) + 1, 16896), (1 << 22, 16896)])
def test_single_launch_plan_by_size(n, tile):
    # up to 2^22 keys the default plan is one cooperative launch whose tile
    # (= merge block) depends on n; its rounds still map to one pass each
    T, W, rounds = ms.msort_plan_info(n, ms.MSORT_U32, False)
    assert (T, W) == (tile, tile) and rounds == _rounds(n, tile)
    assert ms.msort_plan_passes(n, ms.MSORT_U32, False) == (2, rounds)
    # the scratch holds the ping-pong copy and the split table, whose first
    # 8 bytes carry the grid barrier
    assert ms.msort_scratch_bytes(n, ms.MSORT_U32, False) >= n * 4 + 8


def test_single_launch_options():
    n = 1 << 20
    assert ms.msort_plan_info(n, ms.MSORT_U64, True)[0] == 4352
    assert ms.msort_plan_info(1 << 16, ms.MSORT_U64, False)[0] == 2816
    assert ms.msort_plan_info(n, ms.MSORT_U64, False)[0] == 8448
    # forced beyond the automatic limit, with a chosen single-launch tile
    assert ms.msort_plan_info(1 << 24, ms.MSORT_U32, False, {"single_launch": 1, "tile": 5632})[0] == 5632
    # options the single launch does not take fall back to the multi-launch plan ...
    assert ms.msort_plan_info(n, ms.MSORT_U32, False, {"tile": 8448})[0] == 8448
    assert ms.msort_plan_passes(n, ms.MSORT_U32, False, {"merge_ways": 4})[0] == 4
    # ... or are refused when the single launch is forced
    for bad in ({"single_launch": 3}, {"single_launch": 1, "tile": 33792}, {"single_launch": 1, "partition_mode": 2},
                {"single_launch": 1, "merge_ways": 4}, {"single_launch": 1, "merge_block": 8448}):
        with pytest.raises(ms.MsortError) as e:
            ms.msort_plan_info(n, ms.MSORT_U32, False, bad)
        assert e.value.status == ms.MSORT_ERR_INVALID_ARG
    with pytest.raises(ms.MsortError):
        ms.msort_plan_info((1 << 28) + 1, ms.MSORT_U32, False, {"single_launch": 1})

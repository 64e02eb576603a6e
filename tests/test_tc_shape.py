"""Host logic of the tensor mode's launch shapes (hot_tc_shape; no GPU): for every size the
GEMM tiles cover their matrices, every K split of the forward GEMM is non-empty and together
they cover K exactly, padding stays bounded, and the shared-memory ring of each tile width fits
the SM.  Plus the shapes of the named workloads (the ones measured in the profiles)."""
import itertools

import pytest


@pytest.fixture(scope="module")
def hot():
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot as h
    return h


SLICE = 64                                   # K elements (FP16) per 128-byte slice
RING = {32: 4 * 40, 64: 4 * 48, 128: 3 * 64, 256: 2 * 96}   # KB: stages x (2 A + 2 B tiles)


def check(s, W, H, M, sms):
    assert s["bn_back"] in RING and s["bn_fwd"] in RING
    assert s["Kb"] % SLICE == 0 and 2 * M <= s["Kb"] < 2 * M + SLICE
    assert s["Kf"] % SLICE == 0 and 2 * W <= s["Kf"] < 2 * W + SLICE
    assert s["rows_h"] % 128 == 0 and H <= s["rows_h"] < H + 128
    assert s["rows_b"] % s["bn_back"] == 0 and 2 * W <= s["rows_b"] < 2 * W + s["bn_back"]
    assert s["rows_f"] % s["bn_fwd"] == 0 and 2 * M <= s["rows_f"] < 2 * M + s["bn_fwd"]
    kc, cps, sp = s["Kf"] // SLICE, s["fwd_slices_per_split"], s["fwd_splits"]
    assert cps >= 1 and sp >= 1 and (sp - 1) * cps < kc <= sp * cps    # every split non-empty
    # a wide tile is chosen only when its padding stays within 1/8 of the 32-wide padding
    for bn, cols in ((s["bn_back"], 2 * W), (s["bn_fwd"], 2 * M)):
        if bn > 32:
            assert 8 * (-(-cols // bn) * bn) <= 9 * (-(-cols // 32) * 32)
    # the forward GEMM's CTAs do not exceed one wave when the K range is split
    tiles = (s["rows_h"] // 128) * (s["rows_f"] // s["bn_fwd"])
    if sp > 1:
        assert tiles * sp <= sms


@pytest.mark.parametrize("sms", [152, 148, 8, 1])
def test_shapes_cover_and_bound(hot, sms):
    sizes = [1, 2, 31, 33, 100, 257, 512, 1152, 1920]
    for W, H, M in itertools.product(sizes, sizes[::2], [1, 7, 100, 129, 1000, 4096]):
        check(hot.hot_tc_shape(W, H, M, sms), W, H, M, sms)


def test_named_workload_shapes(hot):
    s = hot.hot_tc_shape(1920, 1152, 1000, 152)   # profiles/gsw_tc_rand1000_1920.md
    assert (s["bn_back"], s["bn_fwd"], s["fwd_splits"]) == (256, 256, 2)
    s = hot.hot_tc_shape(512, 512, 100, 152)
    assert s["bn_back"] == 32 and s["fwd_splits"] > 1


def test_invalid_arguments(hot):
    with pytest.raises(hot.HotError, match="HOT_EINVAL"):
        hot.hot_tc_shape(0, 8, 8, 152)
    with pytest.raises(hot.HotError, match="HOT_EINVAL"):
        hot.hot_tc_shape(8, 8, 8, 0)

"""Pins of the chunking oracle (Algorithms 2, 3, 4): branch selection on
fabricated sizes, the closed-form copy costs, part invariants, and the
chunked product reproducing the plain product."""
import math

import numpy as np
import pytest

import oracle
from oracle import chunking as CH
from paper_1804_00695_gb300 import inputs as I


def uniform_rp(n, per_row):
    return np.arange(n + 1, dtype=np.int64) * per_row


def check_parts(parts, n, size_fn, psize):
    assert parts[0][0] == 0 and parts[-1][1] == n
    for (a0, a1), (b0, b1) in zip(parts, parts[1:]):
        assert a1 == b0
    for r0, r1 in parts:
        assert r1 > r0
        assert size_fn(r0, r1) <= psize
        if r1 < n:  # greedy: one more row would not fit
            assert size_fn(r0, r1 + 1) > psize


def sizes(rp, v=8):
    return CH.range_bytes(rp, 0, len(rp) - 1, v)


def test_range_bytes():
    rp = np.array([0, 3, 3, 7])
    assert CH.range_bytes(rp, 0, 3, 8) == 4 * 8 + 7 * 12
    assert CH.range_bytes(rp, 1, 2, 4) == 2 * 8


def test_branch1_b_fits():
    a, c, b = uniform_rp(1000, 10), uniform_rp(1000, 20), uniform_rp(500, 5)
    fast = 1_000_000
    pl = CH.partition(a, c, b, 8, fast)
    assert pl.branch == 1 and pl.algorithm == 3 and pl.p_b == [(0, 500)]
    small = 0.25 * fast + 0.75 * fast - sizes(b)
    tot = sizes(a) + sizes(c)
    ps = tot / math.ceil(tot / small)
    check_parts(pl.p_ac, 1000, lambda r0, r1: CH.range_bytes(a, r0, r1, 8) + CH.range_bytes(c, r0, r1, 8), ps)


def test_branch2_ac_fits():
    a, c, b = uniform_rp(100, 10), uniform_rp(100, 20), uniform_rp(5000, 30)
    fast = 1_000_000
    assert sizes(b) > 0.75 * fast and sizes(a) + sizes(c) < 0.75 * fast
    pl = CH.partition(a, c, b, 8, fast)
    assert pl.branch == 2 and pl.algorithm == 2 and pl.p_ac == [(0, 100)]
    small = fast - (sizes(a) + sizes(c))
    ps = sizes(b) / math.ceil(sizes(b) / small)
    check_parts(pl.p_b, 5000, lambda r0, r1: CH.range_bytes(b, r0, r1, 8), ps)
    assert pl.cost_chunk1 == sizes(a) + sizes(c) + sizes(b) * len(pl.p_ac)


@pytest.mark.parametrize("branch", [3, 4])
def test_branch3_4_cost_choice(branch):
    if branch == 3:   # size(A) + 2 size(C) > size(B)
        a, c, b = uniform_rp(4000, 20), uniform_rp(4000, 30), uniform_rp(4000, 25)
    else:
        a, c, b = uniform_rp(4000, 10), uniform_rp(4000, 5), uniform_rp(4000, 60)
    fast = 600_000
    sa, sb, sc = sizes(a), sizes(b), sizes(c)
    assert sb >= 0.75 * fast and sa + sc >= 0.75 * fast
    assert (sa + 2 * sc > sb) == (branch == 3)
    pl = CH.partition(a, c, b, 8, fast)
    assert pl.branch == branch
    assert pl.cost_chunk1 == sa + sc + sb * len(pl.p_ac)
    assert pl.cost_chunk2 == sb + sa * len(pl.p_b) + sc * (len(pl.p_b) - 1)
    assert pl.algorithm == (2 if pl.cost_chunk1 <= pl.cost_chunk2 else 3)
    size_ac = lambda r0, r1: CH.range_bytes(a, r0, r1, 8) + CH.range_bytes(c, r0, r1, 8)
    size_b = lambda r0, r1: CH.range_bytes(b, r0, r1, 8)
    if branch == 3:
        ps = (sa + sc) / math.ceil((sa + sc) / (0.75 * fast))
        check_parts(pl.p_ac, 4000, size_ac, ps)
        used = max(size_ac(*p) for p in pl.p_ac)
        small = 0.25 * fast + 0.75 * fast - used
        check_parts(pl.p_b, 4000, size_b, sb / math.ceil(sb / small))
    else:
        ps = sb / math.ceil(sb / (0.75 * fast))
        check_parts(pl.p_b, 4000, size_b, ps)
        used = max(size_b(*p) for p in pl.p_b)
        small = 0.25 * fast + 0.75 * fast - used
        check_parts(pl.p_ac, 4000, size_ac, (sa + sc) / math.ceil((sa + sc) / small))


def test_row_too_big_is_budget_error():
    a, c, b = uniform_rp(10, 1000), uniform_rp(10, 1000), uniform_rp(10, 1000)
    with pytest.raises(ValueError):
        CH.partition(a, c, b, 8, 10_000)


@pytest.mark.parametrize("fast", [3_000, 6_000, 20_000, 10**9])
def test_chunked_product_equals_plain(fast):
    a = I.random_csr(120, 90, 0.06, 81, shuffle_cols=True)
    b = I.random_csr(90, 110, 0.07, 82, shuffle_cols=True)
    full = oracle.spgemm(a, b)
    pl = CH.partition(a.row_ptr, full.row_ptr, b.row_ptr, 8, fast)
    rp, col, val = CH.chunked_product(a, b, pl, oracle.fma_range)
    assert np.array_equal(rp, full.row_ptr) and np.array_equal(col, full.col)
    assert np.all(np.abs(val - full.val) <= 1e-13 * full.bound)
    if fast < 10_000:
        assert len(pl.p_ac) > 1 or len(pl.p_b) > 1


@pytest.mark.parametrize("alg", [2, 3])
def test_chunked_loop_orders(alg):
    """Both loop orders (A,C in place; B in place) with several parts on
    each side give the plain product."""
    a = I.random_csr(70, 60, 0.1, 91, shuffle_cols=True)
    b = I.random_csr(60, 50, 0.1, 92, shuffle_cols=True)
    full = oracle.spgemm(a, b)
    pl = CH.Plan(alg, 0, [(0, 9), (9, 40), (40, 41), (41, 70)], [(0, 1), (1, 30), (30, 60)])
    rp, col, val = CH.chunked_product(a, b, pl, oracle.fma_range)
    assert np.array_equal(rp, full.row_ptr) and np.array_equal(col, full.col)
    assert np.all(np.abs(val - full.val) <= 1e-13 * full.bound)

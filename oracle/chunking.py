"""Oracle for the chunking decisions of Section 3.3.1 (Algorithms 2, 3, 4).

TEST INFRASTRUCTURE ONLY.  Plain Python, written from the paper's steps in the
paper's order so that the library's native planner can be compared with it
plan for plan.

Readings taken where the paper leaves details open:
  * size(X) of a row range [r0, r1) of a CSR matrix is the bytes of its arrays:
    (r1 - r0 + 1) row offsets of 8 bytes, plus (4 + value bytes) per stored
    entry; for the A/C pair it is the sum of both.
  * BinarySearch(X, pSize) cuts the rows greedily from the top: each part is
    the longest run of rows, starting where the previous part ended, whose
    size does not exceed pSize (found by bisection on the cumulative sizes).
    A single row larger than pSize is a budget error.
  * the balanced part size of a portion: np = ceil(size / portion)
    parts, pSize = size / np.
  * the leftover of the large portion goes to the small one: small += big - used, where used
    is the size of the operand placed whole (branches 1 and 2) or of the
    largest part cut from the big portion (branches 3 and 4).
  * Branch 1 calls Algorithm 3 (B in place) and branch 2 Algorithm 2 (A and C
    in place), as written; branches 3 and 4 take the algorithm with the lower
    copy cost, Algorithm 2 on a tie.
  * Where the text describing Algorithm 2 gives the rest of the fast memory to
    C, it is read as giving it to B (A and C already have the large portion).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def range_bytes(row_ptr: np.ndarray, r0: int, r1: int, vbytes: int) -> int:
    """Bytes of rows [r0, r1) of a CSR matrix: offsets + columns + values."""
    return (r1 - r0 + 1) * 8 + int(row_ptr[r1] - row_ptr[r0]) * (4 + vbytes)


def binary_search(sizes_of_range, nrows: int, psize: float):
    """BinarySearch of Algorithms 1 and 4: list of (r0, r1) row ranges."""
    parts = []
    r0 = 0
    while r0 < nrows:
        if sizes_of_range(r0, r0 + 1) > psize:
            raise ValueError("budget: one row exceeds the partition size")
        lo, hi = r0 + 1, nrows  # largest r1 in [lo, hi] with size <= psize
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if sizes_of_range(r0, mid) <= psize:
                lo = mid
            else:
                hi = mid - 1
        parts.append((r0, lo))
        r0 = lo
    if nrows == 0:
        parts.append((0, 0))
    return parts


@dataclass
class Plan:
    algorithm: int                 # 2 = kkmemGPUchunk1 (A,C in place), 3 = kkmemGPUchunk2 (B in place)
    branch: int                    # which branch of Algorithm 4 decided (1..4)
    p_ac: list = field(default_factory=list)
    p_b: list = field(default_factory=list)
    cost_chunk1: int = 0
    cost_chunk2: int = 0


def copy_cost_chunk1(size_a: int, size_b: int, size_c: int, n_ac: int) -> int:
    """Algorithm 2: size(A) + size(C) + size(B) * |P_AC|."""
    return size_a + size_c + size_b * n_ac


def copy_cost_chunk2(size_a: int, size_b: int, size_c: int, n_b: int) -> int:
    """Algorithm 3: size(B) + size(A) * |P_B| + size(C) * (|P_B| - 1)."""
    return size_b + size_a * n_b + size_c * (n_b - 1)


def partition(a_rp, c_rp, b_rp, vbytes: int, fast_size: int, b_vbytes: int | None = None) -> Plan:
    """Algorithm 4 (Partition).  a_rp, c_rp: row offsets of A and C (same
    row count); b_rp: row offsets of B."""
    b_vbytes = vbytes if b_vbytes is None else b_vbytes
    n_ac = len(a_rp) - 1
    n_b = len(b_rp) - 1

    def size_ac(r0, r1):
        return range_bytes(a_rp, r0, r1, vbytes) + range_bytes(c_rp, r0, r1, vbytes)

    def size_bb(r0, r1):
        return range_bytes(b_rp, r0, r1, b_vbytes)

    s_a = range_bytes(a_rp, 0, n_ac, vbytes)
    s_c = range_bytes(c_rp, 0, n_ac, vbytes)
    s_b = size_bb(0, n_b)
    big = 0.75 * fast_size
    small = 0.25 * fast_size

    def balanced(total, portion):
        if portion <= 0:
            raise ValueError("budget: empty portion")
        npart = max(1, math.ceil(total / portion))
        return total / npart

    if s_b < big:
        p_b = [(0, n_b)]
        small += big - s_b
        p_ac = binary_search(size_ac, n_ac, balanced(s_a + s_c, small))
        plan = Plan(3, 1, p_ac, p_b)
    elif s_a + s_c < big:
        p_ac = [(0, n_ac)]
        small += big - (s_a + s_c)
        p_b = binary_search(size_bb, n_b, balanced(s_b, small))
        plan = Plan(2, 2, p_ac, p_b)
    elif s_a + 2 * s_c > s_b:
        p_ac = binary_search(size_ac, n_ac, balanced(s_a + s_c, big))
        used = max(size_ac(r0, r1) for r0, r1 in p_ac)
        small += big - used
        p_b = binary_search(size_bb, n_b, balanced(s_b, small))
        plan = Plan(0, 3, p_ac, p_b)
    else:
        p_b = binary_search(size_bb, n_b, balanced(s_b, big))
        used = max(size_bb(r0, r1) for r0, r1 in p_b)
        small += big - used
        p_ac = binary_search(size_ac, n_ac, balanced(s_a + s_c, small))
        plan = Plan(0, 4, p_ac, p_b)
    plan.cost_chunk1 = copy_cost_chunk1(s_a, s_b, s_c, len(plan.p_ac))
    plan.cost_chunk2 = copy_cost_chunk2(s_a, s_b, s_c, len(plan.p_b))
    if plan.algorithm == 0:
        plan.algorithm = 2 if plan.cost_chunk1 <= plan.cost_chunk2 else 3
    return plan


def chunked_product(a, b, plan: Plan, fma_range):
    """Algorithms 2 and 3 run on the CPU with the Section 3.2.2 fused
    multiply-add (``fma_range`` from the oracle): returns C as
    (row_ptr, col, val).  Only the loop order differs between the two; the
    result is the same product."""
    import numpy as np  # local: keeps the module import light
    from . import _sub_rows, _cat_rows
    parts = {}
    if plan.algorithm == 2:
        for (r0, r1) in plan.p_ac:
            sub = _sub_rows(a, r0, r1)
            cur = None
            for (lo, hi) in plan.p_b:
                cur = fma_range(sub, b, lo, hi, cur)
            parts[(r0, r1)] = cur
    else:
        cur_by = {}
        for (lo, hi) in plan.p_b:
            for (r0, r1) in plan.p_ac:
                sub = _sub_rows(a, r0, r1)
                cur_by[(r0, r1)] = fma_range(sub, b, lo, hi, cur_by.get((r0, r1)))
        parts = cur_by
    return _cat_rows([parts[k] for k in sorted(parts)])

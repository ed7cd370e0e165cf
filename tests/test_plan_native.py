"""The library's native chunk planner (Algorithm 4, host code behind the C
ABI) against the plain Python oracle of the same algorithm: identical plans,
part for part, over fabricated sizes covering all four branches."""
import numpy as np
import pytest

from oracle import chunking as CH
import paper_1804_00695_gb300 as sg


def rand_rp(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, size=n)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    return rp


CASES = []
for seed in range(40):
    rng = np.random.default_rng(1000 + seed)
    n_ac, n_b = int(rng.integers(1, 3000)), int(rng.integers(1, 3000))
    a = rand_rp(n_ac, 0, int(rng.integers(1, 60)), seed)
    c = rand_rp(n_ac, 0, int(rng.integers(1, 90)), seed + 1)
    b = rand_rp(n_b, 0, int(rng.integers(1, 60)), seed + 2)
    vb = int(rng.choice([4, 8, 0]))
    tot = CH.range_bytes(a, 0, n_ac, vb) + CH.range_bytes(c, 0, n_ac, vb) + CH.range_bytes(b, 0, n_b, vb)
    fast = int(tot * float(rng.choice([0.05, 0.2, 0.5, 0.9, 1.5, 3.0])))
    CASES.append((a, c, b, vb, max(fast, 1)))
for seed in range(8):   # A and C small against a large B (branch 2)
    n_ac, n_b = 200 + 37 * seed, 4000 + 11 * seed
    a = rand_rp(n_ac, 0, 5, 500 + seed)
    c = rand_rp(n_ac, 0, 9, 600 + seed)
    b = rand_rp(n_b, 10, 40, 700 + seed)
    sa, sc, sb = (CH.range_bytes(x, 0, len(x) - 1, 8) for x in (a, c, b))
    CASES.append((a, c, b, 8, int((sa + sc) * (1.4 + 0.05 * seed))))


@pytest.mark.parametrize("k", range(len(CASES)))
def test_native_plan_matches_oracle(k):
    a, c, b, vb, fast = CASES[k]
    try:
        ref = CH.partition(a, c, b, vb, fast)
    except ValueError:
        with pytest.raises(sg.SpgemmError) as ei:
            sg.plan_chunks(a, c, b, vb, fast)
        assert ei.value.status == 5
        return
    got = sg.plan_chunks(a, c, b, vb, fast)
    assert got["branch"] == ref.branch
    assert got["algorithm"] == ref.algorithm
    assert got["p_ac"] == [tuple(x) for x in ref.p_ac]
    assert got["p_b"] == [tuple(x) for x in ref.p_b]
    assert got["cost_chunk1"] == ref.cost_chunk1 and got["cost_chunk2"] == ref.cost_chunk2


def test_all_branches_covered():
    branches = set()
    for a, c, b, vb, fast in CASES:
        try:
            branches.add(CH.partition(a, c, b, vb, fast).branch)
        except ValueError:
            pass
    assert branches == {1, 2, 3, 4}


def test_galerkin_256_plan():
    """The chunked 256^3 workload (A = B = 27-point Laplacian, C = A*A, FP64)
    under a 4 GB budget: sizes from the closed forms of the row lengths."""
    n = 256
    l1 = np.array([2] + [3] * (n - 2) + [2])            # 1D row lengths of T
    l2 = np.array([3, 4] + [5] * (n - 4) + [4, 3])      # 1D row lengths of T^2
    la = (l1[:, None, None] * l1[None, :, None] * l1[None, None, :]).reshape(-1)
    lc = (l2[:, None, None] * l2[None, :, None] * l2[None, None, :]).reshape(-1)
    a = np.zeros(n ** 3 + 1, dtype=np.int64); np.cumsum(la, out=a[1:])
    c = np.zeros(n ** 3 + 1, dtype=np.int64); np.cumsum(lc, out=c[1:])
    assert a[-1] == 449455096 and c[-1] == 2067798824
    fast = 4 * 10 ** 9
    ref = CH.partition(a, c, a, 8, fast)
    got = sg.plan_chunks(a, c, a, 8, fast)
    assert got["branch"] == ref.branch == 3 and got["algorithm"] == ref.algorithm == 2
    assert got["p_ac"] == [tuple(x) for x in ref.p_ac] and got["p_b"] == [tuple(x) for x in ref.p_b]

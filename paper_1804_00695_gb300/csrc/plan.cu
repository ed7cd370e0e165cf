// Chunking decision of Section 3.3.1: BinarySearch row partitioning and the
// Partition heuristic (Algorithm 4) choosing between Algorithm 2 (A and C in
// place, B streamed) and Algorithm 3 (B in place, A and C streamed) by their
// copy costs.  Host code only.
//
// Readings where the paper leaves details open:
//  - size(X) of rows [r0, r1) is the bytes of the CSR arrays: (r1-r0+1)
//    offsets of 8 bytes plus (4 + value bytes) per entry; for the A/C pair
//    the sum of both.
//  - BinarySearch cuts greedily from the top: each part is the longest run of
//    rows from the previous cut whose size does not exceed pSize (bisection
//    on the cumulative sizes); a row larger than pSize is a budget error.
//  - the balanced part size of a portion: np = ceil(size/portion) parts,
//    pSize = size/np.
//  - the leftover of the large portion goes to the small one:
//    small += big - used, used =
//    the operand placed whole (branches 1, 2) or the largest part cut from
//    the big portion (branches 3, 4).
//  - Branch 1 calls Algorithm 3 and branch 2 Algorithm 2 as written;
//    branches 3 and 4 take the lower copy cost, Algorithm 2 on a tie.
#include <cmath>
#include <vector>
#include "internal.cuh"

namespace sg {

static int64_t rbytes(const int64_t *rp, int64_t r0, int64_t r1, int vb) {
    return (r1 - r0 + 1) * 8 + (rp[r1] - rp[r0]) * (int64_t)(4 + vb);
}

struct SizeFn {
    const int64_t *rp1, *rp2;   // rp2 may be null (single matrix)
    int vb1, vb2;
    int64_t operator()(int64_t r0, int64_t r1) const {
        int64_t s = rbytes(rp1, r0, r1, vb1);
        if (rp2) s += rbytes(rp2, r0, r1, vb2);
        return s;
    }
};

// Greedy bisection cuts; returns false if one row exceeds psize.
static bool binary_search(const SizeFn &f, int64_t nrows, double psize,
                          std::vector<int64_t> &cuts) {
    cuts.clear();
    int64_t r0 = 0;
    if (nrows == 0) {
        cuts.push_back(0);
        cuts.push_back(0);
        return true;
    }
    cuts.push_back(0);
    while (r0 < nrows) {
        if ((double)f(r0, r0 + 1) > psize) return false;
        int64_t lo = r0 + 1, hi = nrows;
        while (lo < hi) {
            int64_t mid = (lo + hi + 1) / 2;
            if ((double)f(r0, mid) <= psize) lo = mid;
            else hi = mid - 1;
        }
        cuts.push_back(lo);
        r0 = lo;
    }
    return true;
}

bool cut_rows(const int64_t *rp1, const int64_t *rp2, int64_t n, int vb, double psize,
              std::vector<int64_t> &cuts) {
    SizeFn f{rp1, rp2, vb, vb};
    return binary_search(f, n, psize, cuts);
}

static double balanced(int64_t total, double portion) {
    double np = std::ceil((double)total / portion);
    if (np < 1) np = 1;
    return (double)total / np;
}

int plan_chunks(const int64_t *a_rp, int64_t n_ac, const int64_t *c_rp, const int64_t *b_rp,
                int64_t n_b, int vb_ac, int vb_b, int64_t fast, ChunkPlan &p) {
    if (fast <= 0) {
        set_error("chunk plan: budget must be positive");
        return SPGEMM_ERR_BUDGET;
    }
    SizeFn fac{a_rp, c_rp, vb_ac, vb_ac};
    SizeFn fb{b_rp, nullptr, vb_b, 0};
    p.size_a = rbytes(a_rp, 0, n_ac, vb_ac);
    p.size_c = rbytes(c_rp, 0, n_ac, vb_ac);
    p.size_b = rbytes(b_rp, 0, n_b, vb_b);
    const int64_t sa = p.size_a, sb = p.size_b, sc = p.size_c;
    double big = 0.75 * (double)fast, small = 0.25 * (double)fast;
    bool ok = true;
    p.algorithm = 0;
    if ((double)sb < big) {
        p.branch = 1;
        p.b_cuts = {0, n_b};
        small += big - (double)sb;
        ok = binary_search(fac, n_ac, balanced(sa + sc, small), p.ac_cuts);
        p.algorithm = 3;
    } else if ((double)(sa + sc) < big) {
        p.branch = 2;
        p.ac_cuts = {0, n_ac};
        small += big - (double)(sa + sc);
        ok = binary_search(fb, n_b, balanced(sb, small), p.b_cuts);
        p.algorithm = 2;
    } else if (sa + 2 * sc > sb) {
        p.branch = 3;
        ok = binary_search(fac, n_ac, balanced(sa + sc, big), p.ac_cuts);
        if (ok) {
            int64_t used = 0;
            for (size_t j = 0; j + 1 < p.ac_cuts.size(); j++)
                used = std::max(used, fac(p.ac_cuts[j], p.ac_cuts[j + 1]));
            small += big - (double)used;
            ok = binary_search(fb, n_b, balanced(sb, small), p.b_cuts);
        }
    } else {
        p.branch = 4;
        ok = binary_search(fb, n_b, balanced(sb, big), p.b_cuts);
        if (ok) {
            int64_t used = 0;
            for (size_t j = 0; j + 1 < p.b_cuts.size(); j++)
                used = std::max(used, fb(p.b_cuts[j], p.b_cuts[j + 1]));
            small += big - (double)used;
            ok = binary_search(fac, n_ac, balanced(sa + sc, small), p.ac_cuts);
        }
    }
    if (!ok) {
        set_error("chunk plan: a single row does not fit its portion of the %lld-byte budget",
                  (long long)fast);
        return SPGEMM_ERR_BUDGET;
    }
    const int64_t nac = (int64_t)p.ac_cuts.size() - 1, nb = (int64_t)p.b_cuts.size() - 1;
    p.cost1 = sa + sc + sb * nac;                 // Algorithm 2
    p.cost2 = sb + sa * nb + sc * (nb - 1);       // Algorithm 3
    if (p.algorithm == 0) p.algorithm = p.cost1 <= p.cost2 ? 2 : 3;
    return SPGEMM_OK;
}

}  // namespace sg

using namespace sg;

extern "C" int spgemm_plan_chunks(const int64_t *A_row_ptr, int64_t nrows_A, const int64_t *C_row_ptr,
                                  const int64_t *B_row_ptr, int64_t nrows_B, int value_bytes,
                                  int64_t fast_size, spgemm_chunk_plan *plan) {
    if (!A_row_ptr || !C_row_ptr || !B_row_ptr || !plan || nrows_A < 0 || nrows_B < 0 ||
        value_bytes < 0) {
        set_error("spgemm_plan_chunks: bad arguments");
        return SPGEMM_ERR_ARG;
    }
    ChunkPlan p;
    SG_TRY(plan_chunks(A_row_ptr, nrows_A, C_row_ptr, B_row_ptr, nrows_B, value_bytes, value_bytes,
                       fast_size, p));
    plan->algorithm = p.algorithm;
    plan->branch = p.branch;
    plan->n_ac = (int64_t)p.ac_cuts.size() - 1;
    plan->n_b = (int64_t)p.b_cuts.size() - 1;
    plan->size_a = p.size_a;
    plan->size_b = p.size_b;
    plan->size_c = p.size_c;
    plan->cost_chunk1 = p.cost1;
    plan->cost_chunk2 = p.cost2;
    if (plan->ac_cuts && plan->cap_ac >= plan->n_ac + 1)
        for (int64_t j = 0; j <= plan->n_ac; j++) plan->ac_cuts[j] = p.ac_cuts[j];
    if (plan->b_cuts && plan->cap_b >= plan->n_b + 1)
        for (int64_t j = 0; j <= plan->n_b; j++) plan->b_cuts[j] = p.b_cuts[j];
    return SPGEMM_OK;
}

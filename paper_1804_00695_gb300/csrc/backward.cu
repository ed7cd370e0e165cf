// Gradients of a sparse product with respect to the stored values of its
// operands.  With L a scalar function of C = A*B and dC = dL/dC given on the
// pattern of C, the product is bilinear, so
//     dA_ik = sum over stored b_kj of dC_ij * b_kj        (dC * B^T on pattern(A))
//     dB_kj = sum over stored a_ik of a_ik * dC_ij        (A^T * dC on pattern(B))
// Both come out of one pass over the same products as the forward product:
// for each stored a_ik and each stored b_kj, dC_ij is found in row i of C
// (columns ascending) by binary search; the dA terms of a_ik are summed by
// the lanes walking B_k (a segmented sum across the lanes, one update per
// a_ik and step), and the dB terms are added atomically into the slot of
// b_kj (its position in B is the loop index).  No dense intermediate.
// Rows of C with at most BWD_CAP entries are searched in a copy of their
// columns in shared memory (a warp per row, products dealt out over the
// lanes); longer rows are searched in global memory.
#include "internal.cuh"

namespace sg {

// Position of column j in the sorted row col[c0, c1), or -1.
__device__ __forceinline__ int64_t find_col(const int32_t *__restrict__ col, int64_t c0, int64_t c1, int j) {
    int64_t lo = c0, hi = c1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < c1 && col[lo] == j) ? lo : -1;
}

// A warp per row of A whose row of C has at most BWD_CAP entries: the
// columns of C_i are copied to shared memory, the products a_ik * b_kj of
// the row are dealt out over the lanes through prefix sums of nnz(B_k)
// (stored a_ik staged BWD_E at a time), each lane finds dC_ij by binary
// search in the copy, adds its dA term into the staged entry's accumulator
// and its dB term atomically into db.
constexpr int BWD_CAP = 1024, BWD_WPB = 8, BWD_E = 32;

template <typename V>
__global__ void __launch_bounds__(BWD_WPB * 32) k_backward_rows(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const V *__restrict__ aval, const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol,
    const V *__restrict__ bval, const int64_t *__restrict__ crp, const int32_t *__restrict__ ccol,
    const V *__restrict__ dc, V *__restrict__ da, V *__restrict__ db, int *err) {
    __shared__ int cs_all[BWD_WPB * BWD_CAP];
    __shared__ long long eq0_all[BWD_WPB * BWD_E];
    __shared__ V ea_all[BWD_WPB * BWD_E];
    __shared__ V dacc_all[BWD_WPB * BWD_E];
    __shared__ int pre_all[BWD_WPB * (BWD_E + 1)];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *cs = cs_all + w * BWD_CAP;
    long long *eq0 = eq0_all + w * BWD_E;
    V *ea = ea_all + w * BWD_E;
    V *dacc = dacc_all + w * BWD_E;
    int *pre = pre_all + w * (BWD_E + 1);
    bool missing = false;
    for (int64_t i = (int64_t)blockIdx.x * BWD_WPB + w; i < nrows; i += (int64_t)gridDim.x * BWD_WPB) {
        const int64_t c0 = crp[i];
        const int64_t nc64 = crp[i + 1] - c0;
        if (nc64 > BWD_CAP) continue;   // searched in global memory by k_backward
        const int nc = (int)nc64;
        const int64_t p0 = arp[i];
        const int plen = (int)(arp[i + 1] - p0);
        if (plen == 0) continue;
        for (int x = lane; x < nc; x += 32) cs[x] = ccol[c0 + x];
        __syncwarp();
        for (int pb = 0; pb < plen; pb += BWD_E) {
            int len = 0;
            if (pb + lane < plen) {
                const int k = acol[p0 + pb + lane];
                const int64_t q0 = brp[k];
                eq0[lane] = q0;
                len = (int)(brp[k + 1] - q0);
                ea[lane] = aval ? aval[p0 + pb + lane] : V(0);
            }
            dacc[lane] = V(0);
            int incl = len;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            pre[lane] = incl - len;
            if (lane == 31) pre[BWD_E] = incl;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            int e = 0;
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int t = t0 + lane;
                V term = V(0);
                const bool live = t < total;
                if (live) {
                    while (pre[e + 1] <= t) e++;
                    const int64_t q = eq0[e] + (t - pre[e]);
                    const int j = bcol[q];
                    int lo = 0, hi = nc;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (cs[mid] < j) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo < nc && cs[lo] == j) {
                        const V g = dc[c0 + lo];
                        if (bval) term = g * bval[q];
                        if (db) atomicAdd(&db[q], ea[e] * g);
                    } else {
                        missing = true;
                    }
                }
                if (bval) {
                    // the lanes of one staged a_ik are consecutive: a segmented
                    // sum over them leaves its dA term in the segment's first
                    // lane, which alone updates the entry's accumulator
                    const unsigned grp = __match_any_sync(0xffffffffu, live ? e : -1 - lane);
                    const int last = 31 - __clz(grp);
                    for (int d = 1; d < 32; d <<= 1) {
                        const V y = __shfl_down_sync(0xffffffffu, term, d);
                        if (lane + d <= last) term += y;
                    }
                    if (live && lane == __ffs(grp) - 1) dacc[e] += term;
                    __syncwarp();
                }
            }
            __syncwarp();
            if (da && pb + lane < plen) da[p0 + pb + lane] = dacc[lane];
            __syncwarp();
        }
    }
    if (missing) atomicOr(err, DERR_COUNT);
}

// G lanes per row of A whose row of C has more than skip_cap entries: for
// each stored a_ik in turn the lanes walk B_k, each looks up dC_ij in global
// memory, and the group reduces the dA term.
template <typename V, int G>
__global__ void __launch_bounds__(256, 4) k_backward(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const V *__restrict__ aval, const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol,
    const V *__restrict__ bval, const int64_t *__restrict__ crp, const int32_t *__restrict__ ccol,
    const V *__restrict__ dc, V *__restrict__ da, V *__restrict__ db, int *err, int64_t skip_cap) {
    const int gl = threadIdx.x % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1)));
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    bool missing = false;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < nrows; i += groups) {
        const int64_t c0 = crp[i], c1 = crp[i + 1];
        if (c1 - c0 <= skip_cap) continue;
        for (int64_t p = arp[i]; p < arp[i + 1]; p++) {
            const int k = acol[p];
            const V a = aval ? aval[p] : V(0);
            V acc = V(0);
            for (int64_t q = brp[k] + gl; q < brp[k + 1]; q += G) {
                const int64_t pos = find_col(ccol, c0, c1, bcol[q]);
                if (pos < 0) {
                    missing = true;
                    continue;
                }
                const V g = dc[pos];
                if (bval) acc += g * bval[q];
                if (db) atomicAdd(&db[q], a * g);
            }
            for (int d = G / 2; d > 0; d >>= 1) acc += __shfl_xor_sync(gmask, acc, d, G);
            if (da && gl == 0) da[p] = acc;
        }
    }
    if (missing) atomicOr(err, DERR_COUNT);
}

template <typename V>
static int run_bwd(const spgemm_csr &A, const spgemm_csr &B, const spgemm_csr &C, void *da, void *db,
                   int *err, int G, Ctx &c) {
    if (db) SG_CUDA(cudaMemsetAsync(db, 0, (size_t)B.nnz * sizeof(V), c.s));
    if (A.nrows == 0) return SPGEMM_OK;
    int64_t rblocks = (A.nrows + BWD_WPB - 1) / BWD_WPB;
    rblocks = rblocks < (int64_t)c.nsm * 16 ? rblocks : (int64_t)c.nsm * 16;
    c.begin("backward", A.nrows);
    k_backward_rows<V><<<(unsigned)rblocks, BWD_WPB * 32, 0, c.s>>>(
        A.nrows, A.row_ptr, A.col_idx, (const V *)A.values, B.row_ptr, B.col_idx,
        da ? (const V *)B.values : nullptr, C.row_ptr, C.col_idx, (const V *)C.values, (V *)da, (V *)db, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    int64_t blocks = (A.nrows * G + 255) / 256;
    blocks = blocks < (int64_t)c.nsm * 32 ? blocks : (int64_t)c.nsm * 32;
    c.begin("backward_long", A.nrows);
#define SG_BWD(GG)                                                                                   \
    k_backward<V, GG><<<(unsigned)blocks, 256, 0, c.s>>>(                                            \
        A.nrows, A.row_ptr, A.col_idx, (const V *)A.values, B.row_ptr, B.col_idx,                   \
        da ? (const V *)B.values : nullptr, C.row_ptr, C.col_idx, (const V *)C.values, (V *)da,      \
        (V *)db, err, (int64_t)BWD_CAP)
    switch (G) {
        case 4: SG_BWD(4); break;
        case 8: SG_BWD(8); break;
        case 16: SG_BWD(16); break;
        default: SG_BWD(32);
    }
#undef SG_BWD
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

int launch_backward(int dtype, const spgemm_csr &A, const spgemm_csr &B, const spgemm_csr &C, void *da,
                    void *db, int *err, Ctx &c) {
    const double mean_b = B.nrows ? (double)B.nnz / (double)B.nrows : 1.0;
    int G = 4;
    while (G < 32 && 2 * G <= mean_b) G *= 2;
    return dtype == SPGEMM_F64 ? run_bwd<double>(A, B, C, da, db, err, G, c)
                               : run_bwd<float>(A, B, C, da, db, err, G, c);
}

}  // namespace sg

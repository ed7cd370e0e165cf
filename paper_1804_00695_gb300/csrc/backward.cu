// Gradients of a sparse product with respect to the stored values of its
// operands.  With L a scalar function of C = A*B and dC = dL/dC given on the
// pattern of C, the product is bilinear, so
//     dA_ik = sum over stored b_kj of dC_ij * b_kj        (dC * B^T on pattern(A))
//     dB_kj = sum over stored a_ik of a_ik * dC_ij        (A^T * dC on pattern(B))
// Both come out of one pass over the same products as the forward product:
// for each stored a_ik and each stored b_kj, dC_ij is found in row i of C
// (columns ascending) by binary search; the dA terms of a_ik are summed by
// the lanes walking B_k, and the dB terms are added atomically into the slot
// of b_kj (its position in B is the loop index).  No dense intermediate.
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

// G lanes per row of A: for each stored a_ik in turn the lanes walk B_k,
// each looks up dC_ij, and the group reduces the dA term.
template <typename V, int G>
__global__ void __launch_bounds__(256, 4) k_backward(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const V *__restrict__ aval, const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol,
    const V *__restrict__ bval, const int64_t *__restrict__ crp, const int32_t *__restrict__ ccol,
    const V *__restrict__ dc, V *__restrict__ da, V *__restrict__ db, int *err) {
    const int gl = threadIdx.x % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1)));
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    bool missing = false;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < nrows; i += groups) {
        const int64_t c0 = crp[i], c1 = crp[i + 1];
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
    int64_t blocks = (A.nrows * G + 255) / 256;
    blocks = blocks < (int64_t)c.nsm * 32 ? blocks : (int64_t)c.nsm * 32;
    c.begin("backward", A.nrows);
#define SG_BWD(GG)                                                                                   \
    k_backward<V, GG><<<(unsigned)blocks, 256, 0, c.s>>>(                                            \
        A.nrows, A.row_ptr, A.col_idx, (const V *)A.values, B.row_ptr, B.col_idx,                   \
        da ? (const V *)B.values : nullptr, C.row_ptr, C.col_idx, (const V *)C.values, (V *)da,      \
        (V *)db, err)
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

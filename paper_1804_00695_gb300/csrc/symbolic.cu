// Symbolic phase (Section 2.1): nnz(C_i) = | union over stored a_ik of the
// column set of B_k |, computed on compressed column sets: every set is a
// list of (block = col/32, 32-bit mask) pairs, a union is a hash map from
// block to the OR of its masks, and the count is the sum of popcounts
// (Section 2.1, compression makes union a bitwise operation).  Rows are
// binned by the number of keys their map can hold (Section 3.3): bins 1-3
// give a group of 8, 16 or 32 lanes to a row, bins 4-5 a whole block with a
// shared-memory map, bin 6 a block with a dense bitmap over all blocks of
// columns (shared memory when it fits, otherwise global memory).
#include <climits>
#include "internal.cuh"

namespace sg {

template <int S>
__device__ __forceinline__ bool sym_insert(int *keys, unsigned *masks, int blk, unsigned m) {
    constexpr int L = __builtin_ctz(S);
    unsigned h = hash_slot(blk, L);
#pragma unroll 1
    for (int probe = 0; probe < S; probe++) {
        int k = ((volatile int *)keys)[h];
        if (k == blk) {
            atomicOr(&masks[h], m);
            return true;
        }
        if (k == -1) {
            int old = atomicCAS(&keys[h], -1, blk);
            if (old == -1 || old == blk) {
                atomicOr(&masks[h], m);
                return true;
            }
        }
        h = (h + 1) & (S - 1);
    }
    return false;
}

// G lanes per row, S slots per row; each lane walks its share of the row's
// stored a_ik (stride G) and inserts every compressed pair of B_k.
template <int G, int S>
__global__ void __launch_bounds__(256) k_sym_group(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ ccnt,
    const int2 *__restrict__ pairs, const int32_t *__restrict__ rows, int64_t count,
    int64_t *__restrict__ crp, int *err) {
    constexpr int GPB = 256 / G;
    extern __shared__ int smem[];
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    int *keys = smem + g * S;
    unsigned *masks = (unsigned *)(smem + GPB * S) + g * S;
    const unsigned gmask = (G == 32) ? 0xffffffffu
                                     : (((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1)));
    bool fail = false;
    for (int64_t t = (int64_t)blockIdx.x * GPB + g; t < count; t += (int64_t)gridDim.x * GPB) {
        const int i = rows[t];
        for (int s = lane; s < S; s += G) {
            keys[s] = -1;
            masks[s] = 0;
        }
        __syncwarp(gmask);
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + lane; p < pe; p += G) {
            const int k = acol[p];
            const int64_t q0 = brp[k];
            const int n = ccnt[k];
            for (int q = 0; q < n; q++) {
                int2 pr = pairs[q0 + q];
                fail |= !sym_insert<S>(keys, masks, pr.x, (unsigned)pr.y);
            }
        }
        __syncwarp(gmask);
        int c = 0;
        for (int s = lane; s < S; s += G) c += __popc(masks[s]);
        for (int d = G / 2; d > 0; d >>= 1) c += __shfl_xor_sync(gmask, c, d, G);
        if (lane == 0) crp[i + 1] = c;
        __syncwarp(gmask);
    }
    if (fail) atomicOr(err, DERR_PROBE);
}

// A whole block per row; each warp takes stored a_ik in turn and its lanes
// stride over the pairs of B_k.
template <int BS, int S>
__global__ void __launch_bounds__(BS) k_sym_block(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ ccnt,
    const int2 *__restrict__ pairs, const int32_t *__restrict__ rows, int64_t count,
    int64_t *__restrict__ crp, int *err) {
    extern __shared__ int smem[];
    __shared__ int red[BS / 32];
    int *keys = smem;
    unsigned *masks = (unsigned *)(smem + S);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool fail = false;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        for (int s = threadIdx.x; s < S; s += BS) {
            keys[s] = -1;
            masks[s] = 0;
        }
        __syncthreads();
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += BS / 32) {
            const int k = acol[p];
            const int64_t q0 = brp[k];
            const int n = ccnt[k];
            for (int q = lane; q < n; q += 32) {
                int2 pr = pairs[q0 + q];
                fail |= !sym_insert<S>(keys, masks, pr.x, (unsigned)pr.y);
            }
        }
        __syncthreads();
        int c = 0;
        for (int s = threadIdx.x; s < S; s += BS) c += __popc(masks[s]);
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) red[w] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int j = 0; j < BS / 32; j++) tot += red[j];
            crp[i + 1] = tot;
        }
        __syncthreads();
    }
    if (fail) atomicOr(err, DERR_PROBE);
}

// Dense bitmap of all column blocks (one word per block of 32 columns).
template <int BS>
__global__ void __launch_bounds__(BS) k_sym_bitmap(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ ccnt,
    const int2 *__restrict__ pairs, const int32_t *__restrict__ rows, int64_t count,
    int64_t *__restrict__ crp, int64_t nwords, unsigned *gbits) {
    extern __shared__ unsigned sbits[];
    __shared__ long long red[BS / 32];
    unsigned *bits = gbits ? gbits + (size_t)blockIdx.x * (size_t)nwords : sbits;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        for (int64_t s = threadIdx.x; s < nwords; s += BS) bits[s] = 0;
        __syncthreads();
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += BS / 32) {
            const int k = acol[p];
            const int64_t q0 = brp[k];
            const int n = ccnt[k];
            for (int q = lane; q < n; q += 32) {
                int2 pr = pairs[q0 + q];
                atomicOr(&bits[pr.x], (unsigned)pr.y);
            }
        }
        __syncthreads();
        long long c = 0;
        for (int64_t s = threadIdx.x; s < nwords; s += BS) c += __popc(bits[s]);
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) red[w] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tot = 0;
            for (int j = 0; j < BS / 32; j++) tot += red[j];
            crp[i + 1] = tot;
        }
        __syncthreads();
    }
}

constexpr int BITMAP_BS = 512;
constexpr int64_t SMEM_BITMAP_WORDS = 53248;  // 208 KiB of shared memory

size_t symbolic_global_ws(int64_t ncols_b, int nsm) {
    int64_t nwords = (ncols_b + 31) / 32;
    if (nwords <= SMEM_BITMAP_WORDS) return 0;
    return (size_t)nwords * 4 * (size_t)nsm;
}

// Opt in to the dynamic shared memory a launch needs (static shared memory
// comes on top, so the attribute is set for every non-trivial size).
template <typename K>
static int prep(K kern, size_t smem) {
    if (smem > 16 * 1024)
        SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return SPGEMM_OK;
}

static const char *SYM_LABEL[NBINS] = {"", "symbolic.bin1", "symbolic.bin2", "symbolic.bin3",
                                       "symbolic.bin4", "symbolic.bin5", "symbolic.bin6", ""};

template <int G, int S>
static int run_group(const spgemm_csr &A, const int64_t *brp, const int32_t *ccnt, const int2 *pairs,
                     const int32_t *rows, int64_t count, int64_t *crp, int *err, int b, Ctx &c) {
    constexpr int GPB = 256 / G;
    size_t smem = (size_t)GPB * S * 8;
    SG_TRY(prep(k_sym_group<G, S>, smem));
    int64_t blocks = (count + GPB - 1) / GPB;
    blocks = blocks < (int64_t)c.nsm * 64 ? blocks : (int64_t)c.nsm * 64;
    c.begin(SYM_LABEL[b], count);
    k_sym_group<G, S><<<(unsigned)blocks, 256, smem, c.s>>>(A.row_ptr, A.col_idx, brp, ccnt, pairs,
                                                             rows, count, crp, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int BS, int S>
static int run_block(const spgemm_csr &A, const int64_t *brp, const int32_t *ccnt, const int2 *pairs,
                     const int32_t *rows, int64_t count, int64_t *crp, int *err, int b, Ctx &c) {
    size_t smem = (size_t)S * 8;
    SG_TRY(prep(k_sym_block<BS, S>, smem));
    int64_t blocks = count < (int64_t)c.nsm * 16 ? count : (int64_t)c.nsm * 16;
    c.begin(SYM_LABEL[b], count);
    k_sym_block<BS, S><<<(unsigned)blocks, BS, smem, c.s>>>(A.row_ptr, A.col_idx, brp, ccnt, pairs,
                                                            rows, count, crp, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

int launch_symbolic(const spgemm_csr &A, const spgemm_csr &B, const int2 *pairs,
                    const int32_t *ccnt, const int32_t *rows, const long long *counts,
                    int64_t *crp, int *err, void *gws, size_t gws_bytes, Ctx &c) {
    const int nsm = c.nsm;
    int64_t off = 0;
    const int64_t *brp = B.row_ptr;
    for (int b = 1; b < NBINS; b++) {
        int64_t cnt = counts[b];
        const int32_t *r = rows + off;
        off += cnt;
        if (cnt == 0) continue;
        switch (b) {
            case 1: SG_TRY((run_group<8, 32>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c))); break;
            case 2: SG_TRY((run_group<16, 128>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c))); break;
            case 3: SG_TRY((run_group<32, 512>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c))); break;
            case 4: SG_TRY((run_block<128, 2048>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c))); break;
            case 5: SG_TRY((run_block<256, 8192>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c))); break;
            default: {
                int64_t nwords = (B.ncols + 31) / 32;
                bool shared = nwords <= SMEM_BITMAP_WORDS;
                size_t smem = shared ? (size_t)nwords * 4 : 0;
                SG_TRY(prep(k_sym_bitmap<BITMAP_BS>, shared ? smem : 0));
                int64_t blocks = cnt < (int64_t)nsm ? cnt : (int64_t)nsm;
                if (!shared && gws_bytes < (size_t)blocks * (size_t)nwords * 4) {
                    set_error("symbolic: global bitmap workspace too small");
                    return SPGEMM_ERR_INTERNAL;
                }
                c.begin(SYM_LABEL[b], cnt);
                k_sym_bitmap<BITMAP_BS><<<(unsigned)blocks, BITMAP_BS, smem, c.s>>>(
                    A.row_ptr, A.col_idx, brp, ccnt, pairs, r, cnt, crp, nwords,
                    shared ? nullptr : (unsigned *)gws);
                c.end();
                SG_CUDA(cudaGetLastError());
            }
        }
    }
    return SPGEMM_OK;
}

}  // namespace sg

// Numeric phase (Section 2.1): C_i = sum over stored a_ik of a_ik * B_k,
// accumulated in hash maps from column to value (Section 2.1, "sparse
// hashmap-based accumulators"); the first level lives in shared memory and,
// for the largest rows, a second level in global memory takes what the first
// cannot hold (Section 3.3).  Every row's map is sized from its exact count
// (known from the symbolic phase), so bins 1-5 never overflow.  Output rows
// are written with ascending columns: small rows are ranked by counting,
// larger ones sorted with a bitonic network in shared memory, and the
// largest ranked through a bitmap of their columns.
#include <climits>
#include "internal.cuh"

namespace sg {

template <typename V>
__device__ __forceinline__ void atomic_add_v(V *p, V v) { atomicAdd(p, v); }

// Insert (col, v) into a map of 2^L slots; returns false when `limit`
// probes found neither the key nor a free slot.
template <typename V>
__device__ __forceinline__ bool num_insert(int *keys, V *vals, int L, int limit, int col, V v) {
    const unsigned msk = (1u << L) - 1;
    unsigned h = hash_slot(col, L);
#pragma unroll 1
    for (int probe = 0; probe < limit; probe++) {
        int k = ((volatile int *)keys)[h];
        if (k == col) {
            atomic_add_v(&vals[h], v);
            return true;
        }
        if (k == -1) {
            int old = atomicCAS(&keys[h], -1, col);
            if (old == -1 || old == col) {
                atomic_add_v(&vals[h], v);
                return true;
            }
        }
        h = (h + 1) & msk;
    }
    return false;
}

// Bitonic sort of P (power of two) keys with values, in shared memory, by
// NT cooperating threads (tid in [0, NT)); sync() separates the stages.
template <typename V, typename Sync>
__device__ __forceinline__ void bitonic(int *k, V *v, int P, int tid, int NT, Sync sync) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < P / 2; t += NT) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool asc = (lo & size) == 0;
                int a = k[lo], b = k[hi];
                if ((a > b) == asc) {
                    k[lo] = b;
                    k[hi] = a;
                    V tv = v[lo];
                    v[lo] = v[hi];
                    v[hi] = tv;
                }
            }
            sync();
        }
    }
}

__device__ __forceinline__ int next_pow2(int n) { return n <= 1 ? 1 : 1 << (32 - __clz(n - 1)); }

// G lanes per row, S map slots, S/2 compacted entries.  RANK selects
// ranking by counting (cheap for a handful of entries) over bitonic sorting.
template <int G, int S, bool RANK, typename V>
__global__ void __launch_bounds__(256) k_num_group(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol, const V *__restrict__ aval,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, const V *__restrict__ bval,
    const int64_t *__restrict__ crp, int32_t *__restrict__ ccol, V *__restrict__ cval,
    const int32_t *__restrict__ rows, int64_t count, int *err) {
    constexpr int GPB = 256 / G;
    constexpr int L = __builtin_ctz(S);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *vals_all = (V *)smem_raw;                                   // GPB*S
    V *cv_all = vals_all + GPB * S;                                // GPB*S/2
    int *keys_all = (int *)(cv_all + GPB * S / 2);                 // GPB*S
    int *ck_all = keys_all + GPB * S;                              // GPB*S/2
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    int *keys = keys_all + g * S;
    V *vals = vals_all + g * S;
    int *ck = ck_all + g * (S / 2);
    V *cv = cv_all + g * (S / 2);
    const int gbase = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1) << gbase);
    int flag = 0;
    for (int64_t t = (int64_t)blockIdx.x * GPB + g; t < count; t += (int64_t)gridDim.x * GPB) {
        const int i = rows[t];
        for (int s = lane; s < S; s += G) {
            keys[s] = -1;
            vals[s] = V(0);
        }
        __syncwarp(gmask);
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + lane; p < pe; p += G) {
            const int k = acol[p];
            const V a = aval[p];
            const int64_t q1 = brp[k + 1];
            for (int64_t q = brp[k]; q < q1; q++) {
                if (!num_insert<V>(keys, vals, L, S, bcol[q], a * bval[q])) flag |= DERR_PROBE;
            }
        }
        __syncwarp(gmask);
        // Compact the occupied slots (slot order).
        int n = 0;
        for (int s0 = 0; s0 < S; s0 += G) {
            int s = s0 + lane;
            int key = keys[s];
            bool occ = key != -1;
            unsigned b = __ballot_sync(gmask, occ) >> gbase;
            if (occ) {
                int pos = n + __popc(b & ((1u << lane) - 1));
                if (pos < S / 2) {
                    ck[pos] = key;
                    cv[pos] = vals[s];
                }
            }
            n += __popc(b);
        }
        const int64_t out = crp[i];
        const int expect = (int)(crp[i + 1] - out);
        if (n != expect) {
            flag |= DERR_COUNT;
            n = min(min(n, expect), S / 2);
        }
        __syncwarp(gmask);
        if (RANK) {
            for (int e = lane; e < n; e += G) {
                int key = ck[e];
                int r = 0;
                for (int u = 0; u < n; u++) r += ck[u] < key;
                ccol[out + r] = key;
                cval[out + r] = cv[e];
            }
        } else {
            int P = next_pow2(n);
            for (int e = n + lane; e < P; e += G) ck[e] = INT_MAX;
            __syncwarp(gmask);
            bitonic<V>(ck, cv, P, lane, G, [&] { __syncwarp(gmask); });
            for (int e = lane; e < n; e += G) {
                ccol[out + e] = ck[e];
                cval[out + e] = cv[e];
            }
        }
        __syncwarp(gmask);
    }
    if (flag) atomicOr(err, flag);
}

// A whole block per row, map of S slots in shared memory.
template <int BS, int S, typename V>
__global__ void __launch_bounds__(BS) k_num_block(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol, const V *__restrict__ aval,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, const V *__restrict__ bval,
    const int64_t *__restrict__ crp, int32_t *__restrict__ ccol, V *__restrict__ cval,
    const int32_t *__restrict__ rows, int64_t count, int *err) {
    constexpr int L = __builtin_ctz(S);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *vals = (V *)smem_raw;
    V *cv = vals + S;
    int *keys = (int *)(cv + S / 2);
    int *ck = keys + S;
    __shared__ int nsh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int flag = 0;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        for (int s = threadIdx.x; s < S; s += BS) {
            keys[s] = -1;
            vals[s] = V(0);
        }
        if (threadIdx.x == 0) nsh = 0;
        __syncthreads();
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += BS / 32) {
            const int k = acol[p];
            const V a = aval[p];
            const int64_t q1 = brp[k + 1];
            for (int64_t q = brp[k] + lane; q < q1; q += 32) {
                if (!num_insert<V>(keys, vals, L, S, bcol[q], a * bval[q])) flag |= DERR_PROBE;
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < S; s += BS) {
            int key = keys[s];
            bool occ = key != -1;
            unsigned b = __ballot_sync(0xffffffffu, occ);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(&nsh, __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (occ) {
                int pos = base + __popc(b & ((1u << lane) - 1));
                if (pos < S / 2) {
                    ck[pos] = key;
                    cv[pos] = vals[s];
                }
            }
        }
        __syncthreads();
        int n = nsh;
        const int64_t out = crp[i];
        const int expect = (int)(crp[i + 1] - out);
        if (n != expect) {
            flag |= DERR_COUNT;
            n = min(min(n, expect), S / 2);
        }
        int P = next_pow2(n);
        for (int e = n + threadIdx.x; e < P; e += BS) ck[e] = INT_MAX;
        __syncthreads();
        bitonic<V>(ck, cv, P, threadIdx.x, BS, [] { __syncthreads(); });
        for (int e = threadIdx.x; e < n; e += BS) {
            ccol[out + e] = ck[e];
            cval[out + e] = cv[e];
        }
        __syncthreads();
    }
    if (flag) atomicOr(err, flag);
}

// Largest rows: first-level map in shared memory (bounded probing), second
// level in global memory sized for the row (Section 3.3); then the row's
// columns are marked in a bitmap whose word prefix counts give every entry
// its rank.  Global memory per block: L2 keys/values (l2cap slots), bitmap
// and prefix (nwords words each); each row clears the L2 slots it uses.
constexpr int HUGE_BS = 512, HUGE_L1 = 4096, HUGE_PROBES = 16;

template <typename V>
__global__ void __launch_bounds__(HUGE_BS) k_num_huge(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol, const V *__restrict__ aval,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, const V *__restrict__ bval,
    const int64_t *__restrict__ crp, int32_t *__restrict__ ccol, V *__restrict__ cval,
    const int32_t *__restrict__ rows, int64_t count, int *err, int64_t l2cap, int64_t nwords,
    unsigned char *gws) {
    constexpr int L1 = __builtin_ctz(HUGE_L1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *vals = (V *)smem_raw;
    int *keys = (int *)(vals + HUGE_L1);
    __shared__ int cmin, cmax;
    __shared__ long long red[HUGE_BS / 32];
    const size_t per_block = (size_t)l2cap * (4 + sizeof(V)) + (size_t)nwords * 8;
    unsigned char *mine = gws + per_block * blockIdx.x;
    V *g_vals = (V *)mine;
    int *g_keys = (int *)(g_vals + l2cap);
    unsigned *bits = (unsigned *)(g_keys + l2cap);
    unsigned *pref = bits + nwords;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int flag = 0;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        const int64_t out = crp[i];
        const int64_t expect = crp[i + 1] - out;
        int L2 = 1;
        while ((1LL << L2) < 2 * expect) L2++;
        for (int s = threadIdx.x; s < HUGE_L1; s += HUGE_BS) {
            keys[s] = -1;
            vals[s] = V(0);
        }
        for (int64_t s = threadIdx.x; s < (1LL << L2); s += HUGE_BS) {
            g_keys[s] = -1;
            g_vals[s] = V(0);
        }
        if (threadIdx.x == 0) {
            cmin = INT_MAX;
            cmax = -1;
        }
        __syncthreads();
        int lmin = INT_MAX, lmax = -1;
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += HUGE_BS / 32) {
            const int k = acol[p];
            const V a = aval[p];
            const int64_t q1 = brp[k + 1];
            for (int64_t q = brp[k] + lane; q < q1; q += 32) {
                const int c = bcol[q];
                const V v = a * bval[q];
                lmin = min(lmin, c);
                lmax = max(lmax, c);
                if (!num_insert<V>(keys, vals, L1, HUGE_PROBES, c, v))
                    if (!num_insert<V>(g_keys, g_vals, L2, 1 << L2, c, v)) flag |= DERR_PROBE;
            }
        }
        atomicMin(&cmin, lmin);
        atomicMax(&cmax, lmax);
        __syncthreads();
        for (int s = threadIdx.x; s < HUGE_L1; s += HUGE_BS) {
            int key = keys[s];
            if (key != -1)
                if (!num_insert<V>(g_keys, g_vals, L2, 1 << L2, key, vals[s])) flag |= DERR_PROBE;
        }
        const int64_t w0 = cmin >= 0 && cmin != INT_MAX ? (cmin >> 5) : 0;
        const int64_t w1 = cmax >= 0 ? (cmax >> 5) + 1 : 0;
        for (int64_t x = w0 + threadIdx.x; x < w1; x += HUGE_BS) bits[x] = 0;
        __syncthreads();
        const int64_t slots = 1LL << L2;
        for (int64_t s = threadIdx.x; s < slots; s += HUGE_BS) {
            int key = g_keys[s];
            if (key != -1) atomicOr(&bits[key >> 5], 1u << (key & 31));
        }
        __syncthreads();
        // word prefix: contiguous chunk per thread, block scan of chunk sums
        const int64_t nw = w1 - w0;
        const int64_t chunk = (nw + HUGE_BS - 1) / HUGE_BS;
        const int64_t c0 = w0 + threadIdx.x * chunk;
        const int64_t c1 = min(w1, c0 + chunk);
        long long sum = 0;
        for (int64_t x = c0; x < c1; x++) sum += __popc(bits[x]);
        long long incl = sum;
        for (int d = 1; d < 32; d <<= 1) {
            long long tt = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += tt;
        }
        if (lane == 31) red[w] = incl;
        __syncthreads();
        if (w == 0) {
            long long v = lane < HUGE_BS / 32 ? red[lane] : 0, vi = v;
            for (int d = 1; d < 32; d <<= 1) {
                long long tt = __shfl_up_sync(0xffffffffu, vi, d);
                if (lane >= d) vi += tt;
            }
            if (lane < HUGE_BS / 32) red[lane] = vi - v;
        }
        __syncthreads();
        long long run = red[w] + incl - sum;
        for (int64_t x = c0; x < c1; x++) {
            pref[x] = (unsigned)run;
            run += __popc(bits[x]);
        }
        __syncthreads();
        for (int64_t s = threadIdx.x; s < slots; s += HUGE_BS) {
            int key = g_keys[s];
            if (key != -1) {
                int64_t x = key >> 5;
                int64_t r = (int64_t)pref[x] + __popc(bits[x] & ((1u << (key & 31)) - 1));
                if (r < expect) {
                    ccol[out + r] = key;
                    cval[out + r] = g_vals[s];
                } else {
                    flag |= DERR_COUNT;
                }
            }
        }
        __syncthreads();
    }
    if (flag) atomicOr(err, flag);
}

// Opt in to the dynamic shared memory a launch needs (static shared memory
// comes on top, so the attribute is set for every non-trivial size).
template <typename K>
static int prep(K kern, size_t smem) {
    if (smem > 16 * 1024)
        SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return SPGEMM_OK;
}

template <typename V>
struct NumArgs {
    const int64_t *arp; const int32_t *acol; const V *aval;
    const int64_t *brp; const int32_t *bcol; const V *bval;
    const int64_t *crp; int32_t *ccol; V *cval;
};

static const char *NUM_LABEL[NBINS] = {"", "numeric.bin1", "numeric.bin2", "numeric.bin3",
                                       "numeric.bin4", "numeric.bin5", "numeric.bin6", ""};

template <int G, int S, bool RANK, typename V>
static int run_group(const NumArgs<V> &a, const int32_t *rows, int64_t count, int *err, int b,
                     Ctx &c) {
    constexpr int GPB = 256 / G;
    size_t smem = (size_t)GPB * S * (sizeof(V) + 4) * 3 / 2;
    SG_TRY(prep(k_num_group<G, S, RANK, V>, smem));
    int64_t blocks = (count + GPB - 1) / GPB;
    blocks = blocks < (int64_t)c.nsm * 64 ? blocks : (int64_t)c.nsm * 64;
    c.begin(NUM_LABEL[b], count);
    k_num_group<G, S, RANK, V><<<(unsigned)blocks, 256, smem, c.s>>>(
        a.arp, a.acol, a.aval, a.brp, a.bcol, a.bval, a.crp, a.ccol, a.cval, rows, count, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int BS, int S, typename V>
static int run_block(const NumArgs<V> &a, const int32_t *rows, int64_t count, int *err, int b,
                     Ctx &c) {
    size_t smem = (size_t)S * (sizeof(V) + 4) * 3 / 2;
    SG_TRY(prep(k_num_block<BS, S, V>, smem));
    int64_t blocks = count < (int64_t)c.nsm * 16 ? count : (int64_t)c.nsm * 16;
    c.begin(NUM_LABEL[b], count);
    k_num_block<BS, S, V><<<(unsigned)blocks, BS, smem, c.s>>>(
        a.arp, a.acol, a.aval, a.brp, a.bcol, a.bval, a.crp, a.ccol, a.cval, rows, count, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

static int64_t huge_l2cap(int64_t max_row_nnz) {
    int64_t c = 2;
    while (c < 2 * max_row_nnz) c <<= 1;
    return c;
}

size_t numeric_global_ws(int64_t max_row_nnz, int64_t ncols_b, int nsm, int dtype) {
    int64_t l2 = huge_l2cap(max_row_nnz);
    int64_t nwords = (ncols_b + 31) / 32;
    size_t vb = dtype == SPGEMM_F64 ? 8 : 4;
    return ((size_t)l2 * (4 + vb) + (size_t)nwords * 8) * (size_t)nsm;
}

template <typename V>
static int run_all(const NumArgs<V> &a, const spgemm_csr &B, const int32_t *rows,
                   const long long *counts, int *err, void *gws, size_t gws_bytes,
                   int64_t max_row_nnz, Ctx &c) {
    const int nsm = c.nsm;
    int64_t off = 0;
    for (int b = 1; b < NBINS; b++) {
        int64_t cnt = counts[b];
        const int32_t *r = rows + off;
        off += cnt;
        if (cnt == 0) continue;
        switch (b) {
            case 1: SG_TRY((run_group<8, 32, true, V>(a, r, cnt, err, b, c))); break;
            case 2: SG_TRY((run_group<16, 128, false, V>(a, r, cnt, err, b, c))); break;
            case 3: SG_TRY((run_group<32, 512, false, V>(a, r, cnt, err, b, c))); break;
            case 4: SG_TRY((run_block<128, 2048, V>(a, r, cnt, err, b, c))); break;
            case 5: SG_TRY((run_block<256, 8192, V>(a, r, cnt, err, b, c))); break;
            default: {
                int64_t l2 = huge_l2cap(max_row_nnz);
                int64_t nwords = (B.ncols + 31) / 32;
                int64_t blocks = cnt < (int64_t)nsm ? cnt : (int64_t)nsm;
                size_t need = ((size_t)l2 * (4 + sizeof(V)) + (size_t)nwords * 8) * (size_t)blocks;
                if (need > gws_bytes) {
                    set_error("numeric: global map workspace too small");
                    return SPGEMM_ERR_INTERNAL;
                }
                size_t smem = (size_t)HUGE_L1 * (sizeof(V) + 4);
                SG_TRY(prep(k_num_huge<V>, smem));
                c.begin(NUM_LABEL[b], cnt);
                k_num_huge<V><<<(unsigned)blocks, HUGE_BS, smem, c.s>>>(
                    a.arp, a.acol, a.aval, a.brp, a.bcol, a.bval, a.crp, a.ccol, a.cval, r, cnt, err,
                    l2, nwords, (unsigned char *)gws);
                c.end();
                SG_CUDA(cudaGetLastError());
            }
        }
    }
    return SPGEMM_OK;
}

int launch_numeric(int dtype, const spgemm_csr &A, const spgemm_csr &B, spgemm_csr &C,
                   const int32_t *rows, const long long *counts, int *err, void *gws,
                   size_t gws_bytes, int64_t max_row_nnz, Ctx &c) {
    if (dtype == SPGEMM_F64) {
        NumArgs<double> a{A.row_ptr, A.col_idx, (const double *)A.values, B.row_ptr, B.col_idx,
                          (const double *)B.values, C.row_ptr, C.col_idx, (double *)C.values};
        return run_all<double>(a, B, rows, counts, err, gws, gws_bytes, max_row_nnz, c);
    } else {
        NumArgs<float> a{A.row_ptr, A.col_idx, (const float *)A.values, B.row_ptr, B.col_idx,
                         (const float *)B.values, C.row_ptr, C.col_idx, (float *)C.values};
        return run_all<float>(a, B, rows, counts, err, gws, gws_bytes, max_row_nnz, c);
    }
}

}  // namespace sg

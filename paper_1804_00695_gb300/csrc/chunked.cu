// Multi-memory chunking of Section 3.3.1: operands in host memory are moved
// through a fixed device budget (the fast memory) in row parts chosen by
// Algorithm 4, and multiplied part by part with the row-range fused
// multiply-add of Section 3.2.2: C2_i = sum over stored a_ik with k in the B
// part's row range of a_ik * B_k, plus the partial row C1_i already held.
//
//  * Algorithm 2 (A and C in place): for each A/C part, its rows of A and the
//    offsets of C come in, C starts empty (only offsets are copied, as the
//    paper notes), the B parts stream through, and the finished C part goes
//    back to host memory.  B parts that no column of the A part reaches are
//    skipped (same result, fewer bytes).
//  * Algorithm 3 (B in place): for each B part, every A/C part streams in
//    with its partial C (none before the first B part) and back out.
//
// Partial rows live in the final layout of C (offsets from the symbolic
// phase): the first m slots of a row hold its partial entries (in ascending
// column order once the row's last B part is done), the rest hold column -1.  Copies run on two side streams
// (host to device, device to host) and the streamed operand is double
// buffered: while part t is multiplied, part t+1 is copied in.  Every
// device byte of a call comes out of one arena of exactly the budget.
//
// The symbolic phase is chunked the same way with the pattern only; it keeps
// the pattern of B resident (its Algorithm 4 plan must put all of B in one
// part), compressed on the device into (block, mask) pairs (Section 2.1),
// and streams the rows of A, counting the distinct columns of each row by
// ORing masks per block.  A B with unsorted rows is counted on its columns.
#include <climits>
#include <cstring>
#include <algorithm>
#include "internal.cuh"

namespace sg {

// ------------------------------------------------------------------ kernels
__global__ void k_rebase(int64_t *rp, int64_t n1, int64_t base) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) rp[i] -= base;
}

__global__ void k_col_range(const int32_t *__restrict__ col, int64_t nnz, int *mm) {
    int lo = INT_MAX, hi = -1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        lo = min(lo, col[i]);
        hi = max(hi, col[i]);
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

__global__ void k_init_range(int *mm) {
    mm[0] = INT_MAX;
    mm[1] = -1;
}

__global__ void k_init_ranges(int2 *br, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) br[i] = make_int2(INT_MAX, -1);
}

// Column range of every block of CHUNK_RB rows of A that the resident part
// [r0, r1) touches (a CTA per block; rp rebased to the part, so the entries
// of a block's rows are one contiguous run).  Parts that share a block merge
// through the atomics.
__global__ void __launch_bounds__(256) k_block_range(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                                     int64_t r0, int64_t r1, int2 *br) {
    __shared__ int red[2][8];
    const int64_t b = (r0 >> CHUNK_RB_L) + blockIdx.x;
    const int64_t lo_row = max(b << CHUNK_RB_L, r0) - r0, hi_row = min((b + 1) << CHUNK_RB_L, r1) - r0;
    int lo = INT_MAX, hi = -1;
    for (int64_t p = rp[lo_row] + threadIdx.x; p < rp[hi_row]; p += blockDim.x) {
        const int c = col[p];
        lo = min(lo, c);
        hi = max(hi, c);
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = lo;
        red[1][threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            lo = min(lo, red[0][w]);
            hi = max(hi, red[1][w]);
        }
        if (hi >= 0) {
            atomicMin(&br[b].x, lo);
            atomicMax(&br[b].y, hi);
        }
    }
}

// *mx = max(*mx, max_i cnt[i]), i < n (row counts of C, before their scan).
__global__ void k_max_count(const int64_t *__restrict__ cnt, int64_t n, long long *mx) {
    long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (long long)cnt[i]);
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(mx, m);
}

template <typename V>
__device__ __forceinline__ bool fma_insert(int *keys, V *vals, int L, int col, V v) {
    const unsigned msk = (1u << L) - 1;
    unsigned h = hash_slot(col, L);
#pragma unroll 1
    for (int probe = 0; probe <= (int)msk; probe++) {
        int k = ((volatile int *)keys)[h];
        if (k == -1) {
            k = atomicCAS(&keys[h], -1, col);
            if (k == -1) k = col;
        }
        if (k == col) {
            if (vals) atomicAdd(&vals[h], v);
            return true;
        }
        h = (h + 1) & msk;
    }
    return false;
}

template <typename V, typename Sync>
__device__ __forceinline__ void bitonic_kv(int *k, V *v, int P, int tid, int NT, Sync sync) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < P / 2; t += NT) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool asc = (lo & size) == 0;
                const int x = k[lo], y = k[hi];
                if ((x > y) == asc) {
                    k[lo] = y;
                    k[hi] = x;
                    if (v) {
                        const V tv = v[lo];
                        v[lo] = v[hi];
                        v[hi] = tv;
                    }
                }
            }
            sync();
        }
    }
}

// Fused multiply-add on a row range of B (Section 3.2.2), a warp per row of
// the A/C part with at most FMA_WARP_CAP entries in C: the partial row and
// the products of the stored a_ik with lo <= k < hi (other columns of A are
// skipped; they need not be sorted) are merged in a shared-memory map, then
// written back sorted, padded with -1.
constexpr int FMA_WARP_CAP = 256, FMA_S = 512, FMA_WPB = 8, FMA_BMAP = 64, FMA_BMAP_L = 6;
// mode bits of the multiply-add kernels
constexpr int FMA_FRESH = 1;    // the C part holds no partial entries yet (its first pass)
constexpr int FMA_STRICT = 2;   // every column of A must lie in [lo, hi) (one window of B per part)
constexpr int FMA_BIG_OK = 4;   // rows longer than FMA_WARP_CAP are taken by the block kernel

constexpr int FMA_E = 32;   // stored a_ik staged per batch
template <typename V>
struct FmaLayout {   // per warp: vals[FMA_S], keys[FMA_S], eq0[E], ea[E], pre[E+1]
    static constexpr size_t per_warp =
        ((size_t)FMA_S * (sizeof(V) + 4) + FMA_E * 8 + FMA_E * sizeof(V) + (FMA_E + 1) * 4 + 15) & ~(size_t)15;
};

template <typename V>
__global__ void __launch_bounds__(256) k_fma_warp(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const V *__restrict__ aval, int64_t lo, int64_t hi, const int64_t *__restrict__ brp,
    const int32_t *__restrict__ bcol, const V *__restrict__ bval, const int64_t *__restrict__ crp,
    int32_t *__restrict__ ccol, V *__restrict__ cval, int *err, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const bool fresh = mode & FMA_FRESH;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *base = smem_raw + (size_t)w * FmaLayout<V>::per_warp;
    V *vals = (V *)base;
    int *keys = (int *)(vals + FMA_S);
    long long *eq0 = (long long *)(keys + FMA_S);
    V *ea = (V *)(eq0 + FMA_E);
    int *pre = (int *)(ea + FMA_E);
    int flag = 0;
    for (int64_t i = (int64_t)blockIdx.x * FMA_WPB + w; i < nrows; i += (int64_t)gridDim.x * FMA_WPB) {
        const int64_t c0 = crp[i];
        const int64_t cap64 = crp[i + 1] - c0;
        if (cap64 > FMA_WARP_CAP && !(mode & FMA_BIG_OK)) flag |= DERR_COUNT;
        const int cap = (int)cap64;
        if (cap == 0 || cap64 > FMA_WARP_CAP) continue;
        // Rows with no stored a_ik in this B part keep their partial row as it
        // is.  B parts come in ascending row order, so the pass whose range
        // holds the row's largest a_ik column is its last: only that pass
        // sorts the row; earlier ones leave the partial row unsorted.
        bool final_pass;
        {
            bool any = false, out = false;
            int64_t kmax = -1;
            for (int64_t p = arp[i] + lane; p < arp[i + 1]; p += 32) {
                const int64_t k = acol[p];
                any |= k >= lo && k < hi;
                out |= k < lo || k >= hi;
                kmax = k > kmax ? k : kmax;
            }
            if ((mode & FMA_STRICT) && out) flag |= DERR_WINDOW;
            if (!__any_sync(0xffffffffu, any)) continue;
            for (int d = 16; d > 0; d >>= 1) {
                const int64_t o = __shfl_xor_sync(0xffffffffu, kmax, d);
                kmax = o > kmax ? o : kmax;
            }
            final_pass = kmax < hi;
        }
        int S = 32;
        while (S < 2 * cap) S <<= 1;
        const int L = __ffs(S) - 1;
        for (int s = lane; s < S; s += 32) {
            keys[s] = -1;
            if (cval) vals[s] = V(0);
        }
        __syncwarp();
        if (!fresh) {   // the partial row of earlier parts of B
            for (int t = lane; t < cap; t += 32) {
                const int c = ccol[c0 + t];
                if (c >= 0 && !fma_insert<V>(keys, cval ? vals : nullptr, L, c, cval ? cval[c0 + t] : V(0)))
                    flag |= DERR_PROBE;
            }
        }
        // the products of the stored a_ik in [lo, hi), dealt out over the 32
        // lanes through prefix sums of nnz(B_k) (E stored entries at a time)
        const int64_t ps = arp[i], pe = arp[i + 1];
        for (int64_t pb = ps; pb < pe; pb += FMA_E) {
            int len = 0;
            if (pb + lane < pe) {
                const int64_t k = acol[pb + lane];
                if (k >= lo && k < hi) {
                    eq0[lane] = brp[k - lo];
                    len = (int)(brp[k - lo + 1] - brp[k - lo]);
                    ea[lane] = aval ? aval[pb + lane] : V(0);
                }
            }
            int incl = len;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            pre[lane] = incl - len;
            if (lane == 31) pre[FMA_E] = incl;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            int e = 0;
            for (int t = lane; t < total; t += 32) {
                while (pre[e + 1] <= t) e++;
                const int64_t q = eq0[e] + (t - pre[e]);
                if (!fma_insert<V>(keys, cval ? vals : nullptr, L, bcol[q], cval ? ea[e] * bval[q] : V(0)))
                    flag |= DERR_PROBE;
            }
            __syncwarp();
        }
        // compact in place (read everything first), sort, write back
        constexpr int PER = FMA_S / 32;
        int kq[PER];
        V vq[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int s = lane + 32 * u;
            kq[u] = -1;
            if (32 * u >= S) continue;
            kq[u] = s < S ? keys[s] : -1;
            vq[u] = (s < S && cval) ? vals[s] : V(0);
        }
        __syncwarp();
        int n = 0;
#pragma unroll
        for (int u = 0; u < PER; u++) {
            if (32 * u >= S) break;   // S is the warp's (one row per warp)
            const bool occ = kq[u] != -1;
            const unsigned m = __ballot_sync(0xffffffffu, occ);
            if (occ) {
                const int pos = n + __popc(m & ((1u << lane) - 1));
                keys[pos] = kq[u];
                vals[pos] = vq[u];
            }
            n += __popc(m);
        }
        if (n > cap) {
            flag |= DERR_COUNT;
            n = cap;
        }
        __syncwarp();
        bool written = false;
        if (final_pass && n <= FMA_WARP_CAP && cval) {
            // Sorted write through the row's 32-column blocks (the compressed
            // form of Section 2.1): the blocks of the n columns go into a small
            // map (in the free upper half of keys[]), only the blocks are
            // sorted, and a column's place is the number of columns in smaller
            // blocks plus the popcount of its block's mask below it.
            int *bk = keys + FMA_S / 2;                    // block keys
            unsigned *bm = (unsigned *)(bk + FMA_BMAP);    // block masks
            int *bf = (int *)(bm + FMA_BMAP);              // first place of the block
            int *bx = bf + FMA_BMAP;                       // blocks, sorted
            for (int u = lane; u < FMA_BMAP; u += 32) {
                bk[u] = -1;
                bm[u] = 0;
            }
            __syncwarp();
            bool ok = true;
            for (int e = lane; e < n; e += 32) {
                const int c = keys[e];
                ok &= sym_insert(bk, bm, FMA_BMAP_L, c >> 5, 1u << (c & 31));
            }
            ok = __all_sync(0xffffffffu, ok);
            __syncwarp();
            if (ok) {
                int nb = 0;
#pragma unroll
                for (int u = 0; u < FMA_BMAP / 32; u++) {
                    const int k = bk[lane + 32 * u];
                    const bool occ = k != -1;
                    const unsigned m = __ballot_sync(0xffffffffu, occ);
                    if (occ) bx[nb + __popc(m & ((1u << lane) - 1))] = k;
                    nb += __popc(m);
                }
                int PB = 1;
                while (PB < nb) PB <<= 1;
                for (int e = nb + lane; e < PB; e += 32) bx[e] = INT_MAX;
                __syncwarp();
                bitonic_kv<int>(bx, nullptr, PB, lane, 32, [] { __syncwarp(); });
                // first place of each block: popcounts of the blocks before it
                int run = 0;
                for (int j0 = 0; j0 < nb; j0 += 32) {
                    const int j = j0 + lane;
                    unsigned h = 0;
                    int pc = 0;
                    if (j < nb) {
                        h = hash_slot(bx[j], FMA_BMAP_L);
                        for (int g = 0; g < FMA_BMAP && bk[h] != bx[j]; g++) h = (h + 1) & (FMA_BMAP - 1);
                        pc = __popc(bm[h]);
                    }
                    int incl = pc;
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, d);
                        if (lane >= d) incl += y;
                    }
                    if (j < nb) bf[h] = run + incl - pc;
                    run += __shfl_sync(0xffffffffu, incl, 31);
                }
                __syncwarp();
                for (int e = lane; e < n; e += 32) {
                    const int c = keys[e], blk = c >> 5;
                    unsigned h = hash_slot(blk, FMA_BMAP_L);
                    for (int g = 0; g < FMA_BMAP && bk[h] != blk; g++) h = (h + 1) & (FMA_BMAP - 1);
                    const int place = bf[h] + __popc(bm[h] & ((1u << (c & 31)) - 1));
                    ccol[c0 + place] = c;
                    cval[c0 + place] = vals[e];
                }
                for (int e = n + lane; e < cap; e += 32) {
                    ccol[c0 + e] = -1;
                    cval[c0 + e] = V(0);
                }
                written = true;
            }
        }
        if (!written && final_pass) {
            int P = 1;
            while (P < n) P <<= 1;
            for (int e = n + lane; e < P; e += 32) keys[e] = INT_MAX;
            __syncwarp();
            bitonic_kv<V>(keys, cval ? vals : nullptr, P, lane, 32, [] { __syncwarp(); });
            __syncwarp();
        }
        if (!written) {
            for (int e = lane; e < cap; e += 32) {
                ccol[c0 + e] = e < n ? keys[e] : -1;
                if (cval) cval[c0 + e] = e < n ? vals[e] : V(0);
            }
        }
        __syncwarp();
    }
    if (flag) atomicOr(err, flag);
}

// Same for rows with more than FMA_WARP_CAP entries: a block per row, map
// and sort buffer in global memory (per block: 2^L slots, L from cap_max).
template <typename V>
__global__ void __launch_bounds__(256, 1) k_fma_block(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const V *__restrict__ aval, int64_t lo, int64_t hi, const int64_t *__restrict__ brp,
    const int32_t *__restrict__ bcol, const V *__restrict__ bval, const int64_t *__restrict__ crp,
    int32_t *__restrict__ ccol, V *__restrict__ cval, int *err, int64_t slots, unsigned char *gws) {
    __shared__ int nsh;
    int *keys = (int *)(gws + (size_t)blockIdx.x * (size_t)slots * (8 + 2 * sizeof(V)));
    V *vals = (V *)(keys + slots);
    int *ck = (int *)(vals + slots);
    V *cv = (V *)(ck + slots);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int flag = 0;
    for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        const int64_t c0 = crp[i];
        const int64_t cap = crp[i + 1] - c0;
        if (cap <= FMA_WARP_CAP) continue;
        {   // rows with no stored a_ik in this B part keep their partial row as it is
            if (threadIdx.x == 0) nsh = 0;
            __syncthreads();
            bool any = false;
            for (int64_t p = arp[i] + threadIdx.x; p < arp[i + 1] && !any; p += 256) {
                const int64_t k = acol[p];
                any = k >= lo && k < hi;
            }
            if (any) nsh = 1;
            __syncthreads();
            const bool skip = nsh == 0;
            __syncthreads();
            if (skip) continue;
        }
        int L = 1;
        while ((1LL << L) < 2 * cap) L++;
        const int64_t S = 1LL << L;
        for (int64_t s = threadIdx.x; s < S; s += 256) {
            keys[s] = -1;
            vals[s] = V(0);
        }
        if (threadIdx.x == 0) nsh = 0;
        __syncthreads();
        for (int64_t t = threadIdx.x; t < cap; t += 256) {
            const int c = ccol[c0 + t];
            if (c >= 0 && !fma_insert<V>(keys, cval ? vals : nullptr, L, c, cval ? cval[c0 + t] : V(0)))
                flag |= DERR_PROBE;
        }
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += 8) {
            const int64_t k = acol[p];
            if (k < lo || k >= hi) continue;
            const V av = aval ? aval[p] : V(0);
            const int64_t q1 = brp[k - lo + 1];
            for (int64_t q = brp[k - lo] + lane; q < q1; q += 32)
                if (!fma_insert<V>(keys, cval ? vals : nullptr, L, bcol[q], cval ? av * bval[q] : V(0)))
                    flag |= DERR_PROBE;
        }
        __syncthreads();
        for (int64_t s = threadIdx.x; s < S; s += 256) {
            const int key = keys[s];
            const bool occ = key != -1;
            const unsigned m = __ballot_sync(0xffffffffu, occ);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&nsh, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (occ) {
                const int pos = base + __popc(m & ((1u << lane) - 1));
                if (pos < cap) {
                    ck[pos] = key;
                    cv[pos] = vals[s];
                }
            }
        }
        __syncthreads();
        int n = nsh;
        if (n > cap) {
            flag |= DERR_COUNT;
            n = (int)cap;
        }
        int P = 1;
        while (P < n) P <<= 1;
        for (int e = n + threadIdx.x; e < P; e += 256) ck[e] = INT_MAX;
        __syncthreads();
        bitonic_kv<V>(ck, cval ? cv : nullptr, P, threadIdx.x, 256, [] { __syncthreads(); });
        for (int64_t e = threadIdx.x; e < cap; e += 256) {
            ccol[c0 + e] = e < n ? ck[e] : -1;
            if (cval) cval[c0 + e] = e < n ? cv[e] : V(0);
        }
        __syncthreads();
    }
    if (flag) atomicOr(err, flag);
}

// Symbolic count for a part of A against the resident pattern of B: a warp
// per row, distinct columns counted in a shared-memory set; rows with more
// than CNT_S/2 distinct columns are counted again by a block with a bitmap
// of all columns in global memory.
constexpr int CNT_S = 2048, CNT_WPB = 8;

__global__ void __launch_bounds__(256) k_count_warp(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, int64_t *__restrict__ cnt,
    int *overflow, int64_t nrows_b, int *err) {
    extern __shared__ int skeys[];
    __shared__ int scount[CNT_WPB];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *keys = skeys + w * CNT_S;
    constexpr int L = __builtin_ctz(CNT_S);
    for (int64_t i = (int64_t)blockIdx.x * CNT_WPB + w; i < nrows; i += (int64_t)gridDim.x * CNT_WPB) {
        for (int s = lane; s < CNT_S; s += 32) keys[s] = -1;
        if (lane == 0) scount[w] = 0;
        __syncwarp();
        bool full = false;
        int mine = 0;
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i]; p < pe && !full; p++) {
            const int k = acol[p];
            if (k < 0 || (int64_t)k >= nrows_b) {
                if (lane == 0) atomicOr(err, DERR_COL_RANGE);
                continue;
            }
            const int64_t q1 = brp[k + 1];
            for (int64_t q = brp[k] + lane; q < q1; q += 32) {
                const int col = bcol[q];
                unsigned h = hash_slot(col, L);
                bool done = false;
                for (int probe = 0; probe < CNT_S / 2 && !done; probe++) {
                    const int kk = ((volatile int *)keys)[h];
                    if (kk == col) done = true;
                    else if (kk == -1) {
                        const int old = atomicCAS(&keys[h], -1, col);
                        if (old == -1) { mine++; done = true; }
                        else if (old == col) done = true;
                    }
                    h = (h + 1) & (CNT_S - 1);
                }
                if (!done) full = true;
            }
            full = __any_sync(0xffffffffu, full);
        }
        for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, d);
        if (lane == 0) {
            if (full || mine > CNT_S / 2) {
                cnt[i] = -1;
                atomicAdd(overflow, 1);
            } else {
                cnt[i] = mine;
            }
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_count_bitmap(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ bcol, int64_t *__restrict__ cnt,
    int64_t nwords, unsigned *gbits, const int *overflow, int64_t nrows_b) {
    __shared__ long long red[8];
    if (*(volatile const int *)overflow == 0) return;   // no row overflowed the warp sets
    unsigned *bits = gbits + (size_t)blockIdx.x * (size_t)nwords;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        if (cnt[i] >= 0) continue;
        for (int64_t s = threadIdx.x; s < nwords; s += 256) bits[s] = 0;
        __syncthreads();
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i] + w; p < pe; p += 8) {
            const int k = acol[p];
            if (k < 0 || (int64_t)k >= nrows_b) continue;   // flagged by k_count_warp
            for (int64_t q = brp[k] + lane; q < brp[k + 1]; q += 32) {
                const int col = bcol[q];
                atomicOr(&bits[col >> 5], 1u << (col & 31));
            }
        }
        __syncthreads();
        long long c = 0;
        for (int64_t s = threadIdx.x; s < nwords; s += 256) c += __popc(bits[s]);
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) red[w] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int j = 0; j < 8; j++) t += red[j];
            cnt[i] = t;
        }
        __syncthreads();
    }
}

// ---- compressed pattern of B (Section 2.1): (block = col/32, mask) pairs
// Distinct 32-column blocks of each row of B, a thread per row (columns
// ascending; a row that is not flags the call, which then counts columns).
__global__ void k_pairs_count(int64_t nrows, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              int64_t *__restrict__ poff, int *unsorted) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int n = 0, prev = -1, pc = -1;
    bool bad = false;
    for (int64_t q = rp[r]; q < rp[r + 1]; q++) {
        const int c = col[q];
        bad |= c <= pc;
        pc = c;
        const int b = c >> 5;
        n += b != prev;
        prev = b;
    }
    poff[r + 1] = n;
    if (bad) atomicOr(unsorted, 1);
}

// Pairs of each row at poff[r]..: blocks ascending, masks ORed.
__global__ void k_pairs_write(int64_t nrows, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const int64_t *__restrict__ poff, int2 *__restrict__ pairs) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int64_t o = poff[r] - 1;
    int prev = -1;
    unsigned m = 0;
    for (int64_t q = rp[r]; q < rp[r + 1]; q++) {
        const int c = col[q], b = c >> 5;
        if (b != prev) {
            if (prev >= 0) pairs[o] = make_int2(prev, (int)m);
            o++;
            prev = b;
            m = 0;
        }
        m |= 1u << (c & 31);
    }
    if (prev >= 0) pairs[o] = make_int2(prev, (int)m);
}

// Symbolic count of a part of A against the compressed pattern of B: a warp
// per row ORs the pairs of its B_k into a shared map from block to mask
// (CNTP_S slots), the pairs dealt out over the lanes through prefix sums of
// pairs(B_k); the count is the sum of the masks' popcounts.  Rows whose
// blocks overflow the map are marked -1 for k_count_pairs_bitmap.
constexpr int CNTP_S = 512, CNTP_WPB = 8;

__global__ void __launch_bounds__(256) k_count_pairs(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ poff, const int2 *__restrict__ pairs, int64_t *__restrict__ cnt,
    int *overflow, int64_t nrows_b, int *err) {
    constexpr int E = 32, L = __builtin_ctz(CNTP_S);
    __shared__ int keys_all[CNTP_WPB * CNTP_S];
    __shared__ unsigned masks_all[CNTP_WPB * CNTP_S];
    __shared__ long long eq0_all[CNTP_WPB * E];
    __shared__ int pre_all[CNTP_WPB * (E + 1)];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *keys = keys_all + w * CNTP_S;
    unsigned *masks = masks_all + w * CNTP_S;
    long long *eq0 = eq0_all + w * E;
    int *pre = pre_all + w * (E + 1);
    for (int64_t i = (int64_t)blockIdx.x * CNTP_WPB + w; i < nrows; i += (int64_t)gridDim.x * CNTP_WPB) {
        for (int s = lane; s < CNTP_S; s += 32) {
            keys[s] = -1;
            masks[s] = 0;
        }
        __syncwarp();
        const int64_t p0 = arp[i];
        const int plen = (int)(arp[i + 1] - p0);
        bool fail = false;
        for (int pb = 0; pb < plen; pb += E) {
            int len = 0;
            if (pb + lane < plen) {
                const int k = acol[p0 + pb + lane];
                if (k < 0 || (int64_t)k >= nrows_b) {
                    atomicOr(err, DERR_COL_RANGE);
                } else {
                    eq0[lane] = poff[k];
                    len = (int)(poff[k + 1] - poff[k]);
                }
            }
            int incl = len;
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            pre[lane] = incl - len;
            if (lane == 31) pre[E] = incl;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            __syncwarp();
            int e = 0;
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int t = t0 + lane;
                if (t < total && !fail) {
                    while (pre[e + 1] <= t) e++;
                    const int2 pr = pairs[eq0[e] + (t - pre[e])];
                    fail = !sym_insert(keys, masks, L, pr.x, (unsigned)pr.y);
                }
            }
            fail = __any_sync(0xffffffffu, fail);
            __syncwarp();
            if (fail) break;
        }
        int c = 0;
        for (int s = lane; s < CNTP_S; s += 32) c += __popc(masks[s]);
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) {
            if (fail) {
                cnt[i] = -1;
                atomicAdd(overflow, 1);
            } else {
                cnt[i] = c;
            }
        }
        __syncwarp();
    }
}

// Rows marked -1: a block per row ORs the pairs into a bitmap over all
// column blocks of B (global memory, one per block).
__global__ void __launch_bounds__(256) k_count_pairs_bitmap(
    int64_t nrows, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ poff, const int2 *__restrict__ pairs, int64_t *__restrict__ cnt,
    int64_t nwords, unsigned *gbits, const int *overflow, int64_t nrows_b) {
    __shared__ long long red[8];
    if (*(volatile const int *)overflow == 0) return;
    unsigned *bits = gbits + (size_t)blockIdx.x * (size_t)nwords;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        if (cnt[i] >= 0) continue;
        for (int64_t s = threadIdx.x; s < nwords; s += 256) bits[s] = 0;
        __syncthreads();
        for (int64_t p = arp[i] + w; p < arp[i + 1]; p += 8) {
            const int k = acol[p];
            if (k < 0 || (int64_t)k >= nrows_b) continue;
            for (int64_t q = poff[k] + lane; q < poff[k + 1]; q += 32) {
                const int2 pr = pairs[q];
                atomicOr(&bits[pr.x], (unsigned)pr.y);
            }
        }
        __syncthreads();
        long long c = 0;
        for (int64_t s = threadIdx.x; s < nwords; s += 256) c += __popc(bits[s]);
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) red[w] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long t = 0;
            for (int j = 0; j < 8; j++) t += red[j];
            cnt[i] = t;
        }
        __syncthreads();
    }
}

// Column indices of a resident pattern must lie in [0, ncols).
__global__ void k_check_cols(const int32_t *__restrict__ col, int64_t nnz, int64_t ncols, int *err) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        bad |= col[i] < 0 || (int64_t)col[i] >= ncols;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, DERR_COL_RANGE);
}

// x[0..n] += *cin (the offset where this part of C starts); *cout = x[n].
__global__ void k_add_carry(int64_t *x, int64_t n, const int64_t *cin, int64_t *cout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) {
        const int64_t v = x[i] + *cin;
        x[i] = v;
        if (i == n) *cout = v;
    }
}

// ------------------------------------------------------------------ host side
struct Arena {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    void *take(size_t bytes) {
        size_t a = (used + 255) & ~(size_t)255;
        if (a + bytes > cap) return nullptr;
        used = a + bytes;
        return base + a;
    }
};

static size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

static int64_t part_bytes(const int64_t *rp, int64_t r0, int64_t r1, int vb) {
    return (r1 - r0 + 1) * 8 + (rp[r1] - rp[r0]) * (int64_t)(4 + vb);
}

// Offsets of a part copied in as they are, rebased to 0 on stream s.
static int rebase_rows(int64_t *rp, int64_t rows, int64_t p0, cudaStream_t s) {
    if (rows > 0)
        k_rebase<<<(unsigned)((rows + 1 + 255) / 256), 256, 0, s>>>(rp, rows + 1, p0);
    else
        SG_CUDA(cudaMemsetAsync(rp, 0, 8, s));
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

// Device copy of rows [r0, r1) of a host CSR matrix into (rp, col, val);
// returns the bytes moved.  With `rebase` the offsets are rebased to 0 on the
// copy stream, else the caller rebases them (rebase_rows with p0 =
// M.row_ptr[r0]) on the stream that uses them, so that no kernel waits in the
// copy stream's queue behind the kernels that occupy the GPU.
static int64_t copy_rows_in(const spgemm_csr &M, int64_t r0, int64_t r1, int vb, int64_t *rp,
                            int32_t *col, void *val, cudaStream_t s, int *status, bool rebase = true) {
    const int64_t p0 = M.row_ptr[r0], p1 = M.row_ptr[r1];
    int64_t bytes = (r1 - r0 + 1) * 8;
    cudaError_t e = cudaMemcpyAsync(rp, M.row_ptr + r0, (size_t)(r1 - r0 + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && p1 > p0) {
        e = cudaMemcpyAsync(col, M.col_idx + p0, (size_t)(p1 - p0) * 4, cudaMemcpyHostToDevice, s);
        bytes += (p1 - p0) * 4;
        if (e == cudaSuccess && vb && val) {
            e = cudaMemcpyAsync(val, (const char *)M.values + (size_t)p0 * vb, (size_t)(p1 - p0) * vb,
                                cudaMemcpyHostToDevice, s);
            bytes += (p1 - p0) * vb;
        }
    }
    if (e != cudaSuccess) {
        set_error("chunked copy: %s", cudaGetErrorString(e));
        *status = SPGEMM_ERR_CUDA;
        return bytes;
    }
    if (rebase) *status = rebase_rows(rp, r1 - r0, p0, s);
    return bytes;
}

struct PartBuf {
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    void *val = nullptr;
};

static bool take_part(Arena &ar, PartBuf &b, int64_t rows, int64_t nnz, int vb) {
    b.rp = (int64_t *)ar.take((size_t)(rows + 1) * 8);
    b.col = (int32_t *)ar.take((size_t)std::max<int64_t>(nnz, 1) * 4);
    b.val = vb ? ar.take((size_t)std::max<int64_t>(nnz, 1) * vb) : nullptr;
    return b.rp && b.col && (vb == 0 || b.val);
}

// A buffer laid out for rows (offsets) and nnz entries (columns, values).
static size_t carve_bytes(int64_t rows, int64_t nnz, int vb) {
    return r256((size_t)(rows + 1) * 8) + r256((size_t)std::max<int64_t>(nnz, 1) * 4) +
           (size_t)std::max<int64_t>(nnz, 1) * vb;
}

static PartBuf carve(char *base, int64_t rows, int vb, int64_t nnz) {
    PartBuf b;
    b.rp = (int64_t *)base;
    b.col = (int32_t *)(base + r256((size_t)(rows + 1) * 8));
    b.val = vb ? (void *)((char *)b.col + r256((size_t)std::max<int64_t>(nnz, 1) * 4)) : nullptr;
    return b;
}

template <typename V>
static int launch_fma(const PartBuf &A, int64_t nrows, int64_t lo, int64_t hi, const PartBuf &B,
                      const PartBuf &Cp, bool values, int64_t fma_blocks, int64_t slots, void *gws,
                      int *err, Ctx &c, int mode) {
    const size_t smem = (size_t)FMA_WPB * FmaLayout<V>::per_warp;
    SG_CUDA(cudaFuncSetAttribute(k_fma_warp<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (nrows + FMA_WPB - 1) / FMA_WPB;
    blocks = std::min<int64_t>(blocks, (int64_t)c.nsm * 16);
    if (blocks > 0) {
        c.begin("chunked.fma", nrows);
        k_fma_warp<V><<<(unsigned)blocks, 256, smem, c.s>>>(
            nrows, A.rp, A.col, values ? (const V *)A.val : nullptr, lo, hi, B.rp, B.col,
            values ? (const V *)B.val : nullptr, Cp.rp, Cp.col, values ? (V *)Cp.val : nullptr, err,
            mode | (fma_blocks > 0 ? FMA_BIG_OK : 0));
        c.end();
        SG_CUDA(cudaGetLastError());
    }
    if (fma_blocks > 0 && nrows > 0) {
        int64_t bb = std::min<int64_t>(nrows, fma_blocks);
        c.begin("chunked.fma_block", nrows);
        k_fma_block<V><<<(unsigned)bb, 256, 0, c.s>>>(
            nrows, A.rp, A.col, values ? (const V *)A.val : nullptr, lo, hi, B.rp, B.col,
            values ? (const V *)B.val : nullptr, Cp.rp, Cp.col, values ? (V *)Cp.val : nullptr, err,
            slots, (unsigned char *)gws);
        c.end();
        SG_CUDA(cudaGetLastError());
    }
    return SPGEMM_OK;
}

int chunked_numeric(ChunkEnv &env, int dtype, const spgemm_csr &A, const spgemm_csr &B,
                    spgemm_csr &C, size_t budget, ChunkStats &stats) {
    const int vb = dtype == SPGEMM_F64 ? 8 : 4;
    Ctx &c = *env.ctx;
    const cudaStream_t s = c.s;
    // What the chunked symbolic call of this product recorded: the column
    // ranges of A's row blocks (for A's host arrays) and the longest row of C
    // (for A, B and these offsets of C).
    const ChunkCache *cc = env.cache;
    const bool known_ranges = cc && cc->valid && cc->a_rp == A.row_ptr && cc->a_col == A.col_idx &&
                              cc->a_nrows == A.nrows && cc->a_ncols == A.ncols && cc->a_nnz == A.nnz &&
                              (int64_t)cc->brange.size() == (A.nrows + CHUNK_RB - 1) / CHUNK_RB;
    const bool known_max = known_ranges && cc->b_rp == B.row_ptr && cc->b_col == B.col_idx &&
                           cc->b_nrows == B.nrows && cc->b_ncols == B.ncols && cc->b_nnz == B.nnz &&
                           cc->c_rp == C.row_ptr;
    // the largest row of C decides whether the block kernel and its maps are
    // needed (the kernels flag a longer row than planned for)
    int64_t cap_max = 0;
    if (known_max)
        cap_max = cc->max_row;
    else
        for (int64_t i = 0; i < C.nrows; i++) cap_max = std::max(cap_max, C.row_ptr[i + 1] - C.row_ptr[i]);
    const bool big_rows = cap_max > FMA_WARP_CAP;
    int64_t slots = 2;
    while (slots < 2 * cap_max) slots <<= 1;
    // blocks of the wide-row kernel: as many as an eighth of the budget holds
    const size_t per_block = (size_t)slots * (8 + 2 * vb);
    const int64_t fma_blocks = big_rows ? std::max<int64_t>(1, std::min<int64_t>(c.nsm, (int64_t)(budget / 8 / per_block))) : 0;
    const size_t gws_bytes = (size_t)fma_blocks * per_block;
    const size_t reserve = r256(gws_bytes) + 4096;
    if (budget <= reserve) {
        set_error("chunked: budget %zu below the fixed working set %zu", budget, reserve);
        return SPGEMM_ERR_BUDGET;
    }
    // Algorithm 4 on the budget left after the fixed reserve.  The streamed
    // (inner) operand is double (or triple) buffered, so if the outer part
    // plus nb inner parts exceed the budget, the inner operand is cut again,
    // finer, with BinarySearch: the algorithm and the outer parts stay as
    // Algorithm 4 chose them.
    const int nb = env.nbuf >= 3 ? 3 : 2;
    ChunkPlan p;
    const int64_t avail = (int64_t)(budget - reserve) - 16 * 256;
    SG_TRY(plan_chunks(A.row_ptr, A.nrows, C.row_ptr, B.row_ptr, B.nrows, vb, vb, (int64_t)(budget - reserve), p));
    auto buf_ac = [&](const std::vector<int64_t> &cuts) {
        int64_t mr = 0, ma = 0, mc = 0;
        for (size_t j = 0; j + 1 < cuts.size(); j++) {
            mr = std::max(mr, cuts[j + 1] - cuts[j]);
            ma = std::max(ma, A.row_ptr[cuts[j + 1]] - A.row_ptr[cuts[j]]);
            mc = std::max(mc, C.row_ptr[cuts[j + 1]] - C.row_ptr[cuts[j]]);
        }
        return 2 * (mr + 1) * 8 + (ma + mc) * (int64_t)(4 + vb);
    };
    auto buf_b = [&](const std::vector<int64_t> &cuts) {
        int64_t mr = 0, mb = 0;
        for (size_t t = 0; t + 1 < cuts.size(); t++) {
            mr = std::max(mr, cuts[t + 1] - cuts[t]);
            mb = std::max(mb, B.row_ptr[cuts[t + 1]] - B.row_ptr[cuts[t]]);
        }
        return (mr + 1) * 8 + mb * (int64_t)(4 + vb);
    };
    {
        // Both operands are double (nb = 3: triple) buffered in Algorithm 2
        // (the next A/C part comes in while the current one is multiplied
        // and the previous ones go out), the streamed A/C parts in Algorithm
        // 3.  Parts that do not fit nb times are cut again with BinarySearch
        // (finer parts, same algorithm).  B parts are also cut to at most an
        // eighth of an A/C part so that skipping the parts an A part does not
        // reach is fine grained.
        const bool alg2 = p.algorithm == 2;
        std::vector<int64_t> &outer_cuts = alg2 ? p.ac_cuts : p.b_cuts;
        std::vector<int64_t> &inner_cuts = alg2 ? p.b_cuts : p.ac_cuts;
        auto outer_sz = [&]() { return alg2 ? buf_ac(outer_cuts) : buf_b(outer_cuts); };
        auto inner_sz = [&]() { return alg2 ? buf_b(inner_cuts) : buf_ac(inner_cuts); };
        const int nouter = alg2 ? nb : 1;
        double olimit = (double)avail * 0.60 / nb;
        for (int iter = 0; alg2 && outer_sz() * nouter > (int64_t)((double)avail * 0.62); iter++) {
            const bool ok = iter < 40 && cut_rows(A.row_ptr, C.row_ptr, A.nrows, vb, olimit, outer_cuts);
            if (!ok) {
                set_error("chunked: budget %zu too small for the outer parts", budget);
                return SPGEMM_ERR_BUDGET;
            }
            olimit *= 0.85;
        }
        const int64_t outer = outer_sz() * nouter;
        double limit = (double)(avail - outer) / nb;
        if (alg2) limit = std::min(limit, (double)outer / nouter / 8.0);
        bool first = alg2;   // Algorithm 2: always cut B to the fine size
        for (int iter = 0; first || inner_sz() * nb + outer > avail; iter++) {
            first = false;
            bool cut_ok = limit > 0 && iter < 40 &&
                          (alg2 ? cut_rows(B.row_ptr, nullptr, B.nrows, vb, limit, inner_cuts)
                                : cut_rows(A.row_ptr, C.row_ptr, A.nrows, vb, limit, inner_cuts));
            if (!cut_ok) {
                set_error("chunked: budget %zu too small for a part and %d buffered parts", budget, nb);
                return SPGEMM_ERR_BUDGET;
            }
            limit *= 0.85;
        }
    }
    stats.algorithm = p.algorithm;
    stats.branch = p.branch;
    stats.n_ac = (int64_t)p.ac_cuts.size() - 1;
    stats.n_b = (int64_t)p.b_cuts.size() - 1;
    stats.cost1 = p.cost1;
    stats.cost2 = p.cost2;
    // carve the arena
    Arena ar{(char *)env.arena, budget, 0};
    void *gws = gws_bytes ? ar.take(gws_bytes) : nullptr;
    int *mm = (int *)ar.take(2 * CHUNK_MAX_BUF * sizeof(int));   // column range of each A/C buffer's part
    int64_t max_ac_rows = 0, max_ac_a = 0, max_ac_c = 0, max_b_rows = 0, max_b_nnz = 0;
    for (size_t j = 0; j + 1 < p.ac_cuts.size(); j++) {
        const int64_t r0 = p.ac_cuts[j], r1 = p.ac_cuts[j + 1];
        max_ac_rows = std::max(max_ac_rows, r1 - r0);
        max_ac_a = std::max(max_ac_a, A.row_ptr[r1] - A.row_ptr[r0]);
        max_ac_c = std::max(max_ac_c, C.row_ptr[r1] - C.row_ptr[r0]);
    }
    for (size_t t = 0; t + 1 < p.b_cuts.size(); t++) {
        max_b_rows = std::max(max_b_rows, p.b_cuts[t + 1] - p.b_cuts[t]);
        max_b_nnz = std::max(max_b_nnz, B.row_ptr[p.b_cuts[t + 1]] - B.row_ptr[p.b_cuts[t]]);
    }
    const int nbuf_ac = nb;
    PartBuf Ab[CHUNK_MAX_BUF], Cb[CHUNK_MAX_BUF], Bb[CHUNK_MAX_BUF];
    bool ok = mm != nullptr;
    for (int u = 0; u < nbuf_ac && ok; u++)
        ok = take_part(ar, Ab[u], max_ac_rows, max_ac_a, vb) && take_part(ar, Cb[u], max_ac_rows, max_ac_c, vb);
    // Algorithm 2: nb byte buffers for the streamed rows of B, as large as
    // the budget leaves (at least a fixed part each); a part of B or a window
    // of rows is laid out in them per copy.  Algorithm 3: one fixed part.
    char *binner[CHUNK_MAX_BUF] = {nullptr, nullptr, nullptr};
    size_t inner_cap = 0;
    if (p.algorithm == 2) {
        const size_t need_fixed = carve_bytes(max_b_rows, max_b_nnz, vb);
        const size_t left = budget > ar.used + 4096 ? budget - ar.used - 4096 : 0;
        inner_cap = std::max(need_fixed, (left / nb) & ~(size_t)255);
        for (int u = 0; u < nb && ok; u++) {
            binner[u] = (char *)ar.take(inner_cap);
            ok = binner[u] != nullptr;
        }
    } else {
        ok = ok && take_part(ar, Bb[0], max_b_rows, max_b_nnz, vb);
    }
    if (!ok) {
        set_error("chunked: parts do not fit the %zu-byte budget", budget);
        return SPGEMM_ERR_BUDGET;
    }
    stats.device_bytes = (int64_t)ar.used;
    int st = SPGEMM_OK;
    const cudaStream_t si = env.s_in, so = env.s_out;
    // event groups, one event per buffer: rows of B in, rows of B used, C part
    // out, A part (and the offsets of its C part) in, A part used
    cudaEvent_t *ev = env.ev;
    cudaEvent_t *ev_bin = ev, *ev_bused = ev + CHUNK_MAX_BUF, *ev_cout = ev + 2 * CHUNK_MAX_BUF,
                *ev_ain = ev + 3 * CHUNK_MAX_BUF, *ev_aused = ev + 4 * CHUNK_MAX_BUF;
    int *err = env.err;
    // mode: FMA_* bits (first pass of the C part, one window of B)
    auto fma = [&](const PartBuf &Ap, int64_t rows, int64_t lo, int64_t hi, const PartBuf &Bp,
                   const PartBuf &Cp, int mode) -> int {
        return dtype == SPGEMM_F64
                   ? launch_fma<double>(Ap, rows, lo, hi, Bp, Cp, true, fma_blocks, slots, gws, err, c, mode)
                   : launch_fma<float>(Ap, rows, lo, hi, Bp, Cp, true, fma_blocks, slots, gws, err, c, mode);
    };
    if (p.algorithm == 2) {
        // Buffer slot j % nb of A/C part j, slot t % nb of the t-th copy of
        // rows of B.  ev_ain[slot] also covers, without recorded ranges, the
        // part's column range in pinned host memory.  The A buffer and the offsets
        // of a C buffer are reused once the part's products are done, the
        // entries of a C buffer once they have left the device, so neither
        // waits for the other.  The copy-in stream carries copies only and
        // the copy-out stream only the copies of C out: offsets are rebased,
        // and C cleared, on the compute stream, so no copy waits behind a
        // kernel that waits for the GPU to have room, nor a copy out behind
        // a copy in.
        const size_t nac = p.ac_cuts.size() - 1;
        int *hmm = env.host_mm;
        size_t bcount = 0;
        // column range of part j: from the recorded row blocks (a superset,
        // at block granularity), else measured on the device once the part
        // is in and read back by the host
        auto recorded_range = [&](size_t j, int &lo_c, int &hi_c) {
            const int64_t r0 = p.ac_cuts[j], r1 = p.ac_cuts[j + 1];
            lo_c = INT_MAX;
            hi_c = -1;
            if (r1 <= r0) return;
            for (int64_t b = r0 >> CHUNK_RB_L; b <= (r1 - 1) >> CHUNK_RB_L; b++) {
                lo_c = std::min(lo_c, cc->brange[(size_t)b].x);
                hi_c = std::max(hi_c, cc->brange[(size_t)b].y);
            }
        };
        auto stage_ac = [&](size_t j) -> int {
            const int slot = (int)(j % nb);
            const int64_t r0 = p.ac_cuts[j], r1 = p.ac_cuts[j + 1], rows = r1 - r0;
            if (j >= (size_t)nb) SG_CUDA(cudaStreamWaitEvent(si, ev_aused[slot], 0));
            stats.h2d += copy_rows_in(A, r0, r1, vb, Ab[slot].rp, Ab[slot].col, Ab[slot].val, si, &st, false);
            SG_TRY(st);
            // C starts empty: only its offsets come in
            SG_CUDA(cudaMemcpyAsync(Cb[slot].rp, C.row_ptr + r0, (size_t)(rows + 1) * 8, cudaMemcpyHostToDevice, si));
            stats.h2d += (rows + 1) * 8;
            if (!known_ranges) {
                // column range of the A part decides which rows of B it needs
                const int64_t an = A.row_ptr[r1] - A.row_ptr[r0];
                int *dmm = mm + 2 * slot;
                k_init_range<<<1, 1, 0, si>>>(dmm);
                if (an > 0)
                    k_col_range<<<(unsigned)std::min<int64_t>((an + 255) / 256, (int64_t)c.nsm * 8), 256, 0, si>>>(
                        Ab[slot].col, an, dmm);
                SG_CUDA(cudaMemcpyAsync(hmm + 2 * slot, dmm, 8, cudaMemcpyDeviceToHost, si));
            }
            SG_CUDA(cudaEventRecord(ev_ain[slot], si));
            return SPGEMM_OK;
        };
        if (nac > 0) SG_TRY(stage_ac(0));
        for (size_t j = 0; j < nac; j++) {
            const int slot = (int)(j % nb);
            const int64_t r0 = p.ac_cuts[j], r1 = p.ac_cuts[j + 1], rows = r1 - r0;
            const int64_t cn = C.row_ptr[r1] - C.row_ptr[r0];
            int lo_c, hi_c;
            if (known_ranges) {
                recorded_range(j, lo_c, hi_c);
            } else {
                // the host waits for this part's column range only; the
                // device still has the previous part's products queued
                SG_TRY(host_wait_event(ev_ain[slot], env.wait_ms, "chunked numeric (column range of a part)"));
                lo_c = hmm[2 * slot];
                hi_c = hmm[2 * slot + 1];
                // lo_c == INT_MAX only for a part with no entries (hi_c
                // alone cannot tell: a part whose columns are all negative
                // leaves it at -1)
                if (lo_c != INT_MAX && (lo_c < 0 || (int64_t)hi_c >= B.nrows)) {
                    // a column of A outside the rows of B: stop once the
                    // copies already issued are done with the arena
                    cudaStreamSynchronize(si);
                    cudaStreamSynchronize(so);
                    cudaStreamSynchronize(s);
                    set_error("chunked numeric: a column of A lies outside the %lld rows of B",
                              (long long)B.nrows);
                    return SPGEMM_ERR_INDEX;
                }
            }
            // the rows of B this part reaches, as (r0, r1) copies: one window
            // when it fits a buffer, else the fixed parts it overlaps
            std::vector<std::pair<int64_t, int64_t>> need;
            bool window = false;
            if (hi_c >= 0 && carve_bytes(hi_c + 1 - lo_c, B.row_ptr[hi_c + 1] - B.row_ptr[lo_c], vb) <= inner_cap) {
                need.push_back({(int64_t)lo_c, (int64_t)hi_c + 1});
                stats.b_windows++;
                window = true;
            } else {
                for (size_t t = 0; t + 1 < p.b_cuts.size(); t++)
                    if (hi_c >= 0 && p.b_cuts[t] <= hi_c && p.b_cuts[t + 1] > lo_c)
                        need.push_back({p.b_cuts[t], p.b_cuts[t + 1]});
                stats.skipped_b += (int64_t)(p.b_cuts.size() - 1 - need.size());
            }
            // the A part and the offsets of its C part, rebased on the compute
            // stream once the C part that used the buffer has left
            SG_CUDA(cudaStreamWaitEvent(s, ev_ain[slot], 0));
            if (j >= (size_t)nb) SG_CUDA(cudaStreamWaitEvent(s, ev_cout[slot], 0));
            SG_TRY(rebase_rows(Ab[slot].rp, rows, A.row_ptr[r0], s));
            SG_TRY(rebase_rows(Cb[slot].rp, rows, C.row_ptr[r0], s));
            // One window and no long rows: the single pass writes every entry
            // of the part (its rows are complete and padded), so C is not
            // cleared first.  Otherwise passes merge into a cleared part.
            if (cn > 0 && (!window || fma_blocks > 0)) {
                SG_CUDA(cudaMemsetAsync(Cb[slot].col, 0xff, (size_t)cn * 4, s));
                SG_CUDA(cudaMemsetAsync(Cb[slot].val, 0, (size_t)cn * vb, s));
            }
            // stream the needed rows of B, nb buffers
            for (size_t u = 0; u < need.size(); u++, bcount++) {
                const int bs = (int)(bcount % nb);
                const int64_t b0 = need[u].first, b1 = need[u].second;
                Bb[bs] = carve(binner[bs], b1 - b0, vb, B.row_ptr[b1] - B.row_ptr[b0]);
                if (bcount >= (size_t)nb) SG_CUDA(cudaStreamWaitEvent(si, ev_bused[bs], 0));
                stats.h2d += copy_rows_in(B, b0, b1, vb, Bb[bs].rp, Bb[bs].col, Bb[bs].val, si, &st, false);
                SG_TRY(st);
                SG_CUDA(cudaEventRecord(ev_bin[bs], si));
                SG_CUDA(cudaStreamWaitEvent(s, ev_bin[bs], 0));
                SG_TRY(rebase_rows(Bb[bs].rp, b1 - b0, B.row_ptr[b0], s));
                // a recorded range may be stale if A changed after the
                // symbolic call: a window then checks every column of A
                const int mode = (u == 0 ? FMA_FRESH : 0) | (window && known_ranges ? FMA_STRICT : 0);
                SG_TRY(fma(Ab[slot], rows, b0, b1, Bb[bs], Cb[slot], mode));
                SG_CUDA(cudaEventRecord(ev_bused[bs], s));
            }
            SG_CUDA(cudaEventRecord(ev_aused[slot], s));   // A part used, C part complete
            // the next A part comes in behind this part's rows of B
            if (j + 1 < nac) SG_TRY(stage_ac(j + 1));
            // finished part of C back to host memory
            SG_CUDA(cudaStreamWaitEvent(so, ev_aused[slot], 0));
            if (cn > 0) {
                const int64_t p0 = C.row_ptr[r0];
                SG_CUDA(cudaMemcpyAsync(C.col_idx + p0, Cb[slot].col, (size_t)cn * 4, cudaMemcpyDeviceToHost, so));
                SG_CUDA(cudaMemcpyAsync((char *)C.values + (size_t)p0 * vb, Cb[slot].val, (size_t)cn * vb,
                                        cudaMemcpyDeviceToHost, so));
                stats.d2h += cn * (4 + vb);
            }
            SG_CUDA(cudaEventRecord(ev_cout[slot], so));
        }
        for (int u = 0; u < nb && (size_t)u < nac; u++) SG_CUDA(cudaStreamWaitEvent(s, ev_cout[u], 0));
    } else {
        for (size_t t = 0; t + 1 < p.b_cuts.size(); t++) {
            const int64_t b0 = p.b_cuts[t], b1 = p.b_cuts[t + 1];
            if (t > 0) SG_CUDA(cudaStreamWaitEvent(si, ev_bused[0], 0));
            stats.h2d += copy_rows_in(B, b0, b1, vb, Bb[0].rp, Bb[0].col, Bb[0].val, si, &st);
            SG_TRY(st);
            for (size_t j = 0; j + 1 < p.ac_cuts.size(); j++) {
                const size_t jj = t * (p.ac_cuts.size() - 1) + j;   // A/C parts streamed so far
                const int slot = (int)(jj % nb);
                const int64_t r0 = p.ac_cuts[j], r1 = p.ac_cuts[j + 1], rows = r1 - r0;
                const int64_t cn = C.row_ptr[r1] - C.row_ptr[r0], p0 = C.row_ptr[r0];
                // this buffer's previous C part must have gone out first
                if (jj >= (size_t)nb) SG_CUDA(cudaStreamWaitEvent(si, ev_cout[slot], 0));
                stats.h2d += copy_rows_in(A, r0, r1, vb, Ab[slot].rp, Ab[slot].col, Ab[slot].val, si, &st);
                SG_TRY(st);
                SG_CUDA(cudaMemcpyAsync(Cb[slot].rp, C.row_ptr + r0, (size_t)(rows + 1) * 8, cudaMemcpyHostToDevice, si));
                stats.h2d += (rows + 1) * 8;
                if (rows > 0)
                    k_rebase<<<(unsigned)((rows + 1 + 255) / 256), 256, 0, si>>>(Cb[slot].rp, rows + 1, p0);
                if (cn > 0) {
                    if (t == 0) {
                        SG_CUDA(cudaMemsetAsync(Cb[slot].col, 0xff, (size_t)cn * 4, si));
                        SG_CUDA(cudaMemsetAsync(Cb[slot].val, 0, (size_t)cn * vb, si));
                    } else {   // partial C from the previous B parts
                        SG_CUDA(cudaMemcpyAsync(Cb[slot].col, C.col_idx + p0, (size_t)cn * 4, cudaMemcpyHostToDevice, si));
                        SG_CUDA(cudaMemcpyAsync(Cb[slot].val, (const char *)C.values + (size_t)p0 * vb,
                                                (size_t)cn * vb, cudaMemcpyHostToDevice, si));
                        stats.h2d += cn * (4 + vb);
                    }
                }
                SG_CUDA(cudaEventRecord(ev_ain[slot], si));
                SG_CUDA(cudaStreamWaitEvent(s, ev_ain[slot], 0));
                SG_TRY(fma(Ab[slot], rows, b0, b1, Bb[0], Cb[slot], t == 0 ? FMA_FRESH : 0));
                SG_CUDA(cudaEventRecord(ev_aused[slot], s));
                SG_CUDA(cudaStreamWaitEvent(so, ev_aused[slot], 0));
                if (cn > 0) {
                    SG_CUDA(cudaMemcpyAsync(C.col_idx + p0, Cb[slot].col, (size_t)cn * 4, cudaMemcpyDeviceToHost, so));
                    SG_CUDA(cudaMemcpyAsync((char *)C.values + (size_t)p0 * vb, Cb[slot].val, (size_t)cn * vb,
                                            cudaMemcpyDeviceToHost, so));
                    stats.d2h += cn * (4 + vb);
                }
                SG_CUDA(cudaEventRecord(ev_cout[slot], so));
            }
            // the next B part may only overwrite the buffer once every use of it is done
            SG_CUDA(cudaEventRecord(ev_bused[0], s));
        }
        const size_t streamed = (p.b_cuts.size() - 1) * (p.ac_cuts.size() - 1);
        for (int u = 0; u < nb && (size_t)u < streamed; u++) SG_CUDA(cudaStreamWaitEvent(s, ev_cout[u], 0));
    }
    return SPGEMM_OK;
}

int chunked_symbolic(ChunkEnv &env, const spgemm_csr &A, const spgemm_csr &B, int64_t *C_row_ptr,
                     int64_t *nnz_C, size_t budget, ChunkStats &stats) {
    Ctx &c = *env.ctx;
    const cudaStream_t s = c.s, si = env.s_in, so = env.s_out;
    cudaEvent_t *ev = env.ev;   // [0..1] A part in, [2..3] counted, [4..5] offsets out, [6] B in, [7] B compressed
    const int64_t nwords = (B.ncols + 31) / 32;
    // pattern-only sizes; C contributes its offsets only
    std::vector<int64_t> &zeros = *env.zeros;
    if ((int64_t)zeros.size() < A.nrows + 1) zeros.assign((size_t)A.nrows + 1, 0);
    ChunkPlan p;
    const size_t bitmap = r256((size_t)c.nsm * (size_t)nwords * 4);
    const size_t poff_bytes = r256((size_t)(B.nrows + 1) * 8);
    const size_t btmp_bytes = r256(scan_tmp_bytes(B.nrows));
    const size_t raw_b = r256((size_t)(B.nrows + 1) * 8) + r256((size_t)std::max<int64_t>(B.nnz, 1) * 4);
    // column ranges of A's row blocks and the longest row of C, recorded for
    // the numeric call
    const int64_t nblk = (A.nrows + CHUNK_RB - 1) / CHUNK_RB;
    const size_t brange_bytes = r256((size_t)std::max<int64_t>(nblk, 1) * sizeof(int2));
    const size_t reserve = bitmap + poff_bytes + btmp_bytes + brange_bytes + 8192;
    if (budget <= reserve) {
        set_error("chunked symbolic: budget %zu below the fixed working set %zu", budget, reserve);
        return SPGEMM_ERR_BUDGET;
    }
    int64_t fast = (int64_t)(budget - reserve);
    SG_TRY(plan_chunks(A.row_ptr, A.nrows, zeros.data(), B.row_ptr, B.nrows, 0, 0, fast, p));
    if (p.b_cuts.size() != 2) {
        set_error("chunked symbolic: the pattern of B (%lld bytes) must fit the budget's large portion",
                  (long long)p.size_b);
        return SPGEMM_ERR_BUDGET;
    }
    // A parts are double buffered (with their counts and the scan's scratch):
    // if two of them and the pattern of B do not fit, the parts of A are cut
    // again, finer, with BinarySearch (the plan keeps B whole)
    int64_t max_rows = 0, max_nnz = 0;
    size_t part_bytes = 0;
    auto measure = [&]() {
        max_rows = max_nnz = 0;
        for (size_t j = 0; j + 1 < p.ac_cuts.size(); j++) {
            max_rows = std::max(max_rows, p.ac_cuts[j + 1] - p.ac_cuts[j]);
            max_nnz = std::max(max_nnz, A.row_ptr[p.ac_cuts[j + 1]] - A.row_ptr[p.ac_cuts[j]]);
        }
        part_bytes = r256((size_t)(max_rows + 1) * 8) + r256((size_t)std::max<int64_t>(max_nnz, 1) * 4) +
                     r256((size_t)(max_rows + 1) * 8) + r256(scan_tmp_bytes(max_rows));
    };
    measure();
    const size_t fixed = raw_b + reserve + 8 * 256;
    if (fixed >= budget) {
        set_error("chunked symbolic: budget %zu too small for the pattern of B", budget);
        return SPGEMM_ERR_BUDGET;
    }
    double limit = (double)(budget - fixed) / 2.0 * 0.8;
    for (int iter = 0; fixed + 2 * part_bytes > budget; iter++) {
        if (iter == 40 || limit < 64 || !cut_rows(A.row_ptr, zeros.data(), A.nrows, 0, limit, p.ac_cuts)) {
            set_error("chunked symbolic: budget %zu too small", budget);
            return SPGEMM_ERR_BUDGET;
        }
        measure();
        limit *= 0.85;
    }
    stats.algorithm = p.algorithm;
    stats.branch = p.branch;
    stats.n_ac = (int64_t)p.ac_cuts.size() - 1;
    stats.n_b = 1;
    // arena: fixed scratch from the bottom, the raw pattern of B at the top
    Arena ar{(char *)env.arena, budget, 0};
    unsigned *bits = (unsigned *)ar.take(bitmap);
    int *flags = (int *)ar.take(4 * sizeof(int));   // overflow per slot, unsorted rows of B
    int64_t *carry = (int64_t *)ar.take(5 * sizeof(int64_t));   // running offsets, scan totals, longest row
    int64_t *poff = (int64_t *)ar.take(poff_bytes);
    void *btmp = ar.take(btmp_bytes);
    int2 *brange = (int2 *)ar.take(brange_bytes);
    const size_t top = (budget - raw_b) & ~(size_t)255;
    if (!bits || !flags || !carry || !poff || !btmp || !brange || ar.used > top) {
        set_error("chunked symbolic: budget %zu too small", budget);
        return SPGEMM_ERR_BUDGET;
    }
    PartBuf Bp;
    Bp.rp = (int64_t *)((char *)env.arena + top);
    Bp.col = (int32_t *)((char *)Bp.rp + r256((size_t)(B.nrows + 1) * 8));
    int st = SPGEMM_OK;
    stats.h2d += copy_rows_in(B, 0, B.nrows, 0, Bp.rp, Bp.col, nullptr, si, &st);
    SG_TRY(st);
    if (B.nnz > 0)
        k_check_cols<<<(unsigned)std::min<int64_t>((B.nnz + 255) / 256, (int64_t)c.nsm * 8), 256, 0, si>>>(
            Bp.col, B.nnz, B.ncols, env.err);
    SG_CUDA(cudaEventRecord(ev[6], si));
    SG_CUDA(cudaStreamWaitEvent(s, ev[6], 0));
    // compress the pattern of B into (block, mask) pairs (Section 2.1): count,
    // offsets, and the host learns the pair count (one synchronisation)
    SG_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    SG_CUDA(cudaMemsetAsync(carry, 0, 5 * sizeof(int64_t), s));
    if (nblk > 0) k_init_ranges<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(brange, nblk);
    SG_CUDA(cudaMemsetAsync(poff, 0, 8, s));
    if (B.nrows > 0) {
        k_pairs_count<<<(unsigned)((B.nrows + 255) / 256), 256, 0, s>>>(B.nrows, Bp.rp, Bp.col, poff, &flags[2]);
        SG_CUDA(cudaGetLastError());
        SG_TRY(launch_scan_counts(poff, B.nrows, (long long *)&carry[3], btmp, c));
    }
    long long hbuf[2] = {0, 0};
    SG_CUDA(cudaMemcpyAsync(&hbuf[0], &carry[3], 8, cudaMemcpyDeviceToHost, s));
    int hunsorted = 0;
    SG_CUDA(cudaMemcpyAsync(&hunsorted, &flags[2], 4, cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    const int64_t npairs = hbuf[0];
    const size_t pairs_bytes = r256((size_t)std::max<int64_t>(npairs, 1) * 8);
    bool use_pairs = !hunsorted && ar.used + pairs_bytes + 2 * part_bytes + 8 * 256 <= budget &&
                     ar.used + pairs_bytes <= top;
    int2 *pairs = nullptr;
    if (use_pairs) {
        pairs = (int2 *)ar.take(pairs_bytes);
        if (B.nrows > 0) {
            k_pairs_write<<<(unsigned)((B.nrows + 255) / 256), 256, 0, s>>>(B.nrows, Bp.rp, Bp.col, poff, pairs);
            SG_CUDA(cudaGetLastError());
        }
        // A parts may overwrite the raw pattern from here on
        SG_CUDA(cudaEventRecord(ev[7], s));
        SG_CUDA(cudaStreamWaitEvent(si, ev[7], 0));
    }
    const size_t peak_with_raw = ar.used + (budget - top);
    PartBuf Ap[2];
    int64_t *cnt[2] = {nullptr, nullptr};
    void *tmp[2] = {nullptr, nullptr};
    bool ok = true;
    for (int u = 0; u < 2 && ok; u++) {
        ok = take_part(ar, Ap[u], max_rows, max_nnz, 0);
        cnt[u] = (int64_t *)ar.take((size_t)(max_rows + 1) * 8);
        tmp[u] = ar.take(scan_tmp_bytes(max_rows));
        ok = ok && cnt[u] && tmp[u];
    }
    if (!ok || (!use_pairs && ar.used > top)) {
        set_error("chunked symbolic: parts do not fit the %zu-byte budget", budget);
        return SPGEMM_ERR_BUDGET;
    }
    // peak: the raw pattern of B lived beside the fixed scratch (and the pairs)
    stats.device_bytes = (int64_t)std::max(ar.used, peak_with_raw);
    C_row_ptr[0] = 0;
    const size_t smem = (size_t)CNT_WPB * CNT_S * 4;
    SG_CUDA(cudaFuncSetAttribute(k_count_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const size_t nparts = p.ac_cuts.size() - 1;
    // Part j: A rows in on s_in; counts, scan and running offset on s; the
    // offsets out to C_row_ptr on s_out.  No host synchronisation inside.
    for (size_t j = 0; j < nparts; j++) {
        const int slot = (int)(j & 1);
        const int64_t r0 = p.ac_cuts[j], r1 = p.ac_cuts[j + 1], rows = r1 - r0;
        if (j >= 2) SG_CUDA(cudaStreamWaitEvent(si, ev[4 + slot], 0));   // buffers free again
        stats.h2d += copy_rows_in(A, r0, r1, 0, Ap[slot].rp, Ap[slot].col, nullptr, si, &st, false);
        SG_TRY(st);
        SG_CUDA(cudaEventRecord(ev[slot], si));
        SG_CUDA(cudaStreamWaitEvent(s, ev[slot], 0));
        SG_TRY(rebase_rows(Ap[slot].rp, rows, A.row_ptr[r0], s));
        int64_t *x = cnt[slot];
        SG_CUDA(cudaMemsetAsync(x, 0, 8, s));
        if (rows > 0) {
            SG_CUDA(cudaMemsetAsync(&flags[slot], 0, 4, s));
            if (use_pairs) {
                const int64_t blocks = std::min<int64_t>((rows + CNTP_WPB - 1) / CNTP_WPB, (int64_t)c.nsm * 16);
                c.begin("chunked.count", rows);
                k_count_pairs<<<(unsigned)blocks, 256, 0, s>>>(rows, Ap[slot].rp, Ap[slot].col, poff, pairs, x + 1,
                                                               &flags[slot], B.nrows, env.err);
                c.end();
                SG_CUDA(cudaGetLastError());
                k_count_pairs_bitmap<<<(unsigned)std::min<int64_t>(rows, (int64_t)c.nsm), 256, 0, s>>>(
                    rows, Ap[slot].rp, Ap[slot].col, poff, pairs, x + 1, nwords, bits, &flags[slot], B.nrows);
                SG_CUDA(cudaGetLastError());
            } else {
                const int64_t blocks = std::min<int64_t>((rows + CNT_WPB - 1) / CNT_WPB, (int64_t)c.nsm * 16);
                c.begin("chunked.count", rows);
                k_count_warp<<<(unsigned)blocks, 256, smem, s>>>(rows, Ap[slot].rp, Ap[slot].col, Bp.rp, Bp.col,
                                                                 x + 1, &flags[slot], B.nrows, env.err);
                c.end();
                SG_CUDA(cudaGetLastError());
                k_count_bitmap<<<(unsigned)std::min<int64_t>(rows, (int64_t)c.nsm), 256, 0, s>>>(
                    rows, Ap[slot].rp, Ap[slot].col, Bp.rp, Bp.col, x + 1, nwords, bits, &flags[slot], B.nrows);
                SG_CUDA(cudaGetLastError());
            }
            k_max_count<<<(unsigned)std::min<int64_t>((rows + 255) / 256, (int64_t)c.nsm * 4), 256, 0, s>>>(
                x + 1, rows, (long long *)&carry[4]);
            k_block_range<<<(unsigned)(((r1 - 1) >> CHUNK_RB_L) - (r0 >> CHUNK_RB_L) + 1), 256, 0, s>>>(
                Ap[slot].rp, Ap[slot].col, r0, r1, brange);
            SG_CUDA(cudaGetLastError());
            SG_TRY(launch_scan_counts(x, rows, (long long *)&carry[2], tmp[slot], c));
        }
        k_add_carry<<<(unsigned)((rows + 1 + 255) / 256), 256, 0, s>>>(x, rows, &carry[j & 1],
                                                                       &carry[(j + 1) & 1]);
        SG_CUDA(cudaGetLastError());
        SG_CUDA(cudaEventRecord(ev[2 + slot], s));
        SG_CUDA(cudaStreamWaitEvent(so, ev[2 + slot], 0));
        if (rows > 0)
            SG_CUDA(cudaMemcpyAsync(C_row_ptr + r0 + 1, x + 1, (size_t)rows * 8, cudaMemcpyDeviceToHost, so));
        stats.d2h += rows * 8;
        SG_CUDA(cudaEventRecord(ev[4 + slot], so));
    }
    SG_CUDA(cudaStreamWaitEvent(s, ev[4], 0));
    SG_CUDA(cudaStreamWaitEvent(s, ev[5], 0));
    SG_CUDA(cudaMemcpyAsync(nnz_C, &carry[nparts & 1], 8, cudaMemcpyDeviceToHost, s));
    if (env.cache) {
        ChunkCache &cc = *env.cache;
        cc.brange.resize((size_t)nblk);
        if (nblk > 0)
            SG_CUDA(cudaMemcpyAsync(cc.brange.data(), brange, (size_t)nblk * sizeof(int2), cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaMemcpyAsync(&cc.max_row, &carry[4], 8, cudaMemcpyDeviceToHost, s));
    }
    return SPGEMM_OK;
}

}  // namespace sg

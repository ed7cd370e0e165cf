// Symbolic phase (Section 2.1): nnz(C_i) = | union over stored a_ik of the
// column set of B_k |, computed on compressed column sets: every set is a
// list of (block = col/32, 32-bit mask) pairs, a union is a hash map from
// block to the OR of its masks, and the count is the sum of popcounts
// (Section 2.1: compression turns union into bitwise operations).
//
// Rows are sized by an upper bound on their distinct blocks.  A first pass
// takes every row with bound <= 4096 in row order with a 32-slot map per
// row, G lanes sharing the row's stored a_ik; rows that do not fit are
// marked and, with the rows whose bound exceeds 4096, handled by a second
// pass from row lists.  In bins 2-5 a row whose column blocks span at most
// 2048 blocks takes a warp with a bitmap over its span (k_sym_span); wider
// rows take a warp with a 128- or 512-slot map (bins 2, 3) or a block with
// a 2048- or 8192-slot map (bins 4, 5).  Bin 6 takes a block with a dense
// bitmap over all column blocks (shared memory when it fits, global memory
// otherwise).  Maps live in shared memory (Section 3.3).
#include <climits>
#include "internal.cuh"

namespace sg {


// Per-row-slot layout of k_sym_first in 32-bit words: keys[32], masks[32],
// eq0[E] (int64), pre[E+1]; the stride is padded to G (mod 32) words so that
// the row slots of a warp start on different banks.
template <int G>
struct SymFirstLayout {
    static constexpr int S = SYM_FIRST_SLOTS, E = 32;
    static constexpr int raw = 2 * S + 2 * E + E + 1;
    static constexpr int stride = G == 32 ? ((raw + 1) & ~1) : raw + ((G - raw % 32) + 32) % 32;
    static_assert(stride % 2 == 0, "8-byte arrays need an even stride");
    static constexpr int o_keys = 0, o_masks = S, o_eq0 = 2 * S, o_pre = 2 * S + 2 * E;
};

// First pass: a warp takes 32/G consecutive rows, G lanes per row, 32-slot
// map per row.  The stored a_ik are staged E at a time in shared memory with
// the prefix sums of pairs(B_k); each lane takes a contiguous run of the
// batch's compressed pairs (ceil(total/G) of them), finds its first a_ik
// once by bisection of the prefix sums and walks on in registers, so a pair
// costs one load and one insertion.  Insertions are atomic (CAS on the key,
// OR on the mask).  A row whose map fills up is marked crp[i+1] = -1 and
// counted in its second-pass bin.
// True when the analysis left no row for the first pass (every row empty,
// of the widest bin or narrow: the histogram of the analysis, complete
// before this kernel starts on the same stream); the kernel then returns
// at once instead of reading every row's bin.
__device__ __forceinline__ bool first_pass_empty(const DevState *st) {
    long long m = 0;
#pragma unroll
    for (int b = 1; b < BIN_HUGE; b++) m += *(volatile const long long *)&st->sym_hist[b];
    return m == 0;
}

template <int G>
__global__ void __launch_bounds__(256) k_sym_first(
    int64_t n, const uint8_t *__restrict__ bins, const int64_t *__restrict__ arp,
    const int32_t *__restrict__ acol, const int4 *__restrict__ desc,
    const int2 *__restrict__ pairs, int64_t *__restrict__ crp, DevState *st) {
    using Lay = SymFirstLayout<G>;
    constexpr int S = Lay::S, L = 5, RPW = 32 / G, WPB = 8, PER = S / G;
    constexpr int E = Lay::E, EL = E / G, NR = WPB * RPW;
    __shared__ __align__(16) int sm[NR * Lay::stride];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / G, gl = lane % G, gbase = g * G;
    const int rs = w * RPW + g;
    int *reg = sm + rs * Lay::stride;
    int *keys = reg + Lay::o_keys;
    unsigned *masks = (unsigned *)(reg + Lay::o_masks);
    long long *eq0 = (long long *)(reg + Lay::o_eq0);
    int *pre = reg + Lay::o_pre;
    const unsigned lmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1);
    const int64_t stride = (int64_t)gridDim.x * WPB * RPW;
    if (first_pass_empty(st)) return;
    for (int64_t base = ((int64_t)blockIdx.x * WPB + w) * RPW; base < n; base += stride) {
        const int64_t i = base + g;
        const int b = i < n ? bins[i] : 0;
        const bool active = b != BIN_EMPTY && b != BIN_HUGE && b != BIN_NARROW;
        if (!__any_sync(0xffffffffu, active)) continue;   // rows done elsewhere
        const int64_t p0 = active ? arp[i] : 0;
        const int plen = active ? (int)(arp[i + 1] - p0) : 0;
#pragma unroll
        for (int t = 0; t < PER; t++) {
            keys[gl + t * G] = -1;
            masks[gl + t * G] = 0;
        }
        const int maxlen = __reduce_max_sync(0xffffffffu, plen);
        bool fail = false;
        __syncwarp();
        for (int pb = 0; pb < maxlen; pb += E) {
            int cnt[EL];
            int lsum = 0;
#pragma unroll
            for (int u = 0; u < EL; u++) {
                const int e = gl * EL + u;
                int c = 0;
                if (pb + e < plen) {
                    const int4 d = desc[acol[p0 + pb + e]];
                    c = d.w;
                    eq0[e] = desc_start(d);
                }
                cnt[u] = c;
                lsum += c;
            }
            int incl = lsum;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d, G);
                if (gl >= d) incl += y;
            }
            int run = incl - lsum;
#pragma unroll
            for (int u = 0; u < EL; u++) {
                pre[gl * EL + u] = run;
                run += cnt[u];
            }
            if (gl == G - 1) pre[E] = incl;
            int total = __shfl_sync(0xffffffffu, incl, gbase + G - 1);
            if (fail) total = 0;
            __syncwarp();
            const int chunk = (total + G - 1) / G;
            const int t0 = min(total, gl * chunk), t1 = min(total, t0 + chunk);
            if (t0 < t1) {
                int lo_e = 0, hi_e = E - 1;   // last e with pre[e] <= t0
                while (lo_e < hi_e) {
                    const int mid = (lo_e + hi_e + 1) >> 1;
                    if (pre[mid] <= t0) lo_e = mid; else hi_e = mid - 1;
                }
                int e = lo_e;
                int pe1 = pre[e + 1];
                int64_t q = eq0[e] + (t0 - pre[e]);
                int64_t qend = q + (pe1 - t0);
                for (int t = t0; t < t1 && !fail; t++) {
                    while (q == qend) {
                        e++;
                        const int pa = pre[e];
                        pe1 = pre[e + 1];
                        q = eq0[e];
                        qend = q + (pe1 - pa);
                    }
                    const int2 pr = pairs[q];
                    fail = !sym_insert(keys, masks, L, pr.x, (unsigned)pr.y);
                    q++;
                }
            }
            const unsigned fl = __ballot_sync(0xffffffffu, fail);
            fail = ((fl >> gbase) & lmask) != 0;
            __syncwarp();
        }
        int c = 0;
#pragma unroll
        for (int t = 0; t < PER; t++) c += __popc(masks[gl + t * G]);
        for (int d = G / 2; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (active && gl == 0) {
            if (fail) {
                crp[i + 1] = -1;
                atomicAdd((unsigned long long *)&st->bin_count[0][max(b, 2)], 1ull);
            } else {
                crp[i + 1] = c;
            }
        }
        __syncwarp();
    }
}

// The same first pass with the pairs dealt out in stride (lane l takes the
// t-th pair for t = l, l + G, ...): loads of pairs coalesce within each B_k
// at the cost of a forward-moving cursor in shared memory; faster than the
// contiguous runs when few lanes share a row (G <= 8).
template <int G>
__global__ void __launch_bounds__(256) k_sym_first_strided(
    int64_t n, const uint8_t *__restrict__ bins, const int64_t *__restrict__ arp,
    const int32_t *__restrict__ acol, const int4 *__restrict__ desc,
    const int2 *__restrict__ pairs, int64_t *__restrict__ crp, DevState *st) {
    using Lay = SymFirstLayout<G>;
    constexpr int S = Lay::S, L = 5, RPW = 32 / G, WPB = 8, PER = S / G;
    constexpr int E = Lay::E, EL = E / G, NR = WPB * RPW;
    __shared__ __align__(16) int sm[NR * Lay::stride];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / G, gl = lane % G, gbase = g * G;
    const int rs = w * RPW + g;
    int *reg = sm + rs * Lay::stride;
    int *keys = reg + Lay::o_keys;
    unsigned *masks = (unsigned *)(reg + Lay::o_masks);
    long long *eq0 = (long long *)(reg + Lay::o_eq0);
    int *pre = reg + Lay::o_pre;
    const unsigned lmask = (G == 32) ? 0xffffffffu : ((1u << G) - 1);
    const int64_t stride = (int64_t)gridDim.x * WPB * RPW;
    if (first_pass_empty(st)) return;
    for (int64_t base = ((int64_t)blockIdx.x * WPB + w) * RPW; base < n; base += stride) {
        const int64_t i = base + g;
        const int b = i < n ? bins[i] : 0;
        const bool active = b != BIN_EMPTY && b != BIN_HUGE && b != BIN_NARROW;
        if (!__any_sync(0xffffffffu, active)) continue;   // rows done elsewhere
        const int64_t p0 = active ? arp[i] : 0;
        const int plen = active ? (int)(arp[i + 1] - p0) : 0;
#pragma unroll
        for (int t = 0; t < PER; t++) {
            keys[gl + t * G] = -1;
            masks[gl + t * G] = 0;
        }
        const int maxlen = __reduce_max_sync(0xffffffffu, plen);
        bool fail = false;
        __syncwarp();
        for (int pb = 0; pb < maxlen; pb += E) {
            int cnt[EL];
            int lsum = 0;
#pragma unroll
            for (int u = 0; u < EL; u++) {
                const int e = gl * EL + u;
                int c = 0;
                if (pb + e < plen) {
                    const int4 d = desc[acol[p0 + pb + e]];
                    c = d.w;
                    eq0[e] = desc_start(d);
                }
                cnt[u] = c;
                lsum += c;
            }
            int incl = lsum;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d, G);
                if (gl >= d) incl += y;
            }
            int run = incl - lsum;
#pragma unroll
            for (int u = 0; u < EL; u++) {
                pre[gl * EL + u] = run;
                run += cnt[u];
            }
            if (gl == G - 1) pre[E] = incl;
            int total = __shfl_sync(0xffffffffu, incl, gbase + G - 1);
            if (fail) total = 0;
            __syncwarp();
            int e = 0;
            const int maxtot = __reduce_max_sync(0xffffffffu, total);
            for (int t0 = 0; t0 < maxtot; t0 += G) {
                const int t = t0 + gl;
                if (t < total && !fail) {
                    while (pre[e + 1] <= t) e++;
                    const int2 pr = pairs[eq0[e] + (t - pre[e])];
                    fail = !sym_insert(keys, masks, L, pr.x, (unsigned)pr.y);
                }
            }
            const unsigned fl = __ballot_sync(0xffffffffu, fail);
            fail = ((fl >> gbase) & lmask) != 0;
            __syncwarp();
        }
        int c = 0;
#pragma unroll
        for (int t = 0; t < PER; t++) c += __popc(masks[gl + t * G]);
        for (int d = G / 2; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (active && gl == 0) {
            if (fail) {
                crp[i + 1] = -1;
                atomicAdd((unsigned long long *)&st->bin_count[0][max(b, 2)], 1ull);
            } else {
                crp[i + 1] = c;
            }
        }
        __syncwarp();
    }
}

// Second pass for rows whose column blocks span at most BW blocks: a warp
// per row ORs the compressed pairs into a bitmap over the span (one word
// per block) and counts its bits; a summary bitmap (one bit per word) lists
// the touched words so that the count and the clean-up visit only those.
// The pairs of the row are dealt out over the lanes through prefix sums of
// pairs(B_k), as in the first pass.  A union of compressed sets by bitwise
// OR, with no hash map (Section 2.1).
constexpr int SPAN_U = 4;   // pairs per lane per step in k_sym_span

template <int BW, int WPB>
struct SpanLayout {
    static constexpr int NS = BW / 32, E = 32;
    static constexpr int words = BW + NS + 2 * E + E + 2;   // bits, summ, eq0 (int64), pre
};

template <int BW, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_sym_span(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ ccnt,
    const int2 *__restrict__ pairs, const int2 *__restrict__ spans, const int32_t *__restrict__ rows,
    int64_t count, int64_t *__restrict__ crp) {
    using Lay = SpanLayout<BW, WPB>;
    constexpr int NS = Lay::NS, E = Lay::E;
    extern __shared__ __align__(16) unsigned span_smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned *bits = span_smem + (size_t)w * Lay::words;
    unsigned *summ = bits + BW;
    long long *eq0 = (long long *)(summ + NS);
    int *pre = (int *)(eq0 + E);
    for (int x = lane; x < BW; x += 32) bits[x] = 0;
    for (int x = lane; x < NS; x += 32) summ[x] = 0;
    __syncwarp();
    for (int64_t t = (int64_t)blockIdx.x * WPB + w; t < count; t += (int64_t)gridDim.x * WPB) {
        const int i = rows[t];
        const int2 sp = spans[t];
        const int bmin = sp.x, nw = sp.y;
        if (nw > BW) continue;
        const int64_t p0 = arp[i];
        const int plen = (int)(arp[i + 1] - p0);
        for (int pb = 0; pb < plen; pb += E) {
            int len = 0;
            if (pb + lane < plen) {
                const int k = acol[p0 + pb + lane];
                len = ccnt[k];
                eq0[lane] = brp[k];
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
            // SPAN_U pairs per lane per step, their loads issued together
            int e = 0;
            for (int t0 = 0; t0 < total; t0 += 32 * SPAN_U) {
                int64_t qq[SPAN_U];
                int2 pr[SPAN_U];
#pragma unroll
                for (int u = 0; u < SPAN_U; u++) {
                    const int tt = t0 + u * 32 + lane;
                    qq[u] = -1;
                    if (tt < total) {
                        while (pre[e + 1] <= tt) e++;
                        qq[u] = eq0[e] + (tt - pre[e]);
                    }
                }
#pragma unroll
                for (int u = 0; u < SPAN_U; u++) pr[u] = qq[u] >= 0 ? pairs[qq[u]] : make_int2(0, 0);
#pragma unroll
                for (int u = 0; u < SPAN_U; u++) {
                    if (qq[u] < 0) continue;
                    const int wd = pr[u].x - bmin;
                    if (atomicOr(&bits[wd], (unsigned)pr[u].y) == 0) atomicOr(&summ[wd >> 5], 1u << (wd & 31));
                }
            }
            __syncwarp();
        }
        const int ns = (nw + 31) / 32;
        int c = 0;
        for (int y = lane; y < ns; y += 32) {
            unsigned sw = summ[y];
            while (sw) {
                const int x = y * 32 + __ffs(sw) - 1;
                sw &= sw - 1;
                c += __popc(bits[x]);
                bits[x] = 0;
            }
            summ[y] = 0;
        }
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) crp[i + 1] = c;
        __syncwarp();
    }
}

// A warp per row from a row list, S-slot map, lanes walk the pairs of B_k.
template <int S>
__global__ void __launch_bounds__(256) k_sym_warp(
    const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
    const int64_t *__restrict__ brp, const int32_t *__restrict__ ccnt,
    const int2 *__restrict__ pairs, const int32_t *__restrict__ rows, int64_t count,
    int64_t *__restrict__ crp, int *err, const int2 *__restrict__ spans, int skip_span) {
    constexpr int L = __builtin_ctz(S), WPB = 8;
    extern __shared__ int smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *keys = smem + w * S;
    unsigned *masks = (unsigned *)(smem + WPB * S) + w * S;
    bool fail = false;
    for (int64_t t = (int64_t)blockIdx.x * WPB + w; t < count; t += (int64_t)gridDim.x * WPB) {
        const int i = rows[t];
        if (skip_span > 0 && spans[t].y <= skip_span) continue;
        for (int s = lane; s < S; s += 32) {
            keys[s] = -1;
            masks[s] = 0;
        }
        __syncwarp();
        const int64_t pe = arp[i + 1];
        for (int64_t p = arp[i]; p < pe; p++) {
            const int k = acol[p];
            const int64_t q0 = brp[k];
            const int cnt = ccnt[k];
            for (int u = lane; u < cnt; u += 32) {
                const int2 pr = pairs[q0 + u];
                fail |= !sym_insert(keys, masks, L, pr.x, (unsigned)pr.y);
            }
        }
        __syncwarp();
        int c = 0;
        for (int s = lane; s < S; s += 32) c += __popc(masks[s]);
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) crp[i + 1] = c;
        __syncwarp();
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
    int64_t *__restrict__ crp, int *err, const int2 *__restrict__ spans, int skip_span) {
    constexpr int L = __builtin_ctz(S);
    extern __shared__ int smem[];
    __shared__ int red[BS / 32];
    int *keys = smem;
    unsigned *masks = (unsigned *)(smem + S);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool fail = false;
    for (int64_t t = blockIdx.x; t < count; t += gridDim.x) {
        const int i = rows[t];
        if (skip_span > 0 && spans[t].y <= skip_span) continue;   // uniform over the block
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
                fail |= !sym_insert(keys, masks, L, pr.x, (unsigned)pr.y);
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

template <int G>
static int run_first(const spgemm_csr &A, const uint8_t *bins, const int4 *desc, const int2 *pairs,
                     int64_t *crp, DevState *st, Ctx &c) {
    constexpr int GPB = 256 / G;   // rows per block: 8 warps x 32/G rows
    int64_t blocks = (A.nrows + GPB - 1) / GPB;
    // one resident wave striding over the rows: when the analysis left this
    // pass no row, every block returns at once, and a wave costs one round
    // of block launches where 32 blocks an SM cost several
    const int64_t cap = G <= 8 ? resident_blocks(k_sym_first_strided<G>, 256, c.nsm)
                               : resident_blocks(k_sym_first<G>, 256, c.nsm);
    blocks = blocks < cap ? blocks : cap;
    c.begin("symbolic.first", A.nrows);
    if (G <= 8)
        k_sym_first_strided<G><<<(unsigned)blocks, 256, 0, c.s>>>(A.nrows, bins, A.row_ptr, A.col_idx, desc,
                                                                  pairs, crp, st);
    else
        k_sym_first<G><<<(unsigned)blocks, 256, 0, c.s>>>(A.nrows, bins, A.row_ptr, A.col_idx, desc,
                                                       pairs, crp, st);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

int launch_symbolic_first(const spgemm_csr &A, const uint8_t *bins, const int4 *desc,
                          const int2 *pairs, int64_t *crp, DevState *st, int G, Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    switch (G) {
        case 4: return run_first<4>(A, bins, desc, pairs, crp, st, c);
        case 8: return run_first<8>(A, bins, desc, pairs, crp, st, c);
        case 16: return run_first<16>(A, bins, desc, pairs, crp, st, c);
        default: return run_first<32>(A, bins, desc, pairs, crp, st, c);
    }
}

static const char *SYM_LABEL[NBINS] = {"", "", "symbolic.bin2", "symbolic.bin3",
                                       "symbolic.bin4", "symbolic.bin5", "symbolic.bin6", ""};

template <int S>
static int run_warp(const spgemm_csr &A, const int64_t *brp, const int32_t *ccnt, const int2 *pairs,
                    const int32_t *rows, int64_t count, int64_t *crp, int *err, int b, Ctx &c,
                    const int2 *spans, int skip_span) {
    size_t smem = (size_t)8 * S * 8;
    SG_TRY(prep(k_sym_warp<S>, smem));
    int64_t blocks = (count + 7) / 8;
    blocks = blocks < (int64_t)c.nsm * 32 ? blocks : (int64_t)c.nsm * 32;
    c.begin(SYM_LABEL[b], count);
    k_sym_warp<S><<<(unsigned)blocks, 256, smem, c.s>>>(A.row_ptr, A.col_idx, brp, ccnt, pairs, rows,
                                                         count, crp, err, spans, skip_span);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <int BS, int S>
static int run_block(const spgemm_csr &A, const int64_t *brp, const int32_t *ccnt, const int2 *pairs,
                     const int32_t *rows, int64_t count, int64_t *crp, int *err, int b, Ctx &c,
                     const int2 *spans, int skip_span) {
    size_t smem = (size_t)S * 8;
    SG_TRY(prep(k_sym_block<BS, S>, smem));
    int64_t blocks = count < (int64_t)c.nsm * 16 ? count : (int64_t)c.nsm * 16;
    c.begin(SYM_LABEL[b], count);
    k_sym_block<BS, S><<<(unsigned)blocks, BS, smem, c.s>>>(A.row_ptr, A.col_idx, brp, ccnt, pairs,
                                                            rows, count, crp, err, spans, skip_span);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

static const char *SPAN_LABEL[NBINS] = {"", "", "symbolic.span2", "symbolic.span3",
                                        "symbolic.span4", "symbolic.span5", "", ""};
constexpr int SPAN_BW = 2048;

int launch_symbolic(const spgemm_csr &A, const spgemm_csr &B, const int2 *pairs,
                    const int32_t *ccnt, const int32_t *rows, const long long *counts,
                    int64_t *crp, int *err, void *gws, size_t gws_bytes, const int2 *spans, Ctx &c) {
    const int nsm = c.nsm;
    int64_t off = 0;
    const int64_t *brp = B.row_ptr;
    for (int b = 2; b <= BIN_HUGE; b++) {
        int64_t cnt = counts[b];
        const int32_t *r = rows + off;
        const int2 *sp = spans + off;
        off += cnt;
        if (cnt == 0) continue;
        if (b <= 5) {
            // rows spanning at most SPAN_BW column blocks: bitmap over the span
            constexpr int WPB = 8;
            const size_t smem = (size_t)WPB * SpanLayout<SPAN_BW, WPB>::words * 4;
            SG_TRY(prep(k_sym_span<SPAN_BW, WPB>, smem));
            int64_t blocks = (cnt + WPB - 1) / WPB;
            blocks = blocks < (int64_t)nsm * 32 ? blocks : (int64_t)nsm * 32;
            c.begin(SPAN_LABEL[b], cnt);
            k_sym_span<SPAN_BW, WPB><<<(unsigned)blocks, WPB * 32, smem, c.s>>>(
                A.row_ptr, A.col_idx, brp, ccnt, pairs, sp, r, cnt, crp);
            c.end();
            SG_CUDA(cudaGetLastError());
        }
        switch (b) {
            case 2: SG_TRY((run_warp<128>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c, sp, SPAN_BW))); break;
            case 3: SG_TRY((run_warp<512>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c, sp, SPAN_BW))); break;
            case 4: SG_TRY((run_block<128, 2048>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c, sp, SPAN_BW))); break;
            case 5: SG_TRY((run_block<256, 8192>(A, brp, ccnt, pairs, r, cnt, crp, err, b, c, sp, SPAN_BW))); break;
            default: {
                int64_t nwords = (B.ncols + 31) / 32;
                bool shared = nwords <= SMEM_BITMAP_WORDS;
                size_t smem = shared ? (size_t)nwords * 4 : 0;
                SG_TRY(prep(k_sym_bitmap<BITMAP_BS>, smem));
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

// Narrow rows: rows of C whose columns all fall within a window of
// NARROW_W consecutive blocks of 32 columns (4096 columns), the common case
// of banded and stencil-like products such as the multigrid Galerkin
// operators of Section 3.2.
//
// Section 2.1 compresses each row of B into (block, 32-bit mask) pairs so
// that the union of column sets becomes bitwise ORs.  Over a narrow window
// the union needs no hash at all: a dense table of NARROW_W masks, indexed
// by block minus the window's first block, holds it exactly.
//
// * Symbolic (k_sym_narrow): one pass over every row of A computes the
//   row's products (Section 3.1: accumulator insertions = multiplications),
//   its compressed pairs and its column window from the first/last block of
//   each B_k; rows that fit the window OR their pairs into the table and
//   count popcounts (nnz(C_i)); every other row gets the analysis the hash
//   kernels need (symbolic bin, -1 marks for the second pass).
// * Numeric (k_num_narrow): the table is rebuilt from the same pairs, and
//   prefix counts of its masks give every column of the row its rank in the
//   sorted output: rank(c) = base[w] + popc(mask[w] & bits below c), with
//   w = c/32 - first block.  The dense accumulator of Section 3.1 is then
//   indexed by rank, so the row is written in column order with no hash
//   probe and no sort.  Products are taken one stored a_ik at a time, the
//   G lanes of a row on consecutive entries of B_k: entries of one row of B
//   have distinct columns, so within a step no two lanes of a row add to the
//   same rank and the update is a plain read-modify-write of shared memory.
#include <climits>
#include <type_traits>
#include "internal.cuh"

namespace sg {

// Quad (four words) of a row's window that lane gl of its G lanes takes in
// its j-th turn: rounds of G*P consecutive quads, P consecutive ones per
// lane (with G = 4, P = 2 puts the lanes 32 bytes apart, so that the two row
// slots served by one quarter of a warp, 4 words apart, use different banks).
template <int G, int P>
__device__ __forceinline__ int quad_of(int j, int gl) {
    return ((j / P) * G + gl) * P + (j % P);
}

// Stored entries of A are taken a batch of E at a time: every lane of a
// row's G lanes loads E / G of them at once (their loads in flight
// together), so the passes over the batch wait for memory once, not once
// per entry.  A lane keeps the start of B_k (also the start of its
// compressed pairs), its entries and its pairs in registers.
//
// Load the lane's entries pb + gl + G*u (u < E / G) of a row.  Entries past
// plen, with a column of A out of range or a row of B too long for the
// window get no pairs and no entries (and raise `bad` for the latter two).
template <int G, int E>
__device__ __forceinline__ void load_entries(const int32_t *__restrict__ acol, const int4 *__restrict__ desc,
                                             int64_t nrows_b, int64_t p0, int plen, int pb, int gl,
                                             long long (&q0)[E / G], int (&len)[E / G], int (&np)[E / G],
                                             bool &bad) {
    constexpr int EL = E / G;
    int k[EL];
#pragma unroll
    for (int u = 0; u < EL; u++) {
        const int pe = pb + gl + G * u;
        k[u] = pe < plen ? acol[p0 + pe] : -1;
    }
#pragma unroll
    for (int u = 0; u < EL; u++) {
        q0[u] = 0;
        len[u] = 0;
        np[u] = 0;
        if (pb + gl + G * u >= plen) continue;
        if ((unsigned)k[u] >= (unsigned)nrows_b) { bad = true; continue; }
        const int4 d = desc[k[u]];
        if (d.z > NARROW_W * 32 || d.w > NARROW_W) { bad = true; continue; }
        q0[u] = desc_start(d);
        len[u] = d.z;
        np[u] = d.w;
    }
}

// Exclusive prefix of the pair counts of a batch (entry e = gl + G*u is the
// lane's u-th) to pre[0..E], pre[E] = the batch's pairs, and the pair
// starts to q0s[].  Returns the batch's pairs (on every lane of the row).
template <int G, int E>
__device__ __forceinline__ int stage_pairs(const long long (&q0)[E / G], const int (&np)[E / G], long long *q0s,
                                           int *pre, int gl) {
    constexpr int EL = E / G;
    int carry = 0;
#pragma unroll
    for (int u = 0; u < EL; u++) {
        int incl = np[u];
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d, G);
            if (gl >= d) incl += y;
        }
        pre[gl + G * u] = carry + incl - np[u];
        q0s[gl + G * u] = q0[u];
        carry += __shfl_sync(0xffffffffu, incl, G - 1, G);
    }
    if (gl == 0) pre[E] = carry;
    return carry;
}

// OR the compressed pairs of a staged batch into the window table: the
// batch's pairs dealt over the row's lanes (lane gl takes pairs gl, gl + G,
// ...; loads of one B_k coalesce), each lane finding its entry with a
// cursor that only moves forward; four pairs loaded before their ORs
// (lanes of a row may hit the same word: atomic OR).
template <int G>
__device__ __forceinline__ void union_pairs(unsigned *tab, const long long *q0s, const int *pre, int total, int lo,
                                            const int2 *__restrict__ pairs, int gl, int &flag) {
    int e = 0;
    for (int t0 = gl; t0 < total; t0 += 4 * G) {
        int2 x[4];
        bool v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = t0 + u * G;
            v[u] = t < total;
            x[u] = make_int2(0, 0);
            if (v[u]) {
                while (pre[e + 1] <= t) e++;
                x[u] = pairs[q0s[e] + (t - pre[e])];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (!v[u]) continue;
            const unsigned wd = (unsigned)(x[u].x - lo);
            if (wd < (unsigned)NARROW_W) atomicOr(&tab[wd], (unsigned)x[u].y);
            else flag |= DERR_COUNT;
        }
    }
}

// ---------------------------------------------------------------- symbolic
constexpr int NARROW_SYM_E = 32;
constexpr int NARROW_SYM_WPB = 4;

// G lanes per row, 32/G rows per warp.  For row i: flops, pairs and window
// from desc[k] = {start, entries, pairs} and bmm[k] = {first block, last
// block} of every stored a_ik, a batch at a time (the first batch stays in
// registers for the union).  A row is narrow when it has products, no
// column of A out of range, a window of at most NARROW_W blocks and at most
// NARROW_PAIRS pairs; its count goes to crp[i+1], its first block to
// nlo[i] and BIN_NARROW to bins[i].  Other rows get nlo[i] = -1 and the
// symbolic bin of their bound (crp[i+1] = 0 for empty rows, -1 for the
// dense-bitmap bin), exactly as the analysis kernel gives them.
template <int G>
__global__ void __launch_bounds__(NARROW_SYM_WPB * 32) k_sym_narrow(
    int64_t n, int64_t nrows_b, int64_t nwords, const int64_t *__restrict__ arp,
    const int32_t *__restrict__ acol, const int4 *__restrict__ desc, const int2 *__restrict__ bmm,
    const int2 *__restrict__ pairs, int64_t *__restrict__ flops, uint8_t *__restrict__ bins,
    int64_t *__restrict__ crp, int32_t *__restrict__ nlo, DevState *st) {
    constexpr int E = NARROW_SYM_E, WPB = NARROW_SYM_WPB;
    constexpr int RPW = 32 / G, NR = WPB * RPW, QPL = NARROW_W / 4 / G, EL = E / G;
    constexpr int P = G >= 8 ? 1 : 8 / G;
    constexpr int QS = E + 1, PS = E + 2;   // padded row-slot strides of q0s, pre
    __shared__ __align__(16) unsigned tab_all[NR * NARROW_TAB_STRIDE];
    __shared__ long long q0_all[NR * QS];
    __shared__ int pre_all[NR * PS];
    __shared__ unsigned long long hist[NBINS];
    __shared__ unsigned long long fsum, alen_max;
    if (threadIdx.x < NBINS) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) { fsum = 0; alen_max = 0; }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / G, gl = lane % G, gbase = g * G;
    const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1) << gbase);
    const int slot = w * RPW + g;
    unsigned *t = tab_all + slot * NARROW_TAB_STRIDE;
    long long *q0s = q0_all + slot * QS;
    int *pre = pre_all + slot * PS;
    long long wf = 0, wl = 0;
    bool bad = false;
    int flag = 0;
    const int64_t stride = (int64_t)gridDim.x * NR;
    for (int64_t base = (int64_t)blockIdx.x * NR + w * RPW; base < n; base += stride) {
        const int64_t i = base + g;
        const bool live = i < n;
        const int64_t p0 = live ? arp[i] : 0;
        const int plen = live ? (int)(arp[i + 1] - p0) : 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, plen);
        long long f = 0, cp = 0;
        int lo = INT_MAX, hi = INT_MIN;
        bool rowbad = false;
        long long q0[EL];
        int np[EL];
        for (int pb = 0; pb < maxlen; pb += E) {
            int k[EL];
#pragma unroll
            for (int u = 0; u < EL; u++) {
                const int pe = pb + gl + G * u;
                k[u] = pe < plen ? acol[p0 + pe] : -1;
            }
#pragma unroll
            for (int u = 0; u < EL; u++) {
                if (pb == 0) { q0[u] = 0; np[u] = 0; }
                if (pb + gl + G * u >= plen) continue;
                if ((unsigned)k[u] >= (unsigned)nrows_b) { rowbad = true; continue; }
                const int4 d = desc[k[u]];
                const int2 m = bmm[k[u]];
                f += d.z;
                cp += d.w;
                lo = min(lo, m.x);
                hi = max(hi, m.y);
                if (pb == 0 && d.w <= NARROW_W) {
                    q0[u] = desc_start(d);
                    np[u] = d.w;
                }
            }
        }
#pragma unroll
        for (int d = G / 2; d > 0; d >>= 1) {
            f += __shfl_xor_sync(0xffffffffu, f, d, G);
            cp += __shfl_xor_sync(0xffffffffu, cp, d, G);
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d, G));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d, G));
        }
        rowbad = (__ballot_sync(0xffffffffu, rowbad) & gm) != 0;
        bad |= rowbad;
        const bool nar = live && f > 0 && !rowbad && hi >= lo && hi - lo < NARROW_W && cp <= NARROW_PAIRS;
        int cnt = 0;
        if (__any_sync(0xffffffffu, nar)) {
            if (nar) {
#pragma unroll
                for (int j = 0; j < QPL; j++) *(uint4 *)&t[4 * quad_of<G, P>(j, gl)] = make_uint4(0u, 0u, 0u, 0u);
            }
            // batches of the narrow rows (the first one is in registers)
            const int nmax = __reduce_max_sync(0xffffffffu, nar ? plen : 0);
            for (int pb = 0; pb < nmax; pb += E) {
                if (pb > 0) {
                    int len[EL];
                    bool b2 = false;
                    load_entries<G, E>(acol, desc, nrows_b, p0, nar ? plen : 0, pb, gl, q0, len, np, b2);
                }
                if (!nar) {
#pragma unroll
                    for (int u = 0; u < EL; u++) np[u] = 0;
                }
                const int total = stage_pairs<G, E>(q0, np, q0s, pre, gl);
                __syncwarp();
                union_pairs<G>(t, q0s, pre, total, lo, pairs, gl, flag);
                __syncwarp();
            }
            if (nar) {
#pragma unroll
                for (int j = 0; j < QPL; j++) {
                    const uint4 v = *(const uint4 *)&t[4 * quad_of<G, P>(j, gl)];
                    cnt += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                }
            }
#pragma unroll
            for (int d = G / 2; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d, G);
            __syncwarp();
        }
        int b = BIN_EMPTY;
        const bool lead = live && gl == 0;
        if (lead) {
            flops[i] = f;
            wf += f;
            wl = max(wl, (long long)plen);
            if (nar) {
                b = BIN_NARROW;
                bins[i] = (uint8_t)BIN_NARROW;
                crp[i + 1] = cnt;
                nlo[i] = lo;
            } else {
                const long long keys = cp < (long long)nwords ? cp : (long long)nwords;
                b = sym_bin(keys, cp);
                bins[i] = (uint8_t)b;
                if (b == BIN_EMPTY) crp[i + 1] = 0;
                if (b == BIN_HUGE) crp[i + 1] = -1;
                nlo[i] = -1;
            }
        }
        warp_hist(hist, lead, b);
    }
    if (bad) atomicOr(&st->err, DERR_COL_RANGE);
    if (flag) atomicOr(&st->err, flag);
    for (int d = 16; d > 0; d >>= 1) {
        wf += __shfl_xor_sync(0xffffffffu, wf, d);
        wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, d));
    }
    if (lane == 0 && wf) atomicAdd(&fsum, (unsigned long long)wf);
    if (lane == 0 && wl) atomicMax(&alen_max, (unsigned long long)wl);
    __syncthreads();
    if (threadIdx.x == 0 && fsum) atomicAdd((unsigned long long *)&st->flops_total, fsum);
    if (threadIdx.x == 0 && alen_max && alen_max > (unsigned long long)*(volatile long long *)&st->max_alen)
        atomicMax((unsigned long long *)&st->max_alen, alen_max);
    if (threadIdx.x < NBINS && hist[threadIdx.x]) {
        atomicAdd((unsigned long long *)&st->sym_hist[threadIdx.x], hist[threadIdx.x]);
        if (threadIdx.x == BIN_HUGE)
            atomicAdd((unsigned long long *)&st->bin_count[0][BIN_HUGE], hist[threadIdx.x]);
    }
}

// Blocks of `kern` that fit on all SMs at once (at least one per SM): the
// narrow kernels stride over the rows with one resident wave.
template <typename K>
static int64_t resident_blocks(K kern, int threads, int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (int64_t)per_sm * nsm;
}

template <int G>
static int run_sym_narrow(const spgemm_csr &A, const spgemm_csr &B, const int4 *desc, const int2 *bmm,
                          const int2 *pairs, int64_t *flops, uint8_t *bins, int64_t *crp, int32_t *nlo,
                          DevState *st, Ctx &c) {
    constexpr int NT = NARROW_SYM_WPB * 32, NR = NARROW_SYM_WPB * (32 / G);
    int64_t blocks = (A.nrows + NR - 1) / NR;
    const int64_t cap = resident_blocks(k_sym_narrow<G>, NT, c.nsm);
    blocks = blocks < cap ? blocks : cap;
    const int64_t nwords = (B.ncols + 31) / 32;
    c.begin("symbolic.narrow", A.nrows);
    k_sym_narrow<G><<<(unsigned)blocks, NT, 0, c.s>>>(A.nrows, B.nrows, nwords, A.row_ptr, A.col_idx, desc,
                                                      bmm, pairs, flops, bins, crp, nlo, st);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

int launch_sym_narrow(const spgemm_csr &A, const spgemm_csr &B, const int4 *desc, const int2 *bmm,
                      const int2 *pairs, int64_t *flops, uint8_t *bins, int64_t *crp, int32_t *nlo,
                      DevState *st, int G, Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    switch (G) {
        case 4: return run_sym_narrow<4>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, st, c);
        case 8: return run_sym_narrow<8>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, st, c);
        case 16: return run_sym_narrow<16>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, st, c);
        default: return run_sym_narrow<32>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, st, c);
    }
}

// ---------------------------------------------------------------- numeric
struct NarrowP {
    const int64_t *arp; const int32_t *acol; const void *aval;
    const int32_t *bcol; const void *bval;
    const int64_t *crp; int32_t *ccol; void *cval;
    const int4 *bdesc; const int2 *pairs; const int32_t *nlo; const uint8_t *bins;
    int64_t n, nrows_b;
};

// A staged entry of the product pass: the start of B_k in B and a_ik.
template <typename V>
struct __align__(16) NarrowEnt {
    long long q;
    V a;
};

// Shared memory of k_num_narrow, per row slot: the window's masks
// (NARROW_TAB_STRIDE words), the rank of each word's first column (a byte:
// rows hold at most NARROW_NMAX < 256 entries; NARROW_BASE_STRIDE bytes),
// the accumulator by rank (NARROW_ACC_STRIDE values) and the batch of
// stored entries: {start, value}, length, and the prefix of their pair
// counts.  The strides are padded so that the row slots of a warp start on
// different banks: lanes of different rows reading the same word of their
// windows or the same entry do not conflict.
template <int G, int WPB, int E, typename V>
struct NarrowSmem {
    static constexpr int NR = WPB * (32 / G), ES = E + 1, PS = E + 2;
    NarrowEnt<V> ent[NR * ES];
    unsigned tab[NR * NARROW_TAB_STRIDE];
    V acc[NR * NARROW_ACC_STRIDE];
    int elen[NR * ES];
    int pre[NR * PS];
    unsigned char base[NR * NARROW_BASE_STRIDE];
};

// Stage a batch for both passes: {start, a_ik} and length of every entry,
// the pair starts and prefix for the union.  Returns the batch's pairs.
template <int G, int E, typename V>
__device__ __forceinline__ int stage_numeric(const long long (&q0)[E / G], const int (&len)[E / G],
                                             const int (&np)[E / G], const V *__restrict__ aval, int64_t p0,
                                             int plen, int pb, NarrowEnt<V> *ent, int *elen, int *pre, int gl) {
    constexpr int EL = E / G;
    int carry = 0;
#pragma unroll
    for (int u = 0; u < EL; u++) {
        const int e = gl + G * u;
        NarrowEnt<V> x;
        x.q = q0[u];
        x.a = pb + e < plen ? aval[p0 + pb + e] : (V)0;
        ent[e] = x;
        elen[e] = len[u];
        int incl = np[u];
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d, G);
            if (gl >= d) incl += y;
        }
        pre[e] = carry + incl - np[u];
        carry += __shfl_sync(0xffffffffu, incl, G - 1, G);
    }
    if (gl == 0) pre[E] = carry;
    return carry;
}

// OR of the batch's pairs (union_pairs over the staged starts).
template <int G, typename V>
__device__ __forceinline__ void union_staged(unsigned *tab, const NarrowEnt<V> *ent, const int *pre, int total,
                                             int lo, const int2 *__restrict__ pairs, int gl, int &flag) {
    int e = 0;
    for (int t0 = gl; t0 < total; t0 += 4 * G) {
        int2 x[4];
        bool v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = t0 + u * G;
            v[u] = t < total;
            x[u] = make_int2(0, 0);
            if (v[u]) {
                while (pre[e + 1] <= t) e++;
                x[u] = pairs[ent[e].q + (t - pre[e])];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (!v[u]) continue;
            const unsigned wd = (unsigned)(x[u].x - lo);
            if (wd < (unsigned)NARROW_W) atomicOr(&tab[wd], (unsigned)x[u].y);
            else flag |= DERR_COUNT;
        }
    }
}

// Rank of column c in the row (-1 if it is not in the row's window union:
// a pattern changed after the symbolic phase, flagged).
__device__ __forceinline__ int rank_of(int c, int lo, const unsigned *tab, const unsigned char *base, bool ok,
                                       int &flag) {
    const unsigned wd = (unsigned)((c >> 5) - lo);
    const bool in = ok && wd < (unsigned)NARROW_W;
    const unsigned m = in ? tab[wd] : 0u;
    const unsigned bit = 1u << (c & 31);
    flag |= (ok && !(m & bit)) ? DERR_COUNT : 0;
    return in ? base[wd] + __popc(m & (bit - 1u)) : -1;
}

// Chunks per lane and step in the cursor form of the product pass.
constexpr int NARROW_U = 4;

// G lanes per row, 32/G rows per warp, WPB warps per block, batches of E
// stored entries; rows with bins[i] == BIN_NARROW, in row order.  The
// window's words are handled in quads of four, P consecutive quads per lane
// and round (conflict-free 16-byte accesses); ranks run over the quads in
// order, one group scan per round.  Product pass, two forms:
// * G = 4 (rows of B of a few entries): two stored entries per step, their
//   chunks of G entries of B_k in an inner loop bounded by the warp's
//   longest row of B among them; both entries' loads before their updates;
// * G >= 8: a cursor walking the batch chunk by chunk (every lane of a row
//   holding the same cursor), NARROW_U chunks per step, loads first.
// Updates of one step's chunk are conflict-free (the entries of one row of
// B have distinct columns); chunks of different entries are separated by
// __syncwarp.
template <int G, int WPB, int E, typename V>
__global__ void __launch_bounds__(WPB * 32) k_num_narrow(NarrowP a, int *err) {
    using S = NarrowSmem<G, WPB, E, V>;
    constexpr int RPW = 32 / G, NR = WPB * RPW, QPL = NARROW_W / 4 / G, U = NARROW_U, EL = E / G;
    constexpr int P = G >= 8 ? 1 : 8 / G;
    __shared__ __align__(16) S sm;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / G, gl = lane % G;
    const int slot = w * RPW + g;
    unsigned *tab = sm.tab + slot * NARROW_TAB_STRIDE;
    unsigned char *base = sm.base + slot * NARROW_BASE_STRIDE;
    V *acc = sm.acc + slot * NARROW_ACC_STRIDE;
    NarrowEnt<V> *ent = sm.ent + slot * S::ES;
    int *elen = sm.elen + slot * S::ES;
    int *pre = sm.pre + slot * S::PS;
    const V *__restrict__ aval = (const V *)a.aval;
    const V *__restrict__ bval = (const V *)a.bval;
    const int32_t *__restrict__ bcol = a.bcol;
    int flag = 0;
    const int64_t stride = (int64_t)gridDim.x * NR;
    for (int64_t rb = (int64_t)blockIdx.x * NR + w * RPW; rb < a.n; rb += stride) {
        const int64_t i = rb + g;
        bool act = i < a.n && a.bins[i] == BIN_NARROW;
        if (!__any_sync(0xffffffffu, act)) continue;
        const int lo = act ? a.nlo[i] : 0;
        const int64_t p0 = act ? a.arp[i] : 0;
        int plen = act ? (int)(a.arp[i + 1] - p0) : 0;
        const int64_t out = act ? a.crp[i] : 0;
        const int nn = act ? (int)(a.crp[i + 1] - out) : 0;
        if (act && (nn > NARROW_NMAX || lo < 0)) { flag |= DERR_COUNT; act = false; }
        if (!act) plen = 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, plen);
        const int nbatch = (maxlen + E - 1) / E;
        if (act) {
#pragma unroll
            for (int j = 0; j < QPL; j++) *(uint4 *)&tab[4 * quad_of<G, P>(j, gl)] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int r = gl; r < NARROW_NMAX; r += G) acc[r] = (V)0;
        }
        // pass 1: the union of the rows of B the row reaches, over its
        // window, batch by batch; the last batch stays staged for pass 2
        long long q0[EL];
        int len[EL], np[EL];
        bool bad = false;
        for (int b = 0; b < nbatch; b++) {
            load_entries<G, E>(a.acol, a.bdesc, a.nrows_b, p0, plen, b * E, gl, q0, len, np, bad);
            const int total = stage_numeric<G, E, V>(q0, len, np, aval, p0, plen, b * E, ent, elen, pre, gl);
            __syncwarp();
            union_staged<G, V>(tab, ent, pre, total, lo, a.pairs, gl, flag);
            __syncwarp();
        }
        if (bad) flag |= DERR_COL_RANGE;
        // rank of the first column of every word: quads in order; each round
        // the lanes take G*P consecutive quads, P each, and scan their counts
        int carry = 0;
#pragma unroll
        for (int j = 0; j < QPL / P; j++) {
            int cw[4 * P];
            int cl = 0;
#pragma unroll
            for (int pq = 0; pq < P; pq++) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (act) v = *(const uint4 *)&tab[4 * quad_of<G, P>(j * P + pq, gl)];
                cw[4 * pq] = __popc(v.x);
                cw[4 * pq + 1] = __popc(v.y);
                cw[4 * pq + 2] = __popc(v.z);
                cw[4 * pq + 3] = __popc(v.w);
                cl += cw[4 * pq] + cw[4 * pq + 1] + cw[4 * pq + 2] + cw[4 * pq + 3];
            }
            int incl = cl;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d, G);
                if (gl >= d) incl += y;
            }
            int run = carry + incl - cl;
#pragma unroll
            for (int pq = 0; pq < P; pq++) {
                unsigned packed = 0;
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    packed |= (unsigned)run << (8 * u);
                    run += cw[4 * pq + u];
                }
                if (act) *(unsigned *)&base[4 * quad_of<G, P>(j * P + pq, gl)] = packed;
            }
            carry += __shfl_sync(0xffffffffu, incl, G - 1, G);
        }
        if (act && carry != nn) { flag |= DERR_COUNT; act = false; }
        if (!act) plen = 0;
        __syncwarp();
        // pass 2: products, batches in reverse order (the last one is staged)
        for (int b = nbatch - 1; b >= 0; b--) {
            const int pb = b * E;
            if (b != nbatch - 1) {
                bool b2 = false;
                load_entries<G, E>(a.acol, a.bdesc, a.nrows_b, p0, plen, pb, gl, q0, len, np, b2);
                stage_numeric<G, E, V>(q0, len, np, aval, p0, plen, pb, ent, elen, pre, gl);
                __syncwarp();
            }
            const int nb = act ? min(E, plen - pb) : 0;
            if (G == 4) {
                const int nbw = __reduce_max_sync(0xffffffffu, nb > 0 ? nb : 0);
                for (int e0 = 0; e0 < nbw; e0 += 2) {
                    NarrowEnt<V> x0, x1;
                    x0.q = 0; x0.a = 0; x1.q = 0; x1.a = 0;
                    int l0 = 0, l1 = 0;
                    if (e0 < nb) { x0 = ent[e0]; l0 = elen[e0]; }
                    if (e0 + 1 < nb) { x1 = ent[e0 + 1]; l1 = elen[e0 + 1]; }
                    const int chm = __reduce_max_sync(0xffffffffu, max(l0, l1));
                    for (int j = gl; j - gl < chm; j += G) {
                        const bool ok0 = j < l0, ok1 = j < l1;
                        int c0 = 0, c1 = 0;
                        V v0 = 0, v1 = 0;
                        if (ok0) { c0 = bcol[x0.q + j]; v0 = bval[x0.q + j]; }
                        if (ok1) { c1 = bcol[x1.q + j]; v1 = bval[x1.q + j]; }
                        const int r0 = rank_of(c0, lo, tab, base, ok0, flag);
                        const int r1 = rank_of(c1, lo, tab, base, ok1, flag);
                        if (r0 >= 0) acc[r0] = fma(x0.a, v0, acc[r0]);
                        __syncwarp();
                        if (r1 >= 0) acc[r1] = fma(x1.a, v1, acc[r1]);
                        __syncwarp();
                    }
                }
            } else {
                int e = 0, j = 0, clen = 0;
                long long cq = 0;
                V ca = 0;
                if (nb > 0) {
                    const NarrowEnt<V> x = ent[0];
                    cq = x.q + gl;
                    ca = x.a;
                    clen = elen[0];
                }
                while (__any_sync(0xffffffffu, e < nb)) {
                    int c[U];
                    V v[U], av[U];
                    bool ok[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        ok[u] = e < nb && j + gl < clen;
                        c[u] = 0;
                        v[u] = 0;
                        if (ok[u]) {
                            c[u] = bcol[cq + j];
                            v[u] = bval[cq + j];
                        }
                        av[u] = ca;
                        j += G;
                        if (j >= clen && e < nb) {
                            e++;
                            j = 0;
                            if (e < nb) {
                                const NarrowEnt<V> x = ent[e];
                                cq = x.q + gl;
                                ca = x.a;
                                clen = elen[e];
                            }
                        }
                    }
                    int r[U];
#pragma unroll
                    for (int u = 0; u < U; u++) r[u] = rank_of(c[u], lo, tab, base, ok[u], flag);
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        if (r[u] >= 0) acc[r[u]] = fma(av[u], v[u], acc[r[u]]);
                        __syncwarp();
                    }
                }
            }
            __syncwarp();
        }
        // write the row in column order: every lane its quads' columns, from
        // the rank of each word's first column
        if (act) {
#pragma unroll
            for (int jj = 0; jj < QPL; jj++) {
                const int q = quad_of<G, P>(jj, gl);
                const uint4 v = *(const uint4 *)&tab[4 * q];
                const unsigned bq = *(const unsigned *)&base[4 * q];
                const unsigned mw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    unsigned m = mw[u];
                    int rr = (int)((bq >> (8 * u)) & 0xffu);
                    const int col0 = (lo + 4 * q + u) * 32;
                    while (m) {
                        const int bpos = __ffs(m) - 1;
                        m &= m - 1u;
                        a.ccol[out + rr] = col0 + bpos;
                        ((V *)a.cval)[out + rr] = acc[rr];
                        rr++;
                    }
                }
            }
        }
        __syncwarp();
    }
    if (flag) atomicOr(err, flag);
}

template <int G, int E, typename V>
static int run_num_narrow(const NarrowP &p, int *err, Ctx &c) {
    constexpr int WPB = 4, NR = WPB * (32 / G);
    int64_t blocks = (p.n + NR - 1) / NR;
    const int64_t cap = resident_blocks(k_num_narrow<G, WPB, E, V>, WPB * 32, c.nsm);
    blocks = blocks < cap ? blocks : cap;
    c.begin("numeric.narrow", p.n);
    k_num_narrow<G, WPB, E, V><<<(unsigned)blocks, WPB * 32, 0, c.s>>>(p, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

int launch_num_narrow(int dtype, const spgemm_csr &A, const spgemm_csr &B, spgemm_csr &C, const int4 *bdesc,
                      const int2 *pairs, const int32_t *nlo, const uint8_t *bins, int *err, int G, Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    NarrowP p{A.row_ptr, A.col_idx, A.values, B.col_idx, B.values, C.row_ptr, C.col_idx, C.values,
              bdesc, pairs, nlo, bins, A.nrows, B.nrows};
    if (dtype == SPGEMM_F32) {
        switch (G) {
            case 4: return run_num_narrow<4, 16, float>(p, err, c);
            case 8: return run_num_narrow<8, 32, float>(p, err, c);
            default: return run_num_narrow<16, 32, float>(p, err, c);
        }
    }
    switch (G) {
        case 4: return run_num_narrow<4, 16, double>(p, err, c);
        case 8: return run_num_narrow<8, 32, double>(p, err, c);
        default: return run_num_narrow<16, 32, double>(p, err, c);
    }
}

}  // namespace sg

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
//   A narrow row with at most NARROW_NMAX outputs also leaves its union for
//   the numeric phase, as the list of its non-empty words in order, each
//   with its mask and the rank of its first column (prefix counts of the
//   masks).
// * Numeric (k_num_narrow): the row's list is scattered back into the window
//   table, which then gives every column its rank in the sorted output:
//   rank(c) = base[w] + popc(mask[w] & bits below c), w = c/32 - first
//   block.  The dense accumulator of Section 3.1 is indexed by rank, so the
//   row is written in column order with no hash probe and no sort.
//   Products are taken one chunk of G consecutive entries of B_k at a time
//   by the G lanes of a row: entries of one row of B have distinct columns,
//   so within a chunk no two lanes of a row add to the same rank and the
//   update is a plain read-modify-write of shared memory.
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
// per entry.
//
// Load the lane's entries pb + gl + G*u (u < E / G) of a row: the start of
// B_k in B (also the start of its compressed pairs), its entries and pairs.
// Entries past plen, with a column of A out of range or a row of B too long
// for the window get no pairs and no entries (and raise `bad` for the
// latter two).
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

// ---------------------------------------------------------------- symbolic
constexpr int NARROW_SYM_WPB = 8;
constexpr int SYM_EU = 4;   // entries of A per lane whose loads are in flight together

// G lanes per row, 32/G rows per warp.  For row i: flops, pairs and window
// from desc[k] = {start, entries, pairs} and bmm[k] = {first block, last
// block} of every stored a_ik (lanes strided over the entries).  A row is narrow when it has products, no
// column of A out of range, a window of at most NARROW_W blocks and at most
// NARROW_PAIRS pairs; its count goes to crp[i+1], its first block to
// nlo[i] and BIN_NARROW to bins[i]; its non-empty words, in order, to
// ulist[i*NARROW_NMAX ...] as {word | rank of its first column << 8, mask}
// (the first NARROW_NMAX of them) and their number to nwords[i].  Other
// rows get nlo[i] = -1 and the symbolic bin of their bound (crp[i+1] = 0
// for empty rows, -1 for the dense-bitmap bin), exactly as the analysis
// kernel gives them.
template <int G>
__global__ void __launch_bounds__(NARROW_SYM_WPB * 32) k_sym_narrow(
    int64_t n, int64_t nrows_b, int64_t nwords_b, const int64_t *__restrict__ arp,
    const int32_t *__restrict__ acol, const int4 *__restrict__ desc, const int2 *__restrict__ bmm,
    const int2 *__restrict__ pairs, int64_t *__restrict__ flops, uint8_t *__restrict__ bins,
    int64_t *__restrict__ crp, int32_t *__restrict__ nlo, uint8_t *__restrict__ nwords,
    uint2 *__restrict__ ulist, DevState *st) {
    constexpr int WPB = NARROW_SYM_WPB;
    constexpr int RPW = 32 / G, NR = WPB * RPW, QPL = NARROW_W / 4 / G;
    constexpr int P = G >= 8 ? 1 : 8 / G;
    __shared__ __align__(16) unsigned tab_all[NR * NARROW_TAB_STRIDE];
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
        // SYM_EU entries per lane at a time: their loads of A, then of the
        // rows' descriptors, issued together
        for (int e0 = 0; e0 < plen; e0 += G * SYM_EU) {
            int k[SYM_EU];
#pragma unroll
            for (int u = 0; u < SYM_EU; u++) {
                const int e = e0 + gl + G * u;
                k[u] = e < plen ? acol[p0 + e] : -1;
            }
            int4 d[SYM_EU];
            int2 m[SYM_EU];
#pragma unroll
            for (int u = 0; u < SYM_EU; u++) {
                const bool ok = (unsigned)k[u] < (unsigned)nrows_b;
                rowbad |= !ok && e0 + gl + G * u < plen;
                d[u] = ok ? desc[k[u]] : make_int4(0, 0, 0, 0);
                m[u] = ok ? bmm[k[u]] : make_int2(INT_MAX, INT_MIN);
            }
#pragma unroll
            for (int u = 0; u < SYM_EU; u++) {
                f += d[u].z;
                cp += d[u].w;
                lo = min(lo, m[u].x);
                hi = max(hi, m[u].y);
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
        int cnt = 0, nz = 0;
        if (__any_sync(0xffffffffu, nar)) {
            if (nar) {
#pragma unroll
                for (int j = 0; j < QPL; j++) *(uint4 *)&t[4 * quad_of<G, P>(j, gl)] = make_uint4(0u, 0u, 0u, 0u);
            }
            __syncwarp();
            // the union: every lane ORs the pairs of its own entries (lanes of
            // a row may hit the same word: atomic OR), SYM_EU entries at a
            // time, the loads of one pair of each issued together
            if (nar) {
                for (int e0 = 0; e0 < plen; e0 += G * SYM_EU) {
                    int k[SYM_EU];
#pragma unroll
                    for (int u = 0; u < SYM_EU; u++) {
                        const int e = e0 + gl + G * u;
                        k[u] = e < plen ? acol[p0 + e] : -1;
                    }
                    const int2 *pp[SYM_EU];
                    int np[SYM_EU];
                    int npmax = 0;
#pragma unroll
                    for (int u = 0; u < SYM_EU; u++) {
                        const int4 d = k[u] >= 0 ? desc[k[u]] : make_int4(0, 0, 0, 0);
                        pp[u] = pairs + desc_start(d);
                        np[u] = d.w <= NARROW_W ? d.w : 0;
                        npmax = max(npmax, np[u]);
                    }
                    for (int tt = 0; tt < npmax; tt++) {
                        int2 x[SYM_EU];
#pragma unroll
                        for (int u = 0; u < SYM_EU; u++) x[u] = tt < np[u] ? pp[u][tt] : make_int2(lo, 0);
#pragma unroll
                        for (int u = 0; u < SYM_EU; u++) {
                            const unsigned wx = (unsigned)(x[u].x - lo);
                            if (wx < (unsigned)NARROW_W) {
                                if (x[u].y) atomicOr(&t[wx], (unsigned)x[u].y);
                            } else {
                                flag |= DERR_COUNT;
                            }
                        }
                    }
                }
            }
            __syncwarp();
            // count, and the list of non-empty words in order with the rank
            // of each word's first column (quads in order, group scans)
            uint2 *ul = ulist + (live ? i : 0) * NARROW_NMAX;
#pragma unroll
            for (int j = 0; j < QPL / P; j++) {
                uint4 v[P];
                int cl = 0, zl = 0;
#pragma unroll
                for (int pq = 0; pq < P; pq++) {
                    v[pq] = make_uint4(0u, 0u, 0u, 0u);
                    if (nar) v[pq] = *(const uint4 *)&t[4 * quad_of<G, P>(j * P + pq, gl)];
                    cl += __popc(v[pq].x) + __popc(v[pq].y) + __popc(v[pq].z) + __popc(v[pq].w);
                    zl += (v[pq].x != 0) + (v[pq].y != 0) + (v[pq].z != 0) + (v[pq].w != 0);
                }
                int ci = cl, zi = zl;
#pragma unroll
                for (int d = 1; d < G; d <<= 1) {
                    const int y1 = __shfl_up_sync(0xffffffffu, ci, d, G);
                    const int y2 = __shfl_up_sync(0xffffffffu, zi, d, G);
                    if (gl >= d) { ci += y1; zi += y2; }
                }
                int run = cnt + ci - cl, idx = nz + zi - zl;
#pragma unroll
                for (int pq = 0; pq < P; pq++) {
                    const unsigned mw[4] = {v[pq].x, v[pq].y, v[pq].z, v[pq].w};
                    const int w0 = 4 * quad_of<G, P>(j * P + pq, gl);
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        if (nar && mw[u] && idx < NARROW_NMAX)
                            ul[idx] = make_uint2((unsigned)(w0 + u) | ((unsigned)run << 8), mw[u]);
                        idx += mw[u] != 0u;
                        run += __popc(mw[u]);
                    }
                }
                cnt += __shfl_sync(0xffffffffu, ci, G - 1, G);
                nz += __shfl_sync(0xffffffffu, zi, G - 1, G);
            }
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
                nwords[i] = (uint8_t)min(nz, 255);
            } else {
                const long long keys = cp < (long long)nwords_b ? cp : (long long)nwords_b;
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

template <int G>
static int run_sym_narrow(const spgemm_csr &A, const spgemm_csr &B, const int4 *desc, const int2 *bmm,
                          const int2 *pairs, int64_t *flops, uint8_t *bins, int64_t *crp, int32_t *nlo,
                          uint8_t *nwords, uint2 *ulist, DevState *st, Ctx &c) {
    constexpr int NT = NARROW_SYM_WPB * 32, NR = NARROW_SYM_WPB * (32 / G);
    int64_t blocks = (A.nrows + NR - 1) / NR;
    const int64_t cap = resident_blocks(k_sym_narrow<G>, NT, c.nsm);
    blocks = blocks < cap ? blocks : cap;
    const int64_t nwb = (B.ncols + 31) / 32;
    c.begin("symbolic.narrow", A.nrows);
    k_sym_narrow<G><<<(unsigned)blocks, NT, 0, c.s>>>(A.nrows, B.nrows, nwb, A.row_ptr, A.col_idx, desc, bmm,
                                                      pairs, flops, bins, crp, nlo, nwords, ulist, st);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

int launch_sym_narrow(const spgemm_csr &A, const spgemm_csr &B, const int4 *desc, const int2 *bmm,
                      const int2 *pairs, int64_t *flops, uint8_t *bins, int64_t *crp, int32_t *nlo,
                      uint8_t *nwords, uint2 *ulist, DevState *st, int G, Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    switch (G) {
        case 4: return run_sym_narrow<4>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, nwords, ulist, st, c);
        case 8: return run_sym_narrow<8>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, nwords, ulist, st, c);
        case 16: return run_sym_narrow<16>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, nwords, ulist, st, c);
        default: return run_sym_narrow<32>(A, B, desc, bmm, pairs, flops, bins, crp, nlo, nwords, ulist, st, c);
    }
}

// ---------------------------------------------------------------- numeric
struct NarrowP {
    const int64_t *arp; const int32_t *acol; const void *aval;
    const int32_t *bcol; const void *bval;
    const int64_t *crp; int32_t *ccol; void *cval;
    const int4 *bdesc; const int32_t *nlo; const uint8_t *nwords; const uint2 *ulist; const uint8_t *bins;
    int64_t n, nrows_b;
};

// A staged entry of the product pass: the start of B_k in B (as 32-bit
// halves: with fewer than 2^31 entries in B the high half is free and holds
// the length of B_k), and a_ik.
template <typename V>
struct __align__(16) NarrowEnt {
    int q, hl;
    V a;
};

// popc of the bits of m below bit s (0 <= s < 32): m shifted up by 32 - s,
// a shift of 32 giving 0 (the PTX shift clamps its amount).
__device__ __forceinline__ int popc_below(unsigned m, unsigned s) {
    unsigned r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(m), "r"(32u - s));
    return __popc(r);
}

// Shared memory of k_num_narrow.  Per warp, for its 32/G row slots: the
// window's masks and the rank of each word's first column (a byte: rows
// hold at most NARROW_NMAX < 256 entries), word major and row slot minor,
// so that in one instruction the lanes of different row slots never meet on
// a bank whatever words their rows look up; and the accumulator by rank,
// entry r of slot g at r * ACC_RS + g * ACC_GS.  A row's G lanes update G
// distinct ranks per chunk.  With four lanes a row, the slots lie 34
// eight-byte words apart (ranks adjacent within a slot): 270 words a warp,
// small enough for six blocks of four warps an SM (the earlier stride of
// four words per rank and 33 per slot spread a stencil row's neighbouring
// ranks over more banks, but its 356 words a warp left room for five
// blocks; on the 128^3 Galerkin A*P the sixth block gains more than the
// extra conflicts cost).
// Per row slot: the batch of stored entries ({start, value}, length; the
// lengths apart only when B has 2^31 entries or more), padded so that the
// slots of a warp start on different banks.
template <int G, int WPB, int E, typename V, bool IDX32>
struct NarrowSmem {
    static constexpr int RPW = 32 / G, NR = WPB * RPW, ES = E + 1;
    static constexpr int ACC_RS = 1, ACC_GS = G == 4 ? 34 : 40;
    static constexpr int ACC_SZ = (ACC_RS * (NARROW_NMAX - 1) + ACC_GS * (RPW - 1) + 2) & ~1;
    NarrowEnt<V> ent[NR * ES];
    unsigned tab[WPB * NARROW_W * RPW];
    V acc[WPB * ACC_SZ];
    int elen[IDX32 ? 1 : NR * ES];
    unsigned char base[WPB * NARROW_W * RPW];
};

// Chunks per lane and step in the product pass: their loads of B are issued
// before any of their updates (three: with four, the registers of the
// four-lane kernel leave room for five blocks an SM instead of six).
constexpr int NARROW_U = 3;

// Blocks an SM of the four-lane kernel: six (24 warps; 80 registers a
// thread, 37.8 KB of shared memory a block).  The other lane counts leave
// the register count to the compiler (a minimum of 0 blocks): with eight
// lanes it takes 64 registers, eight blocks an SM.
constexpr int NARROW_MINB4 = 6;

// G lanes per row, 32/G rows per warp, WPB warps per block, batches of E
// stored entries; rows with bins[i] == BIN_NARROW, in row order.  The row's
// word list (left by the symbolic phase) is scattered into the window table
// and kept in registers for the output (and to clear the table again after
// the row: the table is cleared once at the start and holds only the
// current rows' words).  The product pass walks a staged batch one chunk of
// G entries of B_k at a time, every lane of a row holding the same cursor
// (the current entry's start, value and length); an idle lane loads the
// first entry of B and skips its update (predicated), and so does a column
// missing from the row's window (flagged).  IDX32: B has fewer than 2^31
// entries (32-bit offsets).
template <int G, int WPB, int E, typename V, bool IDX32>
__global__ void __launch_bounds__(WPB * 32, G == 4 ? NARROW_MINB4 : 0) k_num_narrow(NarrowP a, int *err) {
    using S = NarrowSmem<G, WPB, E, V, IDX32>;
    constexpr int RPW = 32 / G, NR = WPB * RPW, U = NARROW_U, EL = E / G;
    constexpr int LPL = NARROW_NMAX / G;
    __shared__ __align__(16) S sm;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / G, gl = lane % G;
    const int slot = w * RPW + g;
    // this row slot's column of the warp's tables: word wd at tab[wd * RPW]
    unsigned *tab = sm.tab + w * NARROW_W * RPW + g;
    unsigned char *base = sm.base + w * NARROW_W * RPW + g;
    V *acc = sm.acc + w * S::ACC_SZ + g * S::ACC_GS;
    NarrowEnt<V> *ent = sm.ent + slot * S::ES;
    int *elen = sm.elen + slot * S::ES;
    const V *__restrict__ aval = (const V *)a.aval;
    const V *__restrict__ bval = (const V *)a.bval;
    const int32_t *__restrict__ bcol = a.bcol;
    {
        uint4 *t4 = (uint4 *)(sm.tab + w * NARROW_W * RPW);
#pragma unroll
        for (int q = lane; q < NARROW_W * RPW / 4; q += 32) t4[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncwarp();
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
        const int nw = act ? (int)a.nwords[i] : 0;
        if (act && (nn > NARROW_NMAX || nw > nn || lo < 0)) { flag |= DERR_COUNT; act = false; }
        // the row's words: from its list into the window table
        uint2 lw[LPL];
        const uint2 *ul = a.ulist + (act ? i : 0) * NARROW_NMAX;
#pragma unroll
        for (int u = 0; u < LPL; u++) {
            const int x = gl + G * u;
            lw[u] = act && x < nw ? ul[x] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int r = gl; r < NARROW_NMAX; r += G) acc[r * S::ACC_RS] = (V)0;
        int cl = 0;
#pragma unroll
        for (int u = 0; u < LPL; u++) {
            if (lw[u].y == 0u) continue;
            const int wd = (int)(lw[u].x & 0xffu) & (NARROW_W - 1);
            tab[wd * RPW] = lw[u].y;
            base[wd * RPW] = (unsigned char)(lw[u].x >> 8);
            cl += __popc(lw[u].y);
        }
#pragma unroll
        for (int d = G / 2; d > 0; d >>= 1) cl += __shfl_xor_sync(0xffffffffu, cl, d, G);
        if (act && cl != nn) { flag |= DERR_COUNT; act = false; }
        if (!act) plen = 0;
        const int maxlen = __reduce_max_sync(0xffffffffu, plen);
        __syncwarp();
        // products, a batch of stored entries at a time
        bool bad = false;
        unsigned miss = 0;   // set by a column absent from the row's window union
        for (int pb = 0; pb < maxlen; pb += E) {
            long long q0[EL];
            int len[EL], np[EL];
            load_entries<G, E>(a.acol, a.bdesc, a.nrows_b, p0, plen, pb, gl, q0, len, np, bad);
#pragma unroll
            for (int u = 0; u < EL; u++) {
                const int e = gl + G * u;
                NarrowEnt<V> x;
                x.q = (int)(unsigned long long)q0[u];
                x.hl = IDX32 ? len[u] : (int)((unsigned long long)q0[u] >> 32);
                x.a = pb + e < plen ? aval[p0 + pb + e] : (V)0;
                ent[e] = x;
                if (!IDX32) elen[e] = len[u];
            }
            __syncwarp();
            const int nb = min(E, plen - pb);
            int e = 0, j = gl, clen = 0;
            long long cq = 0;
            V ca = 0;
            if (nb > 0) {
                const NarrowEnt<V> x = ent[0];
                cq = IDX32 ? (long long)x.q : (long long)(((unsigned long long)(unsigned)x.hl << 32) | (unsigned)x.q);
                ca = x.a;
                clen = IDX32 ? x.hl : elen[0];
            }
            while (__any_sync(0xffffffffu, e < nb)) {
                int c[U], r[U];
                V v[U], av[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const bool ok = j < clen;
                    r[u] = ok ? 0 : NARROW_NMAX;
                    if (IDX32) {
                        const int q = ok ? (int)cq + j : 0;
                        c[u] = bcol[q];
                        v[u] = bval[q];
                    } else {
                        const long long q = ok ? cq + j : 0;
                        c[u] = bcol[q];
                        v[u] = bval[q];
                    }
                    av[u] = ca;
                    j += G;
                    if (j - gl >= clen && e < nb) {
                        e++;
                        j = gl;
                        clen = 0;
                        if (e < nb) {
                            const NarrowEnt<V> x = ent[e];
                            cq = IDX32 ? (long long)x.q
                                       : (long long)(((unsigned long long)(unsigned)x.hl << 32) | (unsigned)x.q);
                            ca = x.a;
                            clen = IDX32 ? x.hl : elen[e];
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int wd = ((c[u] >> 5) - lo) & (NARROW_W - 1);
                    const unsigned m = tab[wd * RPW];
                    const unsigned sh = (unsigned)c[u] & 31u;
                    const int rk = base[wd * RPW] + popc_below(m, sh);
                    const bool hit = (m >> sh) & 1u;
                    const bool live = r[u] == 0;
                    miss |= live && !hit ? 1u : 0u;
                    r[u] = live && hit ? min(rk, NARROW_NMAX) : NARROW_NMAX;
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (r[u] < NARROW_NMAX) acc[r[u] * S::ACC_RS] = fma(av[u], v[u], acc[r[u] * S::ACC_RS]);
                    __syncwarp();
                }
            }
            __syncwarp();
        }
        if (miss) flag |= DERR_COUNT;
        if (bad) flag |= DERR_COL_RANGE;
        // write the row in column order (every lane its listed words) and
        // clear the row's words from the table
#pragma unroll
        for (int u = 0; u < LPL; u++) {
            unsigned m = lw[u].y;
            if (m == 0u) continue;
            int rr = (int)(lw[u].x >> 8);
            const int wd = (int)(lw[u].x & 0xffu);
            const int col0 = (lo + wd) * 32;
            tab[(wd & (NARROW_W - 1)) * RPW] = 0u;
            if (act) {
                while (m && rr < nn) {
                    const int bpos = __ffs(m) - 1;
                    m &= m - 1u;
                    a.ccol[out + rr] = col0 + bpos;
                    ((V *)a.cval)[out + rr] = acc[rr * S::ACC_RS];
                    rr++;
                }
            }
        }
        __syncwarp();
    }
    if (flag) atomicOr(err, flag);
}

template <int G, int E, typename V, bool IDX32>
static int run_num_narrow(const NarrowP &p, int *err, Ctx &c) {
    constexpr int WPB = 4, NR = WPB * (32 / G);
    int64_t blocks = (p.n + NR - 1) / NR;
    const int64_t cap = resident_blocks(k_num_narrow<G, WPB, E, V, IDX32>, WPB * 32, c.nsm);
    blocks = blocks < cap ? blocks : cap;
    c.begin("numeric.narrow", p.n);
    k_num_narrow<G, WPB, E, V, IDX32><<<(unsigned)blocks, WPB * 32, 0, c.s>>>(p, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

template <typename V, bool IDX32>
static int run_num_narrow_g(const NarrowP &p, int *err, int G, Ctx &c) {
    switch (G) {
        case 4: return run_num_narrow<4, 16, V, IDX32>(p, err, c);
        case 8: return run_num_narrow<8, 32, V, IDX32>(p, err, c);
        default: return run_num_narrow<16, 32, V, IDX32>(p, err, c);
    }
}

int launch_num_narrow(int dtype, const spgemm_csr &A, const spgemm_csr &B, spgemm_csr &C, const int4 *bdesc,
                      const int32_t *nlo, const uint8_t *nwords, const uint2 *ulist, const uint8_t *bins, int *err,
                      int G, Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    NarrowP p{A.row_ptr, A.col_idx, A.values, B.col_idx, B.values, C.row_ptr, C.col_idx, C.values,
              bdesc, nlo, nwords, ulist, bins, A.nrows, B.nrows};
    const bool i32 = B.nnz < ((int64_t)1 << 31);
    if (dtype == SPGEMM_F32)
        return i32 ? run_num_narrow_g<float, true>(p, err, G, c) : run_num_narrow_g<float, false>(p, err, G, c);
    return i32 ? run_num_narrow_g<double, true>(p, err, G, c) : run_num_narrow_g<double, false>(p, err, G, c);
}

}  // namespace sg

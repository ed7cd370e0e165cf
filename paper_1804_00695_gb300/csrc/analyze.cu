// Row analysis: column compression of B (Section 2.1), per-row product
// counts and binning (Section 3.1, Section 3.3), exclusive scan of counts.
#include <climits>
#include "internal.cuh"

namespace sg {

// ---------------------------------------------------------------- compression
// One thread per row of M: consecutive stored columns that fall in the same
// 32-column block are merged into one (block, mask) pair, so that a set of
// columns is held in fewer integers and unions become bitwise ORs (the
// compression of Section 2.1).  Rows need not be sorted; a sorted row yields
// one pair per block, ascending.  The row's descriptors are written
// alongside: desc = {first entry (int64), entries, pairs} for the product
// kernels, ana = {entries, pairs} for the analysis, and the row's first and
// last block (minmax) for the span tests.
//
// A warp takes 32 consecutive rows.  When their entries together number at
// most COMPRESS_STAGE, the warp first copies them into shared memory with
// coalesced asynchronous copies (a lane's row alone is a short run of
// addresses 32 rows apart from its neighbours' in one load instruction), and
// every lane then reads its row from there; otherwise every lane loads its
// own row.
constexpr int64_t COMPRESS_LONG = 128;   // rows longer than this take a warp each
constexpr int COMPRESS_STAGE = 1024;     // staged entries per warp
constexpr int COMPRESS_WPB = 8;

__global__ void __launch_bounds__(COMPRESS_WPB * 32) k_compress(
    int64_t nrows, int64_t ncols, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
    int2 *__restrict__ pairs, int32_t *__restrict__ ccnt, int2 *__restrict__ minmax, int4 *__restrict__ desc,
    int2 *__restrict__ ana, int *err, int *unsorted_flag, int *long_flag) {
    __shared__ int stage_all[COMPRESS_WPB * COMPRESS_STAGE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *stage = stage_all + w * COMPRESS_STAGE;
    const int64_t r0 = ((int64_t)blockIdx.x * COMPRESS_WPB + w) * 32;
    if (r0 >= nrows) return;
    const int64_t r = r0 + lane;
    const bool live = r < nrows;
    const int64_t beg = live ? rp[r] : 0, end = live ? rp[r + 1] : 0;
    const int64_t rlast = min(r0 + 32, nrows);
    const int64_t wbeg = __shfl_sync(0xffffffffu, beg, 0);
    const int64_t wend = rp[rlast];
    const bool staged = wend - wbeg <= COMPRESS_STAGE;
    if (staged) {
        // asynchronous copies global -> shared (cp.async, 4 bytes a lane and
        // step: coalesced, no registers held while they are in flight); each
        // lane waits for its own, the warp barrier then publishes them all
        const int span = (int)(wend - wbeg);
        for (int x = lane; x < span; x += 32) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(stage + x);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(col + wbeg + x) : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    __syncwarp();
    const bool lng = end - beg > COMPRESS_LONG;   // k_compress_long
    if (lng && long_flag) *long_flag = 1;
    if (!live || lng) return;
    const int *src = staged ? stage + (beg - wbeg) : col + beg;
    const int len = (int)(end - beg);
    int cur = -1;
    unsigned m = 0;
    int n = 0, bmin = INT_MAX, bmax = INT_MIN, prev = -1;
    bool bad = false, unsorted = false;
    // four columns at a time, their loads issued together
    for (int p0 = 0; p0 < len; p0 += 4) {
        int cc[4];
#pragma unroll
        for (int u = 0; u < 4; u++) cc[u] = p0 + u < len ? src[p0 + u] : 0;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (p0 + u >= len) break;
            const int c = cc[u];
            if (c < 0 || (int64_t)c >= ncols) { bad = true; continue; }
            unsorted |= c <= prev;
            prev = c;
            const int b = c >> 5;
            if (b != cur) {
                if (cur >= 0 && pairs) pairs[beg + n] = make_int2(cur, (int)m);
                if (cur >= 0) n++;
                cur = b;
                m = 0;
            }
            m |= 1u << (c & 31);
            bmin = min(bmin, b);
            bmax = max(bmax, b);
        }
    }
    if (cur >= 0) {
        if (pairs) pairs[beg + n] = make_int2(cur, (int)m);
        n++;
    }
    if (ccnt) ccnt[r] = n;
    if (minmax) minmax[r] = make_int2(bmin, bmax);
    if (desc) desc[r] = make_int4((int)(unsigned)(uint64_t)beg, (int)((uint64_t)beg >> 32), len, n);
    if (ana) ana[r] = make_int2(len, n);
    if (bad) atomicOr(err, DERR_COL_RANGE);
    if (unsorted && unsorted_flag) atomicOr(unsorted_flag, 1);
}

// The same for the rows longer than COMPRESS_LONG, a warp per row, 32
// consecutive entries at a time: a pair starts where an entry's block
// differs from the previous entry's; the masks of a run are ORed by a
// segmented scan over the lanes; a run that reaches the end of the 32 is
// carried into the next 32 (its pair written once it ends).
__global__ void k_compress_long(int64_t nrows, int64_t ncols, const int64_t *__restrict__ rp,
                                const int32_t *__restrict__ col, int2 *__restrict__ pairs,
                                int32_t *__restrict__ ccnt, int2 *__restrict__ minmax,
                                int4 *__restrict__ desc, int2 *__restrict__ ana, int *err,
                                int *unsorted_flag, const int *long_flag) {
    // k_compress found no long row (the flag is cleared before it runs)
    if (long_flag && *(volatile const int *)long_flag == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    bool bad = false, unsorted = false;
    // a warp tests 32 rows at once and compresses the long ones among them;
    // the rows a warp tests are `warps` apart (row wg + warps * m), so that
    // long rows stored next to each other (the heavy rows of a power-law
    // graph cluster at the low indices) go to different warps
    for (int64_t m0 = 0; wg + warps * m0 < nrows; m0 += 32) {
      const int64_t rl = wg + warps * (m0 + lane);
      unsigned longs = __ballot_sync(0xffffffffu, rl < nrows && rp[rl + 1] - rp[rl] > COMPRESS_LONG);
      while (longs) {
        const int64_t r = wg + warps * (m0 + __ffs(longs) - 1);
        longs &= longs - 1u;
        const int64_t beg = rp[r], end = rp[r + 1];
        int cblk = -1;          // block of the run carried from the previous 32 (-1: none)
        unsigned cmask = 0;
        int npairs = 0;         // runs started so far (the carried one included)
        int prevc = -1;         // last valid column of the previous 32
        int bmin = INT_MAX, bmax = INT_MIN;
        for (int64_t base = beg; base < end; base += 32) {
            const int64_t p = base + lane;
            int c = p < end ? col[p] : -1;
            if (c >= 0 && (int64_t)c >= ncols) { bad = true; c = -1; }
            if (p < end && c < 0) bad = true;
            const bool valid = c >= 0;
            // sortedness against the previous valid entry in storage order
            int pc = __shfl_up_sync(0xffffffffu, c, 1);
            if (lane == 0) pc = prevc;
            unsorted |= valid && pc >= 0 && c <= pc;
            const int b = valid ? c >> 5 : -2;
            int pb = __shfl_up_sync(0xffffffffu, b, 1);
            if (lane == 0) pb = cblk;
            bool start = valid && b != pb;
            unsigned m = valid ? 1u << (c & 31) : 0u;
            if (lane == 0 && valid && !start) m |= cmask;   // continues the carried run
            // invalid lanes (bad columns) break runs: they act as run starts with no bits
            bool seg = start || !valid;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned ym = __shfl_up_sync(0xffffffffu, m, d);
                const bool ys = __shfl_up_sync(0xffffffffu, seg, d);
                if (lane >= d && !seg) m |= ym;
                if (lane >= d) seg = seg || ys;
            }
            const unsigned starts = __ballot_sync(0xffffffffu, start);
            const int idx = npairs + __popc(starts & ((2u << lane) - 1u)) - 1;
            // the carried run, if it ends before this 32 continues it
            if (lane == 0 && cblk >= 0 && !(valid && !start)) {
                if (pairs) pairs[beg + npairs - 1] = make_int2(cblk, (int)cmask);
            }
            const bool nxt_start = __shfl_down_sync(0xffffffffu, start || !valid, 1);
            const bool last_valid = valid && (lane == 31 || nxt_start);
            const unsigned lastm = __ballot_sync(0xffffffffu, valid);
            const int top = lastm ? 31 - __clz(lastm) : -1;   // last valid lane
            // runs that end inside this 32 are written; the one at the last
            // valid lane is carried unless the row ends here
            const bool row_ends = base + 32 >= end;
            if (last_valid && (lane != top || row_ends) && pairs && idx >= 0) pairs[beg + idx] = make_int2(b, (int)m);
            npairs += __popc(starts);
            if (top >= 0) {
                const int tb = __shfl_sync(0xffffffffu, b, top);
                const unsigned tm = __shfl_sync(0xffffffffu, m, top);
                cblk = row_ends ? -1 : tb;
                cmask = row_ends ? 0u : tm;
                prevc = __shfl_sync(0xffffffffu, c, top);
            }
            if (valid) { bmin = min(bmin, b); bmax = max(bmax, b); }
        }
        if (cblk >= 0 && lane == 0 && pairs) pairs[beg + npairs - 1] = make_int2(cblk, (int)cmask);
        for (int d = 16; d > 0; d >>= 1) {
            bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, d));
            bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, d));
        }
        if (lane == 0) {
            const int len = (int)(end - beg);
            if (ccnt) ccnt[r] = npairs;
            if (minmax) minmax[r] = make_int2(bmin, bmax);
            if (desc) desc[r] = make_int4((int)(unsigned)(uint64_t)beg, (int)((uint64_t)beg >> 32), len, npairs);
            if (ana) ana[r] = make_int2(len, npairs);
        }
      }
    }
    unsorted = __any_sync(0xffffffffu, unsorted);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0 && bad) atomicOr(err, DERR_COL_RANGE);
    if (lane == 0 && unsorted && unsorted_flag) atomicOr(unsorted_flag, 1);
}

int launch_compress(const spgemm_csr &M, int2 *pairs, int32_t *ccnt, int2 *minmax, int4 *desc,
                    int2 *ana, int *err, Ctx &c, int *unsorted, int *long_flag) {
    if (M.nrows == 0) return SPGEMM_OK;
    int64_t blocks = (M.nrows + COMPRESS_WPB * 32 - 1) / (COMPRESS_WPB * 32);
    c.begin("compress", M.nrows);
    k_compress<<<(unsigned)blocks, COMPRESS_WPB * 32, 0, c.s>>>(M.nrows, M.ncols, M.row_ptr, M.col_idx, pairs,
                                                    ccnt, minmax, desc, ana, err, unsorted, long_flag);
    c.end();
    // one resident wave (it returns at once when no row is long)
    const int64_t wblocks = std::min<int64_t>((M.nrows + 255) / 256, resident_blocks(k_compress_long, 256, c.nsm));
    c.begin("compress_long", M.nrows);
    k_compress_long<<<(unsigned)wblocks, 256, 0, c.s>>>(M.nrows, M.ncols, M.row_ptr, M.col_idx, pairs, ccnt,
                                                        minmax, desc, ana, err, unsorted, long_flag);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

// ---------------------------------------------------------------- analysis
// Eight lanes per row of A.  For row i: flops_i = sum_k nnz(B_k) (the number
// of accumulator insertions, Section 3.1) and cpairs_i = sum_k pairs(B_k).
// The symbolic accumulator needs at most min(cpairs_i, ceil(ncols/32)) keys
// (the second pass narrows rows down by their column span itself).
// Empty rows get their count (0) here; rows for the dense bitmap (bin 6)
// are marked -1 for the second pass.
constexpr int AN_G = 8;
__global__ void k_analyze(int64_t nrows, int64_t nrows_b, int64_t nwords,
                          const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
                          const int2 *__restrict__ ana, int64_t *__restrict__ flops,
                          uint8_t *__restrict__ bins, int64_t *__restrict__ crp, DevState *st) {
    __shared__ unsigned long long hist[NBINS];
    __shared__ unsigned long long fsum;
    __shared__ unsigned long long alen_max;
    if (threadIdx.x < NBINS) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) { fsum = 0; alen_max = 0; }
    __syncthreads();
    const int lane = threadIdx.x % AN_G;
    const unsigned gmask = ((1u << AN_G) - 1) << ((threadIdx.x & 31) & ~(AN_G - 1));
    // a fixed grid strides over the rows, so the block's totals reach the
    // global counters once per block, not once per 32 rows
    const int64_t rstride = (int64_t)gridDim.x * (blockDim.x / AN_G);
    long long wf = 0, wl = 0;   // this lane's share of the products and the longest row
    bool bad = false;
    for (int64_t i0 = (int64_t)blockIdx.x * (blockDim.x / AN_G); i0 < nrows; i0 += rstride) {
        const int64_t i = i0 + threadIdx.x / AN_G;
        const bool live = i < nrows;
        long long f = 0, cp = 0;
        if (live) {
            for (int64_t p = arp[i] + lane; p < arp[i + 1]; p += AN_G) {
                int k = acol[p];
                if (k < 0 || (int64_t)k >= nrows_b) { bad = true; continue; }
                const int2 d = ana[k];
                f += d.x;
                cp += d.y;
            }
        }
        for (int d = AN_G / 2; d > 0; d >>= 1) {
            f += __shfl_xor_sync(gmask, f, d, AN_G);
            cp += __shfl_xor_sync(gmask, cp, d, AN_G);
        }
        int b = BIN_EMPTY;
        const bool lead = live && lane == 0;
        if (lead) {
            const long long keys = min(cp, (long long)nwords);
            b = sym_bin(keys, cp);
            flops[i] = f;
            bins[i] = (uint8_t)b;
            if (b == BIN_EMPTY) crp[i + 1] = 0;
            if (b == BIN_HUGE) crp[i + 1] = -1;
            wf += f;
            wl = max(wl, (long long)(arp[i + 1] - arp[i]));
        }
        warp_hist(hist, lead, b);
    }
    if (bad) atomicOr(&st->err, DERR_COL_RANGE);
    // products of the warp's rows and its longest row of A
    for (int d = 16; d > 0; d >>= 1) {
        wf += __shfl_xor_sync(0xffffffffu, wf, d);
        wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, d));
    }
    if ((threadIdx.x & 31) == 0 && wf) atomicAdd(&fsum, (unsigned long long)wf);
    if ((threadIdx.x & 31) == 0 && wl) atomicMax(&alen_max, (unsigned long long)wl);
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

int launch_analyze(const spgemm_csr &A, const spgemm_csr &B, const int2 *ana, int64_t *flops,
                   uint8_t *bins, int64_t *crp, DevState *st, Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    int64_t threads = A.nrows * AN_G;
    int64_t blocks = (threads + 255) / 256;
    blocks = std::min<int64_t>(blocks, (int64_t)c.nsm * 16);
    int64_t nwords = (B.ncols + 31) / 32;
    c.begin("analyze", A.nrows);
    k_analyze<<<(unsigned)blocks, 256, 0, c.s>>>(A.nrows, B.nrows, nwords, A.row_ptr, A.col_idx,
                                                   ana, flops, bins, crp, st);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

__global__ void k_list_spans(const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
                             const int2 *__restrict__ bmm, const int32_t *__restrict__ rows, int64_t count,
                             int2 *__restrict__ spans) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < count; t += warps) {
        const int i = rows[t];
        int lo = INT_MAX, hi = -1;
        for (int64_t p = arp[i] + lane; p < arp[i + 1]; p += 32) {
            const int2 m = bmm[acol[p]];
            lo = min(lo, m.x);
            hi = max(hi, m.y);
        }
        for (int d = 16; d > 0; d >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
        }
        if (lane == 0) spans[t] = make_int2(lo, hi >= lo ? hi - lo + 1 : 0);
    }
}

int launch_list_spans(const spgemm_csr &A, const int2 *bmm, const int32_t *rows, int64_t count, int2 *spans,
                      Ctx &c) {
    if (count <= 0) return SPGEMM_OK;
    int64_t blocks = (count + 7) / 8;
    blocks = std::min<int64_t>(blocks, (int64_t)c.nsm * 16);
    c.begin("list_spans", count);
    k_list_spans<<<(unsigned)blocks, 256, 0, c.s>>>(A.row_ptr, A.col_idx, bmm, rows, count, spans);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

// Products per row only (inspection entry point).
__global__ void k_row_flops(int64_t nrows, int64_t nrows_b, const int64_t *__restrict__ arp,
                            const int32_t *__restrict__ acol, const int64_t *__restrict__ brp,
                            int64_t *__restrict__ flops, int *err) {
    const int lane = threadIdx.x % AN_G;
    const unsigned gmask = ((1u << AN_G) - 1) << ((threadIdx.x & 31) & ~(AN_G - 1));
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / AN_G;
    long long f = 0;
    bool bad = false;
    if (i < nrows) {
        for (int64_t p = arp[i] + lane; p < arp[i + 1]; p += AN_G) {
            int k = acol[p];
            if (k < 0 || (int64_t)k >= nrows_b) { bad = true; continue; }
            f += brp[k + 1] - brp[k];
        }
    }
    for (int d = AN_G / 2; d > 0; d >>= 1) f += __shfl_xor_sync(gmask, f, d, AN_G);
    if (bad) atomicOr(err, DERR_COL_RANGE);
    if (i < nrows && lane == 0) flops[i] = f;
}

int launch_row_flops(const spgemm_csr &A, const spgemm_csr &B, int64_t *flops, int *err,
                     Ctx &c) {
    if (A.nrows == 0) return SPGEMM_OK;
    int64_t blocks = (A.nrows * AN_G + 255) / 256;
    c.begin("row_flops", A.nrows);
    k_row_flops<<<(unsigned)blocks, 256, 0, c.s>>>(A.nrows, B.nrows, A.row_ptr, A.col_idx,
                                                     B.row_ptr, flops, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

// ---------------------------------------------------------------- numeric bins
__global__ void k_numeric_binning(int64_t n, const int64_t *__restrict__ crp,
                                  const int64_t *__restrict__ flops, uint8_t *__restrict__ bins,
                                  DevState *st, const int32_t *__restrict__ nlo) {
    __shared__ unsigned long long hist[NBINS];
    if (threadIdx.x < NBINS) hist[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = BIN_EMPTY;
    if (i < n) {
        long long c = crp[i + 1] - crp[i];
        const long long f = flops[i];
        b = c > 0 ? num_bin(c, f) : BIN_EMPTY;
        if (b != BIN_EMPTY && nlo && nlo[i] >= 0 && c <= NARROW_NMAX && f <= NARROW_FLOPS) b = BIN_NARROW;
        bins[i] = (uint8_t)b;
        if (b == BIN_HUGE) atomicMax((unsigned long long *)&st->max_row_nnz, (unsigned long long)c);
    }
    warp_hist(hist, i < n, b);
    __syncthreads();
    if (threadIdx.x < NBINS && hist[threadIdx.x])
        atomicAdd((unsigned long long *)&st->bin_count[1][threadIdx.x], hist[threadIdx.x]);
}

int launch_numeric_binning(int64_t n, const int64_t *crp, const int64_t *flops, uint8_t *bins,
                           DevState *st, Ctx &c, const int32_t *nlo) {
    if (n == 0) return SPGEMM_OK;
    c.begin("numeric_binning", n);
    k_numeric_binning<<<(unsigned)((n + 255) / 256), 256, 0, c.s>>>(n, crp, flops, bins, st, nlo);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

// Row lists for the list-driven kernels.  phase 0 (symbolic second pass):
// rows marked -1 in crp[i+1] (overflowed the first pass, or bin 6), listed by
// max(bins[i], 2).  phase 1 (numeric): rows of bins first_bin..6.  Within a warp the
// lanes with the same bin reserve their slots with one atomic
// (__match_any_sync), so rows stay in ascending order inside each warp.
__global__ void k_scatter_bins(int64_t n, const uint8_t *__restrict__ bins,
                               const int64_t *__restrict__ crp, int32_t *__restrict__ rows,
                               DevState *st, int phase, int first_bin) {
    __shared__ long long off[NBINS];
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int b = 0; b < NBINS; b++) {
            off[b] = o;
            if (b >= (phase == 0 ? 2 : first_bin) && b <= BIN_HUGE) o += st->bin_count[phase][b];
        }
    }
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = BIN_EMPTY;
    if (i < n) {
        if (phase == 0) {
            if (crp[i + 1] < 0) b = max((int)bins[i], 2);
        } else {
            int x = bins[i];
            if (x >= first_bin && x <= BIN_HUGE) b = x;
        }
    }
    unsigned act = __ballot_sync(0xffffffffu, b != BIN_EMPTY);
    if (b == BIN_EMPTY) return;
    unsigned peers = __match_any_sync(act, b);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    long long base = 0;
    if (lane == leader) base = atomicAdd((unsigned long long *)&st->bin_cursor[b],
                                         (unsigned long long)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    int rank = __popc(peers & ((1u << lane) - 1));
    rows[off[b] + base + rank] = (int32_t)i;
}

int launch_scatter_bins(int64_t n, const uint8_t *bins, const int64_t *crp, int32_t *rows,
                        DevState *st, int phase, Ctx &c, int first_bin) {
    if (n == 0) return SPGEMM_OK;
    SG_CUDA(cudaMemsetAsync(st->bin_cursor, 0, sizeof(st->bin_cursor), c.s));
    c.begin("scatter_bins", n);
    k_scatter_bins<<<(unsigned)((n + 255) / 256), 256, 0, c.s>>>(n, bins, crp, rows, st, phase,
                                                                   first_bin);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

// ---------------------------------------------------------------- scan
// Reduce-then-scan over tiles of SCAN_TILE counts: tile sums, one block scans
// the sums (looping with a carry), then every tile is rescanned with its
// offset.  x[0] is set to 0 and x[1..n] becomes the inclusive prefix.
constexpr int SCAN_BS = 256, SCAN_PT = 8, SCAN_TILE = SCAN_BS * SCAN_PT;

size_t scan_tmp_bytes(int64_t n) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(tiles + 1) * sizeof(long long);
}

__device__ __forceinline__ long long block_excl_scan(long long v, long long *sh, long long *total) {
    // sh: SCAN_BS/32 entries
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = v;
    for (int d = 1; d < 32; d <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long s = lane < SCAN_BS / 32 ? sh[lane] : 0;
        long long si = s;
        for (int d = 1; d < 32; d <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, si, d);
            if (lane >= d) si += t;
        }
        if (lane < SCAN_BS / 32) sh[lane] = si - s;
        if (lane == SCAN_BS / 32 - 1) *total = si;
    }
    __syncthreads();
    long long r = sh[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const int64_t *__restrict__ x1, int64_t n, long long *tile_sums) {
    __shared__ long long sh[SCAN_BS / 32];
    __shared__ long long tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PT;
    long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PT; j++)
        if (base + j < n) s += x1[base + j];
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(long long *tile_sums, int64_t tiles, long long *total) {
    __shared__ long long sh[SCAN_BS / 32];
    __shared__ long long tot;
    long long carry = 0;
    for (int64_t b0 = 0; b0 < tiles; b0 += SCAN_BS) {
        int64_t t = b0 + threadIdx.x;
        long long v = t < tiles ? tile_sums[t] : 0;
        long long e = block_excl_scan(v, sh, &tot);
        if (t < tiles) tile_sums[t] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_apply(int64_t *__restrict__ x, int64_t n, const long long *tile_sums) {
    __shared__ long long sh[SCAN_BS / 32];
    __shared__ long long tot;
    int64_t *x1 = x + 1;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PT;
    long long v[SCAN_PT];
    long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PT; j++) {
        v[j] = base + j < n ? x1[base + j] : 0;
        s += v[j];
    }
    long long e = block_excl_scan(s, sh, &tot) + tile_sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_PT; j++) {
        e += v[j];
        if (base + j < n) x1[base + j] = e;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) x[0] = 0;
}

int launch_scan_counts(int64_t *x, int64_t n, long long *total, void *tmp, Ctx &c) {
    if (n == 0) {
        SG_CUDA(cudaMemsetAsync(x, 0, sizeof(int64_t), c.s));
        SG_CUDA(cudaMemsetAsync(total, 0, sizeof(long long), c.s));
        return SPGEMM_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    long long *sums = (long long *)tmp;
    c.begin("scan_tiles", n);
    k_scan_tiles<<<(unsigned)tiles, SCAN_BS, 0, c.s>>>(x + 1, n, sums);
    c.end();
    c.begin("scan_sums", tiles);
    k_scan_sums<<<1, SCAN_BS, 0, c.s>>>(sums, tiles, total);
    c.end();
    c.begin("scan_apply", n);
    k_scan_apply<<<(unsigned)tiles, SCAN_BS, 0, c.s>>>(x, n, sums);
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

}  // namespace sg

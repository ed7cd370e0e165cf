// Triangle counting by a masked sparse product (the triangle-counting
// experiment of Section 4.1, with Wolf et al.'s formulation that the paper
// uses): the vertices of an undirected graph are relabelled in order of
// non-decreasing degree, L is the strictly lower triangle of the relabelled
// pattern, and the number of triangles is the sum of (L * L) masked by L.
// The paper computes L x compressed(L): the right-hand operand is the
// column compression of Section 2.1 (block, 32-bit mask pairs), so a row's
// contribution is, for every stored L_ik, the popcounts of the masks of L_k
// ANDed with row i's own column set held as masks by block.
//
// Steps on the device: degrees and a histogram of them; an exclusive scan
// (bucket starts); labels by atomic cursors per degree (vertices of equal
// degree in any order: the count does not depend on it, and the labels are
// returned); the rows of L counted, scanned and filled; L compressed; rows
// split by work: at most TRI_LIGHT_LEN entries and TRI_LIGHT_WORK pairs to
// look up go to a warp each with a 256-slot map of row i's blocks (shared
// memory), the others to a block each with a dense bitmap of all columns
// (shared memory up to TRI_SMEM_WORDS words, else a bitmap per block in
// global memory), set from row i and cleared again after it.
#include <climits>
#include "internal.cuh"

namespace sg {

constexpr int TRI_LIGHT_LEN = 128;
constexpr long long TRI_LIGHT_WORK = 32768;
constexpr int TRI_MAP_L = 8;             // 256 slots per light row
constexpr int TRI_WPB = 8;
constexpr int TRI_HEAVY_BS = 512;
constexpr int64_t TRI_SMEM_WORDS = 48 * 1024;   // 192 KB of bitmap in shared memory

// deg[u] (clamped to n - 1 for rows with repeated columns) and its histogram
// in hist[1 + deg] (hist[0] stays 0: the scan then gives bucket starts).
__global__ void k_tri_degree(int64_t n, const int64_t *__restrict__ rp, int64_t *__restrict__ deg,
                             int64_t *__restrict__ hist) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t d = rp[u + 1] - rp[u];
        d = d < n - 1 ? d : n - 1;
        deg[u] = d;
        atomicAdd((unsigned long long *)&hist[1 + d], 1ull);
    }
}

// Labels: perm[u] = start of u's degree bucket + its arrival in the bucket.
__global__ void k_tri_label(int64_t n, const int64_t *__restrict__ deg, int64_t *__restrict__ cursor,
                            int64_t *__restrict__ perm, int32_t *__restrict__ iperm) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = (int64_t)atomicAdd((unsigned long long *)&cursor[deg[u]], 1ull);
        perm[u] = p;
        iperm[p] = (int32_t)u;
    }
}

// Entries of row perm[u] of L: the neighbours of u with a smaller label
// (a warp per vertex).  fill = false: their number to lrp[perm[u] + 1];
// true: their labels to lcol from lrp[perm[u]] on, in the order of u's row.
template <bool FILL>
__global__ void k_tri_lower(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const int64_t *__restrict__ perm, int64_t *__restrict__ lrp,
                            int32_t *__restrict__ lcol, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    bool bad = false;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t pu = perm[u];
        const int64_t p0 = rp[u], p1 = rp[u + 1];
        int64_t w = FILL ? lrp[pu] : 0;
        int64_t cnt = 0;
        for (int64_t p = p0; p < p1; p += 32) {
            bool take = false;
            int64_t pv = 0;
            if (p + lane < p1) {
                const int v = col[p + lane];
                if ((unsigned)v >= (unsigned)n) bad = true;
                else {
                    pv = perm[v];
                    take = pv < pu;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, take);
            if (FILL && take) lcol[w + __popc(m & ((1u << lane) - 1u))] = (int32_t)pv;
            w += __popc(m);
            cnt += __popc(m);
        }
        if (!FILL && lane == 0) lrp[pu + 1] = cnt;
    }
    if (bad) atomicOr(err, DERR_COL_RANGE);
}

// Work of every row of L: pairs of the compressed rows it reaches.  Rows
// with entries go to the light list (at most TRI_LIGHT_LEN entries and
// TRI_LIGHT_WORK pairs) or the heavy list; counts in cnt[0], cnt[1].
__global__ void k_tri_bins(int64_t n, const int64_t *__restrict__ lrp, const int32_t *__restrict__ lcol,
                           const int4 *__restrict__ desc, int32_t *__restrict__ light,
                           int32_t *__restrict__ heavy, unsigned long long *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const int64_t p0 = lrp[i], p1 = lrp[i + 1];
        if (p1 == p0) continue;
        long long wk = 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) wk += desc[lcol[p]].w;
        for (int d = 16; d > 0; d >>= 1) wk += __shfl_xor_sync(0xffffffffu, wk, d);
        if (lane == 0) {
            if (p1 - p0 <= TRI_LIGHT_LEN && wk <= TRI_LIGHT_WORK)
                light[atomicAdd(&cnt[0], 1ull)] = (int32_t)i;
            else
                heavy[atomicAdd(&cnt[1], 1ull)] = (int32_t)i;
        }
    }
}

// Light rows: a warp per row.  Row i's column set goes into a map of 256
// slots, block -> OR of its bits (atomic CAS on the key, OR on the mask);
// then the lanes take the row's entries k in turn and, for every pair
// (block, mask) of compressed L_k, add popc(mask & map[block]).
__global__ void __launch_bounds__(TRI_WPB * 32) k_tri_light(
    const int32_t *__restrict__ rows, const unsigned long long *cnt, const int64_t *__restrict__ lrp,
    const int32_t *__restrict__ lcol, const int4 *__restrict__ desc, const int2 *__restrict__ pairs,
    const int32_t *__restrict__ iperm, int64_t *__restrict__ vcount, unsigned long long *total, int *err) {
    constexpr int S = 1 << TRI_MAP_L;
    __shared__ int keys_all[TRI_WPB * S];
    __shared__ unsigned masks_all[TRI_WPB * S];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *keys = keys_all + w * S;
    unsigned *masks = masks_all + w * S;
    const int64_t nrows = (int64_t)cnt[0];
    const int64_t warps = (int64_t)gridDim.x * TRI_WPB;
    unsigned long long wsum = 0;
    bool full = false;
    for (int64_t t = (int64_t)blockIdx.x * TRI_WPB + w; t < nrows; t += warps) {
        const int64_t i = rows[t];
        for (int s = lane; s < S; s += 32) { keys[s] = -1; masks[s] = 0u; }
        __syncwarp();
        const int64_t p0 = lrp[i], p1 = lrp[i + 1];
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int c = lcol[p];
            full |= !sym_insert(keys, masks, TRI_MAP_L, c >> 5, 1u << (c & 31));
        }
        __syncwarp();
        unsigned long long rc = 0;
        for (int64_t p = p0 + lane; p < p1; p += 32) {
            const int4 d = desc[lcol[p]];
            const int2 *pp = pairs + desc_start(d);
            for (int q = 0; q < d.w; q++) {
                const int2 x = pp[q];
                unsigned h = hash_slot(x.x, TRI_MAP_L);
                int probe = 0;
                int key = keys[h];
                while (key != x.x && key != -1 && probe < S) {
                    h = (h + 1) & (S - 1);
                    key = keys[h];
                    probe++;
                }
                if (key == x.x) rc += __popc((unsigned)x.y & masks[h]);
            }
        }
        for (int d = 16; d > 0; d >>= 1) rc += __shfl_xor_sync(0xffffffffu, rc, d);
        if (lane == 0) {
            if (vcount) vcount[iperm[i]] = (int64_t)rc;
            wsum += rc;
        }
        __syncwarp();
    }
    if (full) atomicOr(err, DERR_PROBE);
    if (lane == 0 && wsum) atomicAdd(total, wsum);
}

// Heavy rows: a block per row with a bitmap of all columns (bm: shared
// memory, or this block's region of gbm), all zero between rows: row i's
// bits are set, every warp takes entries k of the row in turn with its
// lanes over the pairs of compressed L_k, then row i's bits are cleared.
template <bool SMEM>
__global__ void __launch_bounds__(TRI_HEAVY_BS) k_tri_heavy(
    const int32_t *__restrict__ rows, const unsigned long long *cnt, const int64_t *__restrict__ lrp,
    const int32_t *__restrict__ lcol, const int4 *__restrict__ desc, const int2 *__restrict__ pairs,
    const int32_t *__restrict__ iperm, int64_t *__restrict__ vcount, unsigned long long *total, int64_t nwords,
    unsigned *gbm) {
    extern __shared__ unsigned tri_smem[];
    __shared__ unsigned long long red[TRI_HEAVY_BS / 32];
    unsigned *bm = SMEM ? tri_smem : gbm + (int64_t)blockIdx.x * nwords;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = TRI_HEAVY_BS / 32;
    for (int64_t x = threadIdx.x; x < nwords; x += TRI_HEAVY_BS) bm[x] = 0u;
    __syncthreads();
    const int64_t nrows = (int64_t)cnt[1];
    unsigned long long bsum = 0;
    for (int64_t t = blockIdx.x; t < nrows; t += gridDim.x) {
        const int64_t i = rows[t];
        const int64_t p0 = lrp[i], p1 = lrp[i + 1];
        for (int64_t p = p0 + threadIdx.x; p < p1; p += TRI_HEAVY_BS) {
            const int c = lcol[p];
            atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        __syncthreads();
        unsigned long long rc = 0;
        for (int64_t p = p0 + w; p < p1; p += NW) {
            const int4 d = desc[lcol[p]];
            const int2 *pp = pairs + desc_start(d);
            for (int q = lane; q < d.w; q += 32) {
                const int2 x = pp[q];
                rc += __popc((unsigned)x.y & bm[x.x]);
            }
        }
        for (int d = 16; d > 0; d >>= 1) rc += __shfl_xor_sync(0xffffffffu, rc, d);
        if (lane == 0) red[w] = rc;
        __syncthreads();
        for (int64_t p = p0 + threadIdx.x; p < p1; p += TRI_HEAVY_BS) bm[lcol[p] >> 5] = 0u;
        if (threadIdx.x == 0) {
            unsigned long long s = 0;
            for (int k = 0; k < NW; k++) s += red[k];
            if (vcount) vcount[iperm[i]] = (int64_t)s;
            bsum += s;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bsum) atomicAdd(total, bsum);
}

size_t triangles_ws(int64_t n, int64_t nnz, int nsm) {
    const int64_t nwords = (n + 31) / 32;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~(size_t)255; };
    add((size_t)n * 8);              // deg
    add((size_t)(n + 1) * 8);        // hist / cursor
    add((size_t)n * 8);              // perm (when the caller passes none)
    add((size_t)n * 4);              // iperm
    add((size_t)(n + 1) * 8);        // lrp
    add((size_t)nnz * 4);            // lcol (at most half of nnz(A) for a symmetric pattern)
    add((size_t)nnz * 8);            // pairs
    add((size_t)n * 4);              // ccnt
    add((size_t)n * 16);             // desc
    add((size_t)n * 4 * 2);          // light and heavy lists
    add(64);                         // counters
    add(scan_tmp_bytes(n));
    if (nwords > TRI_SMEM_WORDS) add((size_t)nsm * (size_t)nwords * 4);
    return b;
}

int launch_triangles(const spgemm_csr &A, void *ws, int64_t *perm_out, int64_t *vcount, unsigned long long *total,
                     int *err, Ctx &c) {
    const int64_t n = A.nrows, nnz = A.nnz, nwords = (n + 31) / 32;
    char *w = (char *)ws;
    auto take = [&](size_t x) { char *p = w; w += (x + 255) & ~(size_t)255; return p; };
    int64_t *deg = (int64_t *)take((size_t)n * 8);
    int64_t *hist = (int64_t *)take((size_t)(n + 1) * 8);
    int64_t *perm = (int64_t *)take((size_t)n * 8);
    if (perm_out) perm = perm_out;
    int32_t *iperm = (int32_t *)take((size_t)n * 4);
    int64_t *lrp = (int64_t *)take((size_t)(n + 1) * 8);
    int32_t *lcol = (int32_t *)take((size_t)nnz * 4);
    int2 *pairs = (int2 *)take((size_t)nnz * 8);
    int32_t *ccnt = (int32_t *)take((size_t)n * 4);
    int4 *desc = (int4 *)take((size_t)n * 16);
    int32_t *light = (int32_t *)take((size_t)n * 4);
    int32_t *heavy = (int32_t *)take((size_t)n * 4);
    unsigned long long *cnt = (unsigned long long *)take(64);
    void *tmp = take(scan_tmp_bytes(n));
    unsigned *gbm = (unsigned *)w;
    const unsigned g1 = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c.nsm * 16);
    const unsigned gw = (unsigned)std::min<int64_t>((n + 7) / 8, (int64_t)c.nsm * 32);
    SG_CUDA(cudaMemsetAsync(hist, 0, (size_t)(n + 1) * 8, c.s));
    SG_CUDA(cudaMemsetAsync(cnt, 0, 64, c.s));
    SG_CUDA(cudaMemsetAsync(total, 0, sizeof(unsigned long long), c.s));
    if (vcount) SG_CUDA(cudaMemsetAsync(vcount, 0, (size_t)n * 8, c.s));
    c.begin("triangles.degree", n);
    k_tri_degree<<<g1, 256, 0, c.s>>>(n, A.row_ptr, deg, hist);
    c.end();
    SG_TRY(launch_scan_counts(hist, n, (long long *)(cnt + 2), tmp, c));   // hist -> bucket starts
    c.begin("triangles.label", n);
    k_tri_label<<<g1, 256, 0, c.s>>>(n, deg, hist, perm, iperm);
    c.end();
    c.begin("triangles.lower_count", n);
    k_tri_lower<false><<<gw, 256, 0, c.s>>>(n, A.row_ptr, A.col_idx, perm, lrp, nullptr, err);
    c.end();
    SG_TRY(launch_scan_counts(lrp, n, (long long *)(cnt + 3), tmp, c));
    c.begin("triangles.lower_fill", n);
    k_tri_lower<true><<<gw, 256, 0, c.s>>>(n, A.row_ptr, A.col_idx, perm, lrp, lcol, err);
    c.end();
    SG_CUDA(cudaGetLastError());
    spgemm_csr L{n, n, nnz, lrp, lcol, nullptr};
    // nnz(L) is on the device; the compression reads the offsets, so the
    // descriptor's entry count only bounds the arrays
    SG_TRY(launch_compress(L, pairs, ccnt, nullptr, desc, nullptr, err, c));
    c.begin("triangles.bins", n);
    k_tri_bins<<<gw, 256, 0, c.s>>>(n, lrp, lcol, desc, light, heavy, cnt);
    c.end();
    c.begin("triangles.light", n);
    k_tri_light<<<(unsigned)((int64_t)c.nsm * 8), TRI_WPB * 32, 0, c.s>>>(light, cnt, lrp, lcol, desc, pairs, iperm,
                                                                         vcount, total, err);
    c.end();
    const bool smem = nwords <= TRI_SMEM_WORDS;
    const size_t sbytes = smem ? (size_t)nwords * 4 : 0;
    if (smem) {
        SG_CUDA(cudaFuncSetAttribute(k_tri_heavy<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sbytes));
        c.begin("triangles.heavy", n);
        k_tri_heavy<true><<<(unsigned)c.nsm, TRI_HEAVY_BS, sbytes, c.s>>>(heavy, cnt, lrp, lcol, desc, pairs, iperm,
                                                                          vcount, total, nwords, nullptr);
    } else {
        c.begin("triangles.heavy", n);
        k_tri_heavy<false><<<(unsigned)c.nsm, TRI_HEAVY_BS, 0, c.s>>>(heavy, cnt, lrp, lcol, desc, pairs, iperm,
                                                                      vcount, total, nwords, gbm);
    }
    c.end();
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

}  // namespace sg

// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <algorithm>
#include "../../include/spgemm.h"

namespace sg {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
#define SG_CUDA(call)                                                          \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            ::sg::set_error("%s failed: %s (%s:%d)", #call,                    \
                            cudaGetErrorString(e_), __FILE__, __LINE__);       \
            return SPGEMM_ERR_CUDA;                                            \
        }                                                                      \
    } while (0)
#define SG_TRY(expr)                                                           \
    do {                                                                       \
        int s_ = (expr);                                                       \
        if (s_ != SPGEMM_OK) return s_;                                        \
    } while (0)

// Device-side error bits (OR-ed into DevState::err by kernels).
enum : int {
    DERR_COL_RANGE = 1,   // a column index of A (>= nrows(B)) or B (>= ncols) out of range
    DERR_PROBE = 2,       // a hash probe sequence exceeded the table
    DERR_COUNT = 4,       // numeric found a different column count than symbolic
    DERR_WINDOW = 8,      // chunked: a column of A outside the rows of B copied for its part
};

struct DevState {          // lives in device memory, one per handle
    int err;
    int b_out_of_range;    // B holds values outside the double-word range
    long long sym_hist[SPGEMM_NBINS];   // rows per symbolic bin (by bound)
    long long nnz;         // nnz(C) written by the scan
    long long bin_count[2][SPGEMM_NBINS];   // [0] symbolic, [1] numeric
    long long bin_cursor[SPGEMM_NBINS];
    long long max_row_nnz;   // largest row of C (numeric binning)
    long long flops_total;   // products of the whole product (analysis)
    int b_unsorted;          // some row of B has columns out of ascending order
    int long_rows;           // the compression met rows for its warp-per-row pass
    long long max_alen;      // longest row of A (analysis)
    unsigned long long triangles;   // spgemm_triangles: the count
};

// ---------------------------------------------------------------- bins
// Rows are binned by the size of the accumulator they need and by their
// product count; each bin has its own kernel shape (Section 3.3: a part of a
// warp, a whole warp or a whole block per row).
constexpr int BIN_EMPTY = 0;
constexpr int BIN_HUGE = 6;     // widest bin: unbounded accumulator
constexpr int NBINS = SPGEMM_NBINS;

// Numeric bins by exact output count (and product count):
//   1: <= 16 entries, 2: <= 32 (both: lanes of a warp, map in shared memory,
//   rows taken in order), 3: <= 128 (a warp), 4: <= 1024, 5: <= 4096 (a
//   block), 6: larger (a block with a global second-level map).
__host__ __device__ constexpr long long num_cap(int b) {
    return b == 1 ? 16 : b == 2 ? 32 : b == 3 ? 128 : b == 4 ? 1024 : b == 5 ? 4096 : (1LL << 40);
}
__host__ __device__ constexpr long long num_flops(int b) {
    return b <= 2 ? 8192 : b == 3 ? 65536 : b == 4 ? 1048576 : b == 5 ? 16777216 : (1LL << 62);
}
__host__ __device__ inline int num_bin(long long nnz, long long flops) {
    if (nnz <= 0) return BIN_EMPTY;
    int b = 1;
    while (b < BIN_HUGE && (nnz > num_cap(b) || flops > num_flops(b))) b++;
    return b;
}

// Symbolic bins by an upper bound on the row's distinct column blocks:
// every row with bound <= 4096 is first tried with a 32-slot map (most rows
// of sparse products have few blocks); rows that overflow it, and rows with
// a larger bound, go to 2: <= 64 keys, 3: <= 256 (a warp), 4: <= 1024,
// 5: <= 4096 (a block), 6: dense bitmap of all blocks (a block).
constexpr int SYM_FIRST_SLOTS = 32;
__host__ __device__ constexpr long long sym_cap(int b) {
    return b == 1 ? 16 : b == 2 ? 64 : b == 3 ? 256 : b == 4 ? 1024 : b == 5 ? 4096 : (1LL << 40);
}
__host__ __device__ inline int sym_bin(long long keys, long long cpairs) {
    if (keys <= 0) return BIN_EMPTY;
    int b = 1;
    while (b < BIN_HUGE && (keys > sym_cap(b) || cpairs > 64 * sym_cap(b))) b++;
    return b;
}

// Narrow rows (narrow.cu): rows of C whose columns all fall within
// NARROW_W consecutive blocks of 32 columns.  The symbolic phase marks them
// BIN_NARROW (their count done by the window table, nlo[i] = the window's
// first block); the numeric phase gives BIN_NARROW to those of them with at
// most NARROW_NMAX outputs and NARROW_FLOPS products.  Bin 7 is otherwise
// unused in both phases.
constexpr int BIN_NARROW = 7;
constexpr int NARROW_W = 128;
constexpr int NARROW_NMAX = 32;
constexpr long long NARROW_FLOPS = 8192;
constexpr long long NARROW_PAIRS = 4096;
// Row-slot strides of the narrow kernels' shared tables, padded so that the
// row slots of a warp start on different banks (words, bytes, values).
constexpr int NARROW_TAB_STRIDE = NARROW_W + 4;
constexpr int NARROW_BASE_STRIDE = NARROW_W + 4;
constexpr int NARROW_ACC_STRIDE = NARROW_NMAX + 1;

// Blocks of `kern` that fit on all SMs at once (at least one per SM): the
// kernels that stride over their rows run one resident wave.
template <typename K>
static inline int64_t resident_blocks(K kern, int threads, int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (int64_t)per_sm * nsm;
}

// Adds this warp's per-bin row counts (bins held by the lanes where `has`)
// to a shared histogram with one ballot per bin.
__device__ __forceinline__ void warp_hist(unsigned long long *hist, bool has, int bin) {
    const unsigned have = __ballot_sync(0xffffffffu, has);
    if (!have) return;
    for (int b = 0; b < NBINS; b++) {
        unsigned m = __ballot_sync(0xffffffffu, has && bin == b);
        if (m && (threadIdx.x & 31) == 0) atomicAdd(&hist[b], (unsigned long long)__popc(m));
    }
}

// Multiplicative hash (Fibonacci) of a non-negative key into [0, 2^log2S).
__device__ __forceinline__ unsigned hash_slot(int key, int log2S) {
    return ((unsigned)key * 0x9E3779B1u) >> (32 - log2S);
}

// Insert block `blk` with mask m into a map of 2^L slots; false if full.
__device__ __forceinline__ bool sym_insert(int *keys, unsigned *masks, int L, int blk, unsigned m) {
    const unsigned msk = (1u << L) - 1;
    unsigned h = hash_slot(blk, L);
#pragma unroll 1
    for (int probe = 0; probe <= (int)msk; probe++) {
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
        h = (h + 1) & msk;
    }
    return false;
}

// ---------------------------------------------------------------- launch context
// Every kernel launch goes through a Ctx: it carries the stream and SM count,
// counts launches, and (when timing is on) brackets each launch with CUDA
// events recorded on the launching stream, labelled "<phase>.<kernel>".
struct TimingRec {
    const char *label;
    long long rows;
    cudaEvent_t e0, e1;
};

struct Ctx {
    cudaStream_t s = nullptr;
    int nsm = 0;
    long long *launches = nullptr;
    int timing = 0;                // 0 off, 1 every kernel, 2 numeric-phase kernels only
    bool open = false;             // begin() recorded the current pair's first event
    TimingRec *recs = nullptr;     // handle-owned ring of event pairs
    int *nrec = nullptr;
    int cap = 0;
    const char *phase = "";
    void begin(const char *label, long long rows);
    void end();
};

// ---------------------------------------------------------------- launchers
// analyze.cu
// Compressed column sets (Section 2.1): pairs of row k sit at
// pairs[M.row_ptr[k] .. M.row_ptr[k] + ccnt[k]), each {block, mask};
// minmax[k] = {first block, last block} ({INT_MAX, INT_MIN} for empty rows);
// desc[k] = {row_ptr[k] low, high 32 bits, entries, pairs};
// ana[k] = {entries, pairs}.  Any output may be NULL.
// `unsorted` (may be null) is set to 1 if a row of M is not strictly ascending.
// `long_flag` (may be null; device, cleared by the caller before the call)
// is set to 1 if a row is long enough for the warp-per-row pass, which
// otherwise returns at once; with null that pass tests every row.
int launch_compress(const spgemm_csr &M, int2 *pairs, int32_t *ccnt, int2 *minmax, int4 *desc,
                    int2 *ana, int *err, Ctx &c, int *unsorted = nullptr, int *long_flag = nullptr);
__device__ __forceinline__ int64_t desc_start(int4 d) {
    return (int64_t)(((uint64_t)(unsigned)d.y << 32) | (uint64_t)(unsigned)d.x);
}
size_t scan_tmp_bytes(int64_t n);
// x[0..n] holds counts in x[1..n]; on return x is the exclusive prefix
// (x[0] = 0); *total (device) = x[n].
int launch_scan_counts(int64_t *x, int64_t n, long long *total, void *tmp, Ctx &c);
// Per row i of A: flops, symbolic bin; empty rows get crp[i+1] = 0.
int launch_analyze(const spgemm_csr &A, const spgemm_csr &B, const int2 *ana, int64_t *flops,
                   uint8_t *bins, int64_t *crp, DevState *st, Ctx &c);
// Numeric bin of every row from its output count crp[i+1]-crp[i] and flops;
// rows the symbolic phase found narrow (nlo[i] >= 0; nlo may be null) that
// fit the narrow numeric kernel get BIN_NARROW.
int launch_numeric_binning(int64_t n, const int64_t *crp, const int64_t *flops, uint8_t *bins,
                           DevState *st, Ctx &c, const int32_t *nlo = nullptr);
// Row lists per bin: rows[offset(b) + t]; offsets from st->bin_count[phase]
// (phase 0: symbolic second pass, phase 1: numeric bins 3..6).
int launch_scatter_bins(int64_t n, const uint8_t *bins, const int64_t *crp, int32_t *rows,
                        DevState *st, int phase, Ctx &c, int first_bin = 3);
int launch_row_flops(const spgemm_csr &A, const spgemm_csr &B, int64_t *flops, int *err, Ctx &c);
// Column-block span of each listed row of C, once for all the kernels that
// choose by it: spans[t] = {first block, number of blocks} of the blocks the
// rows of B reached by row rows[t] of A cover (bmm[k] = {first block, last
// block} of B_k); {INT_MAX, 0} when they cover none.
int launch_list_spans(const spgemm_csr &A, const int2 *bmm, const int32_t *rows, int64_t count, int2 *spans,
                      Ctx &c);

// narrow.cu
// Analysis of every row of A (flops, symbolic bin, as launch_analyze) with
// the count of every narrow row done in the same pass (bins[i] =
// BIN_NARROW, nlo[i] = first block of its window; nlo[i] = -1 otherwise).
// bmm[k] = {first block, last block} of B_k; G lanes per row (4..32).
// A narrow row also leaves its non-empty window words, in order, at
// ulist[i*NARROW_NMAX ...] (first NARROW_NMAX of them; {word | rank of its
// first column << 8, mask}) and their number in nwords[i].
int launch_sym_narrow(const spgemm_csr &A, const spgemm_csr &B, const int4 *desc, const int2 *bmm,
                      const int2 *pairs, int64_t *flops, uint8_t *bins, int64_t *crp, int32_t *nlo,
                      uint8_t *nwords, uint2 *ulist, DevState *st, int G, Ctx &c);
// Numeric phase of the rows with bins[i] == BIN_NARROW (F32 or native F64),
// from the word lists of the symbolic phase; G lanes per row (4, 8 or 16).
int launch_num_narrow(int dtype, const spgemm_csr &A, const spgemm_csr &B, spgemm_csr &C, const int4 *bdesc,
                      const int32_t *nlo, const uint8_t *nwords, const uint2 *ulist, const uint8_t *bins, int *err,
                      int G, Ctx &c);

// symbolic.cu
// First pass over all rows with a 32-slot map and G lanes per row (rows of
// bins EMPTY, HUGE and NARROW are skipped).
int launch_symbolic_first(const spgemm_csr &A, const uint8_t *bins, const int4 *desc,
                          const int2 *pairs, int64_t *crp, DevState *st, int G, Ctx &c);
// Second pass: kernels of bins 2..6; counts[b] = rows in bin b (host),
// rows = concatenated bin lists, spans[t] = span of rows[t] (bins 2..5).
// Writes nnz(C_i) to crp[i+1].
int launch_symbolic(const spgemm_csr &A, const spgemm_csr &B, const int2 *pairs,
                    const int32_t *ccnt, const int32_t *rows, const long long *counts,
                    int64_t *crp, int *err, void *gws, size_t gws_bytes, const int2 *spans, Ctx &c);
size_t symbolic_global_ws(int64_t ncols_b, int nsm);

// numeric.cu
// Runs the numeric kernels: bins 1-2 over all rows in order (bins[i]), bins
// 3..6 from the row lists (counts[b] rows in bin b, host; spans[t] = span of
// rows[t] for the lists of bins up to 4).  FP64 uses double-word
// accumulation unless f64_native; bsplit: room for nnz(B) float2.
// Tunables of the numeric phase: lanes per row of the small-row kernel,
// largest output row it takes (16 or 32; bin 2 rows go to the warp kernel
// when 16), and map slots per output entry (2 or 4).
struct NumTune {
    int G = 8;
    int small_cap = 32;
    int slot_factor = 2;
};
int launch_numeric(int dtype, bool f64_native, const spgemm_csr &A, const spgemm_csr &B,
                   spgemm_csr &C, const uint8_t *bins, const int4 *bdesc, const int2 *spans,
                   const int32_t *rows,
                   const long long *counts, DevState *st, float2 *bsplit, void *gws,
                   size_t gws_bytes, int64_t max_row_nnz, const NumTune &tune, bool b_sorted,
                   int64_t max_alen, Ctx &c);
size_t numeric_global_ws(int64_t max_row_nnz, int64_t ncols_b, int nsm, int dtype);
size_t window_global_ws(int64_t max_alen, int nsm);

// batched.cu: one instance of a batch, with its place in the stacked arrays.
struct BatchInst {
    const int64_t *arp, *brp;
    const int32_t *acol, *bcol;
    const void *aval, *bval;
    int64_t a_rows, a_nnz, b_rows, b_nnz;
    int64_t a_p0, b_p0;                  // row_ptr[0] of each operand
    int64_t a_row_off, a_nnz_off, b_row_off, b_nnz_off;
};
// Stack operand `which` (0 = A, 1 = B) of all instances: offsets and
// (shifted) columns when `pattern`, values when val is not null.
int launch_stack(const BatchInst *dinst, int nb, int64_t max_rows, int64_t max_nnz, int which, bool pattern,
                 int vb, int64_t total_rows, int64_t total_nnz, int64_t *rp, int32_t *col, void *val,
                 Ctx &c);

// triangles.cu: triangles of the undirected graph with the symmetric
// pattern A by the masked product L*L .* L (degree-ordered lower triangle
// L, compressed right-hand operand); the count lands in *total (device);
// perm_out / vcount (device, optional): labels, per-vertex counts.
size_t triangles_ws(int64_t n, int64_t nnz, int nsm);
int launch_triangles(const spgemm_csr &A, void *ws, int64_t *perm_out, int64_t *vcount, unsigned long long *total,
                     int *err, Ctx &c);

// backward.cu: dA on pattern(A), dB on pattern(B) from dC on pattern(C).
int launch_backward(int dtype, const spgemm_csr &A, const spgemm_csr &B, const spgemm_csr &C, void *da,
                    void *db, int *err, Ctx &c);

// plan.cu: Algorithm 4.  Cuts are part boundaries (first 0, last nrows).
struct ChunkPlan {
    int algorithm = 0, branch = 0;
    std::vector<int64_t> ac_cuts, b_cuts;
    int64_t size_a = 0, size_b = 0, size_c = 0, cost1 = 0, cost2 = 0;
};
int plan_chunks(const int64_t *a_rp, int64_t n_ac, const int64_t *c_rp, const int64_t *b_rp,
                int64_t n_b, int vb_ac, int vb_b, int64_t fast, ChunkPlan &p);
// BinarySearch cuts of one matrix (rp2 null) or a row-aligned pair.
bool cut_rows(const int64_t *rp1, const int64_t *rp2, int64_t n, int vb, double psize,
              std::vector<int64_t> &cuts);

// chunked.cu: Algorithms 2 and 3 with host operands.
// What a chunked symbolic call learns about its operands and hands on to the
// chunked numeric call of the same product: the column range of every block
// of CHUNK_RB rows of A (the rows of B each part of A reaches, known before
// the part is copied) and the longest row of C.  Valid only for the same
// host arrays and sizes.
constexpr int CHUNK_RB_L = 10, CHUNK_RB = 1 << CHUNK_RB_L;
struct ChunkCache {
    bool valid = false;
    const void *a_rp = nullptr, *a_col = nullptr, *b_rp = nullptr, *b_col = nullptr, *c_rp = nullptr;
    int64_t a_nrows = 0, a_ncols = 0, a_nnz = 0, b_nrows = 0, b_ncols = 0, b_nnz = 0;
    std::vector<int2> brange;   // per block of CHUNK_RB rows of A: {min, max} column ({INT_MAX, INT_MIN} if none)
    int64_t max_row = 0;        // largest row of C
};
// Events of a chunked call: the numeric call uses five groups of up to
// CHUNK_MAX_BUF (one per buffer of a group), the symbolic call the first 8.
constexpr int CHUNK_MAX_BUF = 3;
constexpr int CHUNK_EVENTS = 5 * CHUNK_MAX_BUF;
// Host waits of the library (for a count, a copied-back state or a part's
// column range): wait_ms <= 0 waits as long as it takes; otherwise the wait
// polls and gives up after wait_ms milliseconds with SPGEMM_ERR_TIMEOUT (the
// queued device work keeps running).
int host_wait_stream(cudaStream_t s, int64_t wait_ms, const char *what);
int host_wait_event(cudaEvent_t e, int64_t wait_ms, const char *what);

struct ChunkEnv {
    Ctx *ctx = nullptr;
    ChunkCache *cache = nullptr;
    void *arena = nullptr;        // exactly the budget, device
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev[CHUNK_EVENTS] = {};
    int nbuf = 2;                 // buffers per streamed operand: 2 (double) or 3 (triple)
    int64_t wait_ms = 0;          // limit of the host's waits (0: none)
    int *err = nullptr;
    std::vector<int64_t> *zeros = nullptr;   // host scratch: offsets of an empty C
    int *host_mm = nullptr;                  // pinned: column ranges of the A parts in the buffers
};
struct ChunkStats {
    int algorithm = 0, branch = 0;
    int64_t n_ac = 0, n_b = 0, cost1 = 0, cost2 = 0, h2d = 0, d2h = 0, skipped_b = 0,
            device_bytes = 0, b_windows = 0;
};
int chunked_numeric(ChunkEnv &env, int dtype, const spgemm_csr &A, const spgemm_csr &B,
                    spgemm_csr &C, size_t budget, ChunkStats &stats);
int chunked_symbolic(ChunkEnv &env, const spgemm_csr &A, const spgemm_csr &B, int64_t *C_row_ptr,
                     int64_t *nnz_C, size_t budget, ChunkStats &stats);

}  // namespace sg

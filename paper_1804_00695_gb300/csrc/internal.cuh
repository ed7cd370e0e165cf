// Internal definitions shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
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
};

struct DevState {          // lives in device memory, one per handle
    int err;
    int pad;
    long long nnz;         // nnz(C) written by the scan
    long long bin_count[2][SPGEMM_NBINS];   // [0] symbolic, [1] numeric
    long long bin_cursor[SPGEMM_NBINS];
    long long max_row_nnz;   // largest row of C (numeric binning)
};

// ---------------------------------------------------------------- bins
// Rows are binned by the size of the accumulator they need and by their
// product count; each bin has its own kernel shape (Section 3.3: a half,
// quarter or whole warp per row, or a whole block).
constexpr int BIN_EMPTY = 0;
constexpr int BIN_HUGE = 6;     // widest bin: unbounded accumulator
constexpr int NBINS = SPGEMM_NBINS;   // bins 1..6 used, 7 spare
// Accumulator capacity of bins 1..5 (distinct keys; bin b's map has
// 2*cap slots); bin 6 is unbounded.
__host__ __device__ constexpr long long bin_cap(int b) {
    return b == 1 ? 16 : b == 2 ? 64 : b == 3 ? 256 : b == 4 ? 1024 : b == 5 ? 4096 : (1LL << 40);
}
// Product counts that promote a row to a wider bin.
__host__ __device__ constexpr long long bin_flops(int b) {
    return b == 1 ? 1024 : b == 2 ? 4096 : b == 3 ? 32768 : b == 4 ? 262144 : b == 5 ? 2097152
                                                                               : (1LL << 62);
}

__host__ __device__ inline int bin_of(long long keys, long long flops) {
    if (keys <= 0) return BIN_EMPTY;
    int b = 1;
    while (b < BIN_HUGE && (keys > bin_cap(b) || flops > bin_flops(b))) b++;
    return b;
}

// Multiplicative hash (Fibonacci) of a non-negative key into [0, 2^log2S).
__device__ __forceinline__ unsigned hash_slot(int key, int log2S) {
    return ((unsigned)key * 0x9E3779B1u) >> (32 - log2S);
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
    bool timing = false;
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
// minmax[k] = {first block, last block} ({INT_MAX, INT_MIN} for empty rows).
int launch_compress(const spgemm_csr &M, int2 *pairs, int32_t *ccnt, int2 *minmax,
                    int *err, Ctx &c);
size_t scan_tmp_bytes(int64_t n);
// x[0..n] holds counts in x[1..n]; on return x is the exclusive prefix
// (x[0] = 0); *total (device) = x[n].
int launch_scan_counts(int64_t *x, int64_t n, long long *total, void *tmp, Ctx &c);
// Per row i of A: flops, symbolic bin; empty rows get crp[i+1] = 0.
int launch_analyze(const spgemm_csr &A, const spgemm_csr &B, const int32_t *ccnt,
                   const int2 *minmax, int64_t *flops, uint8_t *bins, int64_t *crp,
                   DevState *st, Ctx &c);
// Numeric bin of every row from its output count crp[i+1]-crp[i] and flops.
int launch_numeric_binning(int64_t n, const int64_t *crp, const int64_t *flops, uint8_t *bins,
                           DevState *st, Ctx &c);
// Row lists per bin: rows[offset(b) + t]; offsets from st->bin_count[phase].
int launch_scatter_bins(int64_t n, const uint8_t *bins, int32_t *rows, DevState *st, int phase,
                        Ctx &c);
int launch_row_flops(const spgemm_csr &A, const spgemm_csr &B, int64_t *flops, int *err, Ctx &c);

// symbolic.cu
// Runs the symbolic kernels of bins 1..6; counts[b] = rows in bin b (host),
// rows = concatenated bin lists.  Writes nnz(C_i) to crp[i+1].
int launch_symbolic(const spgemm_csr &A, const spgemm_csr &B, const int2 *pairs,
                    const int32_t *ccnt, const int32_t *rows, const long long *counts,
                    int64_t *crp, int *err, void *gws, size_t gws_bytes, Ctx &c);
size_t symbolic_global_ws(int64_t ncols_b, int nsm);

// numeric.cu
// Runs the numeric kernels of bins 1..6 (counts[b] rows in bin b, host).
int launch_numeric(int dtype, const spgemm_csr &A, const spgemm_csr &B, spgemm_csr &C,
                   const int32_t *rows, const long long *counts, int *err, void *gws,
                   size_t gws_bytes, int64_t max_row_nnz, Ctx &c);
size_t numeric_global_ws(int64_t max_row_nnz, int64_t ncols_b, int nsm, int dtype);

}  // namespace sg

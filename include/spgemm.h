/*
 * spgemm.h - C ABI of the GB300 (sm_103a) CSR sparse matrix-matrix multiply
 *            library, C = A * B.
 *
 * Method: Deveci, Hammond, Wolf, Rajamanickam, "Sparse Matrix-Matrix
 * Multiplication on Multilevel Memory Architectures: Algorithms and
 * Experiments" (SAND2018-3428 R).  The product is computed row by row
 * (Section 2.1, the row-wise hierarchical kkmem method) in two phases:
 * a symbolic phase that counts the non-zeros of every row of C and a numeric
 * phase that computes the values (Section 2.1).  Column sets in the symbolic
 * phase are compressed into (column / 32, 32-bit mask) pairs (Section 2.1,
 * "compression"); accumulators are hash maps held in shared memory with a
 * second level in global memory (Section 3.3).  Operands too large for the
 * device are streamed through a fixed device budget by the chunking methods
 * of Section 3.3.1 (Algorithms 2, 3 and 4).
 *
 * Conventions for every call:
 *   - Matrices are CSR: row_ptr holds nrows+1 int64 offsets (row_ptr[0] == 0,
 *     non-decreasing), col_idx holds nnz int32 column indices in
 *     [0, ncols), values holds nnz elements of the call's dtype.  Columns of
 *     an input row may be in any order (Section 3.2.2: the kernel does not
 *     assume sorted columns) but must not repeat; repeated columns are not
 *     detected on the device and make the result undefined.  Output rows
 *     have strictly ascending columns.  The output pattern is structural:
 *     an entry exists when a stored a_ik meets a stored b_kj, even if the
 *     computed value is zero.
 *   - The caller owns every array passed in; the library never frees or
 *     keeps them beyond the call, except that spgemm_numeric requires the
 *     same A, B and C.row_ptr arrays as the preceding spgemm_symbolic on the
 *     same handle.
 *   - "device" arrays are CUDA device pointers of the handle's device;
 *     "host" arrays are host pointers (page-locked memory gives full copy
 *     bandwidth; pageable memory works but is slower).
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device-side calls are asynchronous on that stream except where stated.
 *   - Every call returns a spgemm_status.  On failure, spgemm_last_error()
 *     returns a message for the calling thread.  No call aborts the process.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPGEMM_API __attribute__((visibility("default")))
#else
#define SPGEMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spgemm_status {
    SPGEMM_OK = 0,
    SPGEMM_ERR_ARG = 1,          /* null pointer, negative size, bad dtype */
    SPGEMM_ERR_DIM = 2,          /* A.ncols != B.nrows */
    SPGEMM_ERR_INDEX = 3,        /* column index out of range, or offsets/counts overflow */
    SPGEMM_ERR_NOMEM = 4,        /* a device or pinned allocation failed */
    SPGEMM_ERR_BUDGET = 5,       /* chunked: budget below the minimum working set */
    SPGEMM_ERR_TIMEOUT = 6,      /* a host wait ran out (SPGEMM_OPT_WAIT_LIMIT_MS) */
    SPGEMM_ERR_CUDA = 7,         /* a CUDA runtime call failed */
    SPGEMM_ERR_NOT_SYMBOLIC = 8, /* numeric called without a matching symbolic */
    SPGEMM_ERR_INTERNAL = 9      /* a device-side bound was exceeded (hash probe limit) */
} spgemm_status;

typedef enum spgemm_dtype { SPGEMM_F32 = 0, SPGEMM_F64 = 1 } spgemm_dtype;

/* CSR descriptor; see the conventions above.  values may be NULL where a
 * call only reads the pattern. */
typedef struct spgemm_csr {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    int64_t *row_ptr;
    int32_t *col_idx;
    void *values;
} spgemm_csr;

typedef struct spgemm_handle_s *spgemm_handle;

/* Thread-local message describing the last failure (never NULL). */
SPGEMM_API const char *spgemm_last_error(void);

/* Library version string. */
SPGEMM_API const char *spgemm_version(void);

/* Create a handle bound to CUDA device `device`.  The handle owns a device
 * workspace that grows on demand (stream-ordered allocation on the stream of
 * the call that needs it) and small pinned host buffers.  Not thread-safe:
 * use one handle per host thread. */
SPGEMM_API int spgemm_create(spgemm_handle *handle, int device);
SPGEMM_API int spgemm_destroy(spgemm_handle handle);

/* Symbolic phase (Section 2.1): fills C_row_ptr (device, nrows(A)+1 int64)
 * with the row offsets of C = A*B and stores nnz(C) in *nnz_C (host).
 * Steps: column compression of B (Section 2.1), per-row flop counts and
 * binning, per-row union of compressed column sets in shared-memory hash
 * tables or dense bitmaps, exclusive scan.  Synchronises the stream once to
 * return nnz(C).  A, B: device arrays (values unused, may be NULL).
 * Errors: SPGEMM_ERR_DIM, SPGEMM_ERR_INDEX (column of A outside B's rows or
 * of B outside ncols, int64 overflow), SPGEMM_ERR_NOMEM, SPGEMM_ERR_CUDA. */
SPGEMM_API int spgemm_symbolic(spgemm_handle handle, const spgemm_csr *A, const spgemm_csr *B,
                    int64_t *C_row_ptr, int64_t *nnz_C, void *stream);

/* Numeric phase (Section 2.1, hash accumulators of Section 3.3): with C->row_ptr
 * from spgemm_symbolic on this handle for the same A and B (same arrays and
 * sizes), fills C->col_idx and C->values (device, C->nnz elements each) with
 * ascending columns per row.  Values of A, B, C have type dtype.  Does not
 * synchronise.  Errors: SPGEMM_ERR_NOT_SYMBOLIC, SPGEMM_ERR_ARG. */
SPGEMM_API int spgemm_numeric(spgemm_handle handle, int dtype, const spgemm_csr *A,
                   const spgemm_csr *B, spgemm_csr *C, void *stream);

/* Options of a handle.
 *  SPGEMM_OPT_F64_NATIVE (0/1, default 1): 1 = FP64 products and sums in
 *    native FP64.  0 = double-word accumulation in the FP32 units (pairs of
 *    floats, 48 significand bits, three levels where several lanes add to
 *    one entry), within 1e-12 sum|a_ik||b_kj| of the exact entry; rows of A
 *    (or, for B, the whole call) with a non-zero value outside [2^-32, 2^32)
 *    in magnitude accumulate natively.  Native is the faster of the two on
 *    GB300 for the kernels measured (their time goes to latency, not to the
 *    FP64 units); the chunked calls always accumulate natively.
 *  SPGEMM_OPT_LANES_NUMERIC / SPGEMM_OPT_LANES_SYMBOLIC (0, 4, 8, 16, 32;
 *    default 0 = from the mean products per row): lanes that share a row in
 *    the kernels for rows with few outputs (a warp holds 32/lanes rows).
 *  SPGEMM_OPT_SMALL_CAP (16 or 32, default 32): the largest output row the
 *    small-row numeric kernel takes; larger rows go to a warp each.
 *  SPGEMM_OPT_SLOT_FACTOR (2 or 4, default 2): hash-map slots per output
 *    entry in the small-row numeric kernel.
 *  SPGEMM_OPT_NARROW (0/1, default 1): 1 = rows whose columns all fall
 *    within 128 consecutive blocks of 32 columns are counted and (with at
 *    most 32 outputs and 8192 products) multiplied over a dense window of
 *    the compressed column sets (Section 2.1) instead of hash maps; the
 *    window gives every column its rank, so those rows need no probe and no
 *    sort.  They accumulate in native precision whatever
 *    SPGEMM_OPT_F64_NATIVE says.  Takes effect at the next spgemm_symbolic.
 *  SPGEMM_OPT_LANES_NARROW_SYMBOLIC (0, 4, 8, 16, 32) and
 *    SPGEMM_OPT_LANES_NARROW_NUMERIC (0, 4, 8, 16): lanes per row of the
 *    narrow-row kernels (0 = from the mean length of the rows of A).
 *  SPGEMM_OPT_CHUNK_BUFFERS (2 or 3, default 2): buffers per streamed
 *    operand in spgemm_chunked_numeric / spgemm_chunked: 2 = double
 *    buffering (one part is copied while the other is multiplied), 3 =
 *    triple buffering (the buffering the paper's conclusion of Section 4
 *    names: the budget is cut into three segments per operand, so copies
 *    can run one more part ahead of the multiplications, with parts a
 *    third smaller).  Results are identical; only the plan (parts, copy
 *    bytes) and the overlap change.
 *  SPGEMM_OPT_WAIT_LIMIT_MS (>= 0, default 0 = no limit): the longest the
 *    host waits inside a call for the device (the counts of
 *    spgemm_symbolic, the state read by spgemm_check, the column range of a
 *    part in spgemm_chunked_numeric).  A wait that runs out returns
 *    SPGEMM_ERR_TIMEOUT; the work already queued keeps running, so the
 *    caller synchronises its stream before it reuses or frees the call's
 *    buffers, and runs spgemm_symbolic again before spgemm_numeric.
 * spgemm_autotune picks lanes, small-row cap and slot factor by timing. */
typedef enum spgemm_option {
    SPGEMM_OPT_F64_NATIVE = 1,
    SPGEMM_OPT_LANES_NUMERIC = 2,
    SPGEMM_OPT_LANES_SYMBOLIC = 3,
    SPGEMM_OPT_SMALL_CAP = 4,
    SPGEMM_OPT_SLOT_FACTOR = 5,
    SPGEMM_OPT_NARROW = 6,
    SPGEMM_OPT_LANES_NARROW_SYMBOLIC = 7,
    SPGEMM_OPT_LANES_NARROW_NUMERIC = 8,
    SPGEMM_OPT_CHUNK_BUFFERS = 9,
    SPGEMM_OPT_WAIT_LIMIT_MS = 10
} spgemm_option;
SPGEMM_API int spgemm_set_option(spgemm_handle handle, int option, int64_t value);

/* Chunking plan (Section 3.3.1, Algorithm 4), host only.  A_row_ptr and
 * C_row_ptr (host, nrows_A+1 each) and B_row_ptr (host, nrows_B+1) give the
 * sizes; value_bytes is 4 or 8 (0 to size the pattern only); fast_size is
 * the fast-memory budget in bytes.  Fills `plan`: the algorithm (2 = A and
 * C kept in fast memory while B is streamed, Algorithm 2; 3 = B kept while
 * A and C are streamed, Algorithm 3), the Algorithm 4 branch (1..4), the
 * numbers of row parts, the sizes and both copy costs (Algorithm 2:
 * size(A) + size(C) + size(B)|P_AC|; Algorithm 3: size(B) + size(A)|P_B| +
 * size(C)(|P_B|-1)); and, when ac_cuts / b_cuts have room (cap_ac >= n_ac+1,
 * cap_b >= n_b+1, caller-owned host arrays), the part boundaries.  Sizes of a
 * row range are its CSR bytes: 8 per offset, 4 + value_bytes per entry.
 * SPGEMM_ERR_BUDGET if one row exceeds its portion of the budget. */
typedef struct spgemm_chunk_plan {
    int algorithm;
    int branch;
    int64_t n_ac, n_b;
    int64_t size_a, size_b, size_c;
    int64_t cost_chunk1, cost_chunk2;
    int64_t *ac_cuts, *b_cuts;   /* in: caller arrays (may be NULL); out: boundaries */
    int64_t cap_ac, cap_b;       /* in: capacities of those arrays */
} spgemm_chunk_plan;
SPGEMM_API int spgemm_plan_chunks(const int64_t *A_row_ptr, int64_t nrows_A, const int64_t *C_row_ptr,
                                  const int64_t *B_row_ptr, int64_t nrows_B, int value_bytes,
                                  int64_t fast_size, spgemm_chunk_plan *plan);

/* Chunked product for operands in host memory (Section 3.3.1).  A, B and C
 * are host CSR arrays (page-locked memory gives full copy bandwidth); every
 * device byte the call uses comes out of one allocation of exactly
 * fast_mem_budget bytes, kept by the handle between calls of equal budget.
 *
 * spgemm_chunked_symbolic fills C_row_ptr (host, nrows(A)+1) and *nnz_C.
 * The pattern of B stays resident while the rows of A stream through, so
 * Algorithm 4 must be able to place the pattern of B (offsets and columns)
 * in the large (75%) portion; otherwise SPGEMM_ERR_BUDGET.  It also records
 * in the handle the column range of every 1024-row block of A and the
 * longest row of C, for the numeric call of the same arrays.  Synchronises.
 *
 * spgemm_chunked_numeric fills C->col_idx and C->values (host, C->nnz each,
 * C->row_ptr from spgemm_chunked_symbolic).  Algorithm 4 chooses the row
 * parts and between Algorithm 2 (parts of A and C stay while the parts of B
 * stream; parts of B that the part of A does not reach are skipped) and
 * Algorithm 3 (parts of B stay while A and C stream, partial C going out
 * and in).  Each step is the row-range fused multiply-add of Section 3.2.2.
 * In Algorithm 2, when the rows of B a part of A reaches fit one streaming
 * buffer, that window of rows is copied once instead of the fixed parts and
 * the part is multiplied in one pass (same result, fewer bytes and passes).
 * The streamed operand is double buffered on side streams.  Values of C are
 * accumulated natively (FP64 or FP32).  The rows of B each part of A reaches
 * come from the row-block column ranges that spgemm_chunked_symbolic recorded
 * on this handle for the same host arrays of A (those of B and C_row_ptr too
 * for the longest row); a window pass checks every column of A against them
 * (SPGEMM_ERR_NOT_SYMBOLIC from spgemm_check if A changed).  Without them the
 * range of each part is measured on the device and the host waits for it
 * once per part.  The call returns once all copies and kernels are enqueued;
 * synchronise `stream` before reading C, then spgemm_check.
 * Errors: SPGEMM_ERR_BUDGET (a row or the double-buffered parts do not fit),
 * SPGEMM_ERR_NOMEM (the budget cannot be allocated), SPGEMM_ERR_DIM,
 * SPGEMM_ERR_INDEX (symbolic: a column out of range), SPGEMM_ERR_ARG.
 *
 * spgemm_chunked_stats reports the last chunked call: algorithm (2 or 3),
 * Algorithm 4 branch, parts, both copy-cost formulas, bytes actually copied
 * each way, B parts skipped, device bytes in use, and the parts of A whose
 * rows of B came as one window. */
typedef struct spgemm_chunk_stats {
    int algorithm, branch;
    int64_t n_ac, n_b;
    int64_t cost_chunk1, cost_chunk2;
    int64_t h2d_bytes, d2h_bytes;
    int64_t skipped_b_parts;
    int64_t device_bytes;
    int64_t b_windows;
} spgemm_chunk_stats;
SPGEMM_API int spgemm_chunked_symbolic(spgemm_handle handle, const spgemm_csr *A, const spgemm_csr *B,
                                       int64_t *C_row_ptr, int64_t *nnz_C, size_t fast_mem_budget,
                                       void *stream);
SPGEMM_API int spgemm_chunked_numeric(spgemm_handle handle, int dtype, const spgemm_csr *A,
                                      const spgemm_csr *B, spgemm_csr *C, size_t fast_mem_budget,
                                      void *stream);
SPGEMM_API int spgemm_chunked_stats(spgemm_handle handle, spgemm_chunk_stats *out);

/* Allocator of the one-call chunked product: given nnz(C), points *col_idx
 * and *values at host arrays of nnz elements (int32 columns; values of the
 * call's dtype) that the call fills; pinned memory gives full-speed copies.
 * Returns 0 on success. */
typedef int (*spgemm_alloc_fn)(void *user, int64_t nnz, int32_t **col_idx, void **values);

/* Both chunked phases in one call (kkmem(A, B, C, FastSize) of Section 3.3.1):
 * the symbolic phase fills C->row_ptr (host, nrows(A)+1 int64, caller-
 * allocated), `alloc(user, nnz(C), ...)` is called once for the entries, the
 * numeric phase fills them; C->nrows, ncols, nnz, col_idx and values are set.
 * The numeric phase takes the column ranges the symbolic phase recorded.
 * Synchronises `stream` (C is complete on return).
 * Errors: those of the two phases; SPGEMM_ERR_NOMEM if alloc fails or returns
 * NULL arrays for nnz(C) > 0. */
SPGEMM_API int spgemm_chunked(spgemm_handle handle, int dtype, const spgemm_csr *A, const spgemm_csr *B,
                              spgemm_csr *C, spgemm_alloc_fn alloc, void *user, size_t fast_mem_budget,
                              void *stream);

/* The two-phase product with operands in host memory (the paper's problem
 * statement C = A*B with A, B and C where the caller keeps them): A (and B,
 * unless flags has SPGEMM_HOST_B_ON_DEVICE) are host CSR arrays, pinned for
 * full-speed copies.  The call copies them to the device (patterns first,
 * values on a side stream while the symbolic phase runs), runs
 * spgemm_symbolic and spgemm_numeric on the device copies (the same kernels
 * as the device calls), and returns C: C->row_ptr (nrows(A)+1 int64,
 * caller-allocated) filled; `alloc(user, nnz(C), ...)` called once for the
 * entries; C->nrows, ncols, nnz, col_idx, values set.  C is on the host (its
 * offsets copied out while the numeric phase runs, then its entries) unless
 * flags has SPGEMM_HOST_C_ON_DEVICE, in which case C->row_ptr and the
 * allocator's arrays are device memory and nothing is copied out.  The
 * handle keeps the device copies (grown on demand, reused by later calls).
 * Synchronises `stream` (C is complete on return).  Not in the paper as an
 * entry point: its copies are what the chunked calls do when everything
 * fits the fast memory.  Errors: those of the two phases; SPGEMM_ERR_NOMEM
 * if a device copy cannot be allocated or alloc fails. */
#define SPGEMM_HOST_B_ON_DEVICE 1
#define SPGEMM_HOST_C_ON_DEVICE 2
SPGEMM_API int spgemm_host(spgemm_handle handle, int dtype, const spgemm_csr *A, const spgemm_csr *B,
                           spgemm_csr *C, spgemm_alloc_fn alloc, void *user, int flags, void *stream);

/* Placement of the operands (the comparators of Table 3, Section 3.3.1).
 * The device calls (spgemm_symbolic, spgemm_numeric, spgemm_backward, the
 * batched calls, spgemm_triangles) dereference A, B and C through whatever
 * pointers the caller passes: device memory (the default, "HBM"), pinned
 * host memory (cudaHostAlloc / cudaHostRegister: read and written in place
 * over the host link, "Pin" in Table 3), or managed memory (migrated to the
 * device on demand, "UVM").  The library's own workspace is always device
 * memory.  A placement changes only where the bytes travel, never the
 * result.  spgemm_managed_alloc / spgemm_managed_free: managed memory for a
 * caller placing operands there (cudaMallocManaged, cudaMemAttachGlobal;
 * the pages start wherever they are first touched).  Errors:
 * SPGEMM_ERR_NOMEM, SPGEMM_ERR_CUDA. */
SPGEMM_API int spgemm_managed_alloc(size_t bytes, void **ptr);
SPGEMM_API int spgemm_managed_free(void *ptr);

/* Triangles of an undirected graph by a masked sparse product (the
 * triangle-counting experiment of Section 4.1, after Wolf et al.): the
 * vertices are relabelled in order of non-decreasing degree, L is the
 * strictly lower triangle of the relabelled pattern, and the number of
 * triangles is the sum of (L*L) masked by L, computed as L x compressed(L)
 * (Section 2.1's column compression of the right-hand operand).
 * A: device CSR, the symmetric pattern of the graph without self loops
 * (values unused; a self loop is ignored).  *total (host): the number of
 * triangles.  perm (device, nrows int64, may be NULL): the label of every
 * vertex (degrees non-decreasing along the labels; vertices of equal degree
 * in an unspecified order).  vertex_counts (device, nrows int64, may be
 * NULL): for every vertex u, the triangles whose highest-labelled vertex is
 * u (they sum to *total).  The handle keeps the workspace (grown on demand).
 * Synchronises `stream`.  Errors: SPGEMM_ERR_DIM (not square),
 * SPGEMM_ERR_INDEX (a column out of range), SPGEMM_ERR_NOMEM. */
SPGEMM_API int spgemm_triangles(spgemm_handle handle, const spgemm_csr *A, int64_t *total, int64_t *perm,
                                int64_t *vertex_counts, void *stream);

/* Backward of C = A*B for a scalar loss L with dC = dL/dC given on the
 * pattern of C: the product is bilinear, so
 *   dA_ik = sum over stored b_kj of dC_ij b_kj   (dC B^T restricted to the pattern of A)
 *   dB_kj = sum over stored a_ik of a_ik dC_ij   (A^T dC restricted to the pattern of B)
 * A, B: device CSR (values of B needed for dA, values of A for dB); C: the
 * pattern of A*B as produced by spgemm_numeric (ascending columns) with
 * C->values = dC.  dA_values (A->nnz) and dB_values (B->nnz) are device
 * outputs, either may be NULL; both are overwritten.  One pass over the
 * forward products, each dC_ij found by binary search in row i of C; dB is
 * accumulated with atomic adds.  Asynchronous; a product missing from the
 * pattern of C is reported by spgemm_check (SPGEMM_ERR_INTERNAL). */
SPGEMM_API int spgemm_backward(spgemm_handle handle, int dtype, const spgemm_csr *A, const spgemm_csr *B,
                               const spgemm_csr *C, void *dA_values, void *dB_values, void *stream);

/* Batched products C_i = A_i * B_i, i < nbatch (<= 65535), run as one
 * product of block-diagonal operands so that every kernel takes all
 * instances in one launch.  A and B are host arrays of nbatch descriptors of
 * device matrices (row_ptr[0] == 0).  The output is the stacked C: rows of
 * instance i follow those of instance i-1, columns are local to the
 * instance; C_row_ptr: device, sum of nrows(A_i) + 1 int64.
 * spgemm_batched_symbolic also returns nnz(C) in *nnz_total and, if inst_nnz
 * (host, nbatch) is not NULL, nnz(C_i) per instance; synchronises.
 * spgemm_batched_numeric needs the same instance patterns as the symbolic
 * call on this handle; values may live in other arrays between calls (the
 * instance table is re-sent then).  With unchanged arrays it issues only
 * kernel launches on `stream` (no synchronisation, no allocation), so it can
 * be captured in a CUDA graph and replayed.
 * spgemm_batched_backward: dA and dB (stacked over instances, device) for
 * dC given as C->values on the stacked pattern of the last batched product. */
SPGEMM_API int spgemm_batched_symbolic(spgemm_handle handle, int nbatch, const spgemm_csr *A,
                                       const spgemm_csr *B, int64_t *C_row_ptr, int64_t *nnz_total,
                                       int64_t *inst_nnz, void *stream);
SPGEMM_API int spgemm_batched_numeric(spgemm_handle handle, int dtype, int nbatch, const spgemm_csr *A,
                                      const spgemm_csr *B, spgemm_csr *C, void *stream);
SPGEMM_API int spgemm_batched_backward(spgemm_handle handle, int dtype, const spgemm_csr *C,
                                       void *dA_values, void *dB_values, void *stream);

/* Autotuner: times `reps` runs of the last spgemm_numeric call on this handle
 * (same arguments; C is overwritten) under every combination of lanes per row
 * (8, 16, 32), small-row cap (16, 32) and map slots per entry (2, 4), keeps
 * the fastest as the handle's options and leaves C computed with it.
 * choice (host, 3): lanes, cap, slots; *best_ms: its time.  Synchronises. */
SPGEMM_API int spgemm_autotune(spgemm_handle handle, int reps, int64_t *choice, float *best_ms, void *stream);

/* Row offsets from per-row counts, allocating nothing (this entry point
 * has no counterpart in the paper; it exposes the symbolic phase's scan step
 * for callers that may not allocate device memory: programs whose device
 * memory is wholly owned by another allocator, such as a framework's caching
 * pool or an arena reserved up front, and latency-critical paths that cannot
 * afford the implicit device-wide synchronisation of cudaMalloc/cudaFree).
 * row_ptr: device, nrows+1 int64, the count of row i in row_ptr[i+1]
 * (row_ptr[0] is ignored); on completion row_ptr holds the exclusive prefix
 * (row_ptr[0] = 0, row_ptr[nrows] = total).  No handle is needed.  The
 * scratch is a fixed device array of 512 KiB that every device loading the
 * library holds until exit; it serves up to
 * spgemm_row_offsets_noalloc_max_rows() rows (about 134 million); a larger
 * nrows is rejected with SPGEMM_ERR_ARG before anything runs.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.
 * The stream must belong to the current device.  Asynchronous; calls share
 * the scratch, so calls that overlap on the GPU (different streams, not
 * ordered) race and must be avoided; each call overwrites all the scratch it
 * reads, so nothing needs clearing between calls.  Calls no cudaMalloc,
 * cudaFree or allocating routine. */
SPGEMM_API int spgemm_row_offsets_noalloc(int64_t *row_ptr, int64_t nrows, void *stream);
SPGEMM_API int64_t spgemm_row_offsets_noalloc_max_rows(void);

/* Synchronises `stream` and reports device-side errors raised by earlier
 * asynchronous calls on this handle (SPGEMM_ERR_INTERNAL if a hash probe
 * bound was exceeded or a row's column count disagreed with the symbolic
 * phase), then clears them. */
SPGEMM_API int spgemm_check(spgemm_handle handle, void *stream);

/* Inspection of the first two steps, for tests and tuning.
 * spgemm_row_flops: flops[i] (device, nrows(A) int64) = number of products
 * a_ik*b_kj of row i (Section 3.1: accumulator insertions = multiplications).
 * spgemm_compress: the compressed column sets of M (Section 2.1): for every
 * row k, count[k] (device int32) pairs {block = col/32, mask} stored as two
 * uint32 each at pairs[2*(M.row_ptr[k] + t)], t < count[k] (pairs: device,
 * room for 2*nnz(M) uint32).  Consecutive stored columns that share a block
 * are merged, so a sorted row gives one pair per block, ascending. */
SPGEMM_API int spgemm_row_flops(spgemm_handle handle, const spgemm_csr *A, const spgemm_csr *B,
                     int64_t *flops, void *stream);
SPGEMM_API int spgemm_compress(spgemm_handle handle, const spgemm_csr *M, int32_t *count,
                    uint32_t *pairs, void *stream);

/* Per-bin row counts of the last symbolic and numeric phases on this handle
 * (host array of at least SPGEMM_NBINS int64 each), for tests and tuning.
 * Index 7 counts the narrow rows (SPGEMM_OPT_NARROW): in the symbolic
 * array the rows counted over a window, in the numeric array the rows
 * multiplied over one. */
#define SPGEMM_NBINS 8
SPGEMM_API int spgemm_bin_counts(spgemm_handle handle, int64_t *symbolic_bins, int64_t *numeric_bins);

/* Numeric bin (0..6) of a row with `keys` output entries taking `flops`
 * products (0 = empty row): 1 <= 16 entries, 2 <= 32, 3 <= 128, 4 <= 1024,
 * 5 <= 4096, 6 larger; rows with many products move to wider bins.  Host
 * only. */
SPGEMM_API int spgemm_bin_of(int64_t keys, int64_t flops);

/* Instrumentation.  spgemm_launch_count: kernels launched through this
 * handle since it was created.  spgemm_set_timing(h, 1) brackets every
 * kernel launch with CUDA events on its stream, spgemm_set_timing(h, 2) only
 * the launches of the numeric phase (labels "numeric..."), whose events then
 * add less host work to a timed sequence of calls, and
 * spgemm_set_timing(h, 0) none (other modes: SPGEMM_ERR_ARG); spgemm_timings synchronises
 * on those events and returns per-kernel totals (label "<phase>.<kernel>",
 * launches, rows processed, milliseconds) accumulated since the last
 * spgemm_reset_timings; *count = number of labels (up to cap written). */
typedef struct spgemm_timing {
    char label[32];
    int64_t launches;
    int64_t rows;
    double ms;
} spgemm_timing;
SPGEMM_API int spgemm_launch_count(spgemm_handle handle, int64_t *launches);
SPGEMM_API int spgemm_set_timing(spgemm_handle handle, int on);
SPGEMM_API int spgemm_timings(spgemm_handle handle, spgemm_timing *out, int cap, int *count);
SPGEMM_API int spgemm_reset_timings(spgemm_handle handle);

#ifdef __cplusplus
}
#endif
#endif /* SPGEMM_GB300_H */

// C ABI: handle, workspace and the two phases of Section 2.1.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "internal.cuh"

namespace sg {

static thread_local char g_err[1024] = "no error";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

void Ctx::begin(const char *label, long long rows) {
    if (launches) (*launches)++;
    if (!timing || !recs || *nrec >= cap) return;
    TimingRec &r = recs[*nrec];
    if (!r.e0) {
        if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    r.label = label;
    r.rows = rows;
    cudaEventRecord(r.e0, s);
}

void Ctx::end() {
    if (!timing || !recs || *nrec >= cap) return;
    TimingRec &r = recs[*nrec];
    if (!r.e0) return;
    cudaEventRecord(r.e1, s);
    (*nrec)++;
}

}  // namespace sg

using namespace sg;

struct TimingAgg {
    std::string label;
    long long launches = 0, rows = 0;
    double ms = 0;
};

struct spgemm_handle_s {
    int device = 0;
    int nsm = 0;
    DevState *dstate = nullptr;   // device
    DevState *hstate = nullptr;   // pinned mirror
    char *ws = nullptr;           // device workspace (grow only)
    size_t ws_cap = 0;
    // state carried from symbolic to numeric
    bool sym_valid = false;
    const int64_t *a_rp = nullptr, *b_rp = nullptr, *c_rp = nullptr;
    const int32_t *a_col = nullptr, *b_col = nullptr;
    int64_t a_n = 0, a_m = 0, a_nnz = 0, b_n = 0, b_m = 0, b_nnz = 0, c_nnz = 0;
    long long sym_counts[NBINS] = {0};
    long long num_counts[NBINS] = {0};
    int64_t max_row_nnz = 0;
    size_t num_gws = 0;   // bytes of the second-level maps numeric needs
    bool num_lists = false;   // numeric row lists built for this symbolic result
    // options
    bool f64_native = false;
    int g_numeric = 0, g_symbolic = 0;   // lanes per row (0 = from the mean products per row)
    double mean_flops = 0;
    // chunked calls: budget arena, side streams, events, last statistics
    void *arena = nullptr;
    size_t arena_cap = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev[8] = {};
    ChunkStats cstats;
    float chunk_ms = 0;
    // launch counting and CUDA-event timing
    long long launches = 0;
    bool timing = false;
    std::vector<TimingRec> recs;
    int nrec = 0;
    std::vector<TimingAgg> agg;

    Ctx ctx(cudaStream_t s, const char *phase = "") {
        Ctx c;
        c.s = s;
        c.nsm = nsm;
        c.launches = &launches;
        c.timing = timing;
        c.recs = recs.empty() ? nullptr : recs.data();
        c.nrec = &nrec;
        c.cap = (int)recs.size();
        c.phase = phase;
        return c;
    }
};

static int ws_reserve(spgemm_handle h, size_t bytes, cudaStream_t s, size_t keep = 0) {
    if (bytes <= h->ws_cap) return SPGEMM_OK;
    size_t cap = bytes + bytes / 8;
    char *p = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&p, cap, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("workspace allocation of %zu bytes failed: %s", cap, cudaGetErrorString(e));
        return SPGEMM_ERR_NOMEM;
    }
    if (keep && h->ws) SG_CUDA(cudaMemcpyAsync(p, h->ws, keep, cudaMemcpyDeviceToDevice, s));
    if (h->ws) SG_CUDA(cudaFreeAsync(h->ws, s));
    h->ws = p;
    h->ws_cap = cap;
    return SPGEMM_OK;
}

static int check_csr(const spgemm_csr *m, const char *name, bool need_vals) {
    if (!m) { set_error("%s is NULL", name); return SPGEMM_ERR_ARG; }
    if (m->nrows < 0 || m->ncols < 0 || m->nnz < 0) {
        set_error("%s has a negative size", name);
        return SPGEMM_ERR_ARG;
    }
    if (m->nrows >= (1LL << 31) || m->ncols > (1LL << 31)) {
        set_error("%s: dimensions must fit int32 column indices", name);
        return SPGEMM_ERR_INDEX;
    }
    if (!m->row_ptr) { set_error("%s.row_ptr is NULL", name); return SPGEMM_ERR_ARG; }
    if (m->nnz > 0 && !m->col_idx) { set_error("%s.col_idx is NULL", name); return SPGEMM_ERR_ARG; }
    if (need_vals && m->nnz > 0 && !m->values) {
        set_error("%s.values is NULL", name);
        return SPGEMM_ERR_ARG;
    }
    return SPGEMM_OK;
}

static int fetch_state(spgemm_handle h, cudaStream_t s) {
    SG_CUDA(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    SG_CUDA(cudaStreamSynchronize(s));
    return SPGEMM_OK;
}

static int device_errors(int err) {
    if (err & DERR_COL_RANGE) {
        set_error("column index out of range (A column >= nrows(B) or B column >= ncols(B))");
        return SPGEMM_ERR_INDEX;
    }
    if (err & (DERR_PROBE | DERR_COUNT)) {
        set_error("device bound exceeded (hash probe limit or row count mismatch), code %d", err);
        return SPGEMM_ERR_INTERNAL;
    }
    return SPGEMM_OK;
}

extern "C" {

const char *spgemm_last_error(void) { return g_err; }

const char *spgemm_version(void) { return "gb300-spgemm 0.1 (sm_103a)"; }

int spgemm_create(spgemm_handle *handle, int device) {
    if (!handle) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    *handle = nullptr;
    SG_CUDA(cudaSetDevice(device));
    spgemm_handle h = new spgemm_handle_s();
    h->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->dstate, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hstate, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemset(h->dstate, 0, sizeof(DevState));
    if (e != cudaSuccess) {
        set_error("spgemm_create: %s", cudaGetErrorString(e));
        if (h->dstate) cudaFree(h->dstate);
        if (h->hstate) cudaFreeHost(h->hstate);
        delete h;
        return SPGEMM_ERR_CUDA;
    }
    memset(h->hstate, 0, sizeof(DevState));
    *handle = h;
    return SPGEMM_OK;
}

int spgemm_destroy(spgemm_handle h) {
    if (!h) return SPGEMM_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->ws) cudaFree(h->ws);
    for (auto &r : h->recs) {
        if (r.e0) cudaEventDestroy(r.e0);
        if (r.e1) cudaEventDestroy(r.e1);
    }
    if (h->arena) cudaFree(h->arena);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->dstate) cudaFree(h->dstate);
    if (h->hstate) cudaFreeHost(h->hstate);
    delete h;
    return SPGEMM_OK;
}

int spgemm_check(spgemm_handle h, void *stream) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    SG_TRY(fetch_state(h, s));
    int err = h->hstate->err;
    if (err) SG_CUDA(cudaMemsetAsync(&h->dstate->err, 0, sizeof(int), s));
    SG_CUDA(cudaStreamSynchronize(s));
    return device_errors(err);
}

// Largest power of two <= x, clamped to [lo, 32].
static int lanes_for(double x, int lo = 8) {
    int g = lo;
    while (g < 32 && 2 * g <= x) g *= 2;
    return g;
}

// Workspace: [bins | rows | B descriptors] persist from symbolic to numeric;
// after them the symbolic scratch, or (later) the numeric scratch, which may
// overlap it.
static size_t ws_persist(int64_t n, int64_t nb) {
    return align_up((size_t)n) + align_up((size_t)n * 4) + align_up((size_t)nb * 16);
}

int spgemm_symbolic(spgemm_handle h, const spgemm_csr *A, const spgemm_csr *B, int64_t *C_row_ptr,
                    int64_t *nnz_C, void *stream) {
    if (!h || !C_row_ptr || !nnz_C) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", false));
    SG_TRY(check_csr(B, "B", false));
    if (A->ncols != B->nrows) {
        set_error("dimension mismatch: A is %lld x %lld, B is %lld x %lld", (long long)A->nrows,
                  (long long)A->ncols, (long long)B->nrows, (long long)B->ncols);
        return SPGEMM_ERR_DIM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    h->sym_valid = false;
    const int64_t n = A->nrows;
    SG_CUDA(cudaMemsetAsync(h->dstate, 0, sizeof(DevState), s));
    if (n == 0) {
        SG_CUDA(cudaMemsetAsync(C_row_ptr, 0, sizeof(int64_t), s));
        *nnz_C = 0;
        memset(h->sym_counts, 0, sizeof(h->sym_counts));
        memset(h->num_counts, 0, sizeof(h->num_counts));
    } else {
        const size_t o_bins = 0;
        const size_t o_rows = align_up((size_t)n);
        const size_t o_desc = o_rows + align_up((size_t)n * 4);
        const size_t o_ana = ws_persist(n, B->nrows);
        const size_t o_flops = o_ana + align_up((size_t)B->nrows * 16);
        const size_t o_pairs = o_flops + align_up((size_t)n * 8);
        const size_t o_ccnt = o_pairs + align_up((size_t)B->nnz * 8);
        const size_t o_mm = o_ccnt + align_up((size_t)B->nrows * 4);
        const size_t o_tmp = o_mm + align_up((size_t)B->nrows * 8);
        const size_t o_gws = o_tmp + align_up(scan_tmp_bytes(n));
        const size_t gws_bytes = symbolic_global_ws(B->ncols, h->nsm);
        SG_TRY(ws_reserve(h, o_gws + gws_bytes, s));
        char *w = h->ws;
        uint8_t *bins = (uint8_t *)(w + o_bins);
        int32_t *rows = (int32_t *)(w + o_rows);
        int64_t *flops = (int64_t *)(w + o_flops);
        int2 *pairs = (int2 *)(w + o_pairs);
        int32_t *ccnt = (int32_t *)(w + o_ccnt);
        int2 *minmax = (int2 *)(w + o_mm);
        int4 *desc = (int4 *)(w + o_desc);
        int4 *ana = (int4 *)(w + o_ana);
        Ctx c = h->ctx(s);
        // lanes per row from the mean number of compressed pairs a row visits
        const double mean_pairs = (double)A->nnz / (double)n *
                                  ((double)B->nnz / (double)(B->nrows > 0 ? B->nrows : 1)) * 0.6;
        const int gs = h->g_symbolic ? h->g_symbolic : lanes_for(mean_pairs / 8.0);
        SG_TRY(launch_compress(*B, pairs, ccnt, minmax, desc, ana, &h->dstate->err, c));
        SG_TRY(launch_analyze(*A, *B, ana, flops, bins, C_row_ptr, h->dstate, c));
        SG_TRY(launch_symbolic_first(*A, bins, desc, pairs, C_row_ptr, h->dstate, gs, c));
        SG_TRY(fetch_state(h, s));
        SG_TRY(device_errors(h->hstate->err));
        long long second = 0;
        for (int b = 2; b <= BIN_HUGE; b++) second += h->hstate->bin_count[0][b];
        long long first = 0;
        for (int b = 1; b < BIN_HUGE; b++) first += h->hstate->sym_hist[b];
        h->sym_counts[0] = h->hstate->sym_hist[0];
        h->sym_counts[1] = first - (second - h->hstate->bin_count[0][BIN_HUGE]);
        for (int b = 2; b < NBINS; b++) h->sym_counts[b] = h->hstate->bin_count[0][b];
        if (second > 0) {
            SG_TRY(launch_scatter_bins(n, bins, C_row_ptr, rows, h->dstate, 0, c));
            SG_TRY(launch_symbolic(*A, *B, pairs, ccnt, rows, h->hstate->bin_count[0], C_row_ptr,
                                   &h->dstate->err, w + o_gws, gws_bytes, c));
        }
        SG_TRY(launch_scan_counts(C_row_ptr, n, &h->dstate->nnz, w + o_tmp, c));
        SG_TRY(launch_numeric_binning(n, C_row_ptr, flops, bins, h->dstate, c));
        SG_TRY(fetch_state(h, s));
        SG_TRY(device_errors(h->hstate->err));
        *nnz_C = h->hstate->nnz;
        h->mean_flops = (double)h->hstate->flops_total / (double)n;
        memcpy(h->num_counts, h->hstate->bin_count[1], sizeof(h->num_counts));
        h->max_row_nnz = h->hstate->max_row_nnz;
        h->num_gws = h->num_counts[BIN_HUGE]
                         ? numeric_global_ws(h->max_row_nnz, B->ncols, h->nsm, SPGEMM_F64)
                         : 0;
        h->num_lists = false;
        // numeric scratch: B split into double-words, then the second-level maps
        SG_TRY(ws_reserve(h, ws_persist(n, B->nrows) + align_up((size_t)B->nnz * 8) + h->num_gws, s,
                          ws_persist(n, B->nrows)));
    }
    h->a_rp = A->row_ptr; h->a_col = A->col_idx; h->a_n = A->nrows; h->a_m = A->ncols;
    h->a_nnz = A->nnz;
    h->b_rp = B->row_ptr; h->b_col = B->col_idx; h->b_n = B->nrows; h->b_m = B->ncols;
    h->b_nnz = B->nnz;
    h->c_rp = C_row_ptr;
    h->c_nnz = *nnz_C;
    h->sym_valid = true;
    return SPGEMM_OK;
}

int spgemm_numeric(spgemm_handle h, int dtype, const spgemm_csr *A, const spgemm_csr *B,
                   spgemm_csr *C, void *stream) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) { set_error("bad dtype %d", dtype); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", true));
    SG_TRY(check_csr(B, "B", true));
    SG_TRY(check_csr(C, "C", true));
    if (!h->sym_valid || A->row_ptr != h->a_rp || A->col_idx != h->a_col || A->nrows != h->a_n ||
        A->ncols != h->a_m || A->nnz != h->a_nnz || B->row_ptr != h->b_rp || B->col_idx != h->b_col ||
        B->nrows != h->b_n || B->ncols != h->b_m || B->nnz != h->b_nnz || C->row_ptr != h->c_rp ||
        C->nnz != h->c_nnz || C->nrows != A->nrows || C->ncols != B->ncols) {
        set_error("spgemm_numeric: no matching spgemm_symbolic on this handle");
        return SPGEMM_ERR_NOT_SYMBOLIC;
    }
    if (A->nrows == 0 || C->nnz == 0) return SPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    const int64_t n = A->nrows;
    uint8_t *bins = (uint8_t *)h->ws;
    int32_t *rows = (int32_t *)(h->ws + align_up((size_t)n));
    const int4 *bdesc = (const int4 *)(h->ws + align_up((size_t)n) + align_up((size_t)n * 4));
    float2 *bsplit = (float2 *)(h->ws + ws_persist(n, B->nrows));
    char *gws = h->ws + ws_persist(n, B->nrows) + align_up((size_t)B->nnz * 8);
    Ctx c = h->ctx(s);
    long long listed = 0;
    for (int b = 3; b <= BIN_HUGE; b++) listed += h->num_counts[b];
    if (listed > 0 && !h->num_lists) {
        SG_TRY(launch_scatter_bins(n, bins, C->row_ptr, rows, h->dstate, 1, c));
        h->num_lists = true;
    }
    const int gn = h->g_numeric ? h->g_numeric : lanes_for(h->mean_flops / 12.0);
    return launch_numeric(dtype, h->f64_native, *A, *B, *C, bins, bdesc, rows, h->num_counts,
                          h->dstate, bsplit, gws, h->num_gws, h->max_row_nnz, gn, c);
}

// Side streams, events and the budget arena of the chunked calls.
static int chunk_env(spgemm_handle h, size_t budget, cudaStream_t s, ChunkEnv &env, Ctx &c) {
    if (!h->s_in) {
        SG_CUDA(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
        SG_CUDA(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
        for (auto &e : h->ev) SG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (h->arena_cap != budget) {
        if (h->arena) {
            SG_CUDA(cudaStreamSynchronize(s));
            SG_CUDA(cudaFree(h->arena));
            h->arena = nullptr;
            h->arena_cap = 0;
        }
        cudaError_t e = cudaMalloc(&h->arena, budget);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("chunked: cannot allocate the %zu-byte budget: %s", budget, cudaGetErrorString(e));
            return SPGEMM_ERR_NOMEM;
        }
        h->arena_cap = budget;
    }
    // work issued before this call on the caller's stream comes first
    SG_CUDA(cudaEventRecord(h->ev[7], s));
    SG_CUDA(cudaStreamWaitEvent(h->s_in, h->ev[7], 0));
    SG_CUDA(cudaStreamWaitEvent(h->s_out, h->ev[7], 0));
    env.ctx = &c;
    env.arena = h->arena;
    env.s_in = h->s_in;
    env.s_out = h->s_out;
    for (int k = 0; k < 8; k++) env.ev[k] = h->ev[k];
    env.err = &h->dstate->err;
    return SPGEMM_OK;
}

int spgemm_chunked_symbolic(spgemm_handle h, const spgemm_csr *A, const spgemm_csr *B,
                            int64_t *C_row_ptr, int64_t *nnz_C, size_t fast_mem_budget, void *stream) {
    if (!h || !C_row_ptr || !nnz_C) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", false));
    SG_TRY(check_csr(B, "B", false));
    if (A->ncols != B->nrows) { set_error("dimension mismatch"); return SPGEMM_ERR_DIM; }
    for (int64_t k = 0; k < A->nnz; k++)
        if (A->col_idx[k] < 0 || A->col_idx[k] >= B->nrows) {
            set_error("column %lld of A out of range", (long long)k);
            return SPGEMM_ERR_INDEX;
        }
    for (int64_t k = 0; k < B->nnz; k++)
        if (B->col_idx[k] < 0 || B->col_idx[k] >= B->ncols) {
            set_error("column %lld of B out of range", (long long)k);
            return SPGEMM_ERR_INDEX;
        }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    Ctx c = h->ctx(s);
    ChunkEnv env;
    SG_TRY(chunk_env(h, fast_mem_budget, s, env, c));
    h->cstats = ChunkStats();
    SG_TRY(chunked_symbolic(env, *A, *B, C_row_ptr, nnz_C, fast_mem_budget, h->cstats));
    SG_CUDA(cudaStreamSynchronize(s));
    SG_TRY(fetch_state(h, s));
    return device_errors(h->hstate->err);
}

int spgemm_chunked_numeric(spgemm_handle h, int dtype, const spgemm_csr *A, const spgemm_csr *B,
                           spgemm_csr *C, size_t fast_mem_budget, void *stream) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) { set_error("bad dtype %d", dtype); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", true));
    SG_TRY(check_csr(B, "B", true));
    SG_TRY(check_csr(C, "C", true));
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) {
        set_error("dimension mismatch");
        return SPGEMM_ERR_DIM;
    }
    if (C->row_ptr[C->nrows] != C->nnz) {
        set_error("C.row_ptr does not end at C.nnz");
        return SPGEMM_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    Ctx c = h->ctx(s);
    ChunkEnv env;
    SG_TRY(chunk_env(h, fast_mem_budget, s, env, c));
    h->cstats = ChunkStats();
    return chunked_numeric(env, dtype, *A, *B, *C, fast_mem_budget, h->cstats);
}

int spgemm_chunked_stats(spgemm_handle h, spgemm_chunk_stats *out) {
    if (!h || !out) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    const ChunkStats &x = h->cstats;
    out->algorithm = x.algorithm;
    out->branch = x.branch;
    out->n_ac = x.n_ac;
    out->n_b = x.n_b;
    out->cost_chunk1 = x.cost1;
    out->cost_chunk2 = x.cost2;
    out->h2d_bytes = x.h2d;
    out->d2h_bytes = x.d2h;
    out->skipped_b_parts = x.skipped_b;
    out->device_bytes = x.device_bytes;
    return SPGEMM_OK;
}

int spgemm_backward(spgemm_handle h, int dtype, const spgemm_csr *A, const spgemm_csr *B,
                    const spgemm_csr *C, void *dA_values, void *dB_values, void *stream) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) { set_error("bad dtype %d", dtype); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", dB_values != nullptr));
    SG_TRY(check_csr(B, "B", dA_values != nullptr));
    SG_TRY(check_csr(C, "C (values = dC)", true));
    if (A->ncols != B->nrows || C->nrows != A->nrows || C->ncols != B->ncols) {
        set_error("dimension mismatch");
        return SPGEMM_ERR_DIM;
    }
    if (!dA_values && !dB_values) return SPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    Ctx c = h->ctx(s);
    return launch_backward(dtype, *A, *B, *C, dA_values, dB_values, &h->dstate->err, c);
}

int spgemm_set_option(spgemm_handle h, int option, int64_t value) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    switch (option) {
        case SPGEMM_OPT_F64_NATIVE: h->f64_native = value != 0; return SPGEMM_OK;
        case SPGEMM_OPT_LANES_NUMERIC:
        case SPGEMM_OPT_LANES_SYMBOLIC:
            if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32) {
                set_error("lanes per row must be 0 (automatic), 4, 8, 16 or 32");
                return SPGEMM_ERR_ARG;
            }
            (option == SPGEMM_OPT_LANES_NUMERIC ? h->g_numeric : h->g_symbolic) = (int)value;
            return SPGEMM_OK;
        default: set_error("unknown option %d", option); return SPGEMM_ERR_ARG;
    }
}

int spgemm_row_flops(spgemm_handle h, const spgemm_csr *A, const spgemm_csr *B, int64_t *flops,
                     void *stream) {
    if (!h || !flops) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", false));
    SG_TRY(check_csr(B, "B", false));
    if (A->ncols != B->nrows) { set_error("dimension mismatch"); return SPGEMM_ERR_DIM; }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    Ctx c = h->ctx(s);
    SG_TRY(launch_row_flops(*A, *B, flops, &h->dstate->err, c));
    return SPGEMM_OK;
}

int spgemm_compress(spgemm_handle h, const spgemm_csr *M, int32_t *count, uint32_t *pairs,
                    void *stream) {
    if (!h || !count || (!pairs && M && M->nnz)) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(M, "M", false));
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    size_t need = align_up((size_t)M->nrows * 8);
    SG_TRY(ws_reserve(h, need, s));
    h->sym_valid = false;
    Ctx c = h->ctx(s);
    SG_TRY(launch_compress(*M, (int2 *)pairs, count, (int2 *)h->ws, nullptr, nullptr,
                           &h->dstate->err, c));
    return SPGEMM_OK;
}

int spgemm_set_timing(spgemm_handle h, int on) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    h->timing = on != 0;
    if (h->timing && h->recs.empty()) h->recs.resize(8192, TimingRec{nullptr, 0, nullptr, nullptr});
    return SPGEMM_OK;
}

int spgemm_timings(spgemm_handle h, spgemm_timing *out, int cap, int *count) {
    if (!h || !count) { set_error("NULL handle or count"); return SPGEMM_ERR_ARG; }
    SG_CUDA(cudaSetDevice(h->device));
    for (int k = 0; k < h->nrec; k++) {
        TimingRec &r = h->recs[k];
        SG_CUDA(cudaEventSynchronize(r.e1));
        float ms = 0;
        SG_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
        TimingAgg *a = nullptr;
        for (auto &x : h->agg)
            if (x.label == r.label) a = &x;
        if (!a) {
            h->agg.push_back(TimingAgg());
            a = &h->agg.back();
            a->label = r.label;
        }
        a->launches++;
        a->rows += r.rows;
        a->ms += ms;
    }
    h->nrec = 0;
    int n = (int)h->agg.size();
    for (int k = 0; k < n && k < cap && out; k++) {
        memset(out[k].label, 0, sizeof(out[k].label));
        strncpy(out[k].label, h->agg[k].label.c_str(), sizeof(out[k].label) - 1);
        out[k].launches = h->agg[k].launches;
        out[k].rows = h->agg[k].rows;
        out[k].ms = h->agg[k].ms;
    }
    *count = n;
    return SPGEMM_OK;
}

int spgemm_reset_timings(spgemm_handle h) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    h->agg.clear();
    h->nrec = 0;
    return SPGEMM_OK;
}

int spgemm_launch_count(spgemm_handle h, int64_t *launches) {
    if (!h || !launches) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    *launches = h->launches;
    return SPGEMM_OK;
}

int spgemm_bin_of(int64_t keys, int64_t flops) { return num_bin(keys, flops); }

int spgemm_bin_counts(spgemm_handle h, int64_t *symbolic_bins, int64_t *numeric_bins) {
    if (!h) { set_error("handle is NULL"); return SPGEMM_ERR_ARG; }
    for (int b = 0; b < NBINS; b++) {
        if (symbolic_bins) symbolic_bins[b] = h->sym_counts[b];
        if (numeric_bins) numeric_bins[b] = h->num_counts[b];
    }
    return SPGEMM_OK;
}

}  // extern "C"

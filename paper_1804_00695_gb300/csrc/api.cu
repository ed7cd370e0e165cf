// C ABI: handle, workspace and the two phases of Section 2.1.
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
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
    open = false;
    if (!timing || !recs || *nrec >= cap) return;
    if (timing == 2 && strncmp(label, "numeric", 7) != 0) return;
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
    open = true;
}

void Ctx::end() {
    if (!open) return;
    open = false;
    cudaEventRecord(recs[*nrec].e1, s);
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
    int num_lists = 0;        // first bin of the numeric row lists built (0 = none)
    bool b_sorted = false;    // every row of B strictly ascending (symbolic)
    int64_t max_alen = 0;     // longest row of A
    int small_cap = 32, slot_factor = 2;
    // options
    bool f64_native = true;
    bool narrow = true;                  // window-table kernels for narrow rows
    int g_narrow_sym = 0, g_narrow_num = 0;   // their lanes per row (0 = automatic)
    bool sym_narrow_used = false;        // the last symbolic call ran them
    int g_numeric = 0, g_symbolic = 0;   // lanes per row (0 = from the mean products per row)
    double mean_flops = 0;
    // chunked calls: budget arena, side streams, events, last statistics
    void *arena = nullptr;
    size_t arena_cap = 0;
    cudaStream_t s_in = nullptr, s_out = nullptr;
    // [0, CHUNK_EVENTS) chunked calls, then the ordering of a chunked call
    // against the caller's stream (3), then spgemm_host (2)
    static constexpr int EV_ORDER = CHUNK_EVENTS, EV_HOST = CHUNK_EVENTS + 3;
    cudaEvent_t ev[CHUNK_EVENTS + 5] = {};
    int chunk_nbuf = 2;                  // buffers per streamed operand of the chunked numeric call
    int64_t wait_ms = 0;                 // limit of the host's waits (0: none)
    std::vector<int64_t> zeros;   // offsets of an empty C (chunked symbolic plan)
    int *host_mm = nullptr;       // pinned, column ranges of A parts (chunked numeric)
    ChunkStats cstats;
    ChunkCache ccache;            // recorded by the last chunked symbolic call
    float chunk_ms = 0;
    // batched calls: stacked operands and the instance table
    char *bws = nullptr;
    size_t bws_cap = 0;
    std::vector<BatchInst> inst;
    BatchInst *dinst = nullptr;
    spgemm_csr As{}, Bs{};
    int64_t *inst_out = nullptr;   // device, nbatch+1 offsets gathered from C
    int64_t max_ar = 0, max_an = 0, max_br = 0, max_bn = 0;
    // spgemm_triangles: workspace, grown on demand
    char *tws = nullptr;
    size_t tws_cap = 0;
    // spgemm_host: device copies of A, B (and C's entries), grown on demand
    char *hbuf = nullptr, *hbufc = nullptr;
    size_t hbuf_cap = 0, hbufc_cap = 0;
    // last numeric call (for the autotuner)
    bool have_last = false;
    int last_dtype = 0;
    spgemm_csr lastA{}, lastB{}, lastC{};
    // launch counting and CUDA-event timing
    long long launches = 0;
    int timing = 0;
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

template <typename Q>
static int poll_until(Q query, int64_t wait_ms, const char *what) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = query();
        if (e == cudaSuccess) return SPGEMM_OK;
        if (e != cudaErrorNotReady) {
            set_error("%s: %s", what, cudaGetErrorString(e));
            return SPGEMM_ERR_CUDA;
        }
        if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(wait_ms)) {
            set_error("%s: the device work did not finish within %lld ms", what, (long long)wait_ms);
            return SPGEMM_ERR_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int sg::host_wait_stream(cudaStream_t s, int64_t wait_ms, const char *what) {
    if (wait_ms <= 0) {
        SG_CUDA(cudaStreamSynchronize(s));
        return SPGEMM_OK;
    }
    return poll_until([s] { return cudaStreamQuery(s); }, wait_ms, what);
}

int sg::host_wait_event(cudaEvent_t e, int64_t wait_ms, const char *what) {
    if (wait_ms <= 0) {
        SG_CUDA(cudaEventSynchronize(e));
        return SPGEMM_OK;
    }
    return poll_until([e] { return cudaEventQuery(e); }, wait_ms, what);
}

static int fetch_state(spgemm_handle h, cudaStream_t s) {
    SG_CUDA(cudaMemcpyAsync(h->hstate, h->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    return host_wait_stream(s, h->wait_ms, "waiting for the device state");
}

static int device_errors(int err) {
    if (err & DERR_COL_RANGE) {
        set_error("column index out of range (A column >= nrows(B) or B column >= ncols(B))");
        return SPGEMM_ERR_INDEX;
    }
    if (err & DERR_WINDOW) {
        set_error("chunked numeric: a column of A lies outside the rows of B copied for its part "
                  "(A changed after spgemm_chunked_symbolic)");
        return SPGEMM_ERR_NOT_SYMBOLIC;
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
    if (h->bws) cudaFree(h->bws);
    if (h->hbuf) cudaFree(h->hbuf);
    if (h->tws) cudaFree(h->tws);
    if (h->hbufc) cudaFree(h->hbufc);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    if (h->host_mm) cudaFreeHost(h->host_mm);
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

// Workspace offsets.  [bins | rows | B descriptors | B block ranges | spans
// of the listed rows | first window block of every row | window words of
// the narrow rows (count, list)] persist from symbolic to numeric; after
// them the symbolic scratch, or (later) the numeric scratch, which may
// overlap it.
struct WsLayout {
    size_t bins, rows, desc, mm, spans, nlo, nwords, ulist, persist;   // persistent
    size_t ana, flops, pairs, ccnt, tmp, gws;                          // symbolic scratch
};
static WsLayout ws_layout(int64_t n, int64_t nb, int64_t nnzb) {
    WsLayout L;
    L.bins = 0;
    L.rows = L.bins + align_up((size_t)n);
    L.desc = L.rows + align_up((size_t)n * 4);
    L.mm = L.desc + align_up((size_t)nb * 16);
    L.spans = L.mm + align_up((size_t)nb * 8);
    L.nlo = L.spans + align_up((size_t)n * 8);
    L.nwords = L.nlo + align_up((size_t)n * 4);
    L.ulist = L.nwords + align_up((size_t)n);
    L.persist = L.ulist + align_up((size_t)n * NARROW_NMAX * 8);
    L.ana = L.persist;
    L.pairs = L.ana + align_up((size_t)nb * 8);
    L.flops = L.pairs + align_up((size_t)nnzb * 8);
    L.ccnt = L.flops + align_up((size_t)n * 8);
    L.tmp = L.ccnt + align_up((size_t)nb * 4);
    L.gws = L.tmp + align_up(scan_tmp_bytes(n));
    return L;
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
        const WsLayout L = ws_layout(n, B->nrows, B->nnz);
        const size_t gws_bytes = symbolic_global_ws(B->ncols, h->nsm);
        SG_TRY(ws_reserve(h, L.gws + gws_bytes, s));
        char *w = h->ws;
        uint8_t *bins = (uint8_t *)(w + L.bins);
        int32_t *rows = (int32_t *)(w + L.rows);
        int64_t *flops = (int64_t *)(w + L.flops);
        int2 *pairs = (int2 *)(w + L.pairs);
        int32_t *ccnt = (int32_t *)(w + L.ccnt);
        int2 *minmax = (int2 *)(w + L.mm);
        int4 *desc = (int4 *)(w + L.desc);
        int2 *ana = (int2 *)(w + L.ana);
        int32_t *nlo = (int32_t *)(w + L.nlo);
        uint8_t *nwords = (uint8_t *)(w + L.nwords);
        uint2 *ulist = (uint2 *)(w + L.ulist);
        Ctx c = h->ctx(s);
        // lanes per row from the mean number of compressed pairs a row visits
        const double mean_alen = (double)A->nnz / (double)n;
        const double mean_pairs = mean_alen * ((double)B->nnz / (double)(B->nrows > 0 ? B->nrows : 1)) * 0.6;
        const int gs = h->g_symbolic ? h->g_symbolic : lanes_for(mean_pairs / 64.0);
        SG_TRY(launch_compress(*B, pairs, ccnt, minmax, desc, ana, &h->dstate->err, c,
                               &h->dstate->b_unsorted, &h->dstate->long_rows));
        h->sym_narrow_used = h->narrow;
        if (h->narrow) {
            // analysis and the narrow rows' counts in one pass; the first
            // pass below takes the other rows
            // lanes per row: rows of A longer than 32 entries take 8
            const int gn = h->g_narrow_sym ? h->g_narrow_sym : (mean_alen <= 32.0 ? 4 : 8);
            SG_TRY(launch_sym_narrow(*A, *B, desc, minmax, pairs, flops, bins, C_row_ptr, nlo, nwords, ulist,
                                     h->dstate, gn, c));
        } else {
            SG_TRY(launch_analyze(*A, *B, ana, flops, bins, C_row_ptr, h->dstate, c));
        }
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
        h->sym_counts[BIN_NARROW] = h->hstate->sym_hist[BIN_NARROW];
        if (second > 0) {
            SG_TRY(launch_scatter_bins(n, bins, C_row_ptr, rows, h->dstate, 0, c));
            // spans of the rows of bins 2..5 (the lists come in bin order)
            int2 *spans = (int2 *)(w + L.spans);
            long long spanned = 0;
            for (int b = 2; b < BIN_HUGE; b++) spanned += h->hstate->bin_count[0][b];
            SG_TRY(launch_list_spans(*A, minmax, rows, spanned, spans, c));
            SG_TRY(launch_symbolic(*A, *B, pairs, ccnt, rows, h->hstate->bin_count[0], C_row_ptr,
                                   &h->dstate->err, w + L.gws, gws_bytes, spans, c));
        }
        SG_TRY(launch_scan_counts(C_row_ptr, n, &h->dstate->nnz, w + L.tmp, c));
        SG_TRY(launch_numeric_binning(n, C_row_ptr, flops, bins, h->dstate, c, h->narrow ? nlo : nullptr));
        SG_TRY(fetch_state(h, s));
        SG_TRY(device_errors(h->hstate->err));
        *nnz_C = h->hstate->nnz;
        h->mean_flops = (double)h->hstate->flops_total / (double)n;
        memcpy(h->num_counts, h->hstate->bin_count[1], sizeof(h->num_counts));
        h->max_row_nnz = h->hstate->max_row_nnz;
        h->b_sorted = h->hstate->b_unsorted == 0;
        h->max_alen = h->hstate->max_alen;
        h->num_gws = h->num_counts[BIN_HUGE]
                         ? std::max(numeric_global_ws(h->max_row_nnz, B->ncols, h->nsm, SPGEMM_F64),
                                    window_global_ws(h->max_alen, h->nsm))
                         : 0;
        h->num_lists = 0;
        // numeric scratch: B split into double-words, then the second-level maps
        SG_TRY(ws_reserve(h, L.persist + align_up((size_t)B->nnz * 8) + h->num_gws, s, L.persist));
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
    const WsLayout L = ws_layout(n, B->nrows, B->nnz);
    uint8_t *bins = (uint8_t *)(h->ws + L.bins);
    int32_t *rows = (int32_t *)(h->ws + L.rows);
    const int4 *bdesc = (const int4 *)(h->ws + L.desc);
    const int2 *bmm = (const int2 *)(h->ws + L.mm);
    int2 *spans = (int2 *)(h->ws + L.spans);
    const int32_t *nlo = (const int32_t *)(h->ws + L.nlo);
    const uint8_t *nwords = (const uint8_t *)(h->ws + L.nwords);
    const uint2 *ulist = (const uint2 *)(h->ws + L.ulist);
    float2 *bsplit = (float2 *)(h->ws + L.persist);
    char *gws = h->ws + L.persist + align_up((size_t)B->nnz * 8);
    Ctx c = h->ctx(s);
    h->have_last = true;
    h->last_dtype = dtype;
    h->lastA = *A;
    h->lastB = *B;
    h->lastC = *C;
    NumTune tune;
    tune.G = h->g_numeric ? h->g_numeric : lanes_for(h->mean_flops / 80.0);
    tune.small_cap = h->small_cap;
    tune.slot_factor = h->slot_factor;
    const int first_list = tune.small_cap >= 32 ? 3 : 2;
    long long listed = 0;
    for (int b = first_list; b <= BIN_HUGE; b++) listed += h->num_counts[b];
    if (listed > 0 && h->num_lists != first_list) {
        SG_TRY(launch_scatter_bins(n, bins, C->row_ptr, rows, h->dstate, 1, c, first_list));
        // spans of the listed rows up to bin 4 (the kernels that choose by span)
        long long spanned = 0;
        for (int b = first_list; b <= 4; b++) spanned += h->num_counts[b];
        SG_TRY(launch_list_spans(*A, bmm, rows, spanned, spans, c));
        h->num_lists = first_list;
    }
    if (h->num_counts[BIN_NARROW] > 0) {
        // lanes per row: a chunk of G consecutive entries of a row of B per
        // step, so G follows the mean length of the rows of B
        const double mean_blen = (double)B->nnz / (double)(B->nrows > 0 ? B->nrows : 1);
        const int gn = h->g_narrow_num ? h->g_narrow_num : (mean_blen <= 8.0 ? 4 : 8);
        SG_TRY(launch_num_narrow(dtype, *A, *B, *C, bdesc, nlo, nwords, ulist, bins, &h->dstate->err, gn, c));
    }
    return launch_numeric(dtype, h->f64_native, *A, *B, *C, bins, bdesc, spans, rows, h->num_counts,
                          h->dstate, bsplit, gws, h->num_gws, h->max_row_nnz, tune, h->b_sorted,
                          h->max_alen, c);
}

// Side streams and events of the calls with host operands.
static int side_streams(spgemm_handle h) {
    if (!h->s_in) {
        SG_CUDA(cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking));
        SG_CUDA(cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking));
        for (auto &e : h->ev) SG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        SG_CUDA(cudaMallocHost(&h->host_mm, 2 * CHUNK_MAX_BUF * sizeof(int)));
    }
    return SPGEMM_OK;
}

// Side streams, events and the budget arena of the chunked calls.
static int chunk_env(spgemm_handle h, size_t budget, cudaStream_t s, ChunkEnv &env, Ctx &c) {
    SG_TRY(side_streams(h));
    // work a previous call left on the side streams (one that returned an
    // error part-way) finishes before this call reuses or frees the arena
    SG_CUDA(cudaEventRecord(h->ev[h->EV_ORDER + 1], h->s_in));
    SG_CUDA(cudaStreamWaitEvent(s, h->ev[h->EV_ORDER + 1], 0));
    SG_CUDA(cudaEventRecord(h->ev[h->EV_ORDER + 2], h->s_out));
    SG_CUDA(cudaStreamWaitEvent(s, h->ev[h->EV_ORDER + 2], 0));
    if (h->arena_cap != budget) {
        if (h->arena) {
            // s now waits for both side streams: nothing queued touches the
            // arena once it is done
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
    SG_CUDA(cudaEventRecord(h->ev[h->EV_ORDER], s));
    SG_CUDA(cudaStreamWaitEvent(h->s_in, h->ev[h->EV_ORDER], 0));
    SG_CUDA(cudaStreamWaitEvent(h->s_out, h->ev[h->EV_ORDER], 0));
    env.ctx = &c;
    env.cache = &h->ccache;
    env.arena = h->arena;
    env.s_in = h->s_in;
    env.s_out = h->s_out;
    for (int k = 0; k < CHUNK_EVENTS; k++) env.ev[k] = h->ev[k];
    env.nbuf = h->chunk_nbuf;
    env.wait_ms = h->wait_ms;
    env.err = &h->dstate->err;
    env.zeros = &h->zeros;
    env.host_mm = h->host_mm;
    return SPGEMM_OK;
}

int spgemm_chunked_symbolic(spgemm_handle h, const spgemm_csr *A, const spgemm_csr *B,
                            int64_t *C_row_ptr, int64_t *nnz_C, size_t fast_mem_budget, void *stream) {
    if (!h || !C_row_ptr || !nnz_C) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", false));
    SG_TRY(check_csr(B, "B", false));
    if (A->ncols != B->nrows) { set_error("dimension mismatch"); return SPGEMM_ERR_DIM; }
    // column ranges are checked on the device as the parts arrive
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    Ctx c = h->ctx(s);
    ChunkEnv env;
    SG_TRY(chunk_env(h, fast_mem_budget, s, env, c));
    SG_CUDA(cudaMemsetAsync(h->dstate, 0, sizeof(DevState), s));
    h->cstats = ChunkStats();
    ChunkCache &cc = h->ccache;
    cc.valid = false;
    SG_TRY(chunked_symbolic(env, *A, *B, C_row_ptr, nnz_C, fast_mem_budget, h->cstats));
    SG_CUDA(cudaStreamSynchronize(s));
    SG_TRY(fetch_state(h, s));
    SG_TRY(device_errors(h->hstate->err));
    cc.a_rp = A->row_ptr;
    cc.a_col = A->col_idx;
    cc.a_nrows = A->nrows;
    cc.a_ncols = A->ncols;
    cc.a_nnz = A->nnz;
    cc.b_rp = B->row_ptr;
    cc.b_col = B->col_idx;
    cc.b_nrows = B->nrows;
    cc.b_ncols = B->ncols;
    cc.b_nnz = B->nnz;
    cc.c_rp = C_row_ptr;
    cc.valid = true;
    return SPGEMM_OK;
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

int spgemm_chunked(spgemm_handle h, int dtype, const spgemm_csr *A, const spgemm_csr *B, spgemm_csr *C,
                   spgemm_alloc_fn alloc, void *user, size_t fast_mem_budget, void *stream) {
    if (!h || !C || !alloc || !A || !B) { set_error("NULL handle, operand, C or allocator"); return SPGEMM_ERR_ARG; }
    if (!C->row_ptr) { set_error("C.row_ptr is NULL"); return SPGEMM_ERR_ARG; }
    int64_t nnz = 0;
    SG_TRY(spgemm_chunked_symbolic(h, A, B, C->row_ptr, &nnz, fast_mem_budget, stream));
    int32_t *col = nullptr;
    void *val = nullptr;
    if (alloc(user, nnz, &col, &val) != 0 || (nnz > 0 && (!col || !val))) {
        set_error("chunked: the allocator failed for %lld entries of C", (long long)nnz);
        return SPGEMM_ERR_NOMEM;
    }
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->nnz = nnz;
    C->col_idx = col;
    C->values = val;
    SG_TRY(spgemm_chunked_numeric(h, dtype, A, B, C, fast_mem_budget, stream));
    SG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return spgemm_check(h, stream);
}

// Grow-only device buffer of the host-operand calls (previous contents not kept).
static int host_buf(char *&buf, size_t &cap, size_t bytes, cudaStream_t s) {
    if (bytes <= cap) return SPGEMM_OK;
    if (buf) SG_CUDA(cudaFreeAsync(buf, s));
    buf = nullptr;
    cap = 0;
    const size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMallocAsync((void **)&buf, want, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        buf = nullptr;
        set_error("spgemm_host: device copy of %zu bytes failed: %s", want, cudaGetErrorString(e));
        return SPGEMM_ERR_NOMEM;
    }
    cap = want;
    return SPGEMM_OK;
}

int spgemm_host(spgemm_handle h, int dtype, const spgemm_csr *A, const spgemm_csr *B, spgemm_csr *C,
                spgemm_alloc_fn alloc, void *user, int flags, void *stream) {
    if (!h || !C || !alloc || !A || !B) { set_error("NULL handle, operand, C or allocator"); return SPGEMM_ERR_ARG; }
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) { set_error("bad dtype %d", dtype); return SPGEMM_ERR_ARG; }
    if (!C->row_ptr) { set_error("C.row_ptr is NULL"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", true));
    SG_TRY(check_csr(B, "B", true));
    if (A->ncols != B->nrows) { set_error("dimension mismatch"); return SPGEMM_ERR_DIM; }
    const bool b_dev = (flags & SPGEMM_HOST_B_ON_DEVICE) != 0, c_dev = (flags & SPGEMM_HOST_C_ON_DEVICE) != 0;
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    SG_TRY(side_streams(h));
    const size_t vb = dtype == SPGEMM_F32 ? 4 : 8;
    auto part = [](size_t x) { return align_up(x); };
    // device copies: [A row_ptr | A col | A val | B row_ptr | B col | B val | C row_ptr]
    const size_t oa_rp = 0, oa_col = oa_rp + part((size_t)(A->nrows + 1) * 8),
                 oa_val = oa_col + part((size_t)A->nnz * 4), ob_rp = oa_val + part((size_t)A->nnz * vb);
    const size_t ob_col = ob_rp + (b_dev ? 0 : part((size_t)(B->nrows + 1) * 8));
    const size_t ob_val = ob_col + (b_dev ? 0 : part((size_t)B->nnz * 4));
    const size_t oc_rp = ob_val + (b_dev ? 0 : part((size_t)B->nnz * vb));
    const size_t total = oc_rp + part((size_t)(A->nrows + 1) * 8);
    SG_TRY(host_buf(h->hbuf, h->hbuf_cap, total, s));
    char *d = h->hbuf;
    spgemm_csr Ad = *A, Bd = *B;
    Ad.row_ptr = (int64_t *)(d + oa_rp);
    Ad.col_idx = (int32_t *)(d + oa_col);
    Ad.values = d + oa_val;
    if (!b_dev) {
        Bd.row_ptr = (int64_t *)(d + ob_rp);
        Bd.col_idx = (int32_t *)(d + ob_col);
        Bd.values = d + ob_val;
    }
    int64_t *crp = c_dev ? C->row_ptr : (int64_t *)(d + oc_rp);
    // patterns on the caller's stream; values on the copy-in stream, after
    // the work already queued on the caller's stream
    SG_CUDA(cudaEventRecord(h->ev[h->EV_HOST], s));
    SG_CUDA(cudaStreamWaitEvent(h->s_in, h->ev[h->EV_HOST], 0));
    SG_CUDA(cudaMemcpyAsync(Ad.row_ptr, A->row_ptr, (size_t)(A->nrows + 1) * 8, cudaMemcpyHostToDevice, s));
    if (A->nnz) SG_CUDA(cudaMemcpyAsync(Ad.col_idx, A->col_idx, (size_t)A->nnz * 4, cudaMemcpyHostToDevice, s));
    if (!b_dev) {
        SG_CUDA(cudaMemcpyAsync(Bd.row_ptr, B->row_ptr, (size_t)(B->nrows + 1) * 8, cudaMemcpyHostToDevice, s));
        if (B->nnz) SG_CUDA(cudaMemcpyAsync(Bd.col_idx, B->col_idx, (size_t)B->nnz * 4, cudaMemcpyHostToDevice, s));
    }
    if (A->nnz)
        SG_CUDA(cudaMemcpyAsync(Ad.values, A->values, (size_t)A->nnz * vb, cudaMemcpyHostToDevice, h->s_in));
    if (!b_dev && B->nnz)
        SG_CUDA(cudaMemcpyAsync(Bd.values, B->values, (size_t)B->nnz * vb, cudaMemcpyHostToDevice, h->s_in));
    SG_CUDA(cudaEventRecord(h->ev[h->EV_HOST + 1], h->s_in));
    int64_t nnz = 0;
    const int st_sym = spgemm_symbolic(h, &Ad, &Bd, crp, &nnz, stream);
    if (st_sym != SPGEMM_OK) {
        cudaStreamSynchronize(h->s_in);
        return st_sym;
    }
    // C's offsets leave while the numeric phase runs
    if (!c_dev) {
        SG_CUDA(cudaEventRecord(h->ev[h->EV_HOST], s));
        SG_CUDA(cudaStreamWaitEvent(h->s_out, h->ev[h->EV_HOST], 0));
        SG_CUDA(cudaMemcpyAsync(C->row_ptr, crp, (size_t)(A->nrows + 1) * 8, cudaMemcpyDeviceToHost, h->s_out));
    }
    int32_t *col = nullptr;
    void *val = nullptr;
    if (alloc(user, nnz, &col, &val) != 0 || (nnz > 0 && (!col || !val))) {
        cudaStreamSynchronize(h->s_in);
        cudaStreamSynchronize(h->s_out);
        set_error("spgemm_host: the allocator failed for %lld entries of C", (long long)nnz);
        return SPGEMM_ERR_NOMEM;
    }
    spgemm_csr Cd{A->nrows, B->ncols, nnz, crp, col, val};
    if (!c_dev) {
        SG_TRY(host_buf(h->hbufc, h->hbufc_cap, part((size_t)nnz * 4) + part((size_t)nnz * vb), s));
        Cd.col_idx = (int32_t *)h->hbufc;
        Cd.values = h->hbufc + part((size_t)nnz * 4);
    }
    SG_CUDA(cudaStreamWaitEvent(s, h->ev[h->EV_HOST + 1], 0));
    SG_TRY(spgemm_numeric(h, dtype, &Ad, &Bd, &Cd, stream));
    if (!c_dev && nnz) {
        SG_CUDA(cudaMemcpyAsync(col, Cd.col_idx, (size_t)nnz * 4, cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaMemcpyAsync(val, Cd.values, (size_t)nnz * vb, cudaMemcpyDeviceToHost, s));
    }
    if (!c_dev) {
        SG_CUDA(cudaEventRecord(h->ev[h->EV_HOST], h->s_out));
        SG_CUDA(cudaStreamWaitEvent(s, h->ev[h->EV_HOST], 0));
    }
    C->nrows = A->nrows;
    C->ncols = B->ncols;
    C->nnz = nnz;
    C->col_idx = col;
    C->values = val;
    SG_CUDA(cudaStreamSynchronize(s));
    return spgemm_check(h, stream);
}

int spgemm_triangles(spgemm_handle h, const spgemm_csr *A, int64_t *total, int64_t *perm, int64_t *vertex_counts,
                     void *stream) {
    if (!h || !total) { set_error("NULL handle or total"); return SPGEMM_ERR_ARG; }
    SG_TRY(check_csr(A, "A", false));
    if (A->nrows != A->ncols) { set_error("the graph's pattern must be square"); return SPGEMM_ERR_DIM; }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    *total = 0;
    if (A->nrows == 0) return SPGEMM_OK;
    SG_TRY(host_buf(h->tws, h->tws_cap, triangles_ws(A->nrows, A->nnz, h->nsm), s));
    SG_CUDA(cudaMemsetAsync(&h->dstate->err, 0, sizeof(int), s));
    Ctx c = h->ctx(s);
    SG_TRY(launch_triangles(*A, h->tws, perm, vertex_counts, &h->dstate->triangles, &h->dstate->err, c));
    SG_TRY(fetch_state(h, s));
    SG_TRY(device_errors(h->hstate->err));
    *total = (int64_t)h->hstate->triangles;
    return SPGEMM_OK;
}

int spgemm_managed_alloc(size_t bytes, void **ptr) {
    if (!ptr) { set_error("NULL ptr"); return SPGEMM_ERR_ARG; }
    *ptr = nullptr;
    cudaError_t e = cudaMallocManaged(ptr, bytes > 0 ? bytes : 1, cudaMemAttachGlobal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocManaged of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return SPGEMM_ERR_NOMEM;
    }
    return SPGEMM_OK;
}

int spgemm_managed_free(void *ptr) {
    if (ptr) SG_CUDA(cudaFree(ptr));
    return SPGEMM_OK;
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
    out->b_windows = x.b_windows;
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

__global__ void k_gather_offsets(const BatchInst *__restrict__ inst, int nb, const int64_t *__restrict__ crp,
                                 int64_t total_rows, int64_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb) out[i] = crp[inst[i].a_row_off];
    if (i == nb) out[nb] = crp[total_rows];
}

// Instance table of a batch; returns totals.  Fills h->inst (host).
static int batch_table(spgemm_handle h, int nbatch, const spgemm_csr *A, const spgemm_csr *B, bool need_vals) {
    if (nbatch < 0 || (nbatch > 0 && (!A || !B))) { set_error("bad batch"); return SPGEMM_ERR_ARG; }
    if (nbatch > 65535) { set_error("at most 65535 instances per batch"); return SPGEMM_ERR_ARG; }
    h->inst.assign((size_t)nbatch, BatchInst{});
    int64_t ar = 0, an = 0, br = 0, bn = 0;
    h->max_ar = h->max_an = h->max_br = h->max_bn = 0;
    for (int i = 0; i < nbatch; i++) {
        SG_TRY(check_csr(&A[i], "A[i]", need_vals));
        SG_TRY(check_csr(&B[i], "B[i]", need_vals));
        if (A[i].ncols != B[i].nrows) {
            set_error("instance %d: dimension mismatch", i);
            return SPGEMM_ERR_DIM;
        }
        BatchInst &d = h->inst[(size_t)i];
        d.arp = A[i].row_ptr; d.acol = A[i].col_idx; d.aval = A[i].values;
        d.brp = B[i].row_ptr; d.bcol = B[i].col_idx; d.bval = B[i].values;
        d.a_rows = A[i].nrows; d.a_nnz = A[i].nnz; d.b_rows = B[i].nrows; d.b_nnz = B[i].nnz;
        d.a_p0 = d.b_p0 = 0;
        d.a_row_off = ar; d.a_nnz_off = an; d.b_row_off = br; d.b_nnz_off = bn;
        ar += A[i].nrows; an += A[i].nnz; br += B[i].nrows; bn += B[i].nnz;
        h->max_ar = std::max(h->max_ar, A[i].nrows); h->max_an = std::max(h->max_an, A[i].nnz);
        h->max_br = std::max(h->max_br, B[i].nrows); h->max_bn = std::max(h->max_bn, B[i].nnz);
    }
    if (br >= (1LL << 31)) { set_error("batch: stacked rows of B exceed int32 columns"); return SPGEMM_ERR_INDEX; }
    int64_t maxcol = 0;
    for (int i = 0; i < nbatch; i++) maxcol = std::max(maxcol, B[i].ncols);
    h->As = spgemm_csr{ar, br, an, nullptr, nullptr, nullptr};
    h->Bs = spgemm_csr{br, maxcol, bn, nullptr, nullptr, nullptr};
    return SPGEMM_OK;
}

int spgemm_batched_symbolic(spgemm_handle h, int nbatch, const spgemm_csr *A, const spgemm_csr *B,
                            int64_t *C_row_ptr, int64_t *nnz_total, int64_t *inst_nnz, void *stream) {
    if (!h || !C_row_ptr || !nnz_total) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    SG_TRY(batch_table(h, nbatch, A, B, false));
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    const int64_t ar = h->As.nrows, an = h->As.nnz, br = h->Bs.nrows, bn = h->Bs.nnz;
    // stacked arrays: table | A rp, col, val | B rp, col, val | instance offsets
    const size_t o_tab = 0;
    const size_t o_arp = align_up((size_t)nbatch * sizeof(BatchInst));
    const size_t o_acol = o_arp + align_up((size_t)(ar + 1) * 8);
    const size_t o_aval = o_acol + align_up((size_t)an * 4);
    const size_t o_brp = o_aval + align_up((size_t)an * 8);
    const size_t o_bcol = o_brp + align_up((size_t)(br + 1) * 8);
    const size_t o_bval = o_bcol + align_up((size_t)bn * 4);
    const size_t o_out = o_bval + align_up((size_t)bn * 8);
    const size_t need = o_out + align_up((size_t)(nbatch + 1) * 8);
    if (need > h->bws_cap) {
        if (h->bws) SG_CUDA(cudaFreeAsync(h->bws, s));
        h->bws = nullptr;
        h->bws_cap = 0;
        cudaError_t e = cudaMallocAsync((void **)&h->bws, need, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("batched: allocation of %zu bytes failed", need);
            return SPGEMM_ERR_NOMEM;
        }
        h->bws_cap = need;
    }
    char *w = h->bws;
    h->dinst = (BatchInst *)(w + o_tab);
    h->As.row_ptr = (int64_t *)(w + o_arp); h->As.col_idx = (int32_t *)(w + o_acol); h->As.values = w + o_aval;
    h->Bs.row_ptr = (int64_t *)(w + o_brp); h->Bs.col_idx = (int32_t *)(w + o_bcol); h->Bs.values = w + o_bval;
    h->inst_out = (int64_t *)(w + o_out);
    if (nbatch > 0)
        SG_CUDA(cudaMemcpyAsync(h->dinst, h->inst.data(), (size_t)nbatch * sizeof(BatchInst),
                                cudaMemcpyHostToDevice, s));
    Ctx c = h->ctx(s);
    if (nbatch > 0) {
        SG_TRY(launch_stack(h->dinst, nbatch, h->max_ar, h->max_an, 0, true, 0, ar, an, h->As.row_ptr,
                            h->As.col_idx, nullptr, c));
        SG_TRY(launch_stack(h->dinst, nbatch, h->max_br, h->max_bn, 1, true, 0, br, bn, h->Bs.row_ptr,
                            h->Bs.col_idx, nullptr, c));
    } else {
        SG_CUDA(cudaMemsetAsync(h->As.row_ptr, 0, 8, s));
        SG_CUDA(cudaMemsetAsync(h->Bs.row_ptr, 0, 8, s));
    }
    SG_TRY(spgemm_symbolic(h, &h->As, &h->Bs, C_row_ptr, nnz_total, stream));
    if (inst_nnz && nbatch > 0) {
        k_gather_offsets<<<(nbatch + 1 + 255) / 256, 256, 0, s>>>(h->dinst, nbatch, C_row_ptr, ar, h->inst_out);
        SG_CUDA(cudaGetLastError());
        std::vector<int64_t> off((size_t)nbatch + 1);
        SG_CUDA(cudaMemcpyAsync(off.data(), h->inst_out, (size_t)(nbatch + 1) * 8, cudaMemcpyDeviceToHost, s));
        SG_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < nbatch; i++) inst_nnz[i] = off[(size_t)i + 1] - off[(size_t)i];
    }
    return SPGEMM_OK;
}

int spgemm_batched_numeric(spgemm_handle h, int dtype, int nbatch, const spgemm_csr *A, const spgemm_csr *B,
                           spgemm_csr *C, void *stream) {
    if (!h || !C) { set_error("NULL handle or output"); return SPGEMM_ERR_ARG; }
    if (dtype != SPGEMM_F32 && dtype != SPGEMM_F64) { set_error("bad dtype %d", dtype); return SPGEMM_ERR_ARG; }
    if (nbatch != (int)h->inst.size()) { set_error("batched numeric: no matching batched symbolic"); return SPGEMM_ERR_NOT_SYMBOLIC; }
    bool vals_changed = false;
    for (int i = 0; i < nbatch; i++) {
        BatchInst &d = h->inst[(size_t)i];
        if (A[i].row_ptr != d.arp || A[i].col_idx != d.acol || B[i].row_ptr != d.brp || B[i].col_idx != d.bcol ||
            A[i].nnz != d.a_nnz || B[i].nnz != d.b_nnz) {
            set_error("batched numeric: instance %d differs from the batched symbolic", i);
            return SPGEMM_ERR_NOT_SYMBOLIC;
        }
        if ((A[i].nnz && !A[i].values) || (B[i].nnz && !B[i].values)) { set_error("instance %d: NULL values", i); return SPGEMM_ERR_ARG; }
        if (A[i].values != d.aval || B[i].values != d.bval) {
            d.aval = A[i].values;
            d.bval = B[i].values;
            vals_changed = true;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    if (vals_changed && nbatch > 0)
        SG_CUDA(cudaMemcpyAsync(h->dinst, h->inst.data(), (size_t)nbatch * sizeof(BatchInst),
                                cudaMemcpyHostToDevice, s));
    Ctx c = h->ctx(s);
    const int vb = dtype == SPGEMM_F64 ? 8 : 4;
    if (nbatch > 0) {
        SG_TRY(launch_stack(h->dinst, nbatch, h->max_ar, h->max_an, 0, false, vb, h->As.nrows, h->As.nnz,
                            nullptr, nullptr, (void *)h->As.values, c));
        SG_TRY(launch_stack(h->dinst, nbatch, h->max_br, h->max_bn, 1, false, vb, h->Bs.nrows, h->Bs.nnz,
                            nullptr, nullptr, (void *)h->Bs.values, c));
    }
    return spgemm_numeric(h, dtype, &h->As, &h->Bs, C, stream);
}

int spgemm_batched_backward(spgemm_handle h, int dtype, const spgemm_csr *C, void *dA_values,
                            void *dB_values, void *stream) {
    if (!h || !C) { set_error("NULL handle or C"); return SPGEMM_ERR_ARG; }
    if (h->inst.empty() && h->As.nrows == 0) return SPGEMM_OK;
    return spgemm_backward(h, dtype, &h->As, &h->Bs, C, dA_values, dB_values, stream);
}

int spgemm_autotune(spgemm_handle h, int reps, int64_t *choice, float *best_ms, void *stream) {
    if (!h || !h->have_last) { set_error("autotune: run spgemm_numeric once first"); return SPGEMM_ERR_ARG; }
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    SG_CUDA(cudaSetDevice(h->device));
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0));
    SG_CUDA(cudaEventCreate(&e1));
    const int saved[3] = {h->g_numeric, h->small_cap, h->slot_factor};
    float best = 1e30f;
    int bg = saved[0], bc = saved[1], bs = saved[2];
    int status = SPGEMM_OK;
    const int gs[3] = {8, 16, 32}, caps[2] = {32, 16}, slots[2] = {2, 4};
    for (int gi = 0; gi < 3 && status == SPGEMM_OK; gi++)
        for (int ci = 0; ci < 2 && status == SPGEMM_OK; ci++)
            for (int si = 0; si < 2 && status == SPGEMM_OK; si++) {
                h->g_numeric = gs[gi];
                h->small_cap = caps[ci];
                h->slot_factor = slots[si];
                status = spgemm_numeric(h, h->last_dtype, &h->lastA, &h->lastB, &h->lastC, stream);
                if (status != SPGEMM_OK) break;
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && status == SPGEMM_OK; r++)
                    status = spgemm_numeric(h, h->last_dtype, &h->lastA, &h->lastB, &h->lastC, stream);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)reps;
                if (ms < best) {
                    best = ms;
                    bg = gs[gi];
                    bc = caps[ci];
                    bs = slots[si];
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != SPGEMM_OK) {
        h->g_numeric = saved[0];
        h->small_cap = saved[1];
        h->slot_factor = saved[2];
        return status;
    }
    h->g_numeric = bg;
    h->small_cap = bc;
    h->slot_factor = bs;
    // leave C holding the product under the chosen settings
    SG_TRY(spgemm_numeric(h, h->last_dtype, &h->lastA, &h->lastB, &h->lastC, stream));
    if (choice) {
        choice[0] = bg;
        choice[1] = bc;
        choice[2] = bs;
    }
    if (best_ms) *best_ms = best;
    return SPGEMM_OK;
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
        case SPGEMM_OPT_SMALL_CAP:
            if (value != 16 && value != 32) { set_error("small-row cap must be 16 or 32"); return SPGEMM_ERR_ARG; }
            h->small_cap = (int)value;
            return SPGEMM_OK;
        case SPGEMM_OPT_SLOT_FACTOR:
            if (value != 2 && value != 4) { set_error("slot factor must be 2 or 4"); return SPGEMM_ERR_ARG; }
            h->slot_factor = (int)value;
            return SPGEMM_OK;
        case SPGEMM_OPT_NARROW: h->narrow = value != 0; return SPGEMM_OK;
        case SPGEMM_OPT_LANES_NARROW_SYMBOLIC:
            if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32) {
                set_error("narrow symbolic lanes per row must be 0 (automatic), 4, 8, 16 or 32");
                return SPGEMM_ERR_ARG;
            }
            h->g_narrow_sym = (int)value;
            return SPGEMM_OK;
        case SPGEMM_OPT_LANES_NARROW_NUMERIC:
            if (value != 0 && value != 4 && value != 8 && value != 16) {
                set_error("narrow numeric lanes per row must be 0 (automatic), 4, 8 or 16");
                return SPGEMM_ERR_ARG;
            }
            h->g_narrow_num = (int)value;
            return SPGEMM_OK;
        case SPGEMM_OPT_CHUNK_BUFFERS:
            if (value != 2 && value != 3) { set_error("chunk buffers must be 2 or 3"); return SPGEMM_ERR_ARG; }
            h->chunk_nbuf = (int)value;
            return SPGEMM_OK;
        case SPGEMM_OPT_WAIT_LIMIT_MS:
            if (value < 0) { set_error("wait limit must be >= 0 ms"); return SPGEMM_ERR_ARG; }
            h->wait_ms = value;
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
    if (on < 0 || on > 2) { set_error("bad timing mode %d", on); return SPGEMM_ERR_ARG; }
    h->timing = on;
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

// Row offsets from per-row counts with no device allocation at all.
//
// Some callers cannot allocate device memory at the point where they need
// this step: programs whose device memory is wholly owned by another
// allocator (a framework's caching pool, or an arena reserved up front that
// leaves nothing for cudaMalloc), and latency-critical paths where
// cudaMalloc and cudaFree would stall other streams with their implicit
// device-wide synchronisation.  For them this entry point runs the same scan
// kernels as the symbolic phase, but their scratch (one partial sum per tile
// of rows, and the total) lives in a fixed, file-scope device array instead
// of the handle's growable workspace, and no handle is needed.
#include <mutex>
#include "internal.cuh"

namespace sg {

// Scratch: the total, then one 8-byte partial sum per tile of 2048 rows, for
// up to 65536 tiles (134,217,728 rows): 512 KiB, held by every device that
// loads the library until the process exits.
constexpr int64_t NOALLOC_SCRATCH_WORDS = 65536 + 8;
static __device__ __align__(256) long long g_offsets_scratch[NOALLOC_SCRATCH_WORDS];

// Device address of the scratch array, per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) by cudaGetSymbolAddress.
constexpr int NOALLOC_MAX_DEVICES = 64;
static long long *g_scratch_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

static int scratch_for_current_device(long long **out) {
    int dev = 0;
    SG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("spgemm_row_offsets_noalloc: device ordinal %d beyond %d", dev, NOALLOC_MAX_DEVICES);
        return SPGEMM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_offsets_scratch);
        if (e != cudaSuccess || !p) {
            set_error("spgemm_row_offsets_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SPGEMM_ERR_CUDA;
        }
        g_scratch_addr[dev] = (long long *)p;
    }
    *out = g_scratch_addr[dev];
    return SPGEMM_OK;
}

int64_t noalloc_max_rows() {
    // largest n whose scan scratch (plus the total) fits the array
    int64_t lo = 0, hi = (int64_t)1 << 40;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if ((int64_t)scan_tmp_bytes(mid) + 8 <= NOALLOC_SCRATCH_WORDS * 8) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace sg

using namespace sg;

extern "C" int spgemm_row_offsets_noalloc(int64_t *row_ptr, int64_t nrows, void *stream) {
    if (!row_ptr || nrows < 0) {
        set_error("spgemm_row_offsets_noalloc: NULL row_ptr or negative row count");
        return SPGEMM_ERR_ARG;
    }
    if ((int64_t)scan_tmp_bytes(nrows) + 8 > NOALLOC_SCRATCH_WORDS * 8) {
        set_error("spgemm_row_offsets_noalloc: %lld rows exceed the fixed scratch (at most %lld rows)",
                  (long long)nrows, (long long)noalloc_max_rows());
        return SPGEMM_ERR_ARG;
    }
    long long *scratch = nullptr;
    SG_TRY(scratch_for_current_device(&scratch));
    Ctx c;
    c.s = (cudaStream_t)stream;
    // scratch[0] receives the total, the tile sums follow
    return launch_scan_counts(row_ptr, nrows, scratch, scratch + 1, c);
}

extern "C" int64_t spgemm_row_offsets_noalloc_max_rows(void) { return noalloc_max_rows(); }

// Batched products: nbatch independent products A_i * B_i run as one
// product of block-diagonal operands.  Rows of all A_i are stacked, and the
// columns of A_i are shifted to the stacked rows of B_i; the columns of B_i
// (and so of C_i) stay local to the instance, which is harmless because every
// row's accumulator belongs to one instance.  Each kernel of both phases then
// takes all instances in one launch.  The stacking itself is one launch per
// array kind, a block row per instance (grid.y = instance).
#include "internal.cuh"

namespace sg {

__global__ void k_stack_rows(const BatchInst *__restrict__ inst, int nb, int which, int64_t *out,
                             int64_t total_rows, int64_t total_nnz) {
    const BatchInst &d = inst[blockIdx.y];
    const int64_t *rp = which == 0 ? d.arp : d.brp;
    const int64_t rows = which == 0 ? d.a_rows : d.b_rows;
    const int64_t roff = which == 0 ? d.a_row_off : d.b_row_off;
    const int64_t noff = which == 0 ? d.a_nnz_off : d.b_nnz_off;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x)
        out[roff + r] = rp[r] - rp[0] + noff;
    if (blockIdx.y == nb - 1 && blockIdx.x == 0 && threadIdx.x == 0) out[total_rows] = total_nnz;
}

__global__ void k_stack_cols(const BatchInst *__restrict__ inst, int which, int32_t *out) {
    const BatchInst &d = inst[blockIdx.y];
    const int32_t *col = which == 0 ? d.acol : d.bcol;
    const int64_t nnz = which == 0 ? d.a_nnz : d.b_nnz;
    const int64_t noff = which == 0 ? d.a_nnz_off : d.b_nnz_off;
    const int64_t p0 = which == 0 ? d.a_p0 : d.b_p0;
    const int shift = which == 0 ? (int)d.b_row_off : 0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        out[noff + p] = col[p0 + p] + shift;
}

template <typename V>
__global__ void k_stack_vals(const BatchInst *__restrict__ inst, int which, V *out) {
    const BatchInst &d = inst[blockIdx.y];
    const V *val = (const V *)(which == 0 ? d.aval : d.bval);
    const int64_t nnz = which == 0 ? d.a_nnz : d.b_nnz;
    const int64_t noff = which == 0 ? d.a_nnz_off : d.b_nnz_off;
    const int64_t p0 = which == 0 ? d.a_p0 : d.b_p0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x)
        out[noff + p] = val[p0 + p];
}

int launch_stack(const BatchInst *dinst, int nb, int64_t max_rows, int64_t max_nnz, int which, bool pattern,
                 int vb, int64_t total_rows, int64_t total_nnz, int64_t *rp, int32_t *col, void *val,
                 Ctx &c) {
    if (nb == 0) return SPGEMM_OK;
    if (pattern) {
        dim3 g1((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_rows + 255) / 256, 64)), (unsigned)nb);
        c.begin(which == 0 ? "batched.stack_a_rows" : "batched.stack_b_rows", total_rows);
        k_stack_rows<<<g1, 256, 0, c.s>>>(dinst, nb, which, rp, total_rows, total_nnz);
        c.end();
        dim3 g2((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_nnz + 255) / 256, 256)), (unsigned)nb);
        c.begin(which == 0 ? "batched.stack_a_cols" : "batched.stack_b_cols", total_nnz);
        k_stack_cols<<<g2, 256, 0, c.s>>>(dinst, which, col);
        c.end();
    }
    if (val) {
        dim3 g2((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_nnz + 255) / 256, 256)), (unsigned)nb);
        c.begin(which == 0 ? "batched.stack_a_vals" : "batched.stack_b_vals", total_nnz);
        if (vb == 8) k_stack_vals<double><<<g2, 256, 0, c.s>>>(dinst, which, (double *)val);
        else k_stack_vals<float><<<g2, 256, 0, c.s>>>(dinst, which, (float *)val);
        c.end();
    }
    SG_CUDA(cudaGetLastError());
    return SPGEMM_OK;
}

}  // namespace sg

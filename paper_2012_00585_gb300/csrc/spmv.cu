// Sparse matrix-vector product y = G x over the assembled matrix, through
// CSR (column index per value) and through CRAC (one (first column, value
// position) pair per run of consecutive columns, §2.2): the consumer of the
// assembled matrix that the paper's outlook names.  One warp per row; each
// lane's products are summed in a fixed order (lane-strided partial sums,
// then a fixed shuffle tree), so results are reproducible run to run.
#include "internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_spmv_csr(int64_t n_rows, const int64_t *__restrict__ row_ptr,
                                                  const int32_t *__restrict__ col_idx,
                                                  const double *__restrict__ values, const double *__restrict__ x,
                                                  double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = fe_warp_id(); i < n_rows; i += fe_warps()) {
        const int64_t a = row_ptr[i], b = row_ptr[i + 1];
        double s = 0.0;
        for (int64_t k = a + lane; k < b; k += 32) s += __ldcs(values + k) * __ldg(x + __ldcs(col_idx + k));
        s = warp_sum(s);
        if (lane == 0) y[i] = s;
    }
}

// The row's pairs are read 32 at a time (lane r holds pair r); the run of
// value position p is the last pair whose position is <= p, found by a
// five-step binary search over the lanes (every lane takes part in every
// shuffle: the loop over positions has the same trip count on all lanes).
__global__ void __launch_bounds__(256) k_spmv_crac(int64_t n_rows, const int64_t *__restrict__ crac_ptr,
                                                   const int32_t *__restrict__ col_align,
                                                   const double *__restrict__ values, const double *__restrict__ x,
                                                   double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = fe_warp_id(); i < n_rows; i += fe_warps()) {
        const int64_t pa = crac_ptr[i], pb = crac_ptr[i + 1];
        const int n_runs = (int)((pb - pa) >> 1);
        double s = 0.0;
        for (int r0 = 0; r0 < n_runs; r0 += 32) {
            const int r = r0 + lane;
            const int last = min(32, n_runs - r0);  // runs in this group
            const int32_t first = r < n_runs ? col_align[pa + 2 * r] : 0;
            const int32_t pos = r < n_runs ? col_align[pa + 2 * r + 1] : INT32_MAX;
            // value positions of the group: from its first run to the next pair's position
            const int32_t p0 = __shfl_sync(0xffffffffu, pos, 0);
            const int32_t pend = col_align[pa + 2 * (r0 + last) + 1];
            for (int32_t base = p0; base < pend; base += 32) {
                const int32_t p = base + lane;
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int cand = lo + step;
                    const int32_t pc = __shfl_sync(0xffffffffu, pos, cand < 32 ? cand : 31);
                    if (cand < last && pc <= p) lo = cand;
                }
                const int32_t f = __shfl_sync(0xffffffffu, first, lo);
                const int32_t ps = __shfl_sync(0xffffffffu, pos, lo);
                if (p < pend) s += __ldcs(values + p) * __ldg(x + f + (p - ps));
            }
        }
        s = warp_sum(s);
        if (lane == 0) y[i] = s;
    }
}

int spmv(fe_ctx *ctx, const fe_pattern *p, const double *values, const double *x, double *y, void *stream, bool crac)
{
    if (!ctx || !p || p->ctx != ctx || (p->nnz > 0 && (!values || !x)) || (p->n_dofs > 0 && !y))
        return FE_ERR_INVALID_ARG;
    if (crac && !p->col_align) return FE_ERR_NOT_BUILT;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->n_dofs > 0) {
        const int grid = fe_grid_for(p->n_dofs * 32, 256, ctx->num_sms, 8);
        if (crac) k_spmv_crac<<<grid, 256, 0, s>>>(p->n_dofs, p->crac_ptr, p->col_align, values, x, y);
        else k_spmv_csr<<<grid, 256, 0, s>>>(p->n_dofs, p->row_ptr, p->col_idx, values, x, y);
        fe_note_launch();
    }
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        fe_set_last_cuda_error(e, "spmv launch", __LINE__);
        return FE_ERR_DEVICE;
    }
    return FE_OK;
}

}  // namespace

extern "C" {

int fe_spmv_csr(fe_ctx *ctx, const fe_pattern *p, const double *values, const double *x, double *y, void *stream)
{
    return spmv(ctx, p, values, x, y, stream, false);
}

int fe_spmv_crac(fe_ctx *ctx, const fe_pattern *p, const double *values, const double *x, double *y, void *stream)
{
    return spmv(ctx, p, values, x, y, stream, true);
}

}  // extern "C"

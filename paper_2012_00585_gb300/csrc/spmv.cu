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

// One warp per row, rows strided by all warps; the next row's pointers are
// loaded one row ahead, and the entries are taken 128 at a time: column
// indices and values of four 32-entry windows first, then the x gathers, then
// the products (in window order, so the sum order is fixed).
__global__ void __launch_bounds__(256) k_spmv_csr(int64_t n_rows, const int64_t *__restrict__ row_ptr,
                                                  const int32_t *__restrict__ col_idx,
                                                  const double *__restrict__ values, const double *__restrict__ x,
                                                  double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = fe_warps();
    int64_t i = fe_warp_id();
    int64_t a = 0, b = 0;
    if (i < n_rows) {
        a = row_ptr[i];
        b = row_ptr[i + 1];
    }
    for (; i < n_rows; i += W) {
        int64_t an = 0, bn = 0;
        if (i + W < n_rows) {
            an = row_ptr[i + W];
            bn = row_ptr[i + W + 1];
        }
        double s = 0.0;
        for (int64_t k0 = a; k0 < b; k0 += 128) {
            int32_t c[4];
            double v[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t k = k0 + 32 * u + lane;
                c[u] = k < b ? __ldcs(col_idx + k) : -1;
                v[u] = k < b ? __ldcs(values + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) s += v[u] * xv[u];
        }
        s = warp_sum(s);
        if (lane == 0) y[i] = s;
        a = an;
        b = bn;
    }
}

// CRAC: the row's value positions are taken 32 at a time, p = base + lane
// (values coalesced).  The pairs of up to 32 runs are held one per lane; the
// run of each position comes from a ballot of the runs starting inside the
// window and a population count (the run holding the window's first position
// is the last one starting at or before it).  Row starts (first value
// position and pair range) are loaded one row ahead.  The product order per
// lane is fixed: reproducible run to run.
__global__ void __launch_bounds__(256) k_spmv_crac(int64_t n_rows, const int64_t *__restrict__ crac_ptr,
                                                   const int32_t *__restrict__ col_align,
                                                   const double *__restrict__ values, const double *__restrict__ x,
                                                   double *__restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = fe_warps();
    int64_t i = fe_warp_id();
    int64_t pa = 0, pb = 0;
    if (i < n_rows) {
        pa = crac_ptr[i];
        pb = crac_ptr[i + 1];
    }
    for (; i < n_rows; i += W) {
        int64_t pan = 0, pbn = 0;
        if (i + W < n_rows) {
            pan = crac_ptr[i + W];
            pbn = crac_ptr[i + W + 1];
        }
        const int n_runs = (int)((pb - pa) >> 1);
        double s = 0.0;
        for (int r0 = 0; r0 < n_runs; r0 += 32) {
            const int r = r0 + lane;
            const int last = min(32, n_runs - r0);  // runs held in this group
            const int32_t first = r < n_runs ? col_align[pa + 2 * r] : 0;
            const int32_t pos = r < n_runs ? col_align[pa + 2 * r + 1] : INT32_MAX;
            const int32_t p0 = __shfl_sync(0xffffffffu, pos, 0);
            const int32_t pend = col_align[pa + 2 * (r0 + last) + 1];  // next pair's position
            for (int32_t base = p0; base < pend; base += 32) {
                // runs of this group starting at or before the window's start, and inside it
                const int before = __popc(__ballot_sync(0xffffffffu, lane < last && pos <= base)) - 1;
                // bit o of `starts` set when a run of the group starts at base + o (o > 0)
                uint32_t starts = 0;
                {
                    const int o = pos - base;
                    const uint32_t mine = (lane < last && o > 0 && o < 32) ? (1u << o) : 0u;
                    starts = __reduce_or_sync(0xffffffffu, mine);
                }
                const int k = before + __popc(starts & ((2u << lane) - 1u));
                const int32_t f = __shfl_sync(0xffffffffu, first, k);
                const int32_t ps = __shfl_sync(0xffffffffu, pos, k);
                const int32_t p = base + lane;
                if (p < pend) s += __ldcs(values + p) * __ldg(x + f + (p - ps));
            }
        }
        s = warp_sum(s);
        if (lane == 0) y[i] = s;
        pa = pan;
        pb = pbn;
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
        if (crac)
            k_spmv_crac<<<fe_grid_resident(k_spmv_crac, p->n_dofs * 32, 256, ctx->num_sms), 256, 0, s>>>(
                p->n_dofs, p->crac_ptr, p->col_align, values, x, y);
        else
            k_spmv_csr<<<fe_grid_resident(k_spmv_csr, p->n_dofs * 32, 256, ctx->num_sms), 256, 0, s>>>(
                p->n_dofs, p->row_ptr, p->col_idx, values, x, y);
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

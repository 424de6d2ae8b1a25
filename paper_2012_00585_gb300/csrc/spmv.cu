// Sparse matrix-vector product y = G x over the assembled matrix, through
// CSR (column index per value) and through CRAC (one (first column, value
// position) pair per run of consecutive columns, §2.2): the consumer of the
// assembled matrix that the paper's outlook names.  A group of lanes per row;
// each lane's products are summed in a fixed order (lane-strided partial
// sums, then a fixed shuffle tree), so results are reproducible run to run.
#include "internal.cuh"

namespace {

// G lanes per row (32/G rows per warp; on GB300 the FP64 pipe limits the
// product: a warp-wide reduction per row costs more adds than the row has
// entries, and fewer lanes per row waste fewer predicated multiply-adds).  Row groups are strided by all warps; the
// next group's pointers are loaded one group ahead.  Each lane sums its
// entries k = a + lane, a + lane + G, ... in order, then a fixed shuffle tree
// over the G lanes: the sum order is fixed (reproducible run to run).
constexpr int SPMV_G = 4;  // default lanes per row (FE_KNOB_SPMV_LANES); fastest of 2/4/8/16 measured

template <int G>
__device__ __forceinline__ double group_sum(double v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int G>
__global__ void __launch_bounds__(256) k_spmv_csr(int64_t n_rows, const int64_t *__restrict__ row_ptr,
                                                  const int32_t *__restrict__ col_idx,
                                                  const double *__restrict__ values, const double *__restrict__ x,
                                                  double *__restrict__ y)
{
    constexpr int R = 32 / G, UNR = G >= 8 ? 4 : 2;  // entries per lane per step
    const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
    const int64_t stride = fe_warps() * R;
    int64_t i = fe_warp_id() * R + sub;
    int64_t a = 0, b = 0;
    if (i < n_rows) {
        a = row_ptr[i];
        b = row_ptr[i + 1];
    }
    for (int64_t base = fe_warp_id() * R; base < n_rows; base += stride, i += stride) {
        int64_t an = 0, bn = 0;
        if (i + stride < n_rows) {
            an = row_ptr[i + stride];
            bn = row_ptr[i + stride + 1];
        }
        double s = 0.0;
        for (int64_t k0 = a + gl; k0 < b; k0 += UNR * G) {
            int32_t c[UNR];
            double v[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int64_t k = k0 + u * G;
                c[u] = k < b ? __ldcs(col_idx + k) : -1;
                v[u] = k < b ? __ldcs(values + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u)
                if (c[u] >= 0) s += v[u] * __ldg(x + c[u]);
        }
        s = group_sum<G>(s);
        if (gl == 0 && i < n_rows) y[i] = s;
        a = an;
        b = bn;
    }
}

// CRAC: the same G lanes per row over the value positions p (coalesced);
// each lane walks the row's runs with its positions (the pairs are read
// through L1; runs are rarely shorter than G, so a lane moves about one run
// per step).  The column of p is first + (p - pos) of its run.
template <int G>
__global__ void __launch_bounds__(256) k_spmv_crac(int64_t n_rows, const int64_t *__restrict__ crac_ptr,
                                                   const int32_t *__restrict__ col_align,
                                                   const double *__restrict__ values, const double *__restrict__ x,
                                                   double *__restrict__ y)
{
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane / G, gl = lane % G;
    const int64_t stride = fe_warps() * R;
    int64_t i = fe_warp_id() * R + sub;
    int64_t pa = 0, pb = 0;
    if (i < n_rows) {
        pa = crac_ptr[i];
        pb = crac_ptr[i + 1];
    }
    for (int64_t base = fe_warp_id() * R; base < n_rows; base += stride, i += stride) {
        int64_t pan = 0, pbn = 0;
        if (i + stride < n_rows) {
            pan = crac_ptr[i + stride];
            pbn = crac_ptr[i + stride + 1];
        }
        double s = 0.0;
        if (pb > pa) {
            // run r: (first, pos) at pa + 2r; its end is the position of the next pair
            // (the next row's first pair, or the final pair, after the last run)
            int64_t r2 = pa;
            int32_t first = __ldg(col_align + r2), pos = __ldg(col_align + r2 + 1);
            int32_t next = __ldg(col_align + r2 + 3);
            const int32_t pend = __ldg(col_align + pb + 1);
            for (int32_t p = pos + gl; p < pend; p += G) {
                while (p >= next) {
                    r2 += 2;
                    first = __ldg(col_align + r2);
                    pos = __ldg(col_align + r2 + 1);
                    next = __ldg(col_align + r2 + 3);
                }
                s += __ldcs(values + p) * __ldg(x + first + (p - pos));
            }
        }
        s = group_sum<G>(s);
        if (gl == 0 && i < n_rows) y[i] = s;
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
        const int G = ctx->knob[FE_KNOB_SPMV_LANES] > 0 ? ctx->knob[FE_KNOB_SPMV_LANES] : SPMV_G;
        const int64_t work = (p->n_dofs + 32 / G - 1) / (32 / G) * 32;  // threads: one warp per row group
        auto go = [&](auto csr_kern, auto crac_kern) {
            if (crac)
                crac_kern<<<fe_grid_resident(crac_kern, work, 256, ctx->num_sms), 256, 0, s>>>(
                    p->n_dofs, p->crac_ptr, p->col_align, values, x, y);
            else
                csr_kern<<<fe_grid_resident(csr_kern, work, 256, ctx->num_sms), 256, 0, s>>>(
                    p->n_dofs, p->row_ptr, p->col_idx, values, x, y);
        };
        switch (G) {
        case 2: go(k_spmv_csr<2>, k_spmv_crac<2>); break;
        case 16: go(k_spmv_csr<16>, k_spmv_crac<16>); break;
        case 8: go(k_spmv_csr<8>, k_spmv_crac<8>); break;
        default: go(k_spmv_csr<4>, k_spmv_crac<4>); break;
        }
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

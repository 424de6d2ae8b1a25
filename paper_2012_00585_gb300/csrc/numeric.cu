// Numeric phase: scatter-add every element-matrix entry into its global slot.
//
//   FE_ATOMIC         element-parallel, FP64 atomic add into the values array
//                     (the atomic parallel assembly of Listing 3); one warp per
//                     element streams K_e with coalesced loads.
//   FE_DETERMINISTIC  row-parallel gather: one warp per row walks the row's
//                     (element, local row) incidences in ascending element
//                     order and adds each K_e(r, :) into per-row accumulators
//                     in shared memory, then writes the row once.  Each value
//                     is summed in exactly the order of Listing 2, so the
//                     result is bit-identical to the sequential assembly.
//
// CSR kernels find the slot of (e, r, c) through a per-entry map (relative to
// the row start).  CRAC kernels use the compressed DOF runs of §2.1: one map
// entry per (e, r, run), the row start taken from the CRAC pairs, and the
// column's offset inside its run (Listing 5's contiguous slices).
#include <algorithm>

#include "internal.cuh"

namespace {

__device__ __forceinline__ int64_t warp_id_global() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t warps_total() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

struct CracArgs {
    const int64_t *crac_ptr;
    const int32_t *col_align;
    const uint32_t *run_mask;
    const int64_t *run_ptr;
    int uniform_R;  // > 0 when every element has this many runs and the same mask
    int mask_words;
};

// First value position of row i, read from the CRAC pairs (pair 0's value
// position; for an empty row the next pair's, which is the same number).
__device__ __forceinline__ int64_t crac_row_base(const CracArgs &ca, int64_t i)
{
    return ca.col_align[ca.crac_ptr[i] + 1];
}

// For column c of an element whose run-start bits (c < 32) are m: the index
// of the run holding c and c's offset inside it.
__device__ __forceinline__ void run_of(uint32_t m, int c, int &k, int &off)
{
    const uint32_t le = m & (0xffffffffu >> (31 - c));
    k = __popc(le) - 1;
    off = c - (31 - __clz(le));
}

// ------------------------------------------------------------ atomic ---
// One warp per element, NLOC <= 32 known at compile time.  All loads of the
// element are issued before its atomics.
template <int NLOC, typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_atomic_small(const double *__restrict__ K, const int32_t *__restrict__ D,
                                                      int64_t n_e, const int64_t *__restrict__ row_ptr,
                                                      const MT *__restrict__ map, CracArgs ca,
                                                      const MT *__restrict__ mapc, double *values)
{
    constexpr int NN = NLOC * NLOC;
    constexpr int IT = (NN + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int64_t e = warp_id_global(); e < n_e; e += warps_total()) {
        const int32_t d = lane < NLOC ? D[e * NLOC + lane] : 0;
        int64_t base = 0;
        int kc = 0, offc = 0, nr = 0;
        int64_t rp = 0;
        if (!CRAC) {
            if (lane < NLOC) base = row_ptr[d];
        } else {
            if (lane < NLOC) base = crac_row_base(ca, d);
            const uint32_t m = ca.uniform_R ? ca.run_mask[0] : ca.run_mask[e];
            if (lane < NLOC) run_of(m, lane, kc, offc);
            if (ca.uniform_R) {
                nr = ca.uniform_R;
                rp = e * nr;
            } else {
                rp = ca.run_ptr[e];
                nr = (int)(ca.run_ptr[e + 1] - rp);
            }
        }
        const double *Ke = K + e * NN;
        double kv[IT];
        int rel[IT];
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int q = lane + 32 * j;
            kv[j] = 0.0;
            rel[j] = 0;
            if (q < NN) {
                kv[j] = __ldcs(Ke + q);
                if (!CRAC) rel[j] = (int)__ldcs(map + e * NN + q);
            }
        }
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int q = lane + 32 * j;
            const int qq = q < NN ? q : 0;
            const int r = qq / NLOC, c = qq % NLOC;
            const int64_t b = __shfl_sync(0xffffffffu, base, r);
            int64_t slot;
            if (!CRAC) {
                slot = b + rel[j];
            } else {
                const int k = __shfl_sync(0xffffffffu, kc, c);
                const int off = __shfl_sync(0xffffffffu, offc, c);
                slot = b + (int64_t)mapc[rp * NLOC + r * nr + k] + off;
            }
            if (q < NN) atomicAdd(values + slot, kv[j]);
        }
    }
}

// Any n_loc <= FE_MAX_NLOC: one warp per (element, local row).
template <typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_atomic_generic(const double *__restrict__ K, const int32_t *__restrict__ D,
                                                        int64_t n_inc, int32_t n_loc,
                                                        const int64_t *__restrict__ row_ptr,
                                                        const MT *__restrict__ map, CracArgs ca,
                                                        const MT *__restrict__ mapc, double *values)
{
    const int lane = threadIdx.x & 31;
    for (int64_t t = warp_id_global(); t < n_inc; t += warps_total()) {
        const int64_t e = (int64_t)((uint32_t)t / (uint32_t)n_loc);
        const int r = (int)(t - e * n_loc);
        const int32_t row = D[t];
        int64_t base, rp = 0;
        int nr = 0;
        if (!CRAC) {
            base = row_ptr[row];
        } else {
            base = crac_row_base(ca, row);
            rp = ca.run_ptr[e];
            nr = (int)(ca.run_ptr[e + 1] - rp);
        }
        int before = 0, last_start = 0;
        for (int c0 = 0; c0 < n_loc; c0 += 32) {
            const int c = c0 + lane;
            int64_t slot = 0;
            if (!CRAC) {
                if (c < n_loc) slot = base + map[t * n_loc + c];
            } else {
                const uint32_t m = ca.run_mask[e * ca.mask_words + (c0 >> 5)];
                const uint32_t le = m & (0xffffffffu >> (31 - lane));
                const int k = before + __popc(le) - 1;
                const int start = le ? c0 + 31 - __clz(le) : last_start;
                if (c < n_loc) slot = base + (int64_t)mapc[rp * n_loc + (int64_t)r * nr + k] + (c - start);
                before += __popc(m);
                if (m) last_start = c0 + 31 - __clz(m);
            }
            if (c < n_loc) atomicAdd(values + slot, __ldcs(K + t * n_loc + c));
        }
    }
}

// ------------------------------------------------------ deterministic ---
// One warp per row; accumulators for the row's values in shared memory.
// Incidences are taken U at a time: their K rows and slots are loaded first,
// then added strictly in ascending order.
template <int NLOC, typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_gather_small(const double *__restrict__ K, int64_t n_dofs,
                                                      const int64_t *__restrict__ adj_ptr,
                                                      const uint32_t *__restrict__ adj,
                                                      const int64_t *__restrict__ row_ptr,
                                                      const MT *__restrict__ map, CracArgs ca,
                                                      const MT *__restrict__ mapc, int cap, int accumulate,
                                                      double *values)
{
    constexpr int U = 8;
    extern __shared__ double acc_all[];
    const int lane = threadIdx.x & 31;
    double *acc = acc_all + (size_t)(threadIdx.x >> 5) * cap;
    int kc = 0, offc = 0;
    if (CRAC && ca.uniform_R && lane < NLOC) run_of(ca.run_mask[0], lane, kc, offc);
    for (int64_t i = warp_id_global(); i < n_dofs; i += warps_total()) {
        int64_t rb, len;
        if (!CRAC) {
            rb = row_ptr[i];
            len = row_ptr[i + 1] - rb;
        } else {
            rb = crac_row_base(ca, i);
            len = ca.col_align[ca.crac_ptr[i + 1] + 1] - rb;
        }
        for (int k = lane; k < len; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        __syncwarp();
        const int64_t a = adj_ptr[i], b = adj_ptr[i + 1];
        for (int64_t s0 = a; s0 < b; s0 += U) {
            double kv[U];
            int slot[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                kv[u] = 0.0;
                slot[u] = 0;
                if (s0 + u < b && lane < NLOC) {
                    const uint32_t t = adj[s0 + u];
                    kv[u] = __ldcs(K + (int64_t)t * NLOC + lane);
                    if (!CRAC) {
                        slot[u] = (int)map[(int64_t)t * NLOC + lane];
                    } else {
                        const uint32_t e = t / NLOC;
                        const int r = (int)(t - e * NLOC);
                        int k = kc, off = offc, nr;
                        int64_t rp;
                        if (ca.uniform_R) {
                            nr = ca.uniform_R;
                            rp = (int64_t)e * nr;
                        } else {
                            run_of(ca.run_mask[e], lane, k, off);
                            rp = ca.run_ptr[e];
                            nr = (int)(ca.run_ptr[e + 1] - rp);
                        }
                        slot[u] = (int)mapc[rp * NLOC + r * nr + k] + off;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (s0 + u < b && lane < NLOC) acc[slot[u]] += kv[u];
                __syncwarp();
            }
        }
        for (int k = lane; k < len; k += 32) values[rb + k] = acc[k];
        __syncwarp();
    }
}

template <typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_gather_generic(const double *__restrict__ K, int64_t n_dofs, int32_t n_loc,
                                                        const int64_t *__restrict__ adj_ptr,
                                                        const uint32_t *__restrict__ adj,
                                                        const int64_t *__restrict__ row_ptr,
                                                        const MT *__restrict__ map, CracArgs ca,
                                                        const MT *__restrict__ mapc, int cap, int accumulate,
                                                        double *values)
{
    extern __shared__ double acc_all[];
    const int lane = threadIdx.x & 31;
    double *acc = acc_all + (size_t)(threadIdx.x >> 5) * cap;
    for (int64_t i = warp_id_global(); i < n_dofs; i += warps_total()) {
        int64_t rb, len;
        if (!CRAC) {
            rb = row_ptr[i];
            len = row_ptr[i + 1] - rb;
        } else {
            rb = crac_row_base(ca, i);
            len = ca.col_align[ca.crac_ptr[i + 1] + 1] - rb;
        }
        for (int k = lane; k < len; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        __syncwarp();
        for (int64_t s = adj_ptr[i]; s < adj_ptr[i + 1]; ++s) {
            const uint32_t t = adj[s];
            const int64_t e = (int64_t)(t / (uint32_t)n_loc);
            const int r = (int)(t - (uint32_t)e * (uint32_t)n_loc);
            int64_t rp = 0;
            int nr = 0;
            if (CRAC) {
                rp = ca.run_ptr[e];
                nr = (int)(ca.run_ptr[e + 1] - rp);
            }
            int before = 0, last_start = 0;
            for (int c0 = 0; c0 < n_loc; c0 += 32) {
                const int c = c0 + lane;
                int sl = 0;
                if (!CRAC) {
                    if (c < n_loc) sl = (int)map[(int64_t)t * n_loc + c];
                } else {
                    const uint32_t m = ca.run_mask[e * ca.mask_words + (c0 >> 5)];
                    const uint32_t le = m & (0xffffffffu >> (31 - lane));
                    const int k = before + __popc(le) - 1;
                    const int start = le ? c0 + 31 - __clz(le) : last_start;
                    if (c < n_loc) sl = (int)mapc[rp * n_loc + (int64_t)r * nr + k] + (c - start);
                    before += __popc(m);
                    if (m) last_start = c0 + 31 - __clz(m);
                }
                if (c < n_loc) acc[sl] += K[(int64_t)t * n_loc + c];
            }
            __syncwarp();
        }
        for (int k = lane; k < len; k += 32) values[rb + k] = acc[k];
        __syncwarp();
    }
}

template <typename KernelT>
int configure_smem(KernelT kernel, size_t bytes)
{
    if (bytes > 48 * 1024) FE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return FE_OK;
}

template <int NLOC, typename MT, bool CRAC>
int launch_atomic(const fe_pattern *p, const double *K, double *values, cudaStream_t s)
{
    const CracArgs ca{p->crac_ptr, p->col_align, p->run_mask, p->run_ptr, p->uniform_runs ? p->runs_per_elem : 0,
                      p->mask_words};
    const int sms = p->ctx->num_sms;
    if constexpr (NLOC > 0) {
        k_atomic_small<NLOC, MT, CRAC><<<fe_grid_for(p->n_e * 32, 256, sms, 8), 256, 0, s>>>(
            K, p->elem_dofs, p->n_e, p->row_ptr, (const MT *)p->map_csr, ca, (const MT *)p->map_crac, values); fe_note_launch();
    } else {
        const int64_t n_inc = p->n_e * p->n_loc;
        k_atomic_generic<MT, CRAC><<<fe_grid_for(n_inc * 32, 256, sms, 8), 256, 0, s>>>(
            K, p->elem_dofs, n_inc, p->n_loc, p->row_ptr, (const MT *)p->map_csr, ca, (const MT *)p->map_crac,
            values); fe_note_launch();
    }
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

template <int NLOC, typename MT, bool CRAC>
int launch_gather(const fe_pattern *p, const double *K, double *values, int accumulate, cudaStream_t s)
{
    const CracArgs ca{p->crac_ptr, p->col_align, p->run_mask, p->run_ptr, p->uniform_runs ? p->runs_per_elem : 0,
                      p->mask_words};
    const int sms = p->ctx->num_sms;
    const int cap = std::max(1, p->max_row_len);
    int W = 8;
    while (W > 1 && (size_t)W * cap * 8 > 64 * 1024) W >>= 1;
    const size_t smem = (size_t)W * cap * 8;
    if (smem > 200 * 1024) return FE_ERR_UNSUPPORTED;
    const int grid = fe_grid_for(p->n_dofs * 32, W * 32, sms, std::max(1, 64 / W));
    if constexpr (NLOC > 0) {
        FE_TRY(configure_smem(k_gather_small<NLOC, MT, CRAC>, smem));
        k_gather_small<NLOC, MT, CRAC><<<grid, W * 32, smem, s>>>(K, p->n_dofs, p->adj_ptr, p->adj, p->row_ptr,
                                                                  (const MT *)p->map_csr, ca,
                                                                  (const MT *)p->map_crac, cap, accumulate, values); fe_note_launch();
    } else {
        FE_TRY(configure_smem(k_gather_generic<MT, CRAC>, smem));
        k_gather_generic<MT, CRAC><<<grid, W * 32, smem, s>>>(K, p->n_dofs, p->n_loc, p->adj_ptr, p->adj,
                                                              p->row_ptr, (const MT *)p->map_csr, ca,
                                                              (const MT *)p->map_crac, cap, accumulate, values); fe_note_launch();
    }
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

template <typename MT, bool CRAC>
int dispatch(const fe_pattern *p, const double *K, double *values, int mode, int accumulate, cudaStream_t s)
{
    if (mode == FE_ATOMIC) {
        if (!accumulate) FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)p->nnz, s));
        if (p->n_e == 0) return FE_OK;
        // the specialised element kernels read one 32-bit run mask per element
        switch (p->n_loc) {
        case 4: return launch_atomic<4, MT, CRAC>(p, K, values, s);
        case 8: return launch_atomic<8, MT, CRAC>(p, K, values, s);
        case 24: return launch_atomic<24, MT, CRAC>(p, K, values, s);
        case 30: return launch_atomic<30, MT, CRAC>(p, K, values, s);
        default: return launch_atomic<0, MT, CRAC>(p, K, values, s);
        }
    }
    if (p->n_dofs == 0) return FE_OK;
    switch (p->n_loc) {
    case 4: return launch_gather<4, MT, CRAC>(p, K, values, accumulate, s);
    case 8: return launch_gather<8, MT, CRAC>(p, K, values, accumulate, s);
    case 24: return launch_gather<24, MT, CRAC>(p, K, values, accumulate, s);
    case 30: return launch_gather<30, MT, CRAC>(p, K, values, accumulate, s);
    default: return launch_gather<0, MT, CRAC>(p, K, values, accumulate, s);
    }
}

int assemble(fe_ctx *ctx, const fe_pattern *p, const double *K, double *values, int mode, int accumulate,
             void *stream, bool crac)
{
    if (!ctx || !p || p->ctx != ctx) return FE_ERR_INVALID_ARG;
    if (mode != FE_ATOMIC && mode != FE_DETERMINISTIC) return FE_ERR_INVALID_ARG;
    if (accumulate != 0 && accumulate != 1) return FE_ERR_INVALID_ARG;
    if ((p->n_e > 0 && !K) || (p->nnz > 0 && !values)) return FE_ERR_INVALID_ARG;
    if (((uintptr_t)K & 7u) || ((uintptr_t)values & 7u)) return FE_ERR_INVALID_ARG;
    if (!crac && !p->map_csr) return FE_ERR_NOT_BUILT;
    if (crac && (!p->map_crac || !p->col_align)) return FE_ERR_NOT_BUILT;
    if (mode == FE_DETERMINISTIC && !p->adj) return FE_ERR_NOT_BUILT;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (p->map_bytes == 1)
        rc = crac ? dispatch<uint8_t, true>(p, K, values, mode, accumulate, s)
                  : dispatch<uint8_t, false>(p, K, values, mode, accumulate, s);
    else
        rc = crac ? dispatch<uint16_t, true>(p, K, values, mode, accumulate, s)
                  : dispatch<uint16_t, false>(p, K, values, mode, accumulate, s);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

}  // namespace

extern "C" {

int fe_assemble_csr(fe_ctx *ctx, const fe_pattern *p, const double *elem_mats, double *values, int mode,
                    int accumulate, void *stream)
{
    return assemble(ctx, p, elem_mats, values, mode, accumulate, stream, false);
}

int fe_assemble_crac(fe_ctx *ctx, const fe_pattern *p, const double *elem_mats, double *values, int mode,
                     int accumulate, void *stream)
{
    return assemble(ctx, p, elem_mats, values, mode, accumulate, stream, true);
}

}  // extern "C"

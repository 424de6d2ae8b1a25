// Device-side pieces shared by the single-mesh kernels (numeric.cu) and the
// batched persistent kernel (batch.cu): pattern geometry, run decoding, and
// the per-element / per-node-row assembly bodies.
#pragma once

#include "internal.cuh"

namespace fe_dev {

struct Geo {
    const int32_t *N;        // block ids per element
    const int64_t *row_ptr;  // CSR
    const int64_t *crac_ptr; // CRAC
    const int32_t *col_align;
    const uint32_t *run_mask;
    const int64_t *run_ptr;
    const int64_t *adj_ptr;
    const uint32_t *adj;
    int uniform_R;  // > 0 when every element has this many runs and the same mask
    int mask_words;
    int64_t nnz;    // values length (index checks of debug builds)
    int *status;    // the context's device status word
    // row starts of the block-map kernels: 0 from row_ptr (CSR), 1 from the
    // value position of each row's first CRAC pair (the CRAC gather)
    int crac_rows = 0;
    // FE_ATOMIC: elements in this order (a locality order), or ascending
    const int32_t *order = nullptr;
};

// Element at position i of the atomic scatter's order.
__device__ __forceinline__ int64_t elem_at(const Geo &g, int64_t i) { return g.order ? (int64_t)g.order[i] : i; }

__device__ __forceinline__ int64_t crac_row_base(const Geo &g, int64_t i) { return g.col_align[g.crac_ptr[i] + 1]; }

// Start of row i in the values array, from the format the kernel was given.
__device__ __forceinline__ int64_t row_start(const Geo &g, int64_t i)
{
    return g.crac_rows ? crac_row_base(g, i) : g.row_ptr[i];
}

// Run index of block kc and kc's offset inside that run, for run-start bits m
// (kc < 32, bit 0 always set).
__device__ __forceinline__ void run_of(uint32_t m, int kc, int &k, int &off)
{
    const uint32_t le = m & (0xffffffffu >> (31 - kc));
    k = __popc(le) - 1;
    off = kc - (31 - __clz(le));
}

// The same for any number of 32-bit mask words.
__device__ __forceinline__ void run_of_multi(const uint32_t *m, int kc, int &k, int &off)
{
    int before = 0, last = 0;
    const int w_end = kc >> 5;
    for (int w = 0; w < w_end; ++w) {
        before += __popc(m[w]);
        if (m[w]) last = 32 * w + 31 - __clz(m[w]);
    }
    const uint32_t le = m[w_end] & (0xffffffffu >> (31 - (kc & 31)));
    k = before + __popc(le) - 1;
    const int start = le ? 32 * w_end + 31 - __clz(le) : last;
    off = kc - start;
}


inline Geo geo_of(const fe_pattern *p)
{
    return Geo{p->node_dofs, p->row_ptr,  p->crac_ptr, p->col_align, p->run_mask,
               p->run_ptr,   p->adj_ptr, p->adj,      p->uniform_runs ? p->runs_per_elem : 0, p->mask_words,
               p->nnz,       p->ctx->d_status, p->crac_rows ? 1 : 0, p->elem_order};
}

// One element of NLN blocks of BB DOFs (NLN*BB <= 32), the warp cooperating:
// every entry of K_e is added into its slot with one FP64 atomic add, or with
// a plain read-modify-write when PLAIN (no other element touching the same
// slots runs concurrently, as within one colour).
template <int NLN, int BB, typename MT, bool CRAC, bool PLAIN = false>
__device__ __forceinline__ void atomic_element(const double *__restrict__ K, int64_t e, const Geo &g,
                                               const MT *__restrict__ map, const MT *__restrict__ mapc,
                                               double *values, int lane)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int IT = (NN + 31) / 32;
    constexpr int CH = 6;
    int kk = 0, koff = 0;
    const int32_t nd = lane < NLN ? g.N[e * NLN + lane] : 0;
    const int32_t rnode = __shfl_sync(0xffffffffu, nd, lane < NLOC ? lane / BB : 0);
    int64_t base = 0;
    if (lane < NLOC) {
        const int64_t row = (int64_t)BB * rnode + lane % BB;
        base = CRAC ? crac_row_base(g, row) : g.row_ptr[row];
    }
    int64_t rp = 0;
    int nr = 0;
    if (CRAC) {
        if (g.uniform_R) {
            nr = g.uniform_R;
            rp = e * nr;
            if (lane < NLN) run_of(g.run_mask[0], lane, kk, koff);
        } else {
            rp = g.run_ptr[e];
            nr = (int)(g.run_ptr[e + 1] - rp);
            if (lane < NLN) run_of(g.run_mask[e], lane, kk, koff);
        }
    }
    const double *Ke = K + e * NN;
#pragma unroll
    for (int j0 = 0; j0 < IT; j0 += CH) {
        double kv[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int q = lane + 32 * (j0 + u);
            kv[u] = (j0 + u < IT && q < NN) ? __ldcs(Ke + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            if (j0 + u < IT) {
                const int q = lane + 32 * (j0 + u);
                const int qq = q < NN ? q : 0;
                const int r = qq / NLOC, c = qq % NLOC;
                const int kc = c / BB;
                const int64_t b = __shfl_sync(0xffffffffu, base, r);
                int pos;
                if (!CRAC) {
                    pos = (int)map[(e * NLN + r / BB) * NLN + kc];
                } else {
                    const int k = __shfl_sync(0xffffffffu, kk, kc);
                    const int off = __shfl_sync(0xffffffffu, koff, kc);
                    pos = (int)mapc[rp * NLN + (r / BB) * nr + k] + off;
                }
                if (q < NN && FE_IN_BOUNDS(b + (int64_t)BB * pos + c % BB, g.nnz, g.status)) {
                    double *dst = values + b + (int64_t)BB * pos + c % BB;
                    if (PLAIN) *dst = *dst + kv[u];
                    else fe_red_add_f64(dst, kv[u]);
                }
            }
        }
    }
}

// Any element size, the warp cooperating; base_s / k_s / off_s are this
// warp's shared tables of at least n_loc and nln entries.
template <typename MT, bool CRAC, bool PLAIN = false>
__device__ __forceinline__ void atomic_element_generic(const double *__restrict__ K, int64_t e, int32_t nln,
                                                       int32_t B, const Geo &g, const MT *__restrict__ map,
                                                       const MT *__restrict__ mapc, double *values, int64_t *base_s,
                                                       int32_t *k_s, int32_t *off_s, int lane)
{
    const int n_loc = nln * B;
    const int64_t NN = (int64_t)n_loc * n_loc;
    int64_t rp = 0;
    int nr = 0;
    if (CRAC) {
        rp = g.run_ptr[e];
        nr = (int)(g.run_ptr[e + 1] - rp);
    }
    for (int r = lane; r < n_loc; r += 32) {
        const int64_t row = (int64_t)B * g.N[e * nln + r / B] + r % B;
        base_s[r] = CRAC ? crac_row_base(g, row) : g.row_ptr[row];
    }
    if (CRAC)
        for (int kc = lane; kc < nln; kc += 32) run_of_multi(g.run_mask + e * g.mask_words, kc, k_s[kc], off_s[kc]);
    __syncwarp();
    const double *Ke = K + e * NN;
    for (int q = lane; q < NN; q += 32) {
        const int r = q / n_loc, c = q - r * n_loc;
        const int kc = c / B;
        int pos;
        if (!CRAC) pos = (int)map[(e * nln + r / B) * nln + kc];
        else pos = (int)mapc[rp * nln + (int64_t)(r / B) * nr + k_s[kc]] + off_s[kc];
        if (!FE_IN_BOUNDS(base_s[r] + (int64_t)B * pos + c % B, g.nnz, g.status)) continue;
        double *dst = values + base_s[r] + (int64_t)B * pos + c % B;
        if (PLAIN) *dst = *dst + __ldcs(Ke + q);
        else fe_red_add_f64(dst, __ldcs(Ke + q));
    }
    __syncwarp();
}

// Node rows v0, v0 + dv, ... < v_end of one mesh (the warp cooperating;
// acc: the warp's accumulator, cap doubles).  One warp per block row; the B
// rows of the node are contiguous in values.  Incidences are taken U at a
// time: their K slices and slots are loaded first, then added strictly in
// ascending element order (bit-identical to the sequential sum).  The slot
// of an entry is row start + B * pos + column % B, pos read from the block
// map (the CSR map, or for the CRAC gather the CRAC run map expanded per
// column block); row starts come from row_ptr or from the CRAC pairs
// (row_start).  Rows of 3+ DOF blocks load the next row's start and
// adjacency range one row ahead (no dependent load at the head of a row:
// this also hides the CRAC pair read behind the pointer read).  Used by the
// single-mesh gather (rows strided over all warps) and by the batched kernel
// (a tile of consecutive rows).
template <int NLN, int BB, typename MT, int U>
__device__ __forceinline__ void gather_node_rows(const double *__restrict__ K, const Geo &g,
                                                 const MT *__restrict__ map, double *acc, int cap, int accumulate,
                                                 double *values, int64_t v0, int64_t v_end, int64_t dv, int lane)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = BB * NLOC;  // doubles of one incidence (B contiguous K rows)
    constexpr int IT = (CHK + 31) / 32;
    static_assert(NLN >= 1, "specialised shapes only");
    // per-entry constants: block row jr, column c
    int jr_[IT], c_[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int q = lane + 32 * j;
        const int qq = q < CHK ? q : 0;
        jr_[j] = qq / NLOC;
        c_[j] = qq % NLOC;
    }
    constexpr bool PF = BB >= 3;
    const int64_t W = dv;
    int64_t p0 = 0, p1 = 0, q0 = 0, q1 = 0;
    if (PF) {
        const int64_t v = v0;
        if (v < v_end) {
            p0 = row_start(g, (int64_t)BB * v);
            p1 = row_start(g, (int64_t)BB * v + 1);
            q0 = g.adj_ptr[v];
            q1 = g.adj_ptr[v + 1];
        }
    }
    for (int64_t v = v0; v < v_end; v += W) {
        int64_t rb, RL, a, b;
        if constexpr (PF) {
            rb = p0;
            RL = p1 - p0;
            a = q0;
            b = q1;
            if (v + W < v_end) {
                p0 = row_start(g, (int64_t)BB * (v + W));
                p1 = row_start(g, (int64_t)BB * (v + W) + 1);
                q0 = g.adj_ptr[v + W];
                q1 = g.adj_ptr[v + W + 1];
            }
        } else {
            const int64_t i0 = (int64_t)BB * v;
            rb = row_start(g, i0);
            RL = row_start(g, i0 + 1) - rb;
            a = g.adj_ptr[v];
            b = g.adj_ptr[v + 1];
        }
        const int total = (int)(BB * RL);
        if (total > 0 && (!FE_IN_BOUNDS(rb + total - 1, g.nnz, g.status) || !FE_IN_BOUNDS(total - 1, cap, g.status)))
            continue;
        for (int k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        __syncwarp();
        for (int64_t s0 = a; s0 < b; s0 += U) {
            double kv[U][IT];
            int rel[U][IT];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool have = s0 + u < b;
                const uint32_t t = have ? g.adj[s0 + u] : 0u;
                const uint32_t e = t / NLN;
                const int kr = (int)(t - e * NLN);
                const double *chunk = K + (int64_t)e * NN + (int64_t)kr * CHK;
#pragma unroll
                for (int j = 0; j < IT; ++j) {
                    const int q = lane + 32 * j;
                    kv[u][j] = 0.0;
                    rel[u][j] = 0;
                    if (have && q < CHK) {
                        kv[u][j] = __ldcs(chunk + q);
                        const int pos = (int)map[(int64_t)t * NLN + c_[j] / BB];
                        rel[u][j] = jr_[j] * (int)RL + BB * pos + c_[j] % BB;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int j = 0; j < IT; ++j)
                    if (s0 + u < b && lane + 32 * j < CHK && FE_IN_BOUNDS(rel[u][j], total, g.status))
                        acc[rel[u][j]] += kv[u][j];
                __syncwarp();
            }
        }
        for (int k = lane; k < total; k += 32) values[rb + k] = acc[k];
        __syncwarp();
    }
}

template <typename MT, bool CRAC>
__device__ __forceinline__ void gather_row_generic(const double *__restrict__ K, int64_t v, int32_t nln, int32_t B,
                                                   const Geo &g, const MT *__restrict__ map,
                                                   const MT *__restrict__ mapc, double *acc, int accumulate,
                                                   double *values, int lane)
{
    const int n_loc = nln * B;
    const int64_t NN = (int64_t)n_loc * n_loc;
    const int chk = B * n_loc;
    const int64_t i0 = (int64_t)B * v;
    int64_t rb, RL;
    if (!CRAC) {
        rb = g.row_ptr[i0];
        RL = g.row_ptr[i0 + 1] - rb;
    } else {
        rb = crac_row_base(g, i0);
        RL = crac_row_base(g, i0 + 1) - rb;
    }
    const int64_t total = B * RL;
    if (total > 0 && !FE_IN_BOUNDS(rb + total - 1, g.nnz, g.status)) return;
    for (int64_t k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
    __syncwarp();
    for (int64_t s = g.adj_ptr[v]; s < g.adj_ptr[v + 1]; ++s) {
        const uint32_t t = g.adj[s];
        const int64_t e = t / (uint32_t)nln;
        const int kr = (int)(t - (uint32_t)e * (uint32_t)nln);
        const double *chunk = K + e * NN + (int64_t)kr * chk;
        int64_t rp = 0;
        int nr = 0;
        if (CRAC) {
            rp = g.run_ptr[e];
            nr = (int)(g.run_ptr[e + 1] - rp);
        }
        for (int q = lane; q < chk; q += 32) {
            const int jr = q / n_loc, c = q - jr * n_loc;
            const int kc = c / B;
            int pos;
            if (!CRAC) {
                pos = (int)map[(int64_t)t * nln + kc];
            } else {
                int k, off;
                run_of_multi(g.run_mask + e * g.mask_words, kc, k, off);
                pos = (int)mapc[rp * nln + (int64_t)kr * nr + k] + off;
            }
            if (FE_IN_BOUNDS(jr * RL + (int64_t)B * pos + c % B, total, g.status))
                acc[jr * RL + (int64_t)B * pos + c % B] += chunk[q];
        }
        __syncwarp();
    }
    for (int64_t k = lane; k < total; k += 32) values[rb + k] = acc[k];
    __syncwarp();
}

}  // namespace fe_dev

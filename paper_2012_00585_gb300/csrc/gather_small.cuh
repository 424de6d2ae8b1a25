// Deterministic row gather for one-DOF elements with at most 16 local nodes
// (B = 1: 2-D and 3-D scalar problems).  A node row then holds one K row of
// NLN entries per incidence, too few for a warp: G = 4, 8 or 16 lanes take
// one row (lane c of the group handles column c), 32 / G rows share a warp,
// each with its own accumulator.  Within a row the incidences are added in
// ascending element order, U at a time loaded first (bit-identical to the
// sequential sum); rows never share an accumulator slot, so the groups add in
// the same instructions.
#pragma once

#include "assemble_body.cuh"

namespace fe_dev {

template <int NLN>
struct SmallRows {
    static constexpr int G = NLN <= 4 ? 4 : (NLN <= 8 ? 8 : 16);  // lanes per row
    static constexpr int RPW = 32 / G;                             // rows per warp
};

// Rows v0 + r * vstep (r = 0 .. RPW-1, those below vend) of one warp;
// acc_warp holds RPW accumulators of cap doubles.
template <int NLN, typename MT, bool CRAC, int U>
__device__ __forceinline__ void gather_rows_small(const double *__restrict__ K, int64_t v0, int64_t vstep,
                                                  int64_t vend, const Geo &g, const MT *__restrict__ map,
                                                  const MT *__restrict__ mapc, double *acc_warp, int cap,
                                                  int accumulate, double *values, int lane)
{
    constexpr int G = SmallRows<NLN>::G;
    constexpr int NN = NLN * NLN;
    const int grp = lane / G, c = lane % G;
    const bool col = c < NLN;
    const int64_t v = v0 + grp * vstep;
    double *acc = acc_warp + (size_t)grp * cap;
    bool row_ok = v < vend;
    int64_t rb = 0, RL = 0, a = 0, b = 0;
    if (row_ok) {
        if (!CRAC) {
            rb = g.row_ptr[v];
            RL = g.row_ptr[v + 1] - rb;
        } else {
            rb = crac_row_base(g, v);
            RL = crac_row_base(g, v + 1) - rb;
        }
        a = g.adj_ptr[v];
        b = g.adj_ptr[v + 1];
        if (RL > 0 && (!FE_IN_BOUNDS(rb + RL - 1, g.nnz, g.status) || !FE_IN_BOUNDS(RL - 1, cap, g.status)))
            row_ok = false;
    }
    if (!row_ok) RL = 0;
    int ku = 0, offu = 0;  // uniform runs: run index / offset of column block c
    if (CRAC && g.uniform_R && col) run_of(g.run_mask[0], c, ku, offu);
    for (int64_t k = c; k < RL; k += G) acc[k] = accumulate ? values[rb + k] : 0.0;
    __syncwarp();
    // the warp's longest row sets the trip count
    int deg = row_ok ? (int)(b - a) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) deg = max(deg, __shfl_xor_sync(0xffffffffu, deg, o));
    const int my_deg = row_ok ? (int)(b - a) : 0;
    for (int s0 = 0; s0 < deg; s0 += U) {
        double kv[U];
        int rel[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            kv[u] = 0.0;
            rel[u] = 0;
            if (col && s0 + u < my_deg) {
                const uint32_t t = g.adj[a + s0 + u];
                const uint32_t e = t / NLN;
                const int kr = (int)(t - e * NLN);
                kv[u] = __ldcs(K + (int64_t)e * NN + (int64_t)kr * NLN + c);
                if (!CRAC) {
                    rel[u] = (int)map[(int64_t)t * NLN + c];
                } else {
                    int64_t rp;
                    int nr;
                    int k = ku, off = offu;
                    if (g.uniform_R) {
                        nr = g.uniform_R;
                        rp = (int64_t)e * nr;
                    } else {
                        rp = g.run_ptr[e];
                        nr = (int)(g.run_ptr[e + 1] - rp);
                        run_of(g.run_mask[e], c, k, off);
                    }
                    rel[u] = (int)mapc[rp * NLN + (int64_t)kr * nr + k] + off;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (col && s0 + u < my_deg && FE_IN_BOUNDS(rel[u], RL, g.status)) acc[rel[u]] += kv[u];
            __syncwarp();
        }
    }
    for (int64_t k = c; k < RL; k += G) values[rb + k] = acc[k];
    __syncwarp();
}

}  // namespace fe_dev

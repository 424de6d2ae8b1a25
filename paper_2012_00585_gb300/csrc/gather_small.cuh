// Deterministic row gather for node rows whose incidence slice (B rows of
// B*NLN entries) holds at most 16 entries: one-DOF elements of up to 16 nodes
// (2-D and 3-D scalar problems) and 4-node elements with 2 DOFs per node (2-D
// elasticity).  Such a slice is too small for a warp: G = 4, 8 or 16 lanes
// take one node row (lane c of the group handles entry c of the slice),
// 32 / G rows share a warp, each with its own accumulator.  Within a row the
// incidences are added in ascending element order, U at a time loaded first
// (bit-identical to the sequential sum); rows never share an accumulator
// slot, so the groups add in the same instructions.
#pragma once

#include "assemble_body.cuh"

namespace fe_dev {

template <int NLN, int BB = 1>
struct SmallRows {
    static constexpr int CHK = BB * NLN * BB;  // entries of one incidence slice
    static_assert(NLN >= 1 && BB >= 1 && CHK <= 16, "one lane per slice entry, 16 lanes at most");
    static constexpr int G = CHK <= 4 ? 4 : (CHK <= 8 ? 8 : 16);  // lanes per row
    static constexpr int RPW = 32 / G;                             // rows per warp
};

// Node rows v0 + r * vstep (r = 0 .. RPW-1, those below vend) of one warp;
// acc_warp holds RPW accumulators of cap doubles (the node's B DOF rows).
template <int NLN, typename MT, bool CRAC, int U, int BB = 1>
__device__ __forceinline__ void gather_rows_small(const double *__restrict__ K, int64_t v0, int64_t vstep,
                                                  int64_t vend, const Geo &g, const MT *__restrict__ map,
                                                  const MT *__restrict__ mapc, double *acc_warp, int cap,
                                                  int accumulate, double *values, int lane)
{
    constexpr int G = SmallRows<NLN, BB>::G;
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = SmallRows<NLN, BB>::CHK;
    const int grp = lane / G, c = lane % G;
    const bool col = c < CHK;
    // slice entry c: DOF row jr of the node, column cc = BB * kc + cb of the element
    const int cq = col ? c : 0;
    const int jr = cq / NLOC, cc = cq % NLOC;
    const int kc = cc / BB, cb = cc % BB;
    const int64_t v = v0 + grp * vstep;
    double *acc = acc_warp + (size_t)grp * cap;
    bool row_ok = v < vend;
    int64_t rb = 0, RL = 0, a = 0, b = 0;
    if (row_ok) {
        if (!CRAC) {
            rb = row_start(g, BB * v);
            RL = row_start(g, BB * v + 1) - rb;
        } else {
            rb = crac_row_base(g, BB * v);
            RL = crac_row_base(g, BB * v + 1) - rb;
        }
        a = g.adj_ptr[v];
        b = g.adj_ptr[v + 1];
        if (RL > 0 &&
            (!FE_IN_BOUNDS(rb + BB * RL - 1, g.nnz, g.status) || !FE_IN_BOUNDS(BB * RL - 1, cap, g.status)))
            row_ok = false;
    }
    if (!row_ok) RL = 0;
    const int64_t total = BB * RL;  // the node's B rows are contiguous in values
    int ku = 0, offu = 0;           // uniform runs: run index / offset of column block kc
    if (CRAC && g.uniform_R && col) run_of(g.run_mask[0], kc, ku, offu);
    for (int64_t k = c; k < total; k += G) acc[k] = accumulate ? values[rb + k] : 0.0;
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
                kv[u] = __ldcs(K + (int64_t)e * NN + (int64_t)kr * CHK + c);
                if (!CRAC) {
                    rel[u] = (int)(jr * RL) + BB * (int)map[(int64_t)t * NLN + kc] + cb;
                } else {
                    int64_t mb;  // the incidence's row of the run map
                    int k = ku, off = offu;
                    if (g.uniform_R) {
                        mb = (int64_t)t * g.uniform_R;  // e R NLN + kr R
                    } else {
                        const int64_t rp = g.run_ptr[e];
                        mb = rp * NLN + (int64_t)kr * (g.run_ptr[e + 1] - rp);
                        run_of(g.run_mask[e], kc, k, off);
                    }
                    rel[u] = (int)(jr * RL) + BB * ((int)mapc[mb + k] + off) + cb;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (col && s0 + u < my_deg && FE_IN_BOUNDS(rel[u], total, g.status)) acc[rel[u]] += kv[u];
            __syncwarp();
        }
    }
    for (int64_t k = c; k < total; k += G) values[rb + k] = acc[k];
    __syncwarp();
}

}  // namespace fe_dev

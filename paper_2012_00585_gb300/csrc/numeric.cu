// Numeric phase: scatter-add every element-matrix entry into its global slot.
//
//   FE_ATOMIC         element-parallel, FP64 atomic add into the values array
//                     (the atomic parallel assembly of Listing 3); one warp per
//                     element streams K_e with coalesced loads.
//   FE_DETERMINISTIC  row-parallel gather: one warp per block row (the B rows
//                     of one node) walks the node's (element, local node)
//                     incidences in ascending element order and adds the B
//                     contiguous rows K_e(B*k .. B*k+B-1, :) into accumulators
//                     in shared memory, then writes the rows once.  Each value
//                     is summed in exactly the order of Listing 2, so the
//                     result is bit-identical to the sequential assembly.
//
// The slot of entry (e, r, c) is row_start(D_e(r)) + B*pos + c%B, where pos
// is the position of column block c/B in the row's block list.  CSR kernels
// read pos from a per (element, row block, column block) map and the row
// start from row_ptr.  CRAC kernels use the runs of consecutive blocks of
// each element (the compressed DOF array of §2.1): one map entry per
// (element, row block, run), the column's offset inside its run, and the
// row start read from the CRAC pairs (Listing 5's contiguous slices).
//
// Kernels (defaults first; the others are schedule knobs, every one
// parity-tested): atomic -- k_atomic_tma (K_e staged by a bulk copy),
// k_atomic_elem, k_atomic_generic; deterministic -- k_gather_node (3-DOF
// and other specialised shapes), k_gather_small (slices of at most 16
// entries, several rows per warp), k_gather_generic (any shape), and the
// variants k_gather_async, k_gather_pipe, k_gather_bulk, k_gather_pair.
// FE_COLOURED and FE_ROWLOCK are in colour.cu and rowlock.cu.
#include "assemble_body.cuh"
#include "internal.cuh"
#include "tma.cuh"
#include "gather_small.cuh"

namespace {

using namespace fe_dev;

// ------------------------------------------------------------ atomic ---
// One warp per element; NLN blocks of BB DOFs, NLN*BB <= 32.
template <int NLN, int BB, typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_atomic_elem(const double *__restrict__ K, int64_t n_e, Geo g,
                                                     const MT *__restrict__ map, const MT *__restrict__ mapc,
                                                     double *values)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int IT = (NN + 31) / 32;
    constexpr int CH = 6;  // loads in flight per lane before their atomics
    const int lane = threadIdx.x & 31;
    int kk = 0, koff = 0;
    if (CRAC && g.uniform_R && lane < NLN) run_of(g.run_mask[0], lane, kk, koff);
    for (int64_t e = fe_warp_id(); e < n_e; e += fe_warps()) {
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
                    if (q < NN) atomicAdd(values + b + (int64_t)BB * pos + c % BB, kv[u]);
                }
            }
        }
    }
}

// Any element size: one warp per element, per-row starts staged in shared
// memory.
template <typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_atomic_generic(const double *__restrict__ K, int64_t n_e, int32_t nln,
                                                        int32_t B, Geo g, const MT *__restrict__ map,
                                                        const MT *__restrict__ mapc, double *values)
{
    __shared__ int64_t base_s[8][FE_MAX_NLOC];
    __shared__ int32_t k_s[8][FE_MAX_NLOC];
    __shared__ int32_t off_s[8][FE_MAX_NLOC];
    const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) & 7;
    const int n_loc = nln * B;
    const int64_t NN = (int64_t)n_loc * n_loc;
    for (int64_t e = fe_warp_id(); e < n_e; e += fe_warps()) {
        int64_t rp = 0;
        int nr = 0;
        if (CRAC) {
            rp = g.run_ptr[e];
            nr = (int)(g.run_ptr[e + 1] - rp);
        }
        for (int r = lane; r < n_loc; r += 32) {
            const int64_t row = (int64_t)B * g.N[e * nln + r / B] + r % B;
            base_s[w][r] = CRAC ? crac_row_base(g, row) : g.row_ptr[row];
        }
        if (CRAC)
            for (int kc = lane; kc < nln; kc += 32)
                run_of_multi(g.run_mask + e * g.mask_words, kc, k_s[w][kc], off_s[w][kc]);
        __syncwarp();
        const double *Ke = K + e * NN;
        for (int q = lane; q < NN; q += 32) {
            const int r = q / n_loc, c = q - r * n_loc;
            const int kc = c / B;
            int pos;
            if (!CRAC) pos = (int)map[(e * nln + r / B) * nln + kc];
            else pos = (int)mapc[rp * nln + (int64_t)(r / B) * nr + k_s[w][kc]] + off_s[w][kc];
            atomicAdd(values + base_s[w][r] + (int64_t)B * pos + c % B, __ldcs(Ke + q));
        }
        __syncwarp();
    }
}

// ------------------------------------------------------ deterministic ---
// One warp per block row; the B rows of the node are contiguous in values.
// Incidences are taken U at a time: their K slices and slots are loaded
// first, then added strictly in ascending element order.
//
// Packed slices (CRAC rows, gather_packs): when a slice is not a multiple of
// 32 entries (3 x 24 for trilinear hexes), the U slices are laid end to end
// over the lanes -- slot s = 32 i + lane holds entry s % CHK of incidence
// s / CHK -- so U x 72 entries take ceil(72 U / 32) load, add and store
// instructions instead of 3 U (9 instead of 12 for U = 4).  One instruction
// then holds the tail of one slice and the head of the next; the two never
// meet in an accumulator slot: entries of one slot share their block row, so
// in the concatenation they lie at least CHK - NLOC + 1 >= 32 slots apart,
// i.e. in different instructions, the earlier incidence first.  The per-slot
// order is unchanged and the result bit-identical.  CRAC rows take the packed
// form whenever it needs no more instruction rows than the unpacked one: it
// holds no per-lane slot tables, which the unpacked CRAC instances spilled
// (64^3 elasticity 615 -> 582 us; P2 tets, 90-entry slices, same row count:
// 7.12 -> 6.25 ms at 64^3).  CSR rows stay unpacked: there the extra shuffles
// and index arithmetic cost more than the saved lanes (413 -> 447 us).
template <int NLN, int BB, bool CRAC, int U>
constexpr bool gather_packs()
{
    constexpr int NLOC = NLN * BB, CHK = BB * NLOC;
    return CRAC && NLN > 0 && NLN <= 32 && (BB - 1) * NLOC + 1 >= 32 && (U * CHK + 31) / 32 <= U * ((CHK + 31) / 32) &&
           U <= 32;
}

template <int NLN, int BB, typename MT, bool CRAC, int U>
__global__ void __launch_bounds__(256, (CRAC && BB == 3 && U == 4) ? 4 : 0) k_gather_node(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                     const MT *__restrict__ map, const MT *__restrict__ mapc, int cap,
                                                     int accumulate, double *values)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = BB * NLOC;  // doubles of one incidence (B contiguous K rows)
    constexpr int IT = (CHK + 31) / 32;
    constexpr int ITP = (U * CHK + 31) / 32;  // slot rows of U packed slices
    constexpr bool PACK = gather_packs<NLN, BB, CRAC, U>();
    static_assert(NLN >= 1 && (!PACK || NLN <= 32), "packed slices: one run-mask word per element");
    constexpr int MW = (NLN + 31) / 32;  // run-start mask words per element
    extern __shared__ double acc_all[];
    const int lane = threadIdx.x & 31;
    double *acc = acc_all + (size_t)(threadIdx.x >> 5) * cap;
    // per-entry constants: block row jr, column c
    int jr_[IT], c_[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int q = lane + 32 * j;
        const int qq = q < CHK ? q : 0;
        jr_[j] = qq / NLOC;
        c_[j] = qq % NLOC;
    }
    int ku[IT], offu[IT];  // run index / offset of the column block (uniform runs)
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        ku[j] = 0;
        offu[j] = 0;
        if (CRAC && g.uniform_R) {
            if constexpr (MW == 1) run_of(g.run_mask[0], c_[j] / BB, ku[j], offu[j]);
            else run_of_multi(g.run_mask, c_[j] / BB, ku[j], offu[j]);
        }
    }
    // CSR rows of 3+ DOF blocks: the next row's pointers and adjacency range
    // are loaded one row ahead (one dependent load fewer on each row's path;
    // measured faster there, slower where the registers cost occupancy)
    constexpr bool PF = !CRAC && BB >= 3;
    const int64_t W = fe_warps();
    int64_t p0 = 0, p1 = 0, q0 = 0, q1 = 0;
    if (PF) {
        const int64_t v = fe_warp_id();
        if (v < n_nodes) {
            p0 = g.row_ptr[(int64_t)BB * v];
            p1 = g.row_ptr[(int64_t)BB * v + 1];
            q0 = g.adj_ptr[v];
            q1 = g.adj_ptr[v + 1];
        }
    }
    for (int64_t v = fe_warp_id(); v < n_nodes; v += W) {
        int64_t rb, RL, a, b;
        if constexpr (PF) {
            rb = p0;
            RL = p1 - p0;
            a = q0;
            b = q1;
            if (v + W < n_nodes) {
                p0 = g.row_ptr[(int64_t)BB * (v + W)];
                p1 = g.row_ptr[(int64_t)BB * (v + W) + 1];
                q0 = g.adj_ptr[v + W];
                q1 = g.adj_ptr[v + W + 1];
            }
        } else {
            const int64_t i0 = (int64_t)BB * v;
            if (!CRAC) {
                rb = g.row_ptr[i0];
                RL = g.row_ptr[i0 + 1] - rb;
            } else {
                rb = crac_row_base(g, i0);
                RL = crac_row_base(g, i0 + 1) - rb;
            }
            a = g.adj_ptr[v];
            b = g.adj_ptr[v + 1];
        }
        const int total = (int)(BB * RL);
        if (total > 0 && (!FE_IN_BOUNDS(rb + total - 1, g.nnz, g.status) || !FE_IN_BOUNDS(total - 1, cap, g.status)))
            continue;
        for (int k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        __syncwarp();
        for (int64_t s0 = a; s0 < b; s0 += U) {
            if constexpr (PACK) {
                // lane u < nu holds incidence s0 + u; slot 32 i + lane reads it
                // by shuffle (its slice starts at K + t * CHK: e NN + kr CHK)
                const int nu = (int)(b - s0 < U ? b - s0 : U);
                uint32_t t_l = 0, m_l = 0;
                int64_t mb_l = 0;  // the incidence's row of the run map (non-uniform runs)
                if (lane < nu) {
                    t_l = g.adj[s0 + lane];
                    if (CRAC && !g.uniform_R) {
                        if (g.inc_off) {
                            mb_l = g.inc_off[s0 + lane];
                            m_l = g.inc_mask[s0 + lane];
                        } else {
                            const uint32_t e = t_l / NLN;
                            const int64_t rp = g.run_ptr[e];
                            mb_l = rp * NLN + (int64_t)(t_l - e * NLN) * (g.run_ptr[e + 1] - rp);
                            m_l = g.run_mask[e];
                        }
                    }
                }
                double kv[ITP];
                int rel[ITP];
                // the lane id read afresh each group: the slot constants below are
                // recomputed instead of held in registers across the row loop
                int ln;
                asm volatile("mov.u32 %0, %%laneid;" : "=r"(ln));
#pragma unroll
                for (int i = 0; i < ITP; ++i) {
                    const int lo = (32 * i) / CHK;  // slot row i spans incidences lo and lo + 1
                    const int sl = ln + 32 * i;
                    const int u = lo + (sl >= (lo + 1) * CHK ? 1 : 0);
                    const int q = sl - u * CHK;
                    const uint32_t t = __shfl_sync(0xffffffffu, t_l, u & 31);
                    int64_t mb = 0;
                    uint32_t m = 0;
                    if (CRAC && !g.uniform_R) {
                        mb = __shfl_sync(0xffffffffu, mb_l, u & 31);
                        m = __shfl_sync(0xffffffffu, m_l, u & 31);
                    }
                    kv[i] = 0.0;
                    rel[i] = -1;
                    if (u < nu) {
                        const int jr = q / NLOC, c = q - jr * NLOC;
                        const int kc = c / BB, cb = c - kc * BB;
                        kv[i] = __ldcs(K + (int64_t)t * CHK + q);
                        int pos;
                        if (!CRAC) {
                            pos = (int)map[(int64_t)t * NLN + kc];
                        } else {
                            int k, off;
                            if (g.uniform_R) {
                                mb = (int64_t)t * g.uniform_R;  // e R NLN + kr R
                                run_of(g.run_mask[0], kc, k, off);
                            } else {
                                run_of(m, kc, k, off);
                            }
                            pos = (int)mapc[mb + k] + off;
                        }
                        rel[i] = jr * (int)RL + BB * pos + cb;
                    }
                }
#pragma unroll
                for (int i = 0; i < ITP; ++i) {
                    if (rel[i] >= 0 && FE_IN_BOUNDS(rel[i], total, g.status)) acc[rel[i]] += kv[i];
                    __syncwarp();
                }
            } else {
                double kv[U][IT];
                int rel[U][IT];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool have = s0 + u < b;
                    const uint32_t t = have ? g.adj[s0 + u] : 0u;
                    const uint32_t e = t / NLN;
                    const int kr = (int)(t - e * NLN);
                    const double *chunk = K + (int64_t)e * NN + (int64_t)kr * CHK;
                    int64_t mb = 0;  // this incidence's row of the run map
                    uint32_t m = 0;
                    if (CRAC && have) {
                        if (g.uniform_R) {
                            mb = (int64_t)t * g.uniform_R;  // e R NLN + kr R
                        } else if (MW == 1 && g.inc_off) {
                            mb = g.inc_off[s0 + u];
                            m = g.inc_mask[s0 + u];
                        } else {
                            const int64_t rp = g.run_ptr[e];
                            mb = rp * NLN + (int64_t)kr * (g.run_ptr[e + 1] - rp);
                            if constexpr (MW == 1) m = g.run_mask[e];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < IT; ++j) {
                        const int q = lane + 32 * j;
                        kv[u][j] = 0.0;
                        rel[u][j] = 0;
                        if (have && q < CHK) {
                            kv[u][j] = __ldcs(chunk + q);
                            const int kc = c_[j] / BB;
                            int pos;
                            if (!CRAC) {
                                pos = (int)map[(int64_t)t * NLN + kc];
                            } else {
                                int k = ku[j], off = offu[j];
                                if (!g.uniform_R) {
                                    if constexpr (MW == 1) run_of(m, kc, k, off);
                                    else run_of_multi(g.run_mask + (int64_t)e * MW, kc, k, off);
                                }
                                pos = (int)mapc[mb + k] + off;
                            }
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
        }
        for (int k = lane; k < total; k += 32) values[rb + k] = acc[k];
        __syncwarp();
    }
}

// Node rows whose incidence slices hold at most 16 entries (one-DOF elements
// of up to 16 nodes, 4-node elements with 2 DOFs per node): 32 / G
// consecutive node rows per warp, G lanes per row (gather_small.cuh).
template <int NLN, typename MT, bool CRAC, int U, int BB = 1>
__global__ void __launch_bounds__(256) k_gather_small(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                      const MT *__restrict__ map, const MT *__restrict__ mapc,
                                                      int cap, int accumulate, double *values)
{
    constexpr int RPW = SmallRows<NLN, BB>::RPW;
    extern __shared__ double acc_all[];
    const int lane = threadIdx.x & 31;
    double *accw = acc_all + (size_t)(threadIdx.x >> 5) * RPW * cap;
    const int64_t W = fe_warps();
    for (int64_t v0 = fe_warp_id() * RPW; v0 < n_nodes; v0 += W * RPW)
        gather_rows_small<NLN, MT, CRAC, U, BB>(K, v0, 1, n_nodes, g, map, mapc, accw, cap, accumulate, values, lane);
}

// Two node rows per warp (nodes 2p and 2p+1, each with its own accumulator):
// the slices of incidence s of both rows share one pass of the lanes, so
// 2 x CHK entries take ceil(2 CHK / 32) FP64 add instructions instead of
// 2 ceil(CHK / 32) (72-entry slices: 5 instead of 6).  The two rows never
// share an accumulator slot, so lanes of both rows add in the same
// instruction; within a row the incidences stay in ascending element order
// (bit-identical to the sequential sum).  Adjacent nodes also read adjacent
// slices of their shared elements.
template <int NLN, int BB, typename MT, bool CRAC, int U>
__global__ void __launch_bounds__(256) k_gather_pair(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                     const MT *__restrict__ map, const MT *__restrict__ mapc, int cap,
                                                     int accumulate, double *values)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = BB * NLOC;
    constexpr int IT = (2 * CHK + 31) / 32;
    extern __shared__ double acc_all[];
    const int lane = threadIdx.x & 31;
    double *acc0 = acc_all + (size_t)(threadIdx.x >> 5) * 2 * cap;
    double *acc1 = acc0 + cap;
    // per lane slot: row of the pair, block row jr, column c
    int row_[IT], jr_[IT], c_[IT], ku[IT], offu[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int q = lane + 32 * j;
        const int qq = q < 2 * CHK ? q : 0;
        row_[j] = qq / CHK;
        const int qr = qq - row_[j] * CHK;
        jr_[j] = qr / NLOC;
        c_[j] = qr % NLOC;
        ku[j] = 0;
        offu[j] = 0;
        if (CRAC && g.uniform_R) run_of(g.run_mask[0], c_[j] / BB, ku[j], offu[j]);
    }
    const int64_t n_pairs = (n_nodes + 1) / 2;
    for (int64_t pr = fe_warp_id(); pr < n_pairs; pr += fe_warps()) {
        const int64_t v0 = 2 * pr, v1 = 2 * pr + 1;
        const bool has1 = v1 < n_nodes;
        int64_t rb0, RL0, rb1 = 0, RL1 = 0;
        if (!CRAC) {
            rb0 = g.row_ptr[BB * v0];
            RL0 = g.row_ptr[BB * v0 + 1] - rb0;
            if (has1) {
                rb1 = g.row_ptr[BB * v1];
                RL1 = g.row_ptr[BB * v1 + 1] - rb1;
            }
        } else {
            rb0 = crac_row_base(g, BB * v0);
            RL0 = crac_row_base(g, BB * v0 + 1) - rb0;
            if (has1) {
                rb1 = crac_row_base(g, BB * v1);
                RL1 = crac_row_base(g, BB * v1 + 1) - rb1;
            }
        }
        const int total0 = (int)(BB * RL0), total1 = (int)(BB * RL1);
        for (int k = lane; k < total0; k += 32) acc0[k] = accumulate ? values[rb0 + k] : 0.0;
        for (int k = lane; k < total1; k += 32) acc1[k] = accumulate ? values[rb1 + k] : 0.0;
        __syncwarp();
        const int64_t a0 = g.adj_ptr[v0], b0 = g.adj_ptr[v0 + 1];
        const int64_t a1 = has1 ? g.adj_ptr[v1] : 0, b1 = has1 ? g.adj_ptr[v1 + 1] : 0;
        const int64_t steps = max(b0 - a0, b1 - a1);
        for (int64_t s0 = 0; s0 < steps; s0 += U) {
            double kv[U][IT];
            int rel[U][IT];
            uint32_t have = 0;  // bit 2u + r: incidence s0+u of row r exists
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool h0 = a0 + s0 + u < b0, h1 = a1 + s0 + u < b1;
                have |= (h0 ? 1u : 0u) << (2 * u) | (h1 ? 1u : 0u) << (2 * u + 1);
                const uint32_t t0 = h0 ? g.adj[a0 + s0 + u] : 0u;
                const uint32_t t1 = h1 ? g.adj[a1 + s0 + u] : 0u;
#pragma unroll
                for (int j = 0; j < IT; ++j) {
                    const int q = lane + 32 * j;
                    const int r = row_[j];
                    const bool h = r == 0 ? h0 : h1;
                    kv[u][j] = 0.0;
                    rel[u][j] = 0;
                    if (q < 2 * CHK && h) {
                        const uint32_t t = r == 0 ? t0 : t1;
                        const uint32_t e = t / NLN;
                        const int kr = (int)(t - e * NLN);
                        kv[u][j] = __ldcs(K + (int64_t)e * NN + (int64_t)kr * CHK + (q - r * CHK));
                        const int kc = c_[j] / BB;
                        int pos;
                        if (!CRAC) {
                            pos = (int)map[(int64_t)t * NLN + kc];
                        } else {
                            int64_t rp;
                            int nr;
                            int k = ku[j], off = offu[j];
                            if (g.uniform_R) {
                                nr = g.uniform_R;
                                rp = (int64_t)e * nr;
                            } else {
                                rp = g.run_ptr[e];
                                nr = (int)(g.run_ptr[e + 1] - rp);
                                run_of(g.run_mask[e], kc, k, off);
                            }
                            pos = (int)mapc[rp * NLN + (int64_t)kr * nr + k] + off;
                        }
                        rel[u][j] = jr_[j] * (int)(r == 0 ? RL0 : RL1) + BB * pos + c_[j] % BB;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int j = 0; j < IT; ++j) {
                    const int r = row_[j];
                    if (lane + 32 * j < 2 * CHK && (have >> (2 * u + r) & 1u)) {
                        double *acc = r == 0 ? acc0 : acc1;
                        acc[rel[u][j]] += kv[u][j];
                    }
                }
                __syncwarp();
            }
        }
        for (int k = lane; k < total0; k += 32) values[rb0 + k] = acc0[k];
        for (int k = lane; k < total1; k += 32) values[rb1 + k] = acc1[k];
        __syncwarp();
    }
}

// Any element shape.  A unit is R of the B DOF rows of a node (R chosen by
// the host so that the accumulator, R x row length doubles, stays small for
// large B); the rows of a node have the same length and are contiguous in
// values, and the unit's part of each incidence's K slice is contiguous too.
// BATCHED (large slices): each lane loads 4 entries' values and slots
// before its 4 adds (the slots of one incidence are distinct).  Incidences
// in ascending element order.
template <typename MT, bool CRAC, bool BATCHED>
__global__ void __launch_bounds__(256) k_gather_generic(const double *__restrict__ K, int64_t n_nodes, int32_t nln,
                                                        int32_t B, int32_t R, Geo g, const MT *__restrict__ map,
                                                        const MT *__restrict__ mapc, int cap, int accumulate,
                                                        double *values)
{
    extern __shared__ double acc_all[];
    const int lane = threadIdx.x & 31;
    double *acc = acc_all + (size_t)(threadIdx.x >> 5) * cap;
    const int n_loc = nln * B;
    const int64_t NN = (int64_t)n_loc * n_loc;
    const int G = BATCHED ? (B + R - 1) / R : 1;  // units per node (one without row groups)
    for (int64_t u = fe_warp_id(); u < n_nodes * G; u += fe_warps()) {
        const int64_t v = BATCHED ? u / G : u;
        const int j0 = BATCHED ? (int)(u - v * G) * R : 0;
        const int nr_rows = BATCHED ? min(R, B - j0) : B;
        const int64_t i0 = (int64_t)B * v;
        int64_t rb, RL;
        if (!CRAC) {
            rb = g.row_ptr[i0];
            RL = g.row_ptr[i0 + 1] - rb;
        } else {
            rb = crac_row_base(g, i0);
            RL = crac_row_base(g, i0 + 1) - rb;
        }
        rb += j0 * RL;
        const int64_t total = nr_rows * RL;
        const int chk = nr_rows * n_loc;
        if (total > 0 && (!FE_IN_BOUNDS(rb + total - 1, g.nnz, g.status) || !FE_IN_BOUNDS(total - 1, cap, g.status)))
            continue;
        for (int64_t k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        __syncwarp();
        for (int64_t s = g.adj_ptr[v]; s < g.adj_ptr[v + 1]; ++s) {
            const uint32_t t = g.adj[s];
            const int64_t e = t / (uint32_t)nln;
            const int kr = (int)(t - (uint32_t)e * (uint32_t)nln);
            const double *chunk = K + e * NN + ((int64_t)kr * B + j0) * n_loc;
            int64_t rp = 0;
            int nr = 0;
            if (CRAC) {
                rp = g.run_ptr[e];
                nr = (int)(g.run_ptr[e + 1] - rp);
            }
            if constexpr (!BATCHED) {
                // one entry per lane at a time (fewer registers: more warps for small slices)
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
            } else {
                for (int q0 = lane; q0 < chk; q0 += 128) {
                    double kv[4];
                    int slot[4];
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int q = q0 + 32 * w;
                        kv[w] = 0.0;
                        slot[w] = -1;
                        if (q < chk) {
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
                            kv[w] = chunk[q];  // plain load: neighbouring rows' slices share lines
                            slot[w] = (int)(jr * RL + (int64_t)B * pos + c % B);
                        }
                    }
#pragma unroll
                    for (int w = 0; w < 4; ++w)
                        if (slot[w] >= 0 && FE_IN_BOUNDS(slot[w], total, g.status)) acc[slot[w]] += kv[w];
                }
            }
            __syncwarp();
        }
        for (int64_t k = lane; k < total; k += 32) values[rb + k] = acc[k];
        __syncwarp();
    }
}


// ------------------------------------------------- staged in smem ---
// The same two assemblies with the element-matrix stream staged in shared
// memory, double buffered: while a warp reduces one row (or element), the
// copies of its next one are in flight.  The gather moves its scattered
// 576..720-byte K slices with per-lane 16-byte asynchronous copies; the
// atomic kernel moves each element's contiguous K with one bulk (TMA) copy
// completed on an mbarrier, L2 evict-first so that values and maps stay
// cached.  Shared memory per warp: two stages, then (gather) the row
// accumulators, then (atomic) the per-element tables and two mbarriers.

constexpr int GATHER_UMAX = 8;  // incidences staged per row (more are loaded directly)

__host__ __device__ inline size_t gather_warp_bytes(int chk, int cap)
{
    const size_t b = ((size_t)2 * GATHER_UMAX * chk + (size_t)cap) * 8 + 16;
    return (b + 127) & ~(size_t)127;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(fe_smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Row gather with the K slices of the next row copied to shared memory by
// per-lane 16-byte asynchronous copies while the current row is reduced.
template <int NLN, int BB, typename MT, bool CRAC>
__global__ void __launch_bounds__(128) k_gather_async(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                      const MT *__restrict__ map, const MT *__restrict__ mapc, int cap,
                                                      int accumulate, double *values)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = BB * NLOC;
    constexpr int IT = (CHK + 31) / 32;
    constexpr int Q16 = CHK / 2;  // 16-byte pieces per slice
    constexpr int STAGE = GATHER_UMAX * CHK;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    double *stage0 = (double *)(smem_raw + (size_t)(threadIdx.x >> 5) * gather_warp_bytes(CHK, cap));
    double *acc = stage0 + 2 * STAGE;
    int jr_[IT], c_[IT], ku[IT], offu[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int q = lane + 32 * j;
        const int qq = q < CHK ? q : 0;
        jr_[j] = qq / NLOC;
        c_[j] = qq % NLOC;
        ku[j] = 0;
        offu[j] = 0;
        if (CRAC && g.uniform_R) run_of(g.run_mask[0], c_[j] / BB, ku[j], offu[j]);
    }
    // copy the first GATHER_UMAX slices of node row v into stage st (one commit group)
    auto issue = [&](int64_t v, int st) -> int {
        const int64_t a = g.adj_ptr[v];
        const int n = (int)min((int64_t)GATHER_UMAX, g.adj_ptr[v + 1] - a);
        const uint32_t t_l = lane < n ? g.adj[a + lane] : 0u;
        for (int base = 0; base < n * Q16; base += 32) {  // same trip count on every lane
            const int idx = base + lane;
            const bool valid = idx < n * Q16;
            const int u = valid ? idx / Q16 : 0, off = idx - u * Q16;
            const uint32_t t = __shfl_sync(0xffffffffu, t_l, u);
            const uint32_t e = t / NLN;
            const uint32_t kr = t - e * NLN;
            if (valid)
                cp_async16(stage0 + st * STAGE + u * CHK + 2 * off, K + (int64_t)e * NN + (int64_t)kr * CHK + 2 * off);
        }
        cp_async_commit();
        return n;
    };
    auto add = [&](uint32_t t, const double *src, bool from_global, int64_t RL) {
        const uint32_t e = t / NLN;
        const int kr = (int)(t - e * NLN);
        int64_t rp = 0;
        int nr = 0;
        uint32_t m = 0;
        if (CRAC) {
            if (g.uniform_R) {
                nr = g.uniform_R;
                rp = (int64_t)e * nr;
            } else {
                rp = g.run_ptr[e];
                nr = (int)(g.run_ptr[e + 1] - rp);
                m = g.run_mask[e];
            }
        }
#pragma unroll
        for (int j = 0; j < IT; ++j) {
            const int q = lane + 32 * j;
            if (q < CHK) {
                const int kc = c_[j] / BB;
                int pos;
                if (!CRAC) {
                    pos = (int)map[(int64_t)t * NLN + kc];
                } else {
                    int k = ku[j], off = offu[j];
                    if (!g.uniform_R) run_of(m, kc, k, off);
                    pos = (int)mapc[rp * NLN + (int64_t)kr * nr + k] + off;
                }
                const double x = from_global ? __ldcs(src + q) : src[q];
                acc[jr_[j] * (int)RL + BB * pos + c_[j] % BB] += x;
            }
        }
        __syncwarp();
    };
    int64_t v = fe_warp_id();
    int st = 0;
    int n_cur = v < n_nodes ? issue(v, 0) : 0;
    while (v < n_nodes) {
        const int64_t vn = v + fe_warps();
        const int n_next = vn < n_nodes ? issue(vn, st ^ 1) : (cp_async_commit(), 0);
        const int64_t i0 = (int64_t)BB * v;
        int64_t rb, RL;
        if (!CRAC) {
            rb = g.row_ptr[i0];
            RL = g.row_ptr[i0 + 1] - rb;
        } else {
            rb = crac_row_base(g, i0);
            RL = crac_row_base(g, i0 + 1) - rb;
        }
        const int total = (int)(BB * RL);
        for (int k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        const int64_t a = g.adj_ptr[v], b = g.adj_ptr[v + 1];
        const uint32_t t_l = lane < n_cur ? g.adj[a + lane] : 0u;
        cp_async_wait<1>();  // this row's group has landed; the next row's may still fly
        __syncwarp();
        const double *stg = stage0 + st * STAGE;
        for (int u = 0; u < n_cur; ++u) add(__shfl_sync(0xffffffffu, t_l, u), stg + u * CHK, false, RL);
        for (int64_t s = a + n_cur; s < b; ++s) {
            const uint32_t t = g.adj[s];
            const uint32_t e = t / NLN;
            const uint32_t kr = t - e * NLN;
            add(t, K + (int64_t)e * NN + (int64_t)kr * CHK, true, RL);
        }
        for (int k = lane; k < total; k += 32) values[rb + k] = acc[k];
        __syncwarp();
        v = vn;
        st ^= 1;
        n_cur = n_next;
    }
    cp_async_wait<0>();
}

__host__ __device__ inline size_t pipe_warp_bytes(int chk, int cap)
{
    const size_t b = ((size_t)2 * GATHER_UMAX * chk + (size_t)cap) * 8 + (size_t)2 * GATHER_UMAX * 8;
    return (b + 127) & ~(size_t)127;
}

__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(fe_smem_u32(dst)), "l"(src) : "memory");
}

// Row gather as a software pipeline over the rows of a warp (stride W):
//   iteration i issues the K slices (and 8-byte CSR map rows) of row v+W by
//   per-lane asynchronous copies, loads the incidence ids of row v+2W and the
//   adjacency pointers of row v+3W, then reduces row v from shared memory.
// No dependent global load stays on the critical path of a row.
template <int NLN, int BB, typename MT, bool CRAC>
__global__ void __launch_bounds__(128) k_gather_pipe(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                     const MT *__restrict__ map, const MT *__restrict__ mapc, int cap,
                                                     int accumulate, double *values)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = BB * NLOC;
    constexpr int IT = (CHK + 31) / 32;
    constexpr int Q16 = CHK / 2;
    constexpr int STAGE = GATHER_UMAX * CHK;
    constexpr bool MAPSTAGE = !CRAC && NLN * sizeof(MT) == 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    double *kst = (double *)(smem_raw + (size_t)(threadIdx.x >> 5) * pipe_warp_bytes(CHK, cap));
    uint64_t *mst = (uint64_t *)(kst + 2 * STAGE);  // [2][GATHER_UMAX] map rows
    double *acc = (double *)(mst + 2 * GATHER_UMAX);
    int jr_[IT], c_[IT], ku[IT], offu[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int q = lane + 32 * j;
        const int qq = q < CHK ? q : 0;
        jr_[j] = qq / NLOC;
        c_[j] = qq % NLOC;
        ku[j] = 0;
        offu[j] = 0;
        if (CRAC && g.uniform_R) run_of(g.run_mask[0], c_[j] / BB, ku[j], offu[j]);
    }
    const int64_t W = fe_warps();
    auto nstaged = [&](int64_t a, int64_t b) { return (int)min((int64_t)GATHER_UMAX, b - a); };
    // copy the staged slices of a row (ids held by lanes 0..n-1) into stage st
    auto issue = [&](uint32_t t_l, int n, int st) {
        for (int base = 0; base < n * Q16; base += 32) {
            const int idx = base + lane;
            const bool valid = idx < n * Q16;
            const int u = valid ? idx / Q16 : 0, off = idx - u * Q16;
            const uint32_t t = __shfl_sync(0xffffffffu, t_l, u);
            const uint32_t e = t / NLN;
            const uint32_t kr = t - e * NLN;
            if (valid)
                cp_async16(kst + st * STAGE + u * CHK + 2 * off, K + (int64_t)e * NN + (int64_t)kr * CHK + 2 * off);
        }
        if (MAPSTAGE && lane < n) cp_async8(mst + st * GATHER_UMAX + lane, map + (int64_t)t_l * NLN);
        cp_async_commit();
    };
    int64_t v = fe_warp_id();
    if (v >= n_nodes) return;
    // prologue: row v (ids + copies), row v+W (ids), row v+2W (pointers)
    int64_t a0 = g.adj_ptr[v], b0 = g.adj_ptr[v + 1];
    int n0 = nstaged(a0, b0);
    uint32_t t0 = lane < n0 ? g.adj[a0 + lane] : 0u;
    issue(t0, n0, 0);
    int64_t a1 = 0, b1 = 0, a2 = 0, b2 = 0;
    uint32_t t1 = 0;
    if (v + W < n_nodes) {
        a1 = g.adj_ptr[v + W];
        b1 = g.adj_ptr[v + W + 1];
        t1 = lane < nstaged(a1, b1) ? g.adj[a1 + lane] : 0u;
    }
    if (v + 2 * W < n_nodes) {
        a2 = g.adj_ptr[v + 2 * W];
        b2 = g.adj_ptr[v + 2 * W + 1];
    }
    int st = 0;
    while (v < n_nodes) {
        // next row's copies, then the geometry two and three rows ahead
        const int n1 = v + W < n_nodes ? nstaged(a1, b1) : 0;
        issue(t1, n1, st ^ 1);
        const int n2 = v + 2 * W < n_nodes ? nstaged(a2, b2) : 0;
        const uint32_t t2 = lane < n2 ? g.adj[a2 + lane] : 0u;
        int64_t a3 = 0, b3 = 0;
        if (v + 3 * W < n_nodes) {
            a3 = g.adj_ptr[v + 3 * W];
            b3 = g.adj_ptr[v + 3 * W + 1];
        }
        const int64_t i0 = (int64_t)BB * v;
        int64_t rb, RL;
        if (!CRAC) {
            rb = g.row_ptr[i0];
            RL = g.row_ptr[i0 + 1] - rb;
        } else {
            rb = crac_row_base(g, i0);
            RL = crac_row_base(g, i0 + 1) - rb;
        }
        const int total = (int)(BB * RL);
        for (int k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        cp_async_wait<1>();  // row v's copies have landed
        __syncwarp();
        const double *stg = kst + st * STAGE;
        for (int s = 0; s < (int)(b0 - a0); ++s) {
            const bool staged = s < n0;
            const uint32_t t = staged ? __shfl_sync(0xffffffffu, t0, s) : g.adj[a0 + s];
            const uint32_t e = t / NLN;
            const int kr = (int)(t - e * NLN);
            const double *src = staged ? stg + s * CHK : K + (int64_t)e * NN + (int64_t)kr * CHK;
            uint64_t mrow = 0;
            if (MAPSTAGE) mrow = staged ? mst[st * GATHER_UMAX + s] : *(const uint64_t *)(map + (int64_t)t * NLN);
            int64_t rp = 0;
            int nr = 0;
            uint32_t m = 0;
            if (CRAC) {
                if (g.uniform_R) {
                    nr = g.uniform_R;
                    rp = (int64_t)e * nr;
                } else {
                    rp = g.run_ptr[e];
                    nr = (int)(g.run_ptr[e + 1] - rp);
                    m = g.run_mask[e];
                }
            }
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const int q = lane + 32 * j;
                if (q < CHK) {
                    const int kc = c_[j] / BB;
                    int pos;
                    if (MAPSTAGE) {
                        pos = (int)((mrow >> (8 * sizeof(MT) * kc)) & ((1ull << (8 * sizeof(MT))) - 1));
                    } else if (!CRAC) {
                        pos = (int)map[(int64_t)t * NLN + kc];
                    } else {
                        int k = ku[j], off = offu[j];
                        if (!g.uniform_R) run_of(m, kc, k, off);
                        pos = (int)mapc[rp * NLN + (int64_t)kr * nr + k] + off;
                    }
                    acc[jr_[j] * (int)RL + BB * pos + c_[j] % BB] += staged ? src[q] : __ldcs(src + q);
                }
            }
            __syncwarp();
        }
        for (int k = lane; k < total; k += 32) values[rb + k] = acc[k];
        __syncwarp();
        // rotate the pipeline
        v += W;
        st ^= 1;
        a0 = a1;
        b0 = b1;
        n0 = n1;
        t0 = t1;
        a1 = a2;
        b1 = b2;
        t1 = t2;
        a2 = a3;
        b2 = b3;
    }
    cp_async_wait<0>();
}

// Shared memory of one warp of k_gather_bulk: S stages of UB slices, S
// mbarriers, per-stage metadata (UB incidence ids; count, adjacency range,
// row start and row length), the row accumulator.
__host__ __device__ inline size_t bulk_warp_bytes(int chk, int cap, int S, int UB)
{
    const size_t b = (size_t)S * UB * chk * 8 + (size_t)S * 8 + (size_t)S * 5 * 8 + (size_t)S * UB * 4 +
                     (size_t)cap * 8 + 8;
    return (b + 127) & ~(size_t)127;
}

// Row gather with the K slices moved by the bulk-copy (TMA) engine: the
// SM's load path streams about half of what bulk copies do.  Each warp walks
// its node rows v0, v0 + W, ... (W = all warps) as a software pipeline:
//   iteration i loads the incidence ids of row i+S+1 and the adjacency and
//   row pointers of row i+S+2 into registers, computes the slots of row i+1
//   from the metadata of its stage, waits for row i's slices, adds them in
//   ascending element order into the row accumulator, writes the row, and
//   refills row i's stage with the slices of row i+S (lanes 0..n-1 issue one
//   bulk copy each; the stage's mbarrier counts the bytes).
// The first UB incidences of a row are staged, further ones (high-degree
// nodes) are read directly.  Bit-identical to the sequential sum.  A wait that
// runs out sets FE_ERR_TIMEOUT, waits (bounded) for the copies in flight and
// ends the warp.
template <int NLN, int BB, typename MT, bool CRAC, int UB>
__global__ void __launch_bounds__(128) k_gather_bulk(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                     const MT *__restrict__ map, const MT *__restrict__ mapc,
                                                     int cap, int S, int accumulate, double *values, int *status)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int CHK = BB * NLOC;
    constexpr int IT = (CHK + 31) / 32;
    constexpr uint32_t CHKB = CHK * 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char *wbase = smem_raw + (size_t)(threadIdx.x >> 5) * bulk_warp_bytes(CHK, cap, S, UB);
    double *kst = (double *)wbase;                             // [S][UB * CHK]
    uint64_t *bar = (uint64_t *)(kst + (size_t)S * UB * CHK);  // [S]
    int64_t *meta = (int64_t *)(bar + S);                      // [S][5]: n, a, b, rb, RL
    uint32_t *meta_t = (uint32_t *)(meta + 5 * S);             // [S][UB]
    double *acc = (double *)(((uintptr_t)(meta_t + S * UB) + 7) & ~(uintptr_t)7);  // [cap]
    int jr_[IT], c_[IT], ku[IT], offu[IT];
#pragma unroll
    for (int j = 0; j < IT; ++j) {
        const int q = lane + 32 * j;
        const int qq = q < CHK ? q : 0;
        jr_[j] = qq / NLOC;
        c_[j] = qq % NLOC;
        ku[j] = 0;
        offu[j] = 0;
        if (CRAC && g.uniform_R) run_of(g.run_mask[0], c_[j] / BB, ku[j], offu[j]);
    }
    const int64_t W = fe_warps(), v0 = fe_warp_id();
    if (v0 >= n_nodes) return;
    const int64_t n_rows = (n_nodes - v0 + W - 1) / W;  // rows of this warp
    if (lane == 0) {
        for (int st = 0; st < S; ++st) fe_mbar_init(&bar[st], 1);
        fe_fence_mbar_init();
    }
    __syncwarp();
    const uint64_t pol = fe_policy_evict_first();

    struct Ptr {
        int64_t a, b, rb, RL;
    };
    auto load_ptr = [&](int64_t i) {
        Ptr p{0, 0, 0, 0};
        if (i < n_rows) {
            const int64_t v = v0 + i * W;
            p.a = g.adj_ptr[v];
            p.b = g.adj_ptr[v + 1];
            const int64_t i0 = (int64_t)BB * v;
            if (!CRAC) {
                p.rb = g.row_ptr[i0];
                p.RL = g.row_ptr[i0 + 1] - p.rb;
            } else {
                p.rb = crac_row_base(g, i0);
                p.RL = crac_row_base(g, i0 + 1) - p.rb;
            }
        }
        return p;
    };
    auto load_ids = [&](const Ptr &p) { return lane < min((int64_t)UB, p.b - p.a) ? g.adj[p.a + lane] : 0u; };
    int64_t issued = 0;
    // row i's stage: metadata, then one bulk copy per staged incidence
    auto issue = [&](int64_t i, const Ptr &p, uint32_t t) {
        if (i >= n_rows) return;
        const int st = (int)(i % S);
        const int n = (int)min((int64_t)UB, p.b - p.a);
        if (lane < n) meta_t[st * UB + lane] = t;
        if (lane == 0) {
            meta[st * 5 + 0] = n;
            meta[st * 5 + 1] = p.a;
            meta[st * 5 + 2] = p.b;
            meta[st * 5 + 3] = p.rb;
            meta[st * 5 + 4] = p.RL;
            fe_fence_proxy_async();
            fe_mbar_expect_tx(&bar[st], (uint32_t)n * CHKB);
        }
        __syncwarp();
        if (lane < n) {
            const uint32_t e = t / NLN;
            const uint32_t kr = t - e * NLN;
            fe_bulk_g2s(kst + ((size_t)st * UB + lane) * CHK, K + (int64_t)e * NN + (int64_t)kr * CHK, CHKB, &bar[st],
                        pol);
        }
        ++issued;
    };
    // slots (relative to the row start) of the staged incidences of row i
    auto slots = [&](int64_t i, int (&rel)[UB][IT]) {
        const int st = (int)(i % S);
        const int n = i < n_rows ? (int)meta[st * 5 + 0] : 0;
        const int RL = i < n_rows ? (int)meta[st * 5 + 4] : 0;
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const uint32_t t = u < n ? meta_t[st * UB + u] : 0u;
            const uint32_t e = t / NLN;
            const int kr = (int)(t - e * NLN);
            int64_t rp = 0;
            int nr = 0;
            uint32_t m = 0;
            if (CRAC && u < n) {
                if (g.uniform_R) {
                    nr = g.uniform_R;
                    rp = (int64_t)e * nr;
                } else {
                    rp = g.run_ptr[e];
                    nr = (int)(g.run_ptr[e + 1] - rp);
                    m = g.run_mask[e];
                }
            }
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                rel[u][j] = 0;
                if (u < n && lane + 32 * j < CHK) {
                    const int kc = c_[j] / BB;
                    int pos;
                    if (!CRAC) {
                        pos = (int)map[(int64_t)t * NLN + kc];
                    } else {
                        int k = ku[j], off = offu[j];
                        if (!g.uniform_R) run_of(m, kc, k, off);
                        pos = (int)mapc[rp * NLN + (int64_t)kr * nr + k] + off;
                    }
                    rel[u][j] = jr_[j] * RL + BB * pos + c_[j] % BB;
                }
            }
        }
    };

    // prologue: rows 0..S-1 staged; ids of row S and pointers of row S+1 in registers
    for (int64_t i = 0; i < S; ++i) {
        const Ptr p = load_ptr(i);
        issue(i, p, load_ids(p));
    }
    Ptr pA = load_ptr(S);
    uint32_t tA = load_ids(pA);
    Ptr pB = load_ptr(S + 1);
    int rel[UB][IT], reln[UB][IT];
    slots(0, rel);

    bool ok = true;
    int64_t i = 0;
    for (; i < n_rows; ++i) {
        const uint32_t tN = load_ids(pB);  // row i+S+1
        const Ptr pN = load_ptr(i + S + 2);
        slots(i + 1, reln);
        const int st = (int)(i % S);
        const int n = (int)meta[st * 5 + 0];
        const int64_t a = meta[st * 5 + 1], b = meta[st * 5 + 2], rb = meta[st * 5 + 3];
        const int RL = (int)meta[st * 5 + 4];
        const int total = BB * RL;
        for (int k = lane; k < total; k += 32) acc[k] = accumulate ? values[rb + k] : 0.0;
        const bool landed = fe_mbar_wait(&bar[st], (uint32_t)((i / S) & 1));
        if (!__all_sync(0xffffffffu, landed)) {
            ok = false;
            break;
        }
        __syncwarp();
        const double *stg = kst + (size_t)st * UB * CHK;
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            if (u < n) {
                double kv[IT], av[IT];
#pragma unroll
                for (int j = 0; j < IT; ++j)
                    if (lane + 32 * j < CHK) kv[j] = stg[u * CHK + lane + 32 * j];
                // the IT slots of one incidence are distinct: load all, then store all
#pragma unroll
                for (int j = 0; j < IT; ++j)
                    if (lane + 32 * j < CHK) av[j] = acc[rel[u][j]];
#pragma unroll
                for (int j = 0; j < IT; ++j)
                    if (lane + 32 * j < CHK) acc[rel[u][j]] = av[j] + kv[j];
            }
            __syncwarp();
        }
        // incidences beyond the staged ones: read directly
        for (int64_t s = a + UB; s < b; ++s) {
            const uint32_t t = g.adj[s];
            const uint32_t e = t / NLN;
            const int kr = (int)(t - e * NLN);
            const double *src = K + (int64_t)e * NN + (int64_t)kr * CHK;
            int64_t rp = 0;
            int nr = 0;
            uint32_t m = 0;
            if (CRAC) {
                if (g.uniform_R) {
                    nr = g.uniform_R;
                    rp = (int64_t)e * nr;
                } else {
                    rp = g.run_ptr[e];
                    nr = (int)(g.run_ptr[e + 1] - rp);
                    m = g.run_mask[e];
                }
            }
#pragma unroll
            for (int j = 0; j < IT; ++j) {
                const int q = lane + 32 * j;
                if (q < CHK) {
                    const int kc = c_[j] / BB;
                    int pos;
                    if (!CRAC) {
                        pos = (int)map[(int64_t)t * NLN + kc];
                    } else {
                        int k = ku[j], off = offu[j];
                        if (!g.uniform_R) run_of(m, kc, k, off);
                        pos = (int)mapc[rp * NLN + (int64_t)kr * nr + k] + off;
                    }
                    const int r = jr_[j] * RL + BB * pos + c_[j] % BB;
                    acc[r] += __ldcs(src + q);
                }
            }
            __syncwarp();
        }
        for (int k = lane; k < total; k += 32) __stcs(values + rb + k, acc[k]);
        __syncwarp();
        issue(i + S, pA, tA);  // row i's stage is free
        pA = pB;
        tA = tN;
        pB = pN;
#pragma unroll
        for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int j = 0; j < IT; ++j) rel[u][j] = reln[u][j];
    }
    if (!ok) {
        if (lane == 0) atomicCAS(status, 0, FE_ERR_TIMEOUT);
        for (; i < issued; ++i) fe_mbar_wait(&bar[i % S], (uint32_t)((i / S) & 1));
    }
}

__host__ __device__ inline size_t atomic_warp_bytes(int nn, int nloc, int nln)
{
    const size_t b = (size_t)2 * nn * 8 + (size_t)nloc * 8 + (size_t)nln * nln * 4 + 2 * (size_t)nln * 4 + 24;
    return (b + 127) & ~(size_t)127;
}

// One warp per element; the element's whole K (NN doubles, contiguous) is one
// bulk copy.  Row starts and block positions are tabulated per element in
// shared memory, then every entry is one atomic add.
template <int NLN, int BB, typename MT, bool CRAC>
__global__ void __launch_bounds__(128) k_atomic_tma(const double *__restrict__ K, int64_t n_e, Geo g,
                                                    const MT *__restrict__ map, const MT *__restrict__ mapc,
                                                    double *values, int *status)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int IT = (NN + 31) / 32;
    constexpr uint32_t NNB = NN * 8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char *wbase = smem_raw + (size_t)(threadIdx.x >> 5) * atomic_warp_bytes(NN, NLOC, NLN);
    double *stage0 = (double *)wbase;
    int64_t *base_s = (int64_t *)(stage0 + 2 * NN);
    int32_t *pos_s = (int32_t *)(base_s + NLOC);    // [NLN*NLN] block positions (CRAC: run starts)
    int32_t *kk_s = pos_s + NLN * NLN;              // CRAC: run index per column block
    int32_t *off_s = kk_s + NLN;                    // CRAC: offset inside the run
    uint64_t *bar = (uint64_t *)(((uintptr_t)(off_s + NLN) + 7) & ~(uintptr_t)7);
    if (lane == 0) {
        fe_mbar_init(&bar[0], 1);
        fe_mbar_init(&bar[1], 1);
        fe_fence_mbar_init();
    }
    __syncwarp();
    const uint64_t pol = fe_policy_evict_first();
    auto issue = [&](int64_t e, int st) {
        if (lane == 0) {
            fe_fence_proxy_async();
            fe_mbar_expect_tx(&bar[st], NNB);
            fe_bulk_g2s(stage0 + st * NN, K + e * NN, NNB, &bar[st], pol);
        }
    };
    int64_t e = fe_warp_id();
    int st = 0;
    uint32_t phase = 0;
    if (e < n_e) issue(e, 0);
    bool ok = true, next_issued = false;
    while (e < n_e) {
        const int64_t en = e + fe_warps();
        next_issued = en < n_e;
        if (next_issued) issue(en, st ^ 1);
        // per-element tables
        if (lane < NLOC) {
            const int64_t row = (int64_t)BB * g.N[e * NLN + lane / BB] + lane % BB;
            base_s[lane] = CRAC ? crac_row_base(g, row) : g.row_ptr[row];
        }
        if (!CRAC) {
            for (int q = lane; q < NLN * NLN; q += 32) pos_s[q] = (int)map[e * NLN * NLN + q];
        } else {
            int64_t rp;
            int nr;
            if (g.uniform_R) {
                nr = g.uniform_R;
                rp = e * nr;
            } else {
                rp = g.run_ptr[e];
                nr = (int)(g.run_ptr[e + 1] - rp);
            }
            const uint32_t m = g.uniform_R ? g.run_mask[0] : g.run_mask[e];
            for (int q = lane; q < NLN * nr; q += 32) pos_s[q] = (int)mapc[rp * NLN + q];
            if (lane < NLN) {
                int k, off;
                run_of(m, lane, k, off);
                kk_s[lane] = k | (nr << 16);  // run index, and the run count as the table's row stride
                off_s[lane] = off;
            }
        }
        bool got = fe_mbar_wait(&bar[st], (phase >> st) & 1u);
        got = __all_sync(0xffffffffu, got);
        phase ^= 1u << st;
        if (!got) {
            ok = false;
            break;
        }
        __syncwarp();
        const double *stg = stage0 + st * NN;
#pragma unroll 6
        for (int j = 0; j < IT; ++j) {
            const int q = lane + 32 * j;
            if (q < NN) {
                const int r = q / NLOC, c = q % NLOC;
                const int kc = c / BB;
                int pos;
                if (!CRAC) {
                    pos = pos_s[(r / BB) * NLN + kc];
                } else {
                    const int kw = kk_s[kc];
                    pos = pos_s[(r / BB) * (kw >> 16) + (kw & 0xffff)] + off_s[kc];
                }
                if (FE_IN_BOUNDS(base_s[r] + BB * pos + c % BB, g.nnz, g.status))
                    atomicAdd(values + base_s[r] + BB * pos + c % BB, stg[q]);
            }
        }
        __syncwarp();
        e = en;
        st ^= 1;
    }
    if (!ok) {
        if (lane == 0) atomicCAS(status, 0, FE_ERR_TIMEOUT);
        fe_mbar_wait(&bar[st], (phase >> st) & 1u);
        if (next_issued) fe_mbar_wait(&bar[st ^ 1], (phase >> (st ^ 1)) & 1u);
    }
}

template <typename KernelT>
int configure_smem(KernelT kernel, size_t bytes)
{
    if (bytes > 48 * 1024) FE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return FE_OK;
}


template <typename KernelT>
int grid_by_occupancy(KernelT kernel, int threads, size_t smem, int sms, int64_t warps_needed, int *grid)
{
    int per_sm = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    if (per_sm < 1) return FE_ERR_UNSUPPORTED;
    const int64_t wpb = threads / 32;
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, (warps_needed + wpb - 1) / wpb));
    return FE_OK;
}

// K slices are moved by bulk copies when their addresses are 16-byte aligned.
inline bool tma_ok(const fe_pattern *p, const double *K, int chk_doubles)
{
    const int64_t nn = (int64_t)p->n_loc * p->n_loc;
    return ((uintptr_t)K & 15u) == 0 && (nn * 8) % 16 == 0 && ((int64_t)chk_doubles * 8) % 16 == 0;
}

template <int NLN, int BB, typename MT, bool CRAC>
int launch_atomic(const fe_pattern *p, const double *K, double *values, cudaStream_t s)
{
    const Geo g = geo_of(p);
    const int sms = p->ctx->num_sms;
    if constexpr (NLN > 0) {
        constexpr int NLOC = NLN * BB;
        if (p->ctx->knob[FE_KNOB_ATOMIC_KERNEL] != 1 && tma_ok(p, K, NLOC * NLOC)) {
            const int W = (p->ctx->knob[FE_KNOB_ATOMIC_WARPS] > 0 && p->ctx->knob[FE_KNOB_ATOMIC_WARPS] <= 4)
                              ? p->ctx->knob[FE_KNOB_ATOMIC_WARPS]
                              : 4;  // launch bound: 128 threads
            const size_t smem = W * atomic_warp_bytes(NLOC * NLOC, NLOC, NLN);
            FE_TRY(configure_smem(k_atomic_tma<NLN, BB, MT, CRAC>, smem));
            int grid;
            FE_TRY(grid_by_occupancy(k_atomic_tma<NLN, BB, MT, CRAC>, W * 32, smem, sms, p->n_e, &grid));
            k_atomic_tma<NLN, BB, MT, CRAC><<<grid, W * 32, smem, s>>>(
                K, p->n_e, g, (const MT *)p->map_csr, (const MT *)p->map_crac, values, p->ctx->d_status);
        } else {
            k_atomic_elem<NLN, BB, MT, CRAC><<<fe_grid_resident(k_atomic_elem<NLN, BB, MT, CRAC>, p->n_e * 32, 256, sms),
                                               256, 0, s>>>(
                K, p->n_e, g, (const MT *)p->map_csr, (const MT *)p->map_crac, values);
        }
    } else {
        k_atomic_generic<MT, CRAC><<<fe_grid_resident(k_atomic_generic<MT, CRAC>, p->n_e * 32, 256, sms), 256, 0, s>>>(
            K, p->n_e, p->nln, p->B, g, (const MT *)p->map_csr, (const MT *)p->map_crac, values);
    }
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

// lean instances take incidences two at a time above this slice size
// (measured on the Q1 d-benchmark, 192^2: d = 5..8 CSR 68 / 77 / 109 / 138
// -> 56 / 66 / 95 / 101 us, CRAC d = 6..8 -> 83 / 130 / 130 us, d <= 4
// unchanged)
constexpr int LEAN_U2_CHK = 64;

// VARIANTS = false: only the default kernels of the shape are instantiated
// (no schedule-knob variants, no U = 8), for shapes added to keep their rows
// off the generic kernel at little compile-time cost.
template <int NLN, int BB, typename MT, bool CRAC, bool VARIANTS = true>
int launch_gather(const fe_pattern *p, const double *K, double *values, int accumulate, cudaStream_t s)
{
    const Geo g = geo_of(p);
    const fe_ctx *ctx = p->ctx;
    const int sms = ctx->num_sms;
    const int cap = std::max(1, p->B * p->max_row_len);
    const int kind = ctx->knob[FE_KNOB_GATHER_KERNEL];
    int W = ctx->knob[FE_KNOB_GATHER_WARPS];
    if constexpr (NLN > 0) {
        constexpr int CHK = BB * NLN * BB;
        if constexpr (CHK <= 16) {
            if (kind == 0 || kind == 6) {  // the default for these shapes
                constexpr int RPW = SmallRows<NLN, BB>::RPW;
                const int Ws = (W > 0 && W <= 8) ? W : 4;
                const size_t ssm = (size_t)Ws * RPW * cap * 8;
                if (ssm <= 200 * 1024) {
                    FE_TRY(configure_smem(k_gather_small<NLN, MT, CRAC, 4, BB>, ssm));
                    const int sgrid = fe_grid_resident(k_gather_small<NLN, MT, CRAC, 4, BB>,
                                                       (p->n_nodes + RPW - 1) / RPW * 32, Ws * 32, sms, ssm);
                    k_gather_small<NLN, MT, CRAC, 4, BB><<<sgrid, Ws * 32, ssm, s>>>(
                        K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, accumulate, values);
                    fe_note_launch();
                    FE_CUDA(cudaGetLastError());
                    return FE_OK;
                }
            }
        }
        if constexpr (VARIANTS) if (kind == 5) {
            constexpr int UP = 2;
            int Wp = (W > 0 && W <= 8) ? W : 2;
            while (Wp > 1 && (size_t)Wp * 2 * cap * 8 > 64 * 1024) Wp >>= 1;
            const size_t psm = (size_t)Wp * 2 * cap * 8;
            if (psm <= 200 * 1024) {
                FE_TRY(configure_smem(k_gather_pair<NLN, BB, MT, CRAC, UP>, psm));
                const int pgrid = fe_grid_resident(k_gather_pair<NLN, BB, MT, CRAC, UP>, (p->n_nodes + 1) / 2 * 32,
                                                   Wp * 32, sms, psm);
                k_gather_pair<NLN, BB, MT, CRAC, UP><<<pgrid, Wp * 32, psm, s>>>(
                    K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, accumulate, values);
                fe_note_launch();
                FE_CUDA(cudaGetLastError());
                return FE_OK;
            }
        }
        if constexpr (VARIANTS) if (kind == 4 && tma_ok(p, K, CHK)) {
            constexpr int UB = 8;
            int S = ctx->knob[FE_KNOB_GATHER_STAGES] > 0 ? ctx->knob[FE_KNOB_GATHER_STAGES] : 4;
            int Wb = (W > 0 && W <= 4) ? W : 4;  // launch bound: 128 threads
            size_t bsmem = (size_t)Wb * bulk_warp_bytes(CHK, cap, S, UB);
            while (bsmem > 200 * 1024 && (Wb > 1 || S > 2)) {
                if (Wb > 1) Wb >>= 1;
                else --S;
                bsmem = (size_t)Wb * bulk_warp_bytes(CHK, cap, S, UB);
            }
            if (bsmem <= 200 * 1024) {
                FE_TRY(configure_smem(k_gather_bulk<NLN, BB, MT, CRAC, UB>, bsmem));
                int bgrid;
                FE_TRY(grid_by_occupancy(k_gather_bulk<NLN, BB, MT, CRAC, UB>, Wb * 32, bsmem, sms, p->n_nodes,
                                         &bgrid));
                k_gather_bulk<NLN, BB, MT, CRAC, UB><<<bgrid, Wb * 32, bsmem, s>>>(
                    K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, S, accumulate, values,
                    ctx->d_status);
                fe_note_launch();
                FE_CUDA(cudaGetLastError());
                return FE_OK;
            }
        }
        if constexpr (VARIANTS) if (kind == 3 && tma_ok(p, K, CHK)) {
            if (W <= 0 || W > 4) W = 4;
            const size_t psmem = (size_t)W * pipe_warp_bytes(CHK, cap);
            if (psmem <= 200 * 1024) {
                FE_TRY(configure_smem(k_gather_pipe<NLN, BB, MT, CRAC>, psmem));
                int pgrid;
                FE_TRY(grid_by_occupancy(k_gather_pipe<NLN, BB, MT, CRAC>, W * 32, psmem, sms, p->n_nodes, &pgrid));
                k_gather_pipe<NLN, BB, MT, CRAC><<<pgrid, W * 32, psmem, s>>>(
                    K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, accumulate, values);
                fe_note_launch();
                FE_CUDA(cudaGetLastError());
                return FE_OK;
            }
            W = ctx->knob[FE_KNOB_GATHER_WARPS];
        }
        if constexpr (VARIANTS) if (kind == 2 && tma_ok(p, K, CHK)) {
            if (W <= 0 || W > 4) W = 4;  // launch bound of the staged kernel: 128 threads
            const size_t tsmem = (size_t)W * gather_warp_bytes(CHK, cap);
            if (tsmem <= 200 * 1024) {
                FE_TRY(configure_smem(k_gather_async<NLN, BB, MT, CRAC>, tsmem));
                int tgrid;
                FE_TRY(grid_by_occupancy(k_gather_async<NLN, BB, MT, CRAC>, W * 32, tsmem, sms, p->n_nodes, &tgrid));
                k_gather_async<NLN, BB, MT, CRAC><<<tgrid, W * 32, tsmem, s>>>(
                    K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, accumulate, values);
                fe_note_launch();
                FE_CUDA(cudaGetLastError());
                return FE_OK;
            }
        }
    }
    // fastest in sweeps of 1..8 warps per block on the 64^3 elasticity mesh:
    // 2 for the unpacked rows, 4 for packed CRAC rows
    if constexpr (NLN > 0) {
        if (W <= 0) W = gather_packs<NLN, BB, CRAC, 4>() ? 4 : 2;
    }
    if (W <= 0) W = 2;
    while (W > 1 && (size_t)W * cap * 8 > 64 * 1024) W >>= 1;
    const size_t smem = (size_t)W * cap * 8;
    if (smem > 200 * 1024) return FE_ERR_UNSUPPORTED;
    const int grid = fe_grid_for(p->n_nodes * 32, W * 32, sms, std::max(1, 64 / W));
    if constexpr (NLN > 0) {
        bool u8 = false;
        if constexpr (VARIANTS) u8 = ctx->knob[FE_KNOB_GATHER_BATCH] == 8;
        if (u8) {
            if constexpr (VARIANTS) {
                FE_TRY(configure_smem(k_gather_node<NLN, BB, MT, CRAC, 8>, smem));
                k_gather_node<NLN, BB, MT, CRAC, 8><<<grid, W * 32, smem, s>>>(
                    K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, accumulate, values);
            }
        } else {
            constexpr int UL = (!VARIANTS && BB * NLN * BB > LEAN_U2_CHK) ? 2 : 4;
            FE_TRY(configure_smem(k_gather_node<NLN, BB, MT, CRAC, UL>, smem));
            k_gather_node<NLN, BB, MT, CRAC, UL><<<grid, W * 32, smem, s>>>(
                K, p->n_nodes, g, (const MT *)p->map_csr, (const MT *)p->map_crac, cap, accumulate, values);
        }
    } else {
        // rows per unit: a node's B rows, split into equal groups when their
        // accumulator would exceed 1024 doubles (large B, e.g. 20 DOF/node)
        const int64_t whole = (int64_t)p->B * std::max(1, p->max_row_len);
        const int groups = (int)std::min<int64_t>(p->B, (whole + 1023) / 1024);
        const int R = (p->B + groups - 1) / groups;
        const int gcap = std::max(1, R * p->max_row_len);
        int GW = ctx->knob[FE_KNOB_GATHER_WARPS] > 0 ? ctx->knob[FE_KNOB_GATHER_WARPS] : 2;
        while (GW > 1 && (size_t)GW * gcap * 8 > 64 * 1024) GW >>= 1;
        const size_t gsmem = (size_t)GW * gcap * 8;
        if (gsmem > 200 * 1024) return FE_ERR_UNSUPPORTED;
        const int64_t units = p->n_nodes * ((p->B + R - 1) / R);
        auto launch = [&](auto kern) -> int {
            FE_TRY(configure_smem(kern, gsmem));
            const int ggrid = fe_grid_resident(kern, units * 32, GW * 32, sms, gsmem);
            kern<<<ggrid, GW * 32, gsmem, s>>>(K, p->n_nodes, p->nln, p->B, R, g, (const MT *)p->map_csr,
                                               (const MT *)p->map_crac, gcap, accumulate, values);
            return FE_OK;
        };
        // without row groups and with small slices: the instance with fewer registers
        if (groups > 1 || R * p->n_loc > 128) FE_TRY(launch(k_gather_generic<MT, CRAC, true>));
        else FE_TRY(launch(k_gather_generic<MT, CRAC, false>));
    }
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

// Element shapes with a specialised kernel: (blocks per element, DOFs per block).
template <typename MT, bool CRAC>
int dispatch(const fe_pattern *p, const double *K, double *values, int mode, int accumulate, cudaStream_t s)
{
    const int nln = p->nln, B = p->B;
    if (mode == FE_ATOMIC) {
        if (!accumulate) FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)p->nnz, s));
        if (p->n_e == 0) return FE_OK;
        if (nln == 4 && B == 1) return launch_atomic<4, 1, MT, CRAC>(p, K, values, s);
        if (nln == 8 && B == 1) return launch_atomic<8, 1, MT, CRAC>(p, K, values, s);
        if (nln == 8 && B == 3) return launch_atomic<8, 3, MT, CRAC>(p, K, values, s);
        if (nln == 10 && B == 3) return launch_atomic<10, 3, MT, CRAC>(p, K, values, s);
        return launch_atomic<0, 0, MT, CRAC>(p, K, values, s);
    }
    if (p->n_nodes == 0) return FE_OK;
    if (nln == 4 && B == 1) return launch_gather<4, 1, MT, CRAC>(p, K, values, accumulate, s);
    if (nln == 8 && B == 1) return launch_gather<8, 1, MT, CRAC>(p, K, values, accumulate, s);
    if (nln == 8 && B == 3) return launch_gather<8, 3, MT, CRAC>(p, K, values, accumulate, s);
    if (nln == 10 && B == 3) return launch_gather<10, 3, MT, CRAC>(p, K, values, accumulate, s);
    if constexpr (std::is_same<MT, uint8_t>::value) {
        // Q2..Q7 scalar quads, Q1 quads with 2..8 DOFs per node and Q2..Q4
        // quads with 4: the several-rows-per-warp and batched-incidence row
        // kernels instead of the generic one, which loads one incidence at a
        // time (elements of more than 32 nodes: multi-word run masks)
        if (nln == 9 && B == 1) return launch_gather<9, 1, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 16 && B == 1) return launch_gather<16, 1, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 25 && B == 1) return launch_gather<25, 1, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 2) return launch_gather<4, 2, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 3) return launch_gather<4, 3, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 4) return launch_gather<4, 4, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 5) return launch_gather<4, 5, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 6) return launch_gather<4, 6, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 7) return launch_gather<4, 7, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 4 && B == 8) return launch_gather<4, 8, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 9 && B == 4) return launch_gather<9, 4, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 16 && B == 4) return launch_gather<16, 4, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 25 && B == 4) return launch_gather<25, 4, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 36 && B == 1) return launch_gather<36, 1, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 49 && B == 1) return launch_gather<49, 1, MT, CRAC, false>(p, K, values, accumulate, s);
        if (nln == 64 && B == 1) return launch_gather<64, 1, MT, CRAC, false>(p, K, values, accumulate, s);
    }
    // Q8 scalar quads: rows of up to 289 nodes, 16-bit slot maps
    if (nln == 81 && B == 1) return launch_gather<81, 1, MT, CRAC, false>(p, K, values, accumulate, s);
    return launch_gather<0, 0, MT, CRAC>(p, K, values, accumulate, s);
}

int assemble(fe_ctx *ctx, const fe_pattern *p, const double *K, double *values, int mode, int accumulate,
             void *stream, bool crac)
{
    if (!ctx || !p || p->ctx != ctx) return FE_ERR_INVALID_ARG;
    if (mode != FE_ATOMIC && mode != FE_DETERMINISTIC && mode != FE_COLOURED && mode != FE_ROWLOCK)
        return FE_ERR_INVALID_ARG;
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
    if (mode == FE_COLOURED || mode == FE_ROWLOCK) {
        rc = mode == FE_COLOURED ? fe_assemble_coloured(p, K, values, accumulate, crac, s)
                                 : fe_assemble_rowlock(p, K, values, accumulate, crac, s);
        if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
        return rc;
    }
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

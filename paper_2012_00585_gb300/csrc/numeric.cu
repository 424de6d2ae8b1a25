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
// parity-tested): atomic -- k_atomic_elem (K_e through registers),
// k_atomic_tma (K_e staged by a bulk copy), k_atomic_generic (any shape);
// deterministic -- k_gather_node (3-DOF and other specialised shapes),
// k_gather_small (slices of at most 16 entries, several rows per warp),
// k_gather_generic (any shape).  Every FP64 add of the atomic kernels is a
// reduction (fe_red_add_f64).  FE_COLOURED and FE_ROWLOCK are in colour.cu
// and rowlock.cu.
#include "assemble_body.cuh"
#include "internal.cuh"
#include "tma.cuh"
#include "gather_small.cuh"

namespace {

using namespace fe_dev;

// ------------------------------------------------------------ atomic ---
// One warp per element; NLN blocks of BB DOFs, NLN*BB <= 32.  (A bound of two
// blocks per SM, 128 registers instead of up to 222 for the 30 x 30
// elements, measured slower: P2 tets 96^3 CSR 21.4 -> 29.8 ms, hex CRAC
// 548 -> 586 us.)
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
    for (int64_t i = fe_warp_id(); i < n_e; i += fe_warps()) {
        const int64_t e = elem_at(g, i);
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
                    if (q < NN) fe_red_add_f64(values + b + (int64_t)BB * pos + c % BB, kv[u]);
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
    for (int64_t i = fe_warp_id(); i < n_e; i += fe_warps()) {
        const int64_t e = elem_at(g, i);
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
            fe_red_add_f64(values + base_s[w][r] + (int64_t)B * pos + c % B, __ldcs(Ke + q));
        }
        __syncwarp();
    }
}

// ------------------------------------------------------ deterministic ---
// One warp per node row, rows strided over all warps (gather_node_rows in
// assemble_body.cuh: ascending-element sums, bit-identical to Listing 2).
template <int NLN, int BB, typename MT, int U>
__global__ void __launch_bounds__(256) k_gather_node(const double *__restrict__ K, int64_t n_nodes, Geo g,
                                                     const MT *__restrict__ map, int cap, int accumulate,
                                                     double *values)
{
    extern __shared__ double acc_all[];
    double *acc = acc_all + (size_t)(threadIdx.x >> 5) * cap;
    gather_node_rows<NLN, BB, MT, U>(K, g, map, acc, cap, accumulate, values, fe_warp_id(), n_nodes, fe_warps(),
                                     threadIdx.x & 31);
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
            rb = row_start(g, i0);
            RL = row_start(g, i0 + 1) - rb;
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


// ------------------------------------------------ staged atomic ---
// The atomic assembly with the element-matrix stream staged in shared
// memory, double buffered: while a warp adds one element, the copy of its
// next one is in flight.  Each element's contiguous K moves with one bulk
// (TMA) copy completed on an mbarrier, L2 evict-first so that values and
// maps stay cached.  Shared memory per warp: two stages, the per-element
// tables and two mbarriers.

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
    int64_t i = fe_warp_id();
    int64_t e = i < n_e ? elem_at(g, i) : 0;
    int st = 0;
    uint32_t phase = 0;
    if (i < n_e) issue(e, 0);
    bool ok = true, next_issued = false;
    while (i < n_e) {
        const int64_t in = i + fe_warps();
        next_issued = in < n_e;
        const int64_t en = next_issued ? elem_at(g, in) : 0;
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
                    fe_red_add_f64(values + base_s[r] + BB * pos + c % BB, stg[q]);
            }
        }
        __syncwarp();
        i = in;
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
        // default: the register kernel (C2 CSR 520 vs 601 us, C3 CSR 21.4 vs
        // 29.5 ms, CRAC 20.5 vs 22.9 ms against the staged kernel, once the
        // adds were issued as reductions); the staged kernel on request
        if (p->ctx->knob[FE_KNOB_ATOMIC_KERNEL] == 2 && tma_ok(p, K, NLOC * NLOC)) {
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
template <int NLN, int BB, typename MT, bool VARIANTS = true>
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
            if (kind == 0 || kind == 2) {  // the default for these shapes
                constexpr int RPW = SmallRows<NLN, BB>::RPW;
                const int Ws = (W > 0 && W <= 8) ? W : 4;
                const size_t ssm = (size_t)Ws * RPW * cap * 8;
                if (ssm <= 200 * 1024) {
                    FE_TRY(configure_smem(k_gather_small<NLN, MT, false, 4, BB>, ssm));
                    const int sgrid = fe_grid_resident(k_gather_small<NLN, MT, false, 4, BB>,
                                                       (p->n_nodes + RPW - 1) / RPW * 32, Ws * 32, sms, ssm);
                    k_gather_small<NLN, MT, false, 4, BB><<<sgrid, Ws * 32, ssm, s>>>(
                        K, p->n_nodes, g, (const MT *)p->map_csr, nullptr, cap, accumulate, values);
                    fe_note_launch();
                    FE_CUDA(cudaGetLastError());
                    return FE_OK;
                }
            }
        }
    }
    // fastest in sweeps of 1..8 warps per block on the 64^3 elasticity mesh:
    // 2 for the unpacked rows, 4 for packed CRAC rows
    if constexpr (NLN > 0) {
        if (W <= 0) W = 2;
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
                FE_TRY(configure_smem(k_gather_node<NLN, BB, MT, 8>, smem));
                k_gather_node<NLN, BB, MT, 8><<<grid, W * 32, smem, s>>>(K, p->n_nodes, g, (const MT *)p->map_csr,
                                                                          cap, accumulate, values);
            }
        } else {
            constexpr int UL = (!VARIANTS && BB * NLN * BB > LEAN_U2_CHK) ? 2 : 4;
            FE_TRY(configure_smem(k_gather_node<NLN, BB, MT, UL>, smem));
            k_gather_node<NLN, BB, MT, UL><<<grid, W * 32, smem, s>>>(K, p->n_nodes, g, (const MT *)p->map_csr, cap,
                                                                       accumulate, values);
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
            kern<<<ggrid, GW * 32, gsmem, s>>>(K, p->n_nodes, p->nln, p->B, R, g, (const MT *)p->map_csr, nullptr,
                                               gcap, accumulate, values);
            return FE_OK;
        };
        // without row groups and with small slices: the instance with fewer registers
        if (groups > 1 || R * p->n_loc > 128) FE_TRY(launch(k_gather_generic<MT, false, true>));
        else FE_TRY(launch(k_gather_generic<MT, false, false>));
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
    // FE_DETERMINISTIC: block-map kernels only (CRAC rows arrive as a view
    // of the pattern with the CRAC block map and CRAC row starts)
    if constexpr (CRAC) {
        return FE_ERR_INVALID_ARG;
    } else {
        if (p->n_nodes == 0) return FE_OK;
        if (nln == 4 && B == 1) return launch_gather<4, 1, MT>(p, K, values, accumulate, s);
        if (nln == 8 && B == 1) return launch_gather<8, 1, MT>(p, K, values, accumulate, s);
        if (nln == 8 && B == 3) return launch_gather<8, 3, MT>(p, K, values, accumulate, s);
        if (nln == 10 && B == 3) return launch_gather<10, 3, MT>(p, K, values, accumulate, s);
        if constexpr (std::is_same<MT, uint8_t>::value) {
            // Q2..Q7 scalar quads, Q1 quads with 2..8 DOFs per node and Q2..Q4
            // quads with 4: the several-rows-per-warp and batched-incidence row
            // kernels instead of the generic one, which loads one incidence at a
            // time (elements of more than 32 nodes: multi-word run masks)
            if (nln == 9 && B == 1) return launch_gather<9, 1, MT, false>(p, K, values, accumulate, s);
            if (nln == 16 && B == 1) return launch_gather<16, 1, MT, false>(p, K, values, accumulate, s);
            if (nln == 25 && B == 1) return launch_gather<25, 1, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 2) return launch_gather<4, 2, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 3) return launch_gather<4, 3, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 4) return launch_gather<4, 4, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 5) return launch_gather<4, 5, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 6) return launch_gather<4, 6, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 7) return launch_gather<4, 7, MT, false>(p, K, values, accumulate, s);
            if (nln == 4 && B == 8) return launch_gather<4, 8, MT, false>(p, K, values, accumulate, s);
            if (nln == 9 && B == 4) return launch_gather<9, 4, MT, false>(p, K, values, accumulate, s);
            if (nln == 16 && B == 4) return launch_gather<16, 4, MT, false>(p, K, values, accumulate, s);
            if (nln == 25 && B == 4) return launch_gather<25, 4, MT, false>(p, K, values, accumulate, s);
            if (nln == 36 && B == 1) return launch_gather<36, 1, MT, false>(p, K, values, accumulate, s);
            if (nln == 49 && B == 1) return launch_gather<49, 1, MT, false>(p, K, values, accumulate, s);
            if (nln == 64 && B == 1) return launch_gather<64, 1, MT, false>(p, K, values, accumulate, s);
        }
        // Q8 scalar quads: rows of up to 289 nodes, 16-bit slot maps
        if (nln == 81 && B == 1) return launch_gather<81, 1, MT, false>(p, K, values, accumulate, s);
        return launch_gather<0, 0, MT>(p, K, values, accumulate, s);
    }
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
    if (crac && mode == FE_DETERMINISTIC) {
        // the CRAC gather: the block-map kernels through a view of the
        // pattern whose block map is the expanded CRAC run map and whose row
        // starts come from the CRAC pairs
        if (!p->map_crac_blk) {
            if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
            return FE_ERR_NOT_BUILT;
        }
        fe_pattern view = *p;
        view.map_csr = p->map_crac_blk;
        view.crac_rows = true;
        rc = p->map_bytes == 1 ? dispatch<uint8_t, false>(&view, K, values, mode, accumulate, s)
                               : dispatch<uint16_t, false>(&view, K, values, mode, accumulate, s);
    } else if (p->map_bytes == 1)
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
    FeRange range("fe_assemble_csr");
    return assemble(ctx, p, elem_mats, values, mode, accumulate, stream, false);
}

int fe_assemble_crac(fe_ctx *ctx, const fe_pattern *p, const double *elem_mats, double *values, int mode,
                     int accumulate, void *stream)
{
    FeRange range("fe_assemble_crac");
    return assemble(ctx, p, elem_mats, values, mode, accumulate, stream, true);
}

}  // extern "C"

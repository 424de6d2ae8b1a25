// Batched assembly: many independent meshes (patterns + element matrices +
// values) in ONE persistent kernel launch.  The launch walks a work list of
// tiles (a tile = `tile` consecutive elements in FE_ATOMIC, `tile`
// consecutive node rows in FE_DETERMINISTIC) of every mesh; warps (or blocks)
// take the next tile from an atomic counter, so meshes of very different
// sizes share the GPU without per-mesh launches or tail effects.  The
// arithmetic per element / node row is the single-mesh one
// (assemble_body.cuh), so a batched result equals the per-mesh result: bit
// for bit in FE_DETERMINISTIC.
//
// Schedules: FE_ATOMIC  -- warp per element (K from global memory, or staged
//                          by bulk copies: the default), thread per entry,
//                          block per element
//            FE_DETERMINISTIC -- warp per node row (one-DOF rows of 4 or 8
//                          nodes: several rows per warp)
// An autotuner times the candidates on the caller's batch and caches the
// fastest per batch signature in the context; a batch can also be captured
// once into a CUDA graph and replayed.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "assemble_body.cuh"
#include "gather_small.cuh"
#include "internal.cuh"
#include "tma.cuh"

using namespace fe_dev;

namespace {

enum Shape { SH_GENERIC = 0, SH_4_1 = 1, SH_8_1 = 2, SH_8_3 = 3, SH_10_3 = 4 };

struct BatchItemDev {
    Geo g;
    const double *K;
    double *values;
    const void *map;
    const void *mapc;
    int64_t units;       // elements (atomic) or node rows (deterministic)
    int64_t nnz;
    int64_t tile_begin;  // first global tile of this item
    int32_t nln, B, shape, map_bytes;
    int32_t staged;      // FE_SCHED_WARP_PER_ELEMENT_TMA: K_e moved by a bulk copy
    uint64_t *times;     // the caller's [first tile started, last tile finished] (ns) or null
};

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per-item timestamps (items with a times array): tc holds two counters per
// item, tiles started and tiles finished; the first start and the last
// finish write the global timer.  Called by one thread per tile.
__device__ __forceinline__ void tile_started(const BatchItemDev &it, int i, unsigned int *tc)
{
    if (it.times && atomicAdd(&tc[2 * i], 1u) == 0) it.times[0] = global_ns();
}

__device__ __forceinline__ void tile_finished(const BatchItemDev &it, int i, unsigned int *tc, int tile)
{
    if (!it.times) return;
    __threadfence();
    const unsigned int n_tiles = (unsigned int)((it.units + tile - 1) / tile);
    if (atomicAdd(&tc[2 * i + 1], 1u) + 1 == n_tiles) it.times[1] = global_ns();
}

int shape_of(const fe_pattern *p)
{
    if (p->nln == 4 && p->B == 1) return SH_4_1;
    if (p->nln == 8 && p->B == 1) return SH_8_1;
    if (p->nln == 8 && p->B == 3) return SH_8_3;
    if (p->nln == 10 && p->B == 3) return SH_10_3;
    return SH_GENERIC;
}

__device__ __forceinline__ int find_item(const BatchItemDev *__restrict__ items, int n_items, int64_t t)
{
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One non-inlined function per element shape, so that the batched kernel
// needs the registers of its largest body, not of all bodies together.
template <int NLN, int BB, typename MT, bool CRAC>
__device__ __noinline__ void atomic_elem_call(const BatchItemDev *__restrict__ it, int64_t e, int lane)
{
    const Geo g = it->g;
    atomic_element<NLN, BB, MT, CRAC>(it->K, e, g, (const MT *)it->map, (const MT *)it->mapc, it->values, lane);
}

// FE_SCHED_WARP_PER_ELEMENT_TMA: elements [u0, u1) of one item through the
// warp's two stages (kst, bar; phase bit s = parity of the next wait on stage
// s).  While element e is added, the copy of e+1 is in flight; the tables
// of e (row starts; block positions, or run positions and the run index /
// offset of every column block) are loaded while its own copy lands, then
// every entry is one atomic add.  tab holds NLN*NLN + 2*NLN ints.  Returns
// false when a wait ran out (after waiting, bounded, for the copy in flight).
template <int NLN, int BB, typename MT, bool CRAC>
__device__ __noinline__ bool staged_tile(const BatchItemDev *__restrict__ it, int64_t u0, int64_t u1, int lane,
                                         double *kst, int stage, uint64_t *bar, uint32_t *phase_io, int64_t *base_s,
                                         int32_t *tab, uint64_t pol)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    constexpr int IT = (NN + 31) / 32;
    constexpr uint32_t NNB = NN * 8;
    const Geo g = it->g;
    const double *K = it->K;
    double *values = it->values;
    const MT *map = (const MT *)it->map;
    const MT *mapc = (const MT *)it->mapc;
    int32_t *pos_s = tab;               // [NLN*NLN] block positions (CRAC: run positions)
    int32_t *kk_s = pos_s + NLN * NLN;  // CRAC: run index | run count << 16, per column block
    int32_t *off_s = kk_s + NLN;        // CRAC: offset inside the run
    uint32_t phase = *phase_io;
    auto issue = [&](int64_t e, int s_) {
        if (lane == 0) {
            fe_fence_proxy_async();
            fe_mbar_expect_tx(&bar[s_], NNB);
            fe_bulk_g2s(kst + (size_t)s_ * stage, K + e * NN, NNB, &bar[s_], pol);
        }
    };
    int st = 0;
    issue(u0, st);
    for (int64_t e = u0; e < u1; ++e) {
        const bool next = e + 1 < u1;
        if (next) issue(e + 1, st ^ 1);
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
                kk_s[lane] = k | (nr << 16);
                off_s[lane] = off;
            }
        }
        if (!__all_sync(0xffffffffu, fe_mbar_wait(&bar[st], (phase >> st) & 1u))) {
            fe_mbar_wait(&bar[st], (phase >> st) & 1u);  // once more, bounded, for the copy itself
            if (next) fe_mbar_wait(&bar[st ^ 1], (phase >> (st ^ 1)) & 1u);
            *phase_io = phase;
            return false;
        }
        phase ^= 1u << st;
        __syncwarp();
        const double *stg = kst + (size_t)st * stage;
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
        st ^= 1;
    }
    *phase_io = phase;
    return true;
}

template <typename MT, bool CRAC>
__device__ __forceinline__ bool staged_tile_any(const BatchItemDev *it, int shape, int64_t u0, int64_t u1, int lane,
                                                double *kst, int stage, uint64_t *bar, uint32_t *phase,
                                                int64_t *base_s, int32_t *tab, uint64_t pol)
{
    switch (shape) {
    case SH_4_1: return staged_tile<4, 1, MT, CRAC>(it, u0, u1, lane, kst, stage, bar, phase, base_s, tab, pol);
    case SH_8_1: return staged_tile<8, 1, MT, CRAC>(it, u0, u1, lane, kst, stage, bar, phase, base_s, tab, pol);
    case SH_8_3: return staged_tile<8, 3, MT, CRAC>(it, u0, u1, lane, kst, stage, bar, phase, base_s, tab, pol);
    default: return staged_tile<10, 3, MT, CRAC>(it, u0, u1, lane, kst, stage, bar, phase, base_s, tab, pol);
    }
}

template <typename MT, bool CRAC>
__device__ __noinline__ void atomic_elem_generic_call(const BatchItemDev *__restrict__ it, int64_t e, int lane,
                                                      int64_t *base_s, int32_t *k_s, int32_t *off_s)
{
    const Geo g = it->g;
    atomic_element_generic<MT, CRAC>(it->K, e, it->nln, it->B, g, (const MT *)it->map, (const MT *)it->mapc,
                                     it->values, base_s, k_s, off_s, lane);
}

// The node rows [u0, u1) of a one-DOF item, RPW at a time with G lanes per
// row (one call per tile).  The warp's accumulator region (cap doubles, cap
// >= RPW x the item's longest row by the plan) is split into RPW per-row
// parts of cap / RPW.
template <int NLN, typename MT, bool CRAC>
__device__ __noinline__ void gather_tile_small(const BatchItemDev *__restrict__ it, int64_t u0, int64_t u1,
                                               double *acc, int cap, int accumulate, int lane)
{
    constexpr int RPW = SmallRows<NLN>::RPW;
    const Geo g = it->g;
    const double *K = it->K;
    double *values = it->values;
    const MT *map = (const MT *)it->map, *mapc = (const MT *)it->mapc;
    for (int64_t v0 = u0; v0 < u1; v0 += RPW)
        gather_rows_small<NLN, MT, CRAC, 4>(K, v0, 1, u1, g, map, mapc, acc, cap / RPW, accumulate, values, lane);
}

// The node rows [u0, u1) of an item with a specialised shape, one call per
// tile: the single-mesh row loop (gather_node_rows, next row's head loaded
// one row ahead) over the tile's consecutive rows, through the item's block
// map (CSR, or the CRAC run map expanded per column block with row starts
// from the CRAC pairs).  Only the fields the loop reads are taken from the
// item, so that they stay in registers.
template <int NLN, int BB, typename MT>
__device__ __noinline__ void gather_tile_node(const BatchItemDev *__restrict__ it, int64_t u0, int64_t u1,
                                              double *acc, int cap, int accumulate, int lane)
{
    Geo g;
    g.row_ptr = it->g.row_ptr;
    g.crac_ptr = it->g.crac_ptr;
    g.col_align = it->g.col_align;
    g.adj_ptr = it->g.adj_ptr;
    g.adj = it->g.adj;
    g.crac_rows = it->g.crac_rows;
    g.nnz = it->g.nnz;
    g.status = it->g.status;
    gather_node_rows<NLN, BB, MT, 4>(it->K, g, (const MT *)it->map, acc, cap, accumulate, it->values, u0, u1, 1,
                                     lane);
}

template <typename MT, bool CRAC>
__device__ __noinline__ void gather_row_generic_call(const BatchItemDev *__restrict__ it, int64_t v, double *acc,
                                                     int accumulate, int lane)
{
    const Geo g = it->g;
    gather_row_generic<MT, CRAC>(it->K, v, it->nln, it->B, g, (const MT *)it->map, (const MT *)it->mapc, acc,
                                 accumulate, it->values, lane);
}

template <typename MT, bool CRAC>
__device__ __forceinline__ void atomic_elem_any(const BatchItemDev *it, int shape, int64_t e, int lane,
                                                int64_t *base_s, int32_t *k_s, int32_t *off_s)
{
    switch (shape) {
    case SH_4_1: atomic_elem_call<4, 1, MT, CRAC>(it, e, lane); break;
    case SH_8_1: atomic_elem_call<8, 1, MT, CRAC>(it, e, lane); break;
    case SH_8_3: atomic_elem_call<8, 3, MT, CRAC>(it, e, lane); break;
    case SH_10_3: atomic_elem_call<10, 3, MT, CRAC>(it, e, lane); break;
    default: atomic_elem_generic_call<MT, CRAC>(it, e, lane, base_s, k_s, off_s);
    }
}

template <typename MT, bool CRAC>
__device__ __forceinline__ void gather_row_any(const BatchItemDev *it, int64_t v, double *acc, int accumulate, int lane)
{
    // shapes without a specialised per-tile path
    gather_row_generic_call<MT, CRAC>(it, v, acc, accumulate, lane);
}

// Slot of entry q of element e for any shape (thread-per-entry schedule).
template <typename MT, bool CRAC>
__device__ __forceinline__ int64_t entry_slot(const BatchItemDev &it, int64_t e, int q)
{
    const int B = it.B, nln = it.nln, n_loc = nln * B;
    const int r = q / n_loc, c = q - r * n_loc;
    const int kc = c / B;
    const int64_t row = (int64_t)B * it.g.N[e * nln + r / B] + r % B;
    int pos;
    int64_t base;
    if (!CRAC) {
        base = it.g.row_ptr[row];
        pos = (int)((const MT *)it.map)[(e * nln + r / B) * nln + kc];
    } else {
        base = crac_row_base(it.g, row);
        const int64_t rp = it.g.run_ptr[e];
        const int nr = (int)(it.g.run_ptr[e + 1] - rp);
        int k, off;
        run_of_multi(it.g.run_mask + e * it.g.mask_words, kc, k, off);
        pos = (int)((const MT *)it.mapc)[rp * nln + (int64_t)(r / B) * nr + k] + off;
    }
    return base + (int64_t)B * pos + c % B;
}

constexpr int SCHED_THREADS = 256;

// Shared memory of the warp-level schedules before the bulk-copy stages:
// per warp FE_MAX_NLOC row starts and 2 x FE_MAX_NLOC run entries.
__host__ __device__ constexpr size_t batch_tables_bytes(int warps)
{
    return (size_t)warps * FE_MAX_NLOC * 8 + (size_t)warps * 2 * FE_MAX_NLOC * 4;
}

// Block size of a schedule: 4-warp blocks for the row gather, 8-warp blocks
// for the others (4-warp blocks of the bulk-copy schedule measured slower).
constexpr int sched_threads(int sched) { return sched == FE_SCHED_WARP_PER_ROW ? 128 : SCHED_THREADS; }

// The row-gather schedule runs 4-warp blocks capped at 73 registers (7 blocks,
// 28 warps per SM): measured on the 256-mesh batch, 6.29 ms, against 6.54 ms
// with 8-warp blocks at 80 registers, 6.73 ms at 64 registers (which spilled
// in the per-tile call) and 7.65 ms at 128.
template <bool CRAC, int SCHED>
__global__ void __launch_bounds__(sched_threads(SCHED), SCHED == FE_SCHED_WARP_PER_ROW ? 7 : 1) k_batch(const BatchItemDev *__restrict__ items, int n_items,
                                                         int64_t t_lo, int64_t total_tiles, int tile, int cap,
                                                         int accumulate, unsigned long long *counter, int stage,
                                                         int *status, unsigned int *tc, int max_tiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long block_tile;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (SCHED == FE_SCHED_BLOCK_PER_ELEMENT) {
        int64_t *base_s = (int64_t *)smem_raw;            // [FE_MAX_NLOC] row starts
        int32_t *k_s = (int32_t *)(base_s + FE_MAX_NLOC);  // [FE_MAX_NLOC] run index (CRAC)
        int32_t *off_s = k_s + FE_MAX_NLOC;                // [FE_MAX_NLOC] offset in run (CRAC)
        for (int nt = 0; nt < max_tiles; ++nt) {
            if (threadIdx.x == 0) block_tile = (unsigned long long)t_lo + atomicAdd(counter, 1ull);
            __syncthreads();
            const unsigned long long t = block_tile;
            __syncthreads();
            if (t >= (unsigned long long)total_tiles) break;
            const int ii = find_item(items, n_items, (int64_t)t);
            const BatchItemDev &it = items[ii];
            const int64_t u0 = ((int64_t)t - it.tile_begin) * tile, u1 = min(u0 + tile, it.units);
            if (threadIdx.x == 0) tile_started(it, ii, tc);
            const int B = it.B, nln = it.nln, n_loc = nln * B;
            const int NN = n_loc * n_loc;
            for (int64_t e = u0; e < u1; ++e) {
                int64_t rp = 0;
                int nr = 0;
                if (CRAC) {
                    rp = it.g.run_ptr[e];
                    nr = (int)(it.g.run_ptr[e + 1] - rp);
                }
                for (int r = threadIdx.x; r < n_loc; r += blockDim.x) {
                    const int64_t row = (int64_t)B * it.g.N[e * nln + r / B] + r % B;
                    base_s[r] = CRAC ? crac_row_base(it.g, row) : it.g.row_ptr[row];
                }
                if (CRAC)
                    for (int kc = threadIdx.x; kc < nln; kc += blockDim.x)
                        run_of_multi(it.g.run_mask + e * it.g.mask_words, kc, k_s[kc], off_s[kc]);
                __syncthreads();
                for (int q = threadIdx.x; q < NN; q += blockDim.x) {
                    const int r = q / n_loc, c = q - r * n_loc;
                    const int kc = c / B;
                    int pos;
                    if (!CRAC) {
                        const int64_t mi = (e * nln + r / B) * nln + kc;
                        pos = it.map_bytes == 1 ? (int)((const uint8_t *)it.map)[mi] : (int)((const uint16_t *)it.map)[mi];
                    } else {
                        const int64_t mi = rp * nln + (int64_t)(r / B) * nr + k_s[kc];
                        pos = (it.map_bytes == 1 ? (int)((const uint8_t *)it.mapc)[mi]
                                                 : (int)((const uint16_t *)it.mapc)[mi]) + off_s[kc];
                    }
                    if (FE_IN_BOUNDS(base_s[r] + (int64_t)B * pos + c % B, it.g.nnz, it.g.status))
                        fe_red_add_f64(it.values + base_s[r] + (int64_t)B * pos + c % B, __ldcs(it.K + e * NN + q));
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) tile_finished(it, ii, tc, tile);
        }
        return;
    }
    // warp-level schedules
    const int nw = blockDim.x >> 5;
    double *acc = (double *)smem_raw + (size_t)wib * cap;                       // deterministic
    int64_t *base_s = (int64_t *)smem_raw + (size_t)wib * FE_MAX_NLOC;          // atomic, generic shapes
    int32_t *k_s = (int32_t *)((int64_t *)smem_raw + (size_t)nw * FE_MAX_NLOC) + (size_t)wib * 2 * FE_MAX_NLOC;
    int32_t *off_s = k_s + FE_MAX_NLOC;
    // FE_SCHED_WARP_PER_ELEMENT_TMA: two stages of `stage` doubles and two
    // mbarriers per warp, after the tables
    double *kst = (double *)(smem_raw + batch_tables_bytes(nw)) + (size_t)wib * 2 * stage;
    uint64_t *bar = (uint64_t *)(smem_raw + batch_tables_bytes(nw) + (size_t)nw * 2 * stage * 8) + 2 * wib;
    if constexpr (SCHED == FE_SCHED_WARP_PER_ELEMENT_TMA) {
        // tiles from the counter; a staged item's tile goes through the
        // warp's two stages in one call, other items take the register path
        if (lane == 0) {
            fe_mbar_init(&bar[0], 1);
            fe_mbar_init(&bar[1], 1);
            fe_fence_mbar_init();
        }
        __syncwarp();
        const uint64_t pol = fe_policy_evict_first();
        uint32_t phase = 0;
        for (int nt = 0; nt < max_tiles; ++nt) {
            unsigned long long t = 0;
            if (lane == 0) t = (unsigned long long)t_lo + atomicAdd(counter, 1ull);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= (unsigned long long)total_tiles) break;
            const int ii = find_item(items, n_items, (int64_t)t);
            const BatchItemDev &it = items[ii];
            const int64_t u0 = ((int64_t)t - it.tile_begin) * tile, u1 = min(u0 + tile, it.units);
            if (lane == 0) tile_started(it, ii, tc);
            if (it.staged) {
                const bool ok = it.map_bytes == 1
                                    ? staged_tile_any<uint8_t, CRAC>(&it, it.shape, u0, u1, lane, kst, stage, bar,
                                                                     &phase, base_s, k_s, pol)
                                    : staged_tile_any<uint16_t, CRAC>(&it, it.shape, u0, u1, lane, kst, stage, bar,
                                                                      &phase, base_s, k_s, pol);
                if (!ok) {
                    if (lane == 0) atomicCAS(status, 0, FE_ERR_TIMEOUT);
                    return;
                }
            } else {
                for (int64_t e = u0; e < u1; ++e) {
                    if (it.map_bytes == 1) atomic_elem_any<uint8_t, CRAC>(&it, it.shape, e, lane, base_s, k_s, off_s);
                    else atomic_elem_any<uint16_t, CRAC>(&it, it.shape, e, lane, base_s, k_s, off_s);
                }
            }
            __syncwarp();
            if (lane == 0) tile_finished(it, ii, tc, tile);
        }
    } else {
        for (int nt = 0; nt < max_tiles; ++nt) {
            unsigned long long t = 0;
            if (lane == 0) t = (unsigned long long)t_lo + atomicAdd(counter, 1ull);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= (unsigned long long)total_tiles) break;
            const int ii = find_item(items, n_items, (int64_t)t);
            const BatchItemDev &it = items[ii];
            const int64_t u0 = ((int64_t)t - it.tile_begin) * tile, u1 = min(u0 + tile, it.units);
            if (lane == 0) tile_started(it, ii, tc);
            if (SCHED == FE_SCHED_WARP_PER_ROW) {
                if (it.shape == SH_4_1 || it.shape == SH_8_1) {
                    // one-DOF rows: several per warp (gather_small.cuh)
                    if (it.shape == SH_4_1) {
                        if (it.map_bytes == 1) gather_tile_small<4, uint8_t, CRAC>(&it, u0, u1, acc, cap, accumulate, lane);
                        else gather_tile_small<4, uint16_t, CRAC>(&it, u0, u1, acc, cap, accumulate, lane);
                    } else {
                        if (it.map_bytes == 1) gather_tile_small<8, uint8_t, CRAC>(&it, u0, u1, acc, cap, accumulate, lane);
                        else gather_tile_small<8, uint16_t, CRAC>(&it, u0, u1, acc, cap, accumulate, lane);
                    }
                } else if (it.shape == SH_8_3 || it.shape == SH_10_3) {
                    if (it.shape == SH_8_3) {
                        if (it.map_bytes == 1) gather_tile_node<8, 3, uint8_t>(&it, u0, u1, acc, cap, accumulate, lane);
                        else gather_tile_node<8, 3, uint16_t>(&it, u0, u1, acc, cap, accumulate, lane);
                    } else {
                        if (it.map_bytes == 1) gather_tile_node<10, 3, uint8_t>(&it, u0, u1, acc, cap, accumulate, lane);
                        else gather_tile_node<10, 3, uint16_t>(&it, u0, u1, acc, cap, accumulate, lane);
                    }
                } else {
                    for (int64_t v = u0; v < u1; ++v) {
                        if (it.map_bytes == 1) gather_row_any<uint8_t, CRAC>(&it, v, acc, accumulate, lane);
                        else gather_row_any<uint16_t, CRAC>(&it, v, acc, accumulate, lane);
                    }
                }
            } else if (SCHED == FE_SCHED_WARP_PER_ELEMENT) {
                for (int64_t e = u0; e < u1; ++e) {
                    if (it.map_bytes == 1) atomic_elem_any<uint8_t, CRAC>(&it, it.shape, e, lane, base_s, k_s, off_s);
                    else atomic_elem_any<uint16_t, CRAC>(&it, it.shape, e, lane, base_s, k_s, off_s);
                }
            } else {  // thread per entry: the tile's entries spread over the lanes
                const int n_loc = it.nln * it.B;
                const int64_t NN = (int64_t)n_loc * n_loc;
                for (int64_t x = u0 * NN + lane; x < u1 * NN; x += 32) {
                    const int64_t e = x / NN;
                    const int q = (int)(x - e * NN);
                    const int64_t slot = it.map_bytes == 1 ? entry_slot<uint8_t, CRAC>(it, e, q)
                                                           : entry_slot<uint16_t, CRAC>(it, e, q);
                    if (FE_IN_BOUNDS(slot, it.g.nnz, it.g.status)) atomicAdd(it.values + slot, __ldcs(it.K + x));
                }
            }
            __syncwarp();
            if (lane == 0) tile_finished(it, ii, tc, tile);
        }
    }
}

// Zero every item's values (FE_ATOMIC without accumulation) in one launch.
__global__ void k_batch_zero(const BatchItemDev *__restrict__ items, int n_items)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int i = 0; i < n_items; ++i) {
        double *v = items[i].values;
        const int64_t n = items[i].nnz;
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) v[k] = 0.0;
    }
}

// FE_DETERMINISTIC items of one specialised 3-DOF shape with one-byte slot
// maps (the bulk of a batch of elasticity meshes): tiles [t_lo, t_hi) of
// items [i_lo, i_hi) through the single-mesh row loop, inlined, so that the
// kernel needs the registers of that loop alone (no per-shape dispatch, no
// call).  Incidences two at a time, 9 blocks of 4 warps per SM (56
// registers): measured on the 256-mesh batch, 5.78 ms, against 5.80 ms at 8
// blocks, 5.76 ms at 10 (more spills), 5.94 ms with four incidences at a
// time and 7 blocks, and 6.28 ms through the general kernel.
template <int NLN, int BB, bool CRAC>
__global__ void __launch_bounds__(128, 9) k_batch_rows(const BatchItemDev *__restrict__ items, int i_lo, int i_hi,
                                                       int64_t t_lo, int64_t t_hi, int tile, int cap, int accumulate,
                                                       unsigned long long *counter, unsigned int *tc, int max_tiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    double *acc = (double *)smem_raw + (size_t)(threadIdx.x >> 5) * cap;
    for (int nt = 0; nt < max_tiles; ++nt) {
        unsigned long long t = 0;
        if (lane == 0) t = (unsigned long long)t_lo + atomicAdd(counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)t_hi) break;
        const int ii = i_lo + find_item(items + i_lo, i_hi - i_lo, (int64_t)t);
        const BatchItemDev &it = items[ii];
        const int64_t u0 = ((int64_t)t - it.tile_begin) * tile, u1 = min(u0 + tile, it.units);
        if (lane == 0) tile_started(it, ii, tc);
        Geo g;
        if (CRAC) {
            g.crac_ptr = it.g.crac_ptr;
            g.col_align = it.g.col_align;
        } else {
            g.row_ptr = it.g.row_ptr;
        }
        g.adj_ptr = it.g.adj_ptr;
        g.adj = it.g.adj;
        g.crac_rows = CRAC ? 1 : 0;
        g.nnz = it.g.nnz;
        g.status = it.g.status;
        gather_node_rows<NLN, BB, uint8_t, 2>(it.K, g, (const uint8_t *)it.map, acc, cap, accumulate, it.values, u0,
                                              u1, 1, lane);
        __syncwarp();
        if (lane == 0) tile_finished(it, ii, tc, tile);
    }
}

// Items of one specialised class occupy a contiguous range of the plan.
struct RowClass {
    int shape = 0;
    int i_lo = 0, i_hi = 0;
    int64_t t_lo = 0, t_hi = 0;
};

struct Plan {
    std::vector<BatchItemDev> host;
    int64_t total_tiles = 0;
    int cap = 1;    // doubles of accumulator per warp (deterministic)
    int stage = 0;  // doubles per bulk-copy stage (FE_SCHED_WARP_PER_ELEMENT_TMA)
    // FE_DETERMINISTIC: the items of the specialised row classes come first,
    // one class after the other; the rest of the tiles [rest_t, total) go to
    // the general kernel
    std::vector<RowClass> classes;
    int64_t rest_t = 0;
};

// Counters of a batched launch: the general kernel's, one per row class,
// then two tile counters per item (per-item timestamps).
constexpr int BATCH_COUNTERS = 3;

// Largest K_e (doubles) a bulk-copy stage holds: 32 x 32.
constexpr int STAGE_MAX = 32 * 32;

int make_plan(fe_ctx *ctx, const fe_batch_item *items, int n, int format, int mode, int tile, Plan &plan)
{
    plan.host.resize(n);
    plan.total_tiles = 0;
    plan.cap = 1;
    plan.classes.clear();
    // FE_DETERMINISTIC: 3-DOF items with one-byte maps first, by shape, for
    // their specialised kernels; the rest keep their order after them
    std::vector<int> order;
    order.reserve(n);
    if (mode == FE_DETERMINISTIC) {
        for (int sh : {SH_8_3, SH_10_3}) {
            RowClass rc;
            rc.shape = sh;
            rc.i_lo = (int)order.size();
            for (int i = 0; i < n; ++i) {
                const fe_pattern *p = items[i].pattern;
                if (p && p->ctx == ctx && shape_of(p) == sh && p->map_bytes == 1) order.push_back(i);
            }
            rc.i_hi = (int)order.size();
            if (rc.i_hi > rc.i_lo) plan.classes.push_back(rc);
        }
    }
    {
        std::vector<char> taken(n, 0);
        for (int i : order) taken[i] = 1;
        for (int i = 0; i < n; ++i)
            if (!taken[i]) order.push_back(i);
    }
    for (int slot = 0; slot < n; ++slot) {
        const int i = order[slot];
        const fe_pattern *p = items[i].pattern;
        if (!p || p->ctx != ctx) return FE_ERR_INVALID_ARG;
        if ((p->n_e > 0 && !items[i].elem_mats) || (p->nnz > 0 && !items[i].values)) return FE_ERR_INVALID_ARG;
        if (((uintptr_t)items[i].elem_mats & 7u) || ((uintptr_t)items[i].values & 7u) ||
            ((uintptr_t)items[i].times_ns & 7u))
            return FE_ERR_INVALID_ARG;
        if (format == FE_FORMAT_CSR && !p->map_csr) return FE_ERR_NOT_BUILT;
        if (format == FE_FORMAT_CRAC && (!p->map_crac || !p->col_align || !p->map_crac_blk)) return FE_ERR_NOT_BUILT;
        if (mode == FE_DETERMINISTIC && !p->adj) return FE_ERR_NOT_BUILT;
        BatchItemDev &d = plan.host[slot];
        d.g = geo_of(p);
        d.K = items[i].elem_mats;
        d.values = items[i].values;
        d.map = p->map_csr;
        d.mapc = p->map_crac;
        d.shape = shape_of(p);
        if (format == FE_FORMAT_CRAC && mode == FE_DETERMINISTIC && (d.shape == SH_8_3 || d.shape == SH_10_3)) {
            // the CRAC gather of these shapes: expanded CRAC block map, CRAC row starts
            d.map = p->map_crac_blk;
            d.g.crac_rows = 1;
        }
        d.units = mode == FE_ATOMIC ? p->n_e : p->n_nodes;
        d.nnz = p->nnz;
        d.tile_begin = plan.total_tiles;
        d.nln = p->nln;
        d.B = p->B;
        d.map_bytes = p->map_bytes;
        const int nn = p->n_loc * p->n_loc;
        d.times = items[i].times_ns;
        d.staged = d.shape != SH_GENERIC && nn <= STAGE_MAX && (nn * 8) % 16 == 0 &&
                   ((uintptr_t)items[i].elem_mats & 15u) == 0;
        if (d.staged) plan.stage = std::max(plan.stage, (nn + 1) & ~1);
        plan.total_tiles += (d.units + tile - 1) / tile;
        plan.cap = std::max(plan.cap, p->B * p->max_row_len);
        // one-DOF rows of 4 or 8 nodes: SmallRows<>::RPW accumulators per warp
        if (d.shape == SH_4_1) plan.cap = std::max(plan.cap, SmallRows<4>::RPW * p->max_row_len);
        if (d.shape == SH_8_1) plan.cap = std::max(plan.cap, SmallRows<8>::RPW * p->max_row_len);
    }
    plan.rest_t = 0;
    for (RowClass &rc : plan.classes) {
        rc.t_lo = plan.host[rc.i_lo].tile_begin;
        rc.t_hi = rc.i_hi < n ? plan.host[rc.i_hi].tile_begin : plan.total_tiles;
        plan.rest_t = rc.t_hi;
    }
    return FE_OK;
}

size_t batch_smem(int mode, int sched, int cap, int stage)
{
    const int W = SCHED_THREADS / 32;
    if (mode == FE_DETERMINISTIC) return (size_t)(sched_threads(FE_SCHED_WARP_PER_ROW) / 32) * cap * 8;
    if (sched == FE_SCHED_BLOCK_PER_ELEMENT) return (size_t)FE_MAX_NLOC * 16;
    if (sched == FE_SCHED_WARP_PER_ELEMENT_TMA) {
        const int w = sched_threads(sched) / 32;
        return batch_tables_bytes(w) + (size_t)w * 2 * stage * 8 + (size_t)w * 16;
    }
    return batch_tables_bytes(W);
}

template <bool CRAC, int SCHED>
int launch_batch_t(fe_ctx *ctx, const BatchItemDev *d_items, int n, int64_t t_lo, int64_t total, int tile, int cap,
                   int acc, unsigned long long *counter, size_t smem, int stage, unsigned int *tc, double frac,
                   int max_tiles, cudaStream_t s)
{
    auto kern = k_batch<CRAC, SCHED>;
    constexpr int threads = sched_threads(SCHED);
    if (smem > 48 * 1024) FE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) return FE_ERR_UNSUPPORTED;
    const int64_t want = SCHED == FE_SCHED_BLOCK_PER_ELEMENT ? total - t_lo
                                                             : (total - t_lo + threads / 32 - 1) / (threads / 32);
    // frac < 1: the persistent grid takes only that share of the resident blocks
    const int64_t resident = std::max<int64_t>(1, (int64_t)((double)ctx->num_sms * per_sm * frac));
    int64_t blocks = std::min<int64_t>(resident, want);
    // max_tiles > 0: every warp (block) takes at most that many tiles, and the
    // grid has as many blocks as the tiles need
    if (max_tiles > 0) blocks = (want + max_tiles - 1) / max_tiles;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, INT32_MAX));
    kern<<<grid, threads, smem, s>>>(d_items, n, t_lo, total, tile, cap, acc, counter, stage, ctx->d_status, tc,
                                     max_tiles > 0 ? max_tiles : INT32_MAX);
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

int launch_batch(fe_ctx *ctx, const BatchItemDev *d_items, int n, int64_t t_lo, int64_t total, int format, int mode,
                 int acc, int sched, int tile, int cap, int stage, unsigned long long *counter, unsigned int *tc,
                 double frac, int max_tiles, cudaStream_t s)
{
    const size_t smem = batch_smem(mode, sched, cap, stage);
    if (smem > 200 * 1024) return FE_ERR_UNSUPPORTED;
    const bool crac = format == FE_FORMAT_CRAC;
    if (mode == FE_DETERMINISTIC)
        return crac ? launch_batch_t<true, FE_SCHED_WARP_PER_ROW>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s)
                    : launch_batch_t<false, FE_SCHED_WARP_PER_ROW>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s);
    switch (sched) {
    case FE_SCHED_THREAD_PER_ENTRY:
        return crac ? launch_batch_t<true, FE_SCHED_THREAD_PER_ENTRY>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s)
                    : launch_batch_t<false, FE_SCHED_THREAD_PER_ENTRY>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s);
    case FE_SCHED_BLOCK_PER_ELEMENT:
        return crac ? launch_batch_t<true, FE_SCHED_BLOCK_PER_ELEMENT>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s)
                    : launch_batch_t<false, FE_SCHED_BLOCK_PER_ELEMENT>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s);
    case FE_SCHED_WARP_PER_ELEMENT_TMA:
        return crac ? launch_batch_t<true, FE_SCHED_WARP_PER_ELEMENT_TMA>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s)
                    : launch_batch_t<false, FE_SCHED_WARP_PER_ELEMENT_TMA>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s);
    default:
        return crac ? launch_batch_t<true, FE_SCHED_WARP_PER_ELEMENT>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s)
                    : launch_batch_t<false, FE_SCHED_WARP_PER_ELEMENT>(ctx, d_items, n, t_lo, total, tile, cap, acc, counter, smem, stage, tc, frac, max_tiles, s);
    }
}

template <int NLN, int BB, bool CRAC>
int launch_rows_t(fe_ctx *ctx, const BatchItemDev *d_items, const RowClass &rc, int tile, int cap, int acc,
                  unsigned long long *counter, unsigned int *tc, double frac, int max_tiles, cudaStream_t s)
{
    auto kern = k_batch_rows<NLN, BB, CRAC>;
    const size_t smem = (size_t)4 * cap * 8;
    if (smem > 200 * 1024) return FE_ERR_UNSUPPORTED;
    if (smem > 48 * 1024) FE_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    if (per_sm < 1) return FE_ERR_UNSUPPORTED;
    const int64_t want = (rc.t_hi - rc.t_lo + 3) / 4;
    const int64_t resident = std::max<int64_t>(1, (int64_t)((double)ctx->num_sms * per_sm * frac));
    int64_t blocks = std::min<int64_t>(resident, want);
    if (max_tiles > 0) blocks = (want + max_tiles - 1) / max_tiles;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, INT32_MAX));
    kern<<<grid, 128, smem, s>>>(d_items, rc.i_lo, rc.i_hi, rc.t_lo, rc.t_hi, tile, cap, acc, counter, tc,
                                 max_tiles > 0 ? max_tiles : INT32_MAX);
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

// Every kernel of a planned batch on stream s: for FE_DETERMINISTIC the
// general kernel on the tiles outside the specialised row classes first
// (those items are the smaller ones of a mixed batch: they complete early),
// then the row classes; counters: BATCH_COUNTERS tile counters, then the
// per-item tile counts.
int launch_plan(fe_ctx *ctx, const BatchItemDev *d_items, int n, const Plan &plan, int format, int mode, int acc,
                const fe_schedule &sc, unsigned long long *counters, double frac, int max_tiles, cudaStream_t s)
{
    unsigned int *tc = (unsigned int *)(counters + BATCH_COUNTERS);
    const int64_t rest = plan.rest_t;
    if (plan.total_tiles > rest)
        FE_TRY(launch_batch(ctx, d_items, n, rest, plan.total_tiles, format, mode, acc, sc.kind, sc.tile, plan.cap,
                            plan.stage, counters, tc, frac, max_tiles, s));
    if (mode != FE_DETERMINISTIC) return FE_OK;
    for (size_t k = 0; k < plan.classes.size(); ++k) {
        const RowClass &rc = plan.classes[k];
        if (rc.t_hi <= rc.t_lo) continue;
        const bool crac = format == FE_FORMAT_CRAC;
        unsigned long long *ctr = counters + 1 + k;
        if (rc.shape == SH_8_3)
            FE_TRY(crac ? (launch_rows_t<8, 3, true>(ctx, d_items, rc, sc.tile, plan.cap, acc, ctr, tc, frac, max_tiles, s))
                        : (launch_rows_t<8, 3, false>(ctx, d_items, rc, sc.tile, plan.cap, acc, ctr, tc, frac, max_tiles, s)));
        else
            FE_TRY(crac ? (launch_rows_t<10, 3, true>(ctx, d_items, rc, sc.tile, plan.cap, acc, ctr, tc, frac, max_tiles, s))
                        : (launch_rows_t<10, 3, false>(ctx, d_items, rc, sc.tile, plan.cap, acc, ctr, tc, frac, max_tiles, s)));
    }
    return FE_OK;
}

bool sched_valid(int mode, const fe_schedule &sc)
{
    if (sc.tile < 1 || sc.tile > (1 << 20)) return false;
    if (mode == FE_DETERMINISTIC) return sc.kind == FE_SCHED_WARP_PER_ROW;
    return sc.kind == FE_SCHED_WARP_PER_ELEMENT || sc.kind == FE_SCHED_THREAD_PER_ENTRY ||
           sc.kind == FE_SCHED_BLOCK_PER_ELEMENT || sc.kind == FE_SCHED_WARP_PER_ELEMENT_TMA;
}

}  // namespace

// ---- per-context state: tuned schedules ----------------------------------

// Item tables reach the device through a ring of pinned host slots: a copy
// from pageable memory may wait for the stream's earlier work (the driver
// stages it), which would stall a caller that launches on several streams,
// such as the server's scheduler.  A slot is reused once the event recorded
// after its copy has completed.
constexpr int UPLOAD_SLOTS = 64;
constexpr size_t UPLOAD_SLOT_BYTES = 64 << 10;

struct fe_batch_state {
    std::mutex mu;
    std::map<std::tuple<int, int, uint64_t, int>, fe_schedule> tuned;  // (format, mode, shapes, size bucket)
    std::mutex up_mu;
    unsigned char *up_host = nullptr;  // UPLOAD_SLOTS x UPLOAD_SLOT_BYTES, pinned
    cudaEvent_t up_done[UPLOAD_SLOTS] = {};
    int up_next = 0;
    bool up_failed = false;
};

void fe_batch_state_destroy(fe_ctx *ctx)
{
    fe_batch_state *st = ctx->batch;
    if (st) {
        for (cudaEvent_t e : st->up_done)
            if (e) {
                cudaEventSynchronize(e);
                cudaEventDestroy(e);
            }
        if (st->up_host) cudaFreeHost(st->up_host);
    }
    delete ctx->batch;
    ctx->batch = nullptr;
}

namespace {

// ---- the autotuner's cache file --------------------------------------------
// With FEASM_TUNE_CACHE set to a path, tuned schedules persist across
// processes: one text line per entry, "<device> <format> <mode> <shapes>
// <size bucket> <kind> <tile>", where <device> names the GPU model and its SM
// count (schedules tuned on one GPU model are not taken on another) and
// <shapes> is the set of element shapes and map widths of the batch.  A
// context reads the entries of its device when it first batches; every
// autotune appends its result (later lines win).
std::string device_key(int device)
{
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string k = prop.name;
    for (char &c : k)
        if (c == ' ' || c == '\t') c = '_';
    return k + "_sm" + std::to_string(prop.multiProcessorCount);
}

void load_tune_cache(fe_ctx *ctx, fe_batch_state *st)
{
    const char *path = getenv("FEASM_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    const std::string key = device_key(ctx->device);
    char dev[256];
    int fmt, mode, bucket, kind, tile;
    unsigned long long shapes;
    while (fscanf(f, "%255s %d %d %llx %d %d %d", dev, &fmt, &mode, &shapes, &bucket, &kind, &tile) == 7) {
        if (key == dev && sched_valid(mode, fe_schedule{kind, tile}))
            st->tuned[std::make_tuple(fmt, mode, (uint64_t)shapes, bucket)] = fe_schedule{kind, tile};
    }
    fclose(f);
}

void store_tune_cache(fe_ctx *ctx, const std::tuple<int, int, uint64_t, int> &sig, const fe_schedule &sc)
{
    const char *path = getenv("FEASM_TUNE_CACHE");
    if (!path || !*path) return;
    static std::mutex file_mu;  // appends from several contexts of this process
    std::lock_guard<std::mutex> lk(file_mu);
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %llx %d %d %d\n", device_key(ctx->device).c_str(), std::get<0>(sig), std::get<1>(sig),
            (unsigned long long)std::get<2>(sig), std::get<3>(sig), sc.kind, sc.tile);
    fclose(f);
}

fe_batch_state *state_of(fe_ctx *ctx)
{
    static std::mutex create_mu;
    std::lock_guard<std::mutex> lk(create_mu);
    if (!ctx->batch) {
        ctx->batch = new fe_batch_state();
        load_tune_cache(ctx, ctx->batch);
    }
    return ctx->batch;
}

std::tuple<int, int, uint64_t, int> signature(const fe_batch_item *items, int n, int format, int mode)
{
    uint64_t shapes = 0;
    int64_t units = 0;
    for (int i = 0; i < n; ++i) {
        const fe_pattern *p = items[i].pattern;
        shapes |= 1ull << (shape_of(p) * 8 + std::min(p->map_bytes, 2));
        units += (int64_t)p->n_e * p->n_loc * p->n_loc;
    }
    int bucket = 0;
    while ((1ll << bucket) < units && bucket < 62) ++bucket;
    return std::make_tuple(format, mode, shapes, bucket / 2);
}

fe_schedule default_schedule(int mode)
{
    // measured on 256 hex meshes (n ~ logU[8,48]): tiles of 8 elements keep the warps on
    // neighbouring elements (atomics hit L2) at few tile fetches
    return mode == FE_DETERMINISTIC ? fe_schedule{FE_SCHED_WARP_PER_ROW, 64}
                                    : fe_schedule{FE_SCHED_WARP_PER_ELEMENT_TMA, 8};
}

struct DeviceScope {
    int prev = -1, dev;
    explicit DeviceScope(int d) : dev(d)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
};

// Copy n bytes of host data to dst on stream s through a pinned slot (the
// pageable copy when the table is larger than a slot or pinned memory could
// not be had).
int upload(fe_ctx *ctx, void *dst, const void *src, size_t n, cudaStream_t s)
{
    fe_batch_state *st = state_of(ctx);
    if (n <= UPLOAD_SLOT_BYTES) {
        std::lock_guard<std::mutex> lk(st->up_mu);
        if (!st->up_host && !st->up_failed) {
            bool ok = cudaHostAlloc((void **)&st->up_host, UPLOAD_SLOTS * UPLOAD_SLOT_BYTES, cudaHostAllocPortable) ==
                      cudaSuccess;
            for (int k = 0; ok && k < UPLOAD_SLOTS; ++k)
                ok = cudaEventCreateWithFlags(&st->up_done[k], cudaEventDisableTiming) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                st->up_failed = true;
            }
        }
        if (st->up_host && !st->up_failed) {
            const int k = st->up_next;
            st->up_next = (k + 1) % UPLOAD_SLOTS;
            FE_CUDA(cudaEventSynchronize(st->up_done[k]));  // the slot's previous copy (long done, normally)
            unsigned char *slot = st->up_host + (size_t)k * UPLOAD_SLOT_BYTES;
            memcpy(slot, src, n);
            FE_CUDA(cudaMemcpyAsync(dst, slot, n, cudaMemcpyHostToDevice, s));
            FE_CUDA(cudaEventRecord(st->up_done[k], s));
            return FE_OK;
        }
    }
    FE_CUDA(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s));
    return FE_OK;
}

// Plan upload + launch on stream s.  The item table and the tile counter are
// stream-ordered allocations freed after the launch.
int run_batch(fe_ctx *ctx, const fe_batch_item *items, int n, int format, int mode, int acc, fe_schedule sc,
              cudaStream_t s, double frac = 1.0, int max_tiles = 0)
{
    Plan plan;
    FE_TRY(make_plan(ctx, items, n, format, mode, sc.tile, plan));
    BatchItemDev *d_items = nullptr;
    unsigned long long *counter = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&d_items, sizeof(BatchItemDev) * n, s));
    // the tile counters, then two tile counters per item (per-item timestamps)
    const size_t cbytes = sizeof(unsigned long long) * BATCH_COUNTERS + sizeof(unsigned int) * 2 * (size_t)n;
    int rc = fe_alloc(ctx, (void **)&counter, cbytes, s);
    if (rc == FE_OK) rc = upload(ctx, d_items, plan.host.data(), sizeof(BatchItemDev) * n, s);
    if (rc == FE_OK && cudaMemsetAsync(counter, 0, cbytes, s) != cudaSuccess) rc = FE_ERR_DEVICE;
    if (rc == FE_OK && mode == FE_ATOMIC && !acc) {
        k_batch_zero<<<ctx->num_sms * 4, 256, 0, s>>>(d_items, n);
        fe_note_launch();
        if (cudaGetLastError() != cudaSuccess) rc = FE_ERR_DEVICE;
    }
    if (rc == FE_OK && plan.total_tiles > 0)
        rc = launch_plan(ctx, d_items, n, plan, format, mode, acc, sc, counter, frac, max_tiles, s);
    fe_free_async(d_items, s);
    fe_free_async(counter, s);
    return rc;
}

}  // namespace

struct fe_batch_graph {
    fe_ctx *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchItemDev *d_items = nullptr;
    unsigned long long *counter = nullptr;
};

extern "C" {

int fe_assemble_batch(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                      int32_t accumulate, const fe_schedule *sched, void *stream)
{
    if (!ctx || n_items < 0 || (n_items > 0 && !items)) return FE_ERR_INVALID_ARG;
    if ((format != FE_FORMAT_CSR && format != FE_FORMAT_CRAC) || (mode != FE_ATOMIC && mode != FE_DETERMINISTIC) ||
        (accumulate != 0 && accumulate != 1))
        return FE_ERR_INVALID_ARG;
    if (n_items == 0) return FE_OK;
    FeRange range("fe_assemble_batch");
    DeviceScope ds(ctx->device);
    fe_schedule sc = default_schedule(mode);
    if (sched) {
        sc = *sched;
        if (!sched_valid(mode, sc)) return FE_ERR_INVALID_ARG;
    } else {
        fe_batch_state *st = state_of(ctx);
        std::lock_guard<std::mutex> lk(st->mu);
        auto it = st->tuned.find(signature(items, n_items, format, mode));
        if (it != st->tuned.end()) sc = it->second;
    }
    return run_batch(ctx, items, n_items, format, mode, accumulate, sc, (cudaStream_t)stream);
}

}  // extern "C"

// fe_assemble_batch (sched = NULL) whose persistent grid takes only `frac` of
// the resident blocks: the server launches large requests this way, so that
// pattern builds and small requests always find free SMs (a persistent grid
// holds every SM until its last tile is done, and a running block is never
// preempted by a higher-priority stream's).
int fe_assemble_batch_share(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                            int32_t accumulate, void *stream, double frac, int max_tiles)
{
    if (!ctx || n_items <= 0 || !items || !(frac > 0.0 && frac <= 1.0)) return FE_ERR_INVALID_ARG;
    if ((format != FE_FORMAT_CSR && format != FE_FORMAT_CRAC) || (mode != FE_ATOMIC && mode != FE_DETERMINISTIC) ||
        (accumulate != 0 && accumulate != 1))
        return FE_ERR_INVALID_ARG;
    FeRange range("fe_assemble_batch (share of the GPU)");
    DeviceScope ds(ctx->device);
    fe_schedule sc = default_schedule(mode);
    {
        fe_batch_state *st = state_of(ctx);
        std::lock_guard<std::mutex> lk(st->mu);
        auto it = st->tuned.find(signature(items, n_items, format, mode));
        if (it != st->tuned.end()) sc = it->second;
    }
    return run_batch(ctx, items, n_items, format, mode, accumulate, sc, (cudaStream_t)stream, frac, max_tiles);
}

extern "C" {

int fe_batch_tuned(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                   fe_schedule *out)
{
    if (!ctx || n_items <= 0 || !items || !out) return FE_ERR_INVALID_ARG;
    if ((format != FE_FORMAT_CSR && format != FE_FORMAT_CRAC) || (mode != FE_ATOMIC && mode != FE_DETERMINISTIC))
        return FE_ERR_INVALID_ARG;
    for (int i = 0; i < n_items; ++i)
        if (!items[i].pattern) return FE_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    fe_batch_state *st = state_of(ctx);
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->tuned.find(signature(items, n_items, format, mode));
    if (it == st->tuned.end()) return FE_ERR_NOT_FOUND;
    *out = it->second;
    return FE_OK;
}

int fe_batch_autotune(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                      void *stream, fe_schedule *best, float *best_ms)
{
    if (!ctx || n_items <= 0 || !items) return FE_ERR_INVALID_ARG;
    if ((format != FE_FORMAT_CSR && format != FE_FORMAT_CRAC) || (mode != FE_ATOMIC && mode != FE_DETERMINISTIC))
        return FE_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<fe_schedule> cands;
    // one atomic tile fetch per warp (or block) per tile: larger tiles mean
    // fewer same-address atomics on the work counter
    if (mode == FE_DETERMINISTIC) {
        for (int t : {4, 16, 64, 256, 1024}) cands.push_back({FE_SCHED_WARP_PER_ROW, t});
    } else {
        for (int t : {4, 16, 64, 256, 1024}) cands.push_back({FE_SCHED_WARP_PER_ELEMENT, t});
        for (int t : {6, 8, 12, 16}) cands.push_back({FE_SCHED_WARP_PER_ELEMENT_TMA, t});
        for (int t : {4, 32}) cands.push_back({FE_SCHED_THREAD_PER_ENTRY, t});
        for (int t : {1, 8}) cands.push_back({FE_SCHED_BLOCK_PER_ELEMENT, t});
    }
    cudaEvent_t e0, e1;
    FE_CUDA(cudaEventCreate(&e0));
    FE_CUDA(cudaEventCreate(&e1));
    fe_schedule win = cands[0];
    float win_ms = 1e30f;
    int rc = FE_OK;
    for (const fe_schedule &sc : cands) {
        rc = run_batch(ctx, items, n_items, format, mode, 0, sc, s);  // warm-up
        if (rc == FE_ERR_UNSUPPORTED) continue;
        if (rc != FE_OK) break;
        float best_rep = 1e30f;
        for (int rep = 0; rep < 3 && rc == FE_OK; ++rep) {
            cudaEventRecord(e0, s);
            rc = run_batch(ctx, items, n_items, format, mode, 0, sc, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = FE_ERR_DEVICE;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best_rep = std::min(best_rep, ms);
        }
        if (rc != FE_OK) break;
        if (best_rep < win_ms) {
            win_ms = best_rep;
            win = sc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != FE_OK) return rc;
    {
        fe_batch_state *st = state_of(ctx);
        const auto sig = signature(items, n_items, format, mode);
        {
            std::lock_guard<std::mutex> lk(st->mu);
            st->tuned[sig] = win;
        }
        store_tune_cache(ctx, sig, win);
    }
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return FE_OK;
}

int fe_batch_graph_create(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                          int32_t accumulate, const fe_schedule *sched, void *stream, fe_batch_graph **out)
{
    if (!ctx || !out || n_items <= 0 || !items) return FE_ERR_INVALID_ARG;
    if ((format != FE_FORMAT_CSR && format != FE_FORMAT_CRAC) || (mode != FE_ATOMIC && mode != FE_DETERMINISTIC) ||
        (accumulate != 0 && accumulate != 1))
        return FE_ERR_INVALID_ARG;
    *out = nullptr;
    DeviceScope ds(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe_schedule sc = default_schedule(mode);
    if (sched) {
        sc = *sched;
        if (!sched_valid(mode, sc)) return FE_ERR_INVALID_ARG;
    } else {
        fe_batch_state *st = state_of(ctx);
        std::lock_guard<std::mutex> lk(st->mu);
        auto it = st->tuned.find(signature(items, n_items, format, mode));
        if (it != st->tuned.end()) sc = it->second;
    }
    Plan plan;
    FE_TRY(make_plan(ctx, items, n_items, format, mode, sc.tile, plan));
    fe_batch_graph *g = new fe_batch_graph();
    g->ctx = ctx;
    int rc = FE_OK;
    // the graph's own item table and counter live as long as the graph
    const size_t cbytes = sizeof(unsigned long long) * BATCH_COUNTERS + sizeof(unsigned int) * 2 * (size_t)n_items;
    if (cudaMalloc((void **)&g->d_items, sizeof(BatchItemDev) * n_items) != cudaSuccess ||
        cudaMalloc((void **)&g->counter, cbytes) != cudaSuccess)
        rc = FE_ERR_OOM;
    // uploaded on the caller's stream (ordered after the work that built the patterns)
    if (rc == FE_OK && (cudaMemcpyAsync(g->d_items, plan.host.data(), sizeof(BatchItemDev) * n_items,
                                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        rc = FE_ERR_DEVICE;
    cudaStream_t cs = nullptr;
    if (rc == FE_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = FE_ERR_DEVICE;
    if (rc == FE_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = FE_ERR_DEVICE;
    if (rc == FE_OK) {
        int lrc = cudaMemsetAsync(g->counter, 0, cbytes, cs) == cudaSuccess ? FE_OK : FE_ERR_DEVICE;
        if (lrc == FE_OK && mode == FE_ATOMIC && !accumulate) {
            k_batch_zero<<<ctx->num_sms * 4, 256, 0, cs>>>(g->d_items, n_items);
            if (cudaGetLastError() != cudaSuccess) lrc = FE_ERR_DEVICE;
        }
        if (lrc == FE_OK && plan.total_tiles > 0)
            lrc = launch_plan(ctx, g->d_items, n_items, plan, format, mode, accumulate, sc, g->counter, 1.0, 0, cs);
        const cudaError_t ec = cudaStreamEndCapture(cs, &g->graph);
        rc = lrc != FE_OK ? lrc : (ec == cudaSuccess ? FE_OK : FE_ERR_DEVICE);
    }
    if (rc == FE_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = FE_ERR_DEVICE;
    if (cs) cudaStreamDestroy(cs);
    if (rc != FE_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->d_items) cudaFree(g->d_items);
        if (g->counter) cudaFree(g->counter);
        delete g;
        return rc;
    }
    *out = g;
    return FE_OK;
}

int fe_batch_graph_launch(fe_batch_graph *g, void *stream)
{
    if (!g) return FE_ERR_INVALID_ARG;
    DeviceScope ds(g->ctx->device);
    FE_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    fe_note_launch();
    return FE_OK;
}

int fe_batch_graph_destroy(fe_batch_graph *g)
{
    if (!g) return FE_ERR_INVALID_ARG;
    DeviceScope ds(g->ctx->device);
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->d_items) cudaFree(g->d_items);
    if (g->counter) cudaFree(g->counter);
    delete g;
    return FE_OK;
}

}  // extern "C"

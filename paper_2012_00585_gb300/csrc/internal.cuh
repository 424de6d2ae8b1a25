// Internal definitions shared by the translation units of libfeasm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstddef>

#include "../../include/feasm.h"

// A named range on a profiler's timeline (NVTX) for the lifetime of the
// object: the library's phases (pattern build steps, numeric assemblies,
// batched launches, the server's launches and builds) show up by name in
// Nsight Systems and can be selected in Nsight Compute (--nvtx).  Without a
// tool attached a range costs a few nanoseconds.
struct FeRange {
    explicit FeRange(const char *name) { nvtxRangePushA(name); }
    ~FeRange() { nvtxRangePop(); }
    FeRange(const FeRange &) = delete;
    FeRange &operator=(const FeRange &) = delete;
};

// Consecutive phases of one call as sibling ranges (next() closes the
// current one and opens the next; early returns close the open one).
struct FePhase {
    explicit FePhase(const char *name) { nvtxRangePushA(name); }
    void next(const char *name)
    {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~FePhase() { nvtxRangePop(); }
    FePhase(const FePhase &) = delete;
    FePhase &operator=(const FePhase &) = delete;
};

#define FE_WARP 32

// Return an FE_* code from the enclosing function when a CUDA call fails.
#define FE_CUDA(call)                                                               \
    do {                                                                            \
        cudaError_t fe_e_ = (call);                                                 \
        if (fe_e_ != cudaSuccess) {                                                 \
            fe_set_last_cuda_error(fe_e_, #call, __LINE__);                         \
            return fe_e_ == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_DEVICE; \
        }                                                                           \
    } while (0)

#define FE_TRY(expr)                        \
    do {                                    \
        int fe_rc_ = (expr);                \
        if (fe_rc_ != FE_OK) return fe_rc_; \
    } while (0)

void fe_set_last_cuda_error(cudaError_t e, const char *what, int line);

struct fe_ctx {
    int device = 0;
    int num_sms = 0;
    size_t hbm_budget = 0;
    size_t pool_limit = 0;  // fe_create_ex: bound on the pool's bytes in use (0 = none)
    cudaMemPool_t pool = nullptr;
    int *d_status = nullptr;  // device status word: first FE_ERR_* a kernel recorded
    int knob[FE_KNOB_COUNT] = {};  // schedule choices (0 = library default)
    struct fe_batch_state *batch = nullptr;  // batching / serving scheduler
};

// A pattern is built at the level of DOF blocks ("nodes"): when every
// element lists its DOFs in groups of B consecutive indices starting at a
// multiple of B (dof = B*node + comp), all B rows of a node share one column
// structure, so adjacency, row unions and slot maps are computed per node and
// expanded.  B = 1 is the general case.
struct fe_pattern {
    fe_ctx *ctx = nullptr;
    int64_t n_e = 0;
    int32_t n_loc = 0;
    int32_t B = 1;            // DOFs per block
    int32_t nln = 0;          // blocks per element = n_loc / B
    int32_t mask_words = 0;   // 32-bit words per element in run_mask (nln bits)
    int64_t n_dofs = 0;
    int64_t n_nodes = 0;      // n_dofs / B
    int64_t nnz = 0;
    int64_t n_ca = 0;
    int64_t n_runs = 0;       // sum over elements of block runs
    int32_t max_row_len = 0;  // DOF-level
    int32_t max_node_len = 0; // blocks per block row
    int32_t max_deg = 0;      // elements sharing one block
    int32_t map_bytes = 1;
    uint32_t flags = 0;
    int64_t device_bytes = 0;
    bool uniform_runs = false;  // every element has the same run mask
    int32_t runs_per_elem = 0;  // valid when uniform_runs

    int32_t *node_dofs = nullptr;  // [n_e * nln] block ids per element
    int64_t *row_ptr = nullptr;    // [n_dofs + 1]
    int32_t *col_idx = nullptr;    // [nnz]
    int64_t *crac_ptr = nullptr;   // [n_dofs + 1], int units
    int32_t *col_align = nullptr;  // [n_ca]
    int64_t *adj_ptr = nullptr;    // [n_nodes + 1]
    uint32_t *adj = nullptr;       // [n_e * nln] ids e*nln + k, ascending per block row
    void *map_csr = nullptr;       // [n_e * nln * nln] uint8/uint16: block position in block row
    uint32_t *run_mask = nullptr;  // [n_e * mask_words] run starts over the element's blocks
    int64_t *run_ptr = nullptr;    // [n_e + 1]
    void *map_crac = nullptr;      // [n_runs * nln] uint8/uint16: run start position in block row
    // [n_e * nln * nln] uint8/uint16: the CRAC run map expanded to one entry
    // per column block (run start + offset in the run), for the CRAC gather
    void *map_crac_blk = nullptr;
    // [n_e] elements grouped by compact clusters of the block graph, the
    // order of the atomic scatter on scattered numberings (null: ascending)
    int32_t *elem_order = nullptr;
    // set only on a numeric-phase view of the pattern: row starts are read
    // from the CRAC pairs (the CRAC gather through map_crac_blk)
    bool crac_rows = false;
    struct fe_colouring *colouring = nullptr;  // greedy element colouring (fe_pattern_colour)
};

void fe_colouring_free(fe_pattern *p, cudaStream_t s);
int fe_assemble_coloured(const fe_pattern *p, const double *K, double *values, int accumulate, bool crac,
                         cudaStream_t s);
int fe_assemble_rowlock(const fe_pattern *p, const double *K, double *values, int accumulate, bool crac,
                        cudaStream_t s);

void fe_batch_state_destroy(fe_ctx *ctx);
// fe_assemble_batch with the persistent grid limited to a share of the GPU
// (batch.cu; used by the server for large requests), or, with max_tiles > 0,
// with blocks that take at most max_tiles tiles per warp and exit (a grid of
// as many blocks as the tiles need), so that the SMs turn over every few
// tiles and kernels of higher-priority streams get them quickly (the
// server's small groups).
int fe_assemble_batch_share(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                            int32_t accumulate, void *stream, double frac, int max_tiles = 0);

// Host-side count of kernel launches made by this library (all threads).
void fe_note_launch();

// Stream-ordered allocation from the context's pool.
int fe_alloc(fe_ctx *ctx, void **p, size_t bytes, cudaStream_t s);
void fe_free_async(void *p, cudaStream_t s);

// Exclusive scan of n counts into out[0..n]; out[n] = total.
int fe_scan_i32_to_i64(fe_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);
int fe_scan_i64(fe_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Debug builds (-DFE_DEBUG) check device indices before the accesses that
// use FE_IN_BOUNDS: an index outside [0, n) records FE_ERR_DEVICE in the
// context's status word and the access is skipped (nothing traps).  Release
// builds compile the checks away.
#ifdef FE_DEBUG
__device__ __forceinline__ bool fe_in_bounds(int64_t i, int64_t n, int *status)
{
    if (i >= 0 && i < n) return true;
    if (status) atomicCAS(status, 0, FE_ERR_DEVICE);
    return false;
}
#define FE_IN_BOUNDS(i, n, st) fe_in_bounds((int64_t)(i), (int64_t)(n), (st))
#else
#define FE_IN_BOUNDS(i, n, st) true
#endif

static inline int fe_grid_for(int64_t work, int threads, int num_sms, int per_sm = 8)
{
    int64_t blocks = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// Resident blocks per SM of a kernel at this block shape (cached per kernel,
// block size and dynamic shared memory; at least 1).
int fe_resident_blocks(const void *kernel, int threads, size_t smem);

// Grid of a grid-strided kernel: enough blocks for `work` threads, at most
// one full wave of resident blocks (a partial second wave would hold a
// share of the strided work at low occupancy).
template <typename KernelT>
inline int fe_grid_resident(KernelT kernel, int64_t work, int threads, int num_sms, size_t smem = 0)
{
    return fe_grid_for(work, threads, num_sms, fe_resident_blocks((const void *)kernel, threads, smem));
}

// FP64 add into global memory whose old value is not needed: issued as a
// reduction (RED, performed in L2, nothing returned), with no compiler
// memory barrier, so independent loads may be scheduled across it.
__device__ __forceinline__ void fe_red_add_f64(double *p, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v));
}

__device__ __forceinline__ int64_t fe_warp_id() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t fe_warps() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

/*
 * feasm.h -- C ABI of a GB300 (sm_103a) library that assembles dense finite
 * element matrices into a global sparse matrix, after Sky et al., "A flexible
 * sparse matrix data format and parallel algorithms for the assembly of
 * sparse matrices in general finite element applications using atomic
 * synchronisation primitives" (arXiv 2012.00585).
 *
 * The problem (§2.1): n_e elements, each with a dense row-major matrix K_e of
 * n_loc x n_loc doubles and an element_dofs_array D_e of n_loc global DOF
 * indices.  Assembly adds K_e(r, c) into G(D_e(r), D_e(c)) for every element
 * (Listing 2).  G is stored in CSR or in CRAC (§2.2, Fig. 1); both share one
 * values array.  The sparsity pattern is built once and reused by every
 * numeric assembly; values are reset between assemblies (§3).
 *
 * Conventions
 *   - Indices are 0-based.  DOFs are int32 in [0, n_dofs); n_dofs rows and
 *     n_dofs columns.
 *   - Pointers documented "device" must point to memory of the context's
 *     device; "host" pointers to host memory.  Sizes are element counts.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without waiting, except
 *     where stated.
 *   - Every call returns FE_OK (0) or a negative FE_ERR_* code; no exception
 *     crosses this boundary and no kernel traps.  fe_strerror() names a code.
 *   - Not thread-safe per context unless stated; distinct contexts are
 *     independent.
 */
#ifndef FEASM_H
#define FEASM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define FE_OK 0
#define FE_ERR_INVALID_ARG (-1)   /* bad pointer, size or flag                 */
#define FE_ERR_DOF_RANGE (-2)     /* a DOF outside [0, n_dofs)                 */
#define FE_ERR_DUP_DOF (-3)       /* a DOF listed twice in one element         */
#define FE_ERR_OVERFLOW (-4)      /* nnz or n_ca >= 2^31, or n_e*n_loc >= 2^32 */
#define FE_ERR_OOM (-5)           /* device allocation failed                  */
#define FE_ERR_ADMISSION (-6)     /* request larger than the HBM budget        */
#define FE_ERR_TIMEOUT (-7)       /* a bounded device or host wait ran out     */
#define FE_ERR_DEVICE (-8)        /* a CUDA call failed                        */
#define FE_ERR_NOT_BUILT (-9)     /* the pattern lacks the requested part      */
#define FE_ERR_UNSUPPORTED (-10)  /* size beyond an implementation limit       */
#define FE_ERR_NOT_FOUND (-11)    /* unknown ticket                            */
#define FE_ERR_CANCELLED (-12)    /* request cancelled before it ran           */

/* Largest element supported (DOFs per element). */
#define FE_MAX_NLOC 128

/* ---- pattern parts (fe_pattern_build flags) ----------------------------- */
#define FE_PATTERN_CSR 0x1u       /* row_ptr + col_idx (always built)          */
#define FE_PATTERN_CRAC 0x2u      /* CRAC row pointers + column alignments     */
#define FE_PATTERN_MAP_CSR 0x4u   /* per-entry slot map for fe_assemble_csr    */
#define FE_PATTERN_MAP_CRAC 0x8u  /* per-run slot map for fe_assemble_crac     */
#define FE_PATTERN_ADJ 0x10u      /* block adjacency (always built; used by
                                     FE_DETERMINISTIC)                        */
#define FE_PATTERN_ALL 0x1Fu

/* ---- numeric modes ------------------------------------------------------ */
#define FE_ATOMIC 0         /* element-parallel scatter with FP64 atomic adds
                               (Listing 3); sum order is unspecified          */
#define FE_DETERMINISTIC 1  /* row-parallel gather, no atomics; every value is
                               summed in ascending element order from +0.0
                               (Listing 2's order), bit-reproducible          */
#define FE_COLOURED 2       /* colour after colour, elements of one colour in
                               parallel with plain adds (Listing 6); needs
                               fe_pattern_colour; every value is summed in
                               colour order (ascending element within a
                               colour), bit-reproducible                      */
#define FE_ROWLOCK 3        /* element-parallel, each row of K_e added under
                               the row's spin_int lock (Listings 3-5): the
                               row pointer itself is the lock (locked value
                               ~v), taken with a bounded spin; sum order
                               unspecified.  The pattern's row pointers change
                               while it runs: no other work on this pattern
                               may run concurrently.                          */

typedef struct fe_ctx fe_ctx;
typedef struct fe_pattern fe_pattern;

typedef struct fe_pattern_info {
    int64_t n_elem;        /* n_e                                          */
    int32_t n_loc;         /* DOFs per element                             */
    int32_t map_bytes;     /* 1 or 2: width of the slot-map entries        */
    int64_t n_dofs;        /* rows = columns                               */
    int64_t nnz;           /* CSR entries = length of the values array     */
    int64_t n_ca;          /* length of the CRAC column-alignments array   */
    int64_t n_elem_runs;   /* sum over elements of maximal DOF runs (§2.1) */
    int32_t max_row_len;   /* longest CSR row                              */
    int32_t max_degree;    /* most elements sharing one DOF                */
    uint32_t flags;        /* parts that were built                        */
    int32_t block;         /* DOFs per block B found in the connectivity:
                              every element lists whole blocks
                              B*node .. B*node+B-1 (1 = no blocking)       */
    int32_t uniform_runs;  /* 1 when all elements share one run layout     */
    int32_t atomic_order;  /* 1 when FE_ATOMIC takes the elements in a
                              locality order (FE_KNOB_ATOMIC_ORDER)        */
    int64_t device_bytes;  /* device memory held by the pattern            */
} fe_pattern_info;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` bounds the
 * device memory the batching/serving scheduler admits at once (0 = 90 % of
 * the device's free memory at creation).  The context owns a stream-ordered
 * memory pool for patterns and workspace.  *out receives the handle. */
int fe_create(fe_ctx **out, int device, size_t hbm_budget_bytes);

/* fe_create with an upper bound on the context's memory pool: every device
 * allocation the library makes for this context (patterns, workspace) comes
 * from the pool, and one that would take it past `pool_limit_bytes` fails
 * with FE_ERR_OOM, cleanly (the call releases what it had allocated; the
 * context stays usable).  0 = no bound beyond the device's. */
int fe_create_ex(fe_ctx **out, int device, size_t hbm_budget_bytes, size_t pool_limit_bytes);

/* Destroy a context: waits for its device work, then frees its memory.  Every
 * pattern created from it must have been freed. */
int fe_destroy(fe_ctx *ctx);

/* Static string for an FE_* code (never NULL). */
const char *fe_strerror(int code);

/* Text of the last CUDA error this thread's calls met (for FE_ERR_DEVICE /
 * FE_ERR_OOM diagnostics); empty when there was none.  Never NULL. */
const char *fe_last_cuda_error(void);

/* Waits for `stream`, then returns the first error a kernel of this context
 * recorded on the device since the last call (FE_OK if none) and clears it.
 * Kernels record instead of trapping: a bounded wait that ran out gives
 * FE_ERR_TIMEOUT and the kernel returns early, leaving its output
 * incomplete. */
int fe_device_status(fe_ctx *ctx, void *stream);

/* Number of kernels this library has launched in this process so far (all
 * contexts and threads); a caller brackets a region with two reads to count
 * the launches inside it. */
uint64_t fe_kernel_launches(void);

/* 1 when this library was built with its device index checks (-DFE_DEBUG;
 * an index outside its array then records FE_ERR_DEVICE in the context's
 * status word and the access is skipped), 0 for the release build. */
int fe_debug_checks(void);

/* ---- schedule knobs ------------------------------------------------------
 * Kernel and launch-shape choices of the numeric phase, per context.  0 means
 * the library's default; an autotuner may set them.  Results do not depend on
 * them (FE_DETERMINISTIC stays bit-identical), only speed does. */
#define FE_KNOB_GATHER_KERNEL 0  /* FE_DETERMINISTIC: 0 default (2 for node
                                    rows whose incidence slices hold <= 16
                                    entries, else 1), 1 one warp per node
                                    row, incidences batched in registers, 2
                                    several node rows per warp (4, 8 or 16
                                    lanes each; slices of <= 16 entries)    */
#define FE_KNOB_GATHER_BATCH 1   /* incidences per register batch: 4 or 8   */
#define FE_KNOB_GATHER_WARPS 2   /* warps per block of the gather: 1..8      */
#define FE_KNOB_ATOMIC_KERNEL 3  /* FE_ATOMIC: 0 default (1), 1 register
                                    warp-per-element, 2 bulk-copy (TMA)
                                    staged warp-per-element                 */
#define FE_KNOB_ATOMIC_WARPS 4   /* warps per block of the staged kernel     */
#define FE_KNOB_ATOMIC_ORDER 5   /* read by fe_pattern_build: the element
                                    order of the FE_ATOMIC scatter.  0 auto
                                    (a locality order when the values exceed
                                    256 MB and the numbering is scattered),
                                    1 always ascending, 2 always the locality
                                    order (clusters of the block graph)      */
#define FE_KNOB_SPMV_LANES 7     /* lanes per row of fe_spmv_*: 2, 4, 8 or 16
                                    (0: 4)                                   */
#define FE_KNOB_LOCK_SPIN 6      /* FE_ROWLOCK: a lock is given up after
                                    2^value compare-and-swap attempts, 4..24
                                    (0: 2^22); the row is then skipped and
                                    FE_ERR_TIMEOUT recorded                  */
#define FE_KNOB_COUNT 8

/* Set / read one schedule knob.  FE_ERR_INVALID_ARG for an unknown knob or a
 * value outside its range. */
int fe_tune_set(fe_ctx *ctx, int knob, int value);
int fe_tune_get(const fe_ctx *ctx, int knob, int *value);

/* ---- symbolic phase ----------------------------------------------------- */

/*
 * Build the sparsity pattern of the matrix assembled from `n_elem` elements
 * with `dofs_per_elem` DOFs each (§3: "initialisation of the sparse matrix",
 * done once; §2.2 for CSR and CRAC).
 *   elem_dofs  device, int32 [n_elem * dofs_per_elem], row-major, element e's
 *              DOFs in local order (the element_dofs_array of §2.1).  Read
 *              only; the pattern keeps its own copy.
 *   n_dofs     number of rows (= columns); DOFs no element lists give empty
 *              rows.
 *   flags      FE_PATTERN_* parts to build (CSR is always built).
 *   stream     all work is ordered on it; the call blocks twice on it to size
 *              the outputs (after validation and after counting the rows),
 *              then returns with the rest enqueued.
 *   out        receives a pattern owned by the library; free with
 *              fe_pattern_free.
 * Errors: FE_ERR_DOF_RANGE / FE_ERR_DUP_DOF for bad connectivity (nothing is
 * allocated), FE_ERR_OVERFLOW, FE_ERR_UNSUPPORTED (dofs_per_elem >
 * FE_MAX_NLOC or a DOF shared by too many elements), FE_ERR_OOM.
 */
int fe_pattern_build(fe_ctx *ctx, int64_t n_elem, int32_t dofs_per_elem, int64_t n_dofs,
                     const int32_t *elem_dofs, uint32_t flags, void *stream,
                     fe_pattern **out);

/*
 * CSR pattern build that allocates no memory (the paper has no counterpart:
 * this entry point exists for callers of this library).
 *
 * Some callers cannot allocate device memory: an application that owns every
 * byte of HBM through its own allocator, a latency-bound loop that cannot
 * accept the implicit device synchronisation of cudaMalloc, or code running
 * where allocation is not permitted.  This call builds the same CSR arrays as
 * fe_pattern_build + fe_pattern_csr, but needs no context and calls no
 * cudaMalloc, cudaFree or allocating routine: its working memory is one fixed
 * 16 MiB device array inside the library, held by every GPU that loads the
 * library until the process exits.
 *
 *   elem_dofs   device, int32 [n_elem * dofs_per_elem] (read only).
 *   row_ptr     device, int64 [n_dofs + 1], written.
 *   col_idx     device, int32 [col_capacity], written when nnz <= capacity.
 *   nnz         host, receives the number of pattern entries (also when the
 *               capacity was too small, so the caller can retry).
 *   stream      work is ordered on it.  The call waits for `stream` three
 *               times (it reads sizes back to the host) and returns after the
 *               last wait, with the outputs complete.
 * Works on the current CUDA device.  The first call on a device does the
 * set-up: it looks up the array's device address (once per device; the
 * address is kept for the life of the process, so after cudaDeviceReset the
 * library must be reloaded before this call is used again).  Make that first
 * call before any stream capture begins.
 * All calls share the one array (its contents persist between calls; this
 * call clears what must start at zero), so calls whose work overlaps on the
 * GPU, from different streams or threads, race: serialise them.
 * Limit: the working arrays are laid out after the DOF block size B is known
 * (see fe_pattern_info.block); they take about 4*n_elem*(dofs_per_elem/B)^2
 * bytes for the row candidates plus 8*n_elem*dofs_per_elem/B bytes of
 * node connectivity and adjacency, 8 bytes per element and 36 bytes per node
 * plus 8 per DOF, which must fit in 16 MiB: e.g. about 39,000 trilinear hexes
 * with 3 DOFs per node (a 34^3 mesh) or 110,000 bilinear quads with one DOF
 * per node (a 330^2 mesh).
 * Errors: FE_ERR_UNSUPPORTED when the mesh needs more than the 16 MiB of
 * scratch or dofs_per_elem > FE_MAX_NLOC; FE_ERR_INVALID_ARG when
 * col_capacity < nnz; FE_ERR_DOF_RANGE / FE_ERR_DUP_DOF for bad connectivity
 * (checked first, whatever the size); FE_ERR_OVERFLOW.
 */
int fe_pattern_csr_noalloc(int64_t n_elem, int32_t dofs_per_elem, int64_t n_dofs, const int32_t *elem_dofs,
                           int64_t *row_ptr, int32_t *col_idx, int64_t col_capacity, int64_t *nnz,
                           void *stream);

/* Release a pattern.  Waits for the device to finish pending work first. */
int fe_pattern_free(fe_pattern *pattern);

/* Stream-ordered release: the pattern's device arrays are freed at the
 * current point of `stream` (no host wait); the handle is invalid on return.
 * Every use of the pattern on other streams must be ordered before that
 * point (e.g. by events) by the caller. */
int fe_pattern_free_async(fe_pattern *pattern, void *stream);

/* Borrowed device pointers to the CSR arrays (§2.2, Fig. 1c): row_ptr int64
 * [n_dofs + 1], col_idx int32 [nnz] sorted ascending within each row.  Valid
 * until fe_pattern_free.  Any output pointer may be NULL. */
int fe_pattern_csr(const fe_pattern *pattern, const int64_t **row_ptr, const int32_t **col_idx,
                   int64_t *nnz);

/* Borrowed device pointers to the CRAC arrays (§2.2, Fig. 1d): row_ptr int64
 * [n_dofs + 1] in int units of col_align; col_align int32 [n_ca] holding, per
 * maximal run of consecutive columns of a row, the pair (first column, value
 * position), followed by the final pair (n_dofs, nnz).  n_ca = 2*(runs+1).
 * FE_ERR_NOT_BUILT without FE_PATTERN_CRAC. */
int fe_pattern_crac(const fe_pattern *pattern, const int64_t **row_ptr, const int32_t **col_align,
                    int64_t *n_ca);

/* Borrowed device pointers to the block adjacency.  *block receives B (see
 * fe_pattern_info.block); blocks are node = dof / B.  adj_ptr int64
 * [n_dofs/B + 1]; adj uint32 [n_elem * dofs_per_elem / B] holding
 * e*(dofs_per_elem/B) + k for every element e whose local block k is the
 * row's block, ascending.  With B = 1 this is the DOF -> (element, local
 * row) adjacency.  Always built. */
int fe_pattern_adjacency(const fe_pattern *pattern, int32_t *block, const int64_t **adj_ptr,
                         const uint32_t **adj);

/*
 * Greedy colouring of the elements (the colouring of Listing 6): elements in
 * ascending order each take the smallest colour not used by an earlier
 * element sharing a DOF, so that elements of one colour share no DOF.
 * Computed on the device in dependency waves; the result equals the
 * sequential first-fit colouring.  Enables mode FE_COLOURED.  Synchronous on
 * `stream`.  *n_colours (may be NULL) receives the number of colours.
 * FE_ERR_UNSUPPORTED beyond 256 colours.
 */
int fe_pattern_colour(fe_ctx *ctx, fe_pattern *pattern, void *stream, int32_t *n_colours);

/* Borrowed device pointer to the colours, int32 [n_elem]. */
int fe_pattern_colours(const fe_pattern *pattern, int32_t *n_colours, const int32_t **colour);

/* Sizes and parts of a pattern. */
int fe_pattern_info_get(const fe_pattern *pattern, fe_pattern_info *out);

/* ---- numeric phase ------------------------------------------------------ */

/*
 * Assemble the element matrices into the CSR values array (Listing 2 for the
 * result; Listing 3 for FE_ATOMIC).
 *   elem_mats  device, double [n_elem * n_loc * n_loc]: K_e row-major, element
 *              after element.  Read only.
 *   values     device, double [nnz], caller-owned; entry k belongs to
 *              (row of k, col_idx[k]).
 *   mode       FE_ATOMIC (needs FE_PATTERN_MAP_CSR), FE_DETERMINISTIC (needs
 *              FE_PATTERN_MAP_CSR and FE_PATTERN_ADJ), FE_COLOURED (needs
 *              FE_PATTERN_MAP_CSR and fe_pattern_colour first, else
 *              FE_ERR_NOT_BUILT) or FE_ROWLOCK (needs FE_PATTERN_MAP_CSR; a
 *              lock spin that runs out leaves the sum incomplete and sets
 *              FE_ERR_TIMEOUT in fe_device_status).
 *   accumulate 0: values are overwritten (reset to zero first, §3);
 *              1: contributions are added to the values already there.
 * Asynchronous on `stream`.  FE_DETERMINISTIC reproduces the oracle's
 * ascending-element sum bit for bit; FE_ATOMIC agrees within rounding.
 */
int fe_assemble_csr(fe_ctx *ctx, const fe_pattern *pattern, const double *elem_mats,
                    double *values, int mode, int accumulate, void *stream);

/*
 * The same assembly located through the CRAC arrays and the compressed DOF
 * runs of each element (§2.1, §2.2, Listing 5's slices): one slot look-up per
 * run of consecutive DOFs instead of one per entry.  The values array has the
 * CSR order (Fig. 1c and 1d share it).  Needs FE_PATTERN_CRAC and
 * FE_PATTERN_MAP_CRAC (and FE_PATTERN_ADJ for FE_DETERMINISTIC).
 */
int fe_assemble_crac(fe_ctx *ctx, const fe_pattern *pattern, const double *elem_mats,
                     double *values, int mode, int accumulate, void *stream);

/* ---- consumers of the assembled matrix ----------------------------------- */

/* y = G x over the CSR arrays (values in CSR order).  x device [n_dofs], y
 * device [n_dofs].  One warp per row, fixed summation order (reproducible run
 * to run; not the left-to-right order of a serial loop).  Asynchronous. */
int fe_spmv_csr(fe_ctx *ctx, const fe_pattern *pattern, const double *values, const double *x, double *y,
                void *stream);

/* The same product through the CRAC arrays (§2.2): every run of consecutive
 * columns multiplies a contiguous slice of values with a contiguous slice of
 * x, so no column index is read per value (the CRAC SpMV of the paper's
 * outlook).  Needs FE_PATTERN_CRAC. */
int fe_spmv_crac(fe_ctx *ctx, const fe_pattern *pattern, const double *values, const double *x, double *y,
                 void *stream);

/* ---- batched assembly (many independent meshes, one launch) --------------
 * Not in the paper: a GPU runs thousands of small assemblies at once when
 * they share one persistent launch.  Every mesh keeps its own pattern, K and
 * values; the result of each is the single-mesh result (bit-identical in
 * FE_DETERMINISTIC). */
#define FE_FORMAT_CSR 0
#define FE_FORMAT_CRAC 1

#define FE_SCHED_WARP_PER_ELEMENT 1  /* FE_ATOMIC: a warp per element          */
#define FE_SCHED_THREAD_PER_ENTRY 2  /* FE_ATOMIC: a thread per K entry        */
#define FE_SCHED_BLOCK_PER_ELEMENT 3 /* FE_ATOMIC: a thread block per element  */
#define FE_SCHED_WARP_PER_ROW 4      /* FE_DETERMINISTIC: a warp per node row  */
#define FE_SCHED_WARP_PER_ELEMENT_TMA 5 /* FE_ATOMIC: a warp per element, K_e
                                       moved into shared memory by one bulk
                                       copy (TMA), double-buffered; items
                                       with n_loc > 32, a generic shape or a
                                       K not 16-byte aligned take the
                                       warp-per-element path               */

typedef struct fe_schedule {
    int32_t kind;  /* FE_SCHED_*                                               */
    int32_t tile;  /* elements (atomic) or node rows (deterministic) per tile  */
} fe_schedule;

typedef struct fe_batch_item {
    const fe_pattern *pattern;  /* built on the same context                     */
    const double *elem_mats;    /* device, [n_elem * n_loc * n_loc], read only    */
    double *values;             /* device, [nnz], written (or added to)           */
    uint64_t *times_ns;         /* device, 2 entries, or NULL: written with the
                                   GPU's global timer (ns) when the first tile of
                                   this item started and when its last tile
                                   finished (per-item latency inside one launch) */
} fe_batch_item;

/* Assemble n_items meshes in one persistent launch on `stream` (plus one
 * zeroing launch in FE_ATOMIC without accumulation).  format: FE_FORMAT_CSR /
 * FE_FORMAT_CRAC; mode, accumulate as in fe_assemble_csr.  sched = NULL uses
 * the schedule fe_batch_autotune found for a batch of this signature (element
 * shapes, format, mode, size class), else a default.  The item array is read
 * during the call only.  Asynchronous. */
int fe_assemble_batch(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                      int32_t accumulate, const fe_schedule *sched, void *stream);

/* Time every candidate schedule (kind x tile) on this batch and remember the
 * fastest for batches of the same signature.  Runs the assemblies (values
 * are overwritten).  Synchronous on `stream`.  *best / *best_ms may be NULL. */
int fe_batch_autotune(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                      void *stream, fe_schedule *best, float *best_ms);

/* The schedule fe_assemble_batch would take for this batch (sched = NULL):
 * the one fe_batch_autotune found for a batch of the same signature, in this
 * context or, with the environment variable FEASM_TUNE_CACHE naming a file,
 * in any earlier process on the same GPU model (the autotuner appends every
 * result to that file, one text line per entry keyed by GPU model and SM
 * count, batch signature and format/mode; a context reads its device's
 * entries when it first batches).  FE_ERR_NOT_FOUND when none is known. */
int fe_batch_tuned(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                   fe_schedule *out);

/* Capture one batched assembly into a CUDA graph (item table copied to the
 * device once); fe_batch_graph_launch replays it on any stream, e.g. after
 * new element values were written into the same K buffers.  The patterns and
 * buffers must outlive the graph. */
typedef struct fe_batch_graph fe_batch_graph;
int fe_batch_graph_create(fe_ctx *ctx, const fe_batch_item *items, int32_t n_items, int32_t format, int32_t mode,
                          int32_t accumulate, const fe_schedule *sched, void *stream, fe_batch_graph **out);
int fe_batch_graph_launch(fe_batch_graph *graph, void *stream);
int fe_batch_graph_destroy(fe_batch_graph *graph);

/* ---- serving: requests admitted by HBM footprint, continuous batching ------
 * Not in the paper.  A server owns a scheduler thread (admission, launches
 * of small requests, completions), a launcher thread for large requests and
 * two pattern-builder threads (each on its own high-priority stream).  Patterns are cached by `pattern_key`; a
 * request for a cached key is numeric-only; when memory runs short, patterns
 * no queued request needs are evicted, meshes used once before meshes used
 * again.  Admitted requests are assembled together (fe_assemble_batch) on one
 * of n_streams streams, so new requests are admitted and run while others are
 * in flight. */
#define FE_STATE_PENDING 0    /* submitted, waiting for admission            */
#define FE_STATE_ADMITTED 1   /* memory reserved, pattern being built/looked up */
#define FE_STATE_RUNNING 2    /* launched                                     */
#define FE_STATE_DONE 3
#define FE_STATE_FAILED 4
#define FE_STATE_CANCELLED 5

typedef struct fe_request {
    uint64_t pattern_key;      /* identity of the mesh for the pattern cache            */
    int64_t n_elem;
    int32_t dofs_per_elem;
    int32_t format;            /* FE_FORMAT_CSR / FE_FORMAT_CRAC                        */
    int64_t n_dofs;
    const int32_t *elem_dofs;  /* device; read when the key is not cached; must stay
                                  valid until the request completes                    */
    const double *elem_mats;   /* device K, or NULL: generate K_e = alpha_e * K_ref   */
    const double *k_ref;       /* device [n_loc*n_loc], used when elem_mats is NULL     */
    uint64_t seed;             /* alpha_e = 0.5 + (splitmix64(seed + e) >> 44) / 2^20   */
    int32_t mode;              /* FE_ATOMIC / FE_DETERMINISTIC                          */
    int32_t reserved;
    void *ready_event;         /* cudaEvent_t the assembly waits for (NULL = none)     */
    double deadline_s;         /* 0 = none; else the request must be launched on the
                                  GPU within this many seconds of its submission: the
                                  server's watchdog fails a request still queued after
                                  that (pending, or admitted and waiting for its
                                  launch) with FE_ERR_TIMEOUT and returns its memory.
                                  Work already launched always completes.             */
} fe_request;

typedef struct fe_result {
    int32_t status;            /* FE_OK or the error of the request                    */
    int32_t state;             /* FE_STATE_*                                           */
    int32_t cold;              /* 1 when the pattern was built for this request        */
    int32_t reserved;
    int64_t nnz;
    const int64_t *row_ptr;    /* device, borrowed from the cached pattern             */
    const int32_t *col_idx;    /* device, borrowed                                     */
    const double *values;      /* device, library-owned until fe_release               */
    double t_submit_us, t_admit_us, t_start_us, t_done_us;  /* host steady clock       */
    double t_ready_us;         /* when its pattern was available (cached: at admission) */
} fe_result;

typedef struct fe_server_stats {
    int64_t submitted, admitted, completed, failed, cancelled;
    int64_t launches, batched_requests, patterns_built, evictions;
    int64_t bytes_in_use, budget_bytes, cached_patterns;
    int64_t rebuilds;  /* builds of a key whose pattern had been evicted       */
    int64_t expired;   /* requests failed by the watchdog (deadline passed)    */
    int64_t admission_waits;    /* times the admission queue found a request that
                                   did not fit the budget                     */
    int64_t peak_bytes_in_use;  /* largest bytes charged at once                */
    double alloc_ms_total, alloc_ms_max;  /* host time in the launches' device
                                   allocations (values, generated K)          */
    /* requests in each stage now: waiting for admission, waiting for a
       pattern build, ready to launch, handed to the large-request launcher,
       launched and not complete; groups in flight */
    int64_t n_pending, n_to_build, n_ready, n_big_jobs, n_running, n_inflight_groups;
} fe_server_stats;

/* One span of device work seen by the server: a launched group of requests
 * (element generation + batched assembly) on one of its streams, or a pattern
 * build on its build stream (stream = -1).  Times are in ms after the server
 * started, from CUDA events recorded on the span's own stream (so start_ms is
 * when that stream reached the work, end_ms when it finished it). */
typedef struct fe_span {
    double start_ms, end_ms;
    int32_t stream;            /* launch stream index, or -1 for a pattern build  */
    int32_t n_requests;        /* requests in the group (1 for a build)           */
} fe_span;

typedef struct fe_server fe_server;

/* Start a server on ctx: n_streams launch streams (1..64), at most max_batch
 * requests per launch, hbm_budget_bytes of device memory for admitted
 * requests and cached patterns (0 = the context's budget).  Requests of at
 * least 2^26 element-matrix entries are launched alone on one of two extra
 * high-priority streams (never grouped with small ones), their kernels on at
 * most 3/4 of the GPU's resident blocks so that pattern builds and small
 * requests always find free SMs; while one runs, small groups take at most
 * 1/4 of them, leaving it most of the memory bandwidth.  n_streams = 1
 * with max_batch = 1 is a strict FIFO: one request at a time from admission
 * to completion on one stream (the one-launch-per-request baseline). */
int fe_server_start(fe_ctx *ctx, int32_t n_streams, int32_t max_batch, size_t hbm_budget_bytes,
                    fe_server **out);
/* Stop the threads, wait for the device, free everything the server owns. */
int fe_server_stop(fe_server *server);
/* Enqueue n requests (thread-safe); tickets[k] identifies request k.  A
 * request whose footprint exceeds the whole budget fails with
 * FE_ERR_ADMISSION; otherwise it waits until memory frees up. */
int fe_batch_submit(fe_server *server, const fe_request *reqs, int32_t n, uint64_t *tickets);
/* Current state of a ticket (never blocks). */
int fe_poll(fe_server *server, uint64_t ticket, fe_result *out);
/* Block until the ticket is done, failed or cancelled, or timeout_s passes
 * (FE_ERR_TIMEOUT). */
int fe_wait(fe_server *server, uint64_t ticket, double timeout_s, fe_result *out);
/* Cancel a request that was not admitted yet. */
int fe_cancel(fe_server *server, uint64_t ticket);
/* Free a finished ticket's values and unpin its pattern. */
int fe_release(fe_server *server, uint64_t ticket);
int fe_server_stats_get(fe_server *server, fe_server_stats *out);
/* Copy spans [first, first + cap) of the server's device timeline (completed
 * groups and builds, in completion order; at most 2^21 are kept) into out;
 * *n_total (may be NULL) receives the number recorded so far.  Callers derive
 * from it how much of the time requests' work from two or more streams was
 * on the device at once. */
int fe_server_timeline(fe_server *server, int64_t first, int64_t cap, fe_span *out, int64_t *n_total);

/* K_e = alpha_e * K_ref for n_elem elements (the generator the server uses
 * for requests without elem_mats), on `stream`. */
int fe_generate_scaled(fe_ctx *ctx, const double *k_ref, int32_t n_loc, int64_t n_elem, uint64_t seed,
                       double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FEASM_H */

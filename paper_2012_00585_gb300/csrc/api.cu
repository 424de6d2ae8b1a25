// Context, memory pool, error strings, and the exclusive scan used by the
// symbolic phase.
#include <atomic>
#include <cstdio>
#include <cstring>

#include <mutex>
#include <vector>

#include "internal.cuh"
#include "tma.cuh"

namespace {
thread_local char g_last_cuda[256] = "";
std::atomic<uint64_t> g_launches{0};

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int64_t SCAN_TILE = (int64_t)SCAN_THREADS * SCAN_ITEMS;

// Inclusive scan over the block; returns this thread's inclusive prefix and
// the block total through *total.
__device__ int64_t block_inclusive_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t warp_tot[SCAN_THREADS / FE_WARP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int64_t w = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    int64_t add = warp > 0 ? warp_tot[warp - 1] : 0;
    *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return v + add;
}

template <typename T>
__global__ void k_tile_reduce(const T *__restrict__ in, int64_t n, int64_t *__restrict__ sums)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x) {
        int64_t idx = base + k;
        if (idx < n) s += (int64_t)in[idx];
    }
    int64_t tot;
    block_inclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// out[i] = offs[tile] + sum(in[tile_base .. i-1]); the thread that owns
// element n-1 also writes out[n].
template <typename T>
__global__ void k_tile_scan(const T *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                            const int64_t *__restrict__ offs)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t x[SCAN_ITEMS];
    int64_t local = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t idx = base + k;
        x[k] = idx < n ? (int64_t)in[idx] : 0;
        local += x[k];
    }
    int64_t tot;
    int64_t incl = block_inclusive_scan(local, &tot);
    int64_t run = incl - local + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = run;
        run += x[k];
        if (idx == n - 1) out[n] = run;
    }
}

__global__ void k_set_zero_i64(int64_t *p) { *p = 0; }

template <typename T>
int scan_impl(fe_ctx *ctx, const T *in, int64_t *out, int64_t n, cudaStream_t s)
{
    if (n <= 0) {
        k_set_zero_i64<<<1, 1, 0, s>>>(out); fe_note_launch();
        FE_CUDA(cudaGetLastError());
        return FE_OK;
    }
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_tile_scan<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr); fe_note_launch();
        FE_CUDA(cudaGetLastError());
        return FE_OK;
    }
    if (tiles > INT32_MAX) return FE_ERR_UNSUPPORTED;
    int64_t *sums = nullptr, *offs = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&sums, sizeof(int64_t) * tiles, s));
    int rc = fe_alloc(ctx, (void **)&offs, sizeof(int64_t) * (tiles + 1), s);
    if (rc != FE_OK) {
        fe_free_async(sums, s);
        return rc;
    }
    k_tile_reduce<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums); fe_note_launch();
    rc = scan_impl<int64_t>(ctx, sums, offs, tiles, s);
    if (rc == FE_OK) k_tile_scan<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs); fe_note_launch();
    fe_free_async(sums, s);
    fe_free_async(offs, s);
    if (rc != FE_OK) return rc;
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

// Keeps the caller's current device and restores it on exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};
}  // namespace

void fe_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void fe_set_last_cuda_error(cudaError_t e, const char *what, int line)
{
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s (%d) at line %d: %s", cudaGetErrorString(e), (int)e,
             line, what);
}

int fe_alloc(fe_ctx *ctx, void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->pool_limit) {  // the context's bound on its pool (bytes handed out, not yet freed)
        uint64_t used = 0;
        if (cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess ||
            used + bytes > ctx->pool_limit) {
            cudaGetLastError();
            return FE_ERR_OOM;
        }
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        fe_set_last_cuda_error(e, "cudaMallocFromPoolAsync", __LINE__);
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_DEVICE;
    }
    return FE_OK;
}

void fe_free_async(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

int fe_scan_i32_to_i64(fe_ctx *ctx, const int32_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    return scan_impl<int32_t>(ctx, in, out, n, s);
}

int fe_scan_i64(fe_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, cudaStream_t s)
{
    return scan_impl<int64_t>(ctx, in, out, n, s);
}

extern "C" {

const char *fe_strerror(int code)
{
    switch (code) {
    case FE_OK: return "ok";
    case FE_ERR_INVALID_ARG: return "invalid argument";
    case FE_ERR_DOF_RANGE: return "DOF index out of range";
    case FE_ERR_DUP_DOF: return "DOF listed twice in one element";
    case FE_ERR_OVERFLOW: return "index overflow (nnz or n_ca >= 2^31, or n_elem*n_loc >= 2^32)";
    case FE_ERR_OOM: return "out of device memory";
    case FE_ERR_ADMISSION: return "request exceeds the HBM budget";
    case FE_ERR_TIMEOUT: return "bounded wait timed out";
    case FE_ERR_DEVICE: return "CUDA error";
    case FE_ERR_NOT_BUILT: return "pattern part not built";
    case FE_ERR_UNSUPPORTED: return "size beyond implementation limit";
    case FE_ERR_NOT_FOUND: return "unknown ticket";
    case FE_ERR_CANCELLED: return "request cancelled";
    default: return "unknown error";
    }
}

const char *fe_last_cuda_error(void) { return g_last_cuda; }

uint64_t fe_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int fe_debug_checks(void)
{
#ifdef FE_DEBUG
    return 1;
#else
    return 0;
#endif
}

int fe_create(fe_ctx **out, int device, size_t hbm_budget_bytes)
{
    return fe_create_ex(out, device, hbm_budget_bytes, 0);
}

int fe_create_ex(fe_ctx **out, int device, size_t hbm_budget_bytes, size_t pool_limit_bytes)
{
    if (!out) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    int n_dev = 0;
    FE_CUDA(cudaGetDeviceCount(&n_dev));
    if (device < 0 || device >= n_dev) return FE_ERR_INVALID_ARG;
    DeviceGuard g(device);
    fe_ctx *ctx = new fe_ctx();
    ctx->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&ctx->pool, &props);
    if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->d_status, 16);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 16);
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;  // keep freed blocks for reuse
        e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        fe_set_last_cuda_error(e, "fe_create", __LINE__);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        if (ctx->d_status) cudaFree(ctx->d_status);
        delete ctx;
        return FE_ERR_DEVICE;
    }
    if (hbm_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        hbm_budget_bytes = (size_t)(0.9 * (double)free_b);
    }
    ctx->hbm_budget = hbm_budget_bytes;
    ctx->pool_limit = pool_limit_bytes;
    *out = ctx;
    return FE_OK;
}

int fe_destroy(fe_ctx *ctx)
{
    if (!ctx) return FE_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    fe_batch_state_destroy(ctx);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return FE_OK;
}

int fe_tune_set(fe_ctx *ctx, int knob, int value)
{
    if (!ctx || knob < 0 || knob >= FE_KNOB_COUNT) return FE_ERR_INVALID_ARG;
    int lo = 0, hi = 0;
    switch (knob) {
    case FE_KNOB_GATHER_KERNEL: hi = 2; break;
    case FE_KNOB_GATHER_BATCH: hi = 8; break;
    case FE_KNOB_GATHER_WARPS: hi = 8; break;
    case FE_KNOB_ATOMIC_KERNEL: hi = 2; break;
    case FE_KNOB_ATOMIC_WARPS: hi = 8; break;
    case FE_KNOB_ATOMIC_ORDER: hi = 2; break;
    case FE_KNOB_LOCK_SPIN: hi = 24; break;
    case FE_KNOB_SPMV_LANES: hi = 16; break;
    default: return FE_ERR_INVALID_ARG;
    }
    if (value < lo || value > hi) return FE_ERR_INVALID_ARG;
    if (knob == FE_KNOB_GATHER_BATCH && value != 0 && value != 4 && value != 8) return FE_ERR_INVALID_ARG;
    if (knob == FE_KNOB_LOCK_SPIN && value != 0 && value < 4) return FE_ERR_INVALID_ARG;
    if (knob == FE_KNOB_SPMV_LANES && value != 0 && value != 2 && value != 4 && value != 8 && value != 16)
        return FE_ERR_INVALID_ARG;
    ctx->knob[knob] = value;
    return FE_OK;
}

int fe_tune_get(const fe_ctx *ctx, int knob, int *value)
{
    if (!ctx || !value || knob < 0 || knob >= FE_KNOB_COUNT) return FE_ERR_INVALID_ARG;
    *value = ctx->knob[knob];
    return FE_OK;
}

}  // extern "C"

int fe_resident_blocks(const void *kernel, int threads, size_t smem)
{
    struct Entry {
        const void *k;
        int threads;
        size_t smem;
        int blocks;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const Entry &e : cache)
            if (e.k == kernel && e.threads == threads && e.smem == smem) return e.blocks;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back({kernel, threads, smem, per_sm});
    return per_sm;
}

extern "C" {

int fe_device_status(fe_ctx *ctx, void *stream)
{
    if (!ctx) return FE_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    FE_CUDA(cudaMemcpyAsync(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s));
    FE_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // extern "C"

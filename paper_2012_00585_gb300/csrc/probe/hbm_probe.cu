// HBM calibration probes for the benchmark (not part of the assembly
// library): the read-only and copy bandwidth of plain 16-byte loads and the
// read-only bandwidth of bulk copies (TMA) into shared memory.  On GB300 the
// SMs' load path streams about half of what the bulk-copy engine does, which
// is why read-dominated kernels are compared with both.  Built into its own
// small library, loaded only by bench.py.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../tma.cuh"

namespace {

// HBM calibration: stream n doubles (read only, or copy to dst), 8
// independent 16-byte accesses in flight per thread.
__global__ void k_hbm_probe(const double2 *__restrict__ src, double2 *__restrict__ dst, int64_t n2, double *sink)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += 8 * stride) {
        double2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i + u * stride < n2 ? __ldcs(src + i + u * stride) : make_double2(0.0, 0.0);
        if (dst) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i + u * stride < n2) __stcs(dst + i + u * stride, v[u]);
        } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u].x + v[u].y;
        }
    }
    if (s == 1.2345e300) *sink = s;  // keeps the loads alive
}

// Read-only stream by 32-byte (256-bit) loads, 4 independent loads in flight
// per thread (src 32-byte aligned, n a multiple of 4).
__global__ void k_hbm_probe_v4(const double *__restrict__ src, int64_t n4, double *sink)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += 4 * stride) {
        double v[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = i + u * stride;
            if (k < n4)
                asm volatile("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                             : "=d"(v[u][0]), "=d"(v[u][1]), "=d"(v[u][2]), "=d"(v[u][3])
                             : "l"(src + 4 * k));
            else
                v[u][0] = v[u][1] = v[u][2] = v[u][3] = 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s += v[u][0] + v[u][1] + v[u][2] + v[u][3];
    }
    if (s == 1.2345e300) *sink = s;  // keeps the loads alive
}

// The same read-only stream moved by the bulk-copy (TMA) engine: chunks of
// PROBE_CHUNK bytes into a ring of PROBE_STAGES shared-memory stages per
// block (one mbarrier each).  Waits are bounded: a wait that runs out sets
// *status to 1, waits (bounded) for the other copies and ends the block.
constexpr int PROBE_CHUNK = 16384, PROBE_STAGES = 4;

__global__ void __launch_bounds__(128) k_hbm_probe_bulk(const char *__restrict__ src, int64_t nbytes, double *sink,
                                                        int *status)
{
    extern __shared__ __align__(128) unsigned char probe_smem[];
    __shared__ uint64_t bar[PROBE_STAGES];
    const int64_t n_chunks = (nbytes + PROBE_CHUNK - 1) / PROBE_CHUNK;
    const uint64_t pol = fe_policy_evict_first();
    if (threadIdx.x == 0) {
        for (int st = 0; st < PROBE_STAGES; ++st) fe_mbar_init(&bar[st], 1);
        fe_fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int st, int64_t c) {
        const uint32_t bytes = (uint32_t)min((int64_t)PROBE_CHUNK, nbytes - c * PROBE_CHUNK);
        fe_fence_proxy_async();
        fe_mbar_expect_tx(&bar[st], bytes);
        fe_bulk_g2s(probe_smem + st * PROBE_CHUNK, src + c * PROBE_CHUNK, bytes, &bar[st], pol);
    };
    if (threadIdx.x == 0)
        for (int st = 0; st < PROBE_STAGES; ++st) {
            const int64_t c = blockIdx.x + (int64_t)st * gridDim.x;
            if (c < n_chunks) issue(st, c);
        }
    double acc = 0.0;
    int64_t it = 0;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x, ++it) {
        const int st = (int)(it % PROBE_STAGES);
        const uint32_t parity = (uint32_t)((it / PROBE_STAGES) & 1);
        if (!__syncthreads_and(fe_mbar_wait(&bar[st], parity))) {
            if (threadIdx.x == 0) atomicCAS(status, 0, 1);
            for (int64_t k = it, cc = c; cc < n_chunks && k < it + PROBE_STAGES; ++k, cc += gridDim.x)
                fe_mbar_wait(&bar[k % PROBE_STAGES], (uint32_t)((k / PROBE_STAGES) & 1));
            return;
        }
        acc += ((const double *)(probe_smem + st * PROBE_CHUNK))[threadIdx.x];  // touch the stage
        __syncthreads();
        const int64_t cn = c + (int64_t)PROBE_STAGES * gridDim.x;
        if (threadIdx.x == 0 && cn < n_chunks) issue(st, cn);
    }
    if (acc == 1.2345e300) *sink = acc;  // keeps the reads alive
}


int sms_of_current()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

}  // namespace

extern "C" {

// Stream n doubles of src (16-byte aligned) through the SMs' loads on
// `stream`: read only (dst = NULL) or copied into dst.  sink: one device
// double the kernel may write (keeps the loads alive).  0 or -1.
int feprobe_stream(const double *src, double *dst, int64_t n, double *sink, void *stream)
{
    const int sms = sms_of_current();
    if (!src || !sink || n < 2 || ((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u) || sms <= 0) return -1;
    k_hbm_probe<<<sms * 8, 256, 0, (cudaStream_t)stream>>>((const double2 *)src, (double2 *)dst, n / 2, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The read-only stream by 32-byte loads (src 32-byte aligned, n a multiple
// of 4).  0 or -1.
int feprobe_stream_v4(const double *src, int64_t n, double *sink, void *stream)
{
    const int sms = sms_of_current();
    if (!src || !sink || n < 4 || (n & 3) || ((uintptr_t)src & 31u) || sms <= 0) return -1;
    k_hbm_probe_v4<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(src, n / 4, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The read-only stream moved by bulk copies (n even).  status: one device
// int, set to 1 when a bounded wait ran out.  0 or -1.
int feprobe_stream_bulk(const double *src, int64_t n, double *sink, int *status, void *stream)
{
    const int sms = sms_of_current();
    if (!src || !sink || !status || n < 2 || (n & 1) || ((uintptr_t)src & 15u) || sms <= 0) return -1;
    const size_t smem = (size_t)PROBE_CHUNK * PROBE_STAGES;
    if (cudaFuncSetAttribute(k_hbm_probe_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_hbm_probe_bulk<<<sms * 2, 128, smem, (cudaStream_t)stream>>>((const char *)src, n * 8, sink, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // extern "C"

// Symbolic phase: the sparsity pattern (CSR and CRAC) and the slot maps that
// the numeric kernels use.  The paper builds the pattern once in
// preprocessing and gives no algorithm for it (§3); the steps here are:
//   A1 validate the element_dofs_array and record each element's maximal
//      runs of consecutive DOFs (the compressed form of §2.1);
//   A2 DOF -> (element, local row) adjacency by counting sort;
//   A3 per-row union of the element DOF lists, sorted and de-duplicated by a
//      warp in shared memory, scanned into row_ptr, then col_idx and the CRAC
//      pairs (§2.2, Fig. 1c/1d) written in one pass;
//   A5 slot maps: per entry (CSR, found by binary search) and per DOF run
//      (CRAC, found by the linear block search of Listing 1).
#include <climits>

#include "internal.cuh"

namespace {

enum { S_ERR = 0, S_MAX_DEG = 1, S_MAX_ROW = 2, S_NONUNIFORM = 3, S_COUNT = 4 };

constexpr int32_t PAD = INT32_MAX;

__device__ __forceinline__ void set_err(int64_t *sc, int code)
{
    atomicCAS((unsigned long long *)&sc[S_ERR], 0ull, (unsigned long long)(int64_t)code);
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t warp_id_global() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t warps_total() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

// ---------------------------------------------------------------- A1 ---
// One warp per element: range and duplicate checks, run-start bits (bit c
// set when D(c) does not continue D(c-1)), runs per element, and whether all
// elements share element 0's run pattern.
__global__ void k_elements(const int32_t *__restrict__ D, int64_t n_e, int32_t n_loc, int64_t n_dofs,
                           int mask_words, uint32_t *__restrict__ run_mask, int32_t *__restrict__ runs,
                           int64_t *sc)
{
    const int lane = threadIdx.x & 31;
    for (int64_t e = warp_id_global(); e < n_e; e += warps_total()) {
        const int32_t *De = D + e * n_loc;
        int nr = 0;
        bool bad_range = false, dup = false, differs = false;
        for (int c0 = 0; c0 < n_loc; c0 += 32) {
            const int c = c0 + lane;
            const bool valid = c < n_loc;
            int32_t d = valid ? De[c] : 0;
            int32_t prev = (valid && c > 0) ? De[c - 1] : 0;
            if (valid && (d < 0 || (int64_t)d >= n_dofs)) bad_range = true;
            if (valid)
                for (int k = 0; k < c; ++k)
                    if (De[k] == d) {
                        dup = true;
                        break;
                    }
            const bool start = valid && (c == 0 || (int64_t)d != (int64_t)prev + 1);
            const unsigned m = __ballot_sync(0xffffffffu, start);
            // element 0's bits for the same lanes
            int32_t d0 = valid ? D[c] : 0;
            int32_t p0 = (valid && c > 0) ? D[c - 1] : 0;
            const bool start0 = valid && (c == 0 || (int64_t)d0 != (int64_t)p0 + 1);
            const unsigned m0 = __ballot_sync(0xffffffffu, start0);
            if (m != m0) differs = true;
            if (lane == 0) run_mask[e * mask_words + (c0 >> 5)] = m;
            nr += __popc(m);
        }
        if (bad_range) set_err(sc, FE_ERR_DOF_RANGE);
        if (dup) set_err(sc, FE_ERR_DUP_DOF);
        if (lane == 0) {
            runs[e] = nr;
            if (differs) sc[S_NONUNIFORM] = 1;
        }
    }
}

// ---------------------------------------------------------------- A2 ---
__global__ void k_count_deg(const int32_t *__restrict__ D, int64_t n_inc, int64_t n_dofs, int32_t *deg)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_inc; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = D[t];
        if (d >= 0 && (int64_t)d < n_dofs) atomicAdd(&deg[d], 1);
    }
}

__global__ void k_max_i32(const int32_t *__restrict__ x, int64_t n, int64_t *out)
{
    int32_t m = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = max(m, x[t]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((long long *)out, (long long)m);
}

__global__ void k_fill_adj(const int32_t *__restrict__ D, int64_t n_inc, const int64_t *__restrict__ adj_ptr,
                           int32_t *cursor, uint32_t *__restrict__ adj)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_inc; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = D[t];
        const int64_t pos = adj_ptr[d] + atomicAdd(&cursor[d], 1);
        adj[pos] = (uint32_t)t;
    }
}

// Each DOF's incidence list, ascending (element-major, since the id is
// e*n_loc + r).  Lists are short (the elements around one node).
__global__ void k_sort_adj(const int64_t *__restrict__ adj_ptr, int64_t n, uint32_t *adj)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = adj_ptr[i], b = adj_ptr[i + 1];
        for (int64_t k = a + 1; k < b; ++k) {
            const uint32_t v = adj[k];
            int64_t j = k - 1;
            while (j >= a && adj[j] > v) {
                adj[j + 1] = adj[j];
                --j;
            }
            adj[j + 1] = v;
        }
    }
}

// ---------------------------------------------------------------- A3 ---
__device__ void warp_bitonic_sort(int32_t *buf, int n, int lane)
{
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (n >> 1); t += 32) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const int32_t x = buf[lo], y = buf[hi];
                if ((x > y) == up) {
                    buf[lo] = y;
                    buf[hi] = x;
                }
            }
            __syncwarp();
        }
    }
}

// One warp per row i: gather D_e(c) for every (e, r) in adj(i), sort,
// de-duplicate.  PASS 1 counts the row length and its maximal column runs;
// PASS 2 writes col_idx and the CRAC pairs (first column, value position).
template <int PASS>
__global__ void k_rows(const int32_t *__restrict__ D, int32_t n_loc, int64_t n_dofs,
                       const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj, int P,
                       int32_t *__restrict__ row_len, int32_t *__restrict__ row_runs2, int64_t *sc,
                       const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ crac_ptr,
                       int32_t *__restrict__ col_idx, int32_t *__restrict__ col_align)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31;
    int32_t *buf = sbuf + (size_t)(threadIdx.x >> 5) * P;
    for (int64_t i = warp_id_global(); i < n_dofs; i += warps_total()) {
        const int64_t a = adj_ptr[i];
        const int n = (int)(adj_ptr[i + 1] - a) * n_loc;
        int Pn = 32;
        while (Pn < n) Pn <<= 1;
        for (int k = lane; k < Pn; k += 32) {
            int32_t v = PAD;
            if (k < n) {
                const int s = k / n_loc;
                const int c = k - s * n_loc;
                const uint32_t t = adj[a + s];
                v = D[(int64_t)(t / (uint32_t)n_loc) * n_loc + c];
            }
            buf[k] = v;
        }
        __syncwarp();
        warp_bitonic_sort(buf, Pn, lane);
        int count = 0, runs = 0;
        int64_t base = 0, cbase = 0;
        if (PASS == 2) {
            base = row_ptr[i];
            if (col_align) cbase = crac_ptr[i];
        }
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const int32_t v = k < n ? buf[k] : PAD;
            const int32_t pv = (k > 0 && k < n) ? buf[k - 1] : PAD;
            const bool keep = k < n && (k == 0 || v != pv);
            const bool rs = keep && (k == 0 || (int64_t)pv != (int64_t)v - 1);
            const unsigned mk = __ballot_sync(0xffffffffu, keep);
            const unsigned mr = __ballot_sync(0xffffffffu, rs);
            if (PASS == 2) {
                const int rank = count + __popc(mk & lanemask_lt());
                if (keep) col_idx[base + rank] = v;
                if (rs && col_align) {
                    const int rr = runs + __popc(mr & lanemask_lt());
                    col_align[cbase + 2 * rr] = v;
                    col_align[cbase + 2 * rr + 1] = (int32_t)(base + rank);
                }
            }
            count += __popc(mk);
            runs += __popc(mr);
        }
        if (PASS == 1 && lane == 0) {
            row_len[i] = count;
            row_runs2[i] = 2 * runs;
            atomicMax((long long *)&sc[S_MAX_ROW], (long long)count);
        }
        __syncwarp();
    }
}

__global__ void k_final_pair(int32_t *col_align, int64_t n_ca, int64_t n_dofs, int64_t nnz)
{
    col_align[n_ca - 2] = (int32_t)n_dofs;
    col_align[n_ca - 1] = (int32_t)nnz;
}

// ---------------------------------------------------------------- A5 ---
// CSR slot map: for every incidence t = e*n_loc + r in row i = D_e(r) and
// every local column c, the position of D_e(c) in the row, relative to
// row_ptr[i].  Warp-cooperative: the row's columns are staged in shared
// memory and each lane binary-searches its own column.
template <typename MT>
__global__ void k_map_csr(const int32_t *__restrict__ D, int32_t n_loc, int64_t n_dofs,
                          const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
                          const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col_idx, int cap,
                          MT *__restrict__ map, int64_t *sc)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31;
    int32_t *cols_s = sbuf + (size_t)(threadIdx.x >> 5) * cap;
    for (int64_t i = warp_id_global(); i < n_dofs; i += warps_total()) {
        const int64_t rb = row_ptr[i];
        const int len = (int)(row_ptr[i + 1] - rb);
        const bool in_smem = len <= cap;
        const int32_t *cols = in_smem ? cols_s : col_idx + rb;
        if (in_smem) {
            for (int k = lane; k < len; k += 32) cols_s[k] = col_idx[rb + k];
            __syncwarp();
        }
        for (int64_t s = adj_ptr[i]; s < adj_ptr[i + 1]; ++s) {
            const uint32_t t = adj[s];
            const int32_t *De = D + (int64_t)(t / (uint32_t)n_loc) * n_loc;
            for (int c = lane; c < n_loc; c += 32) {
                const int32_t j = De[c];
                int lo = 0, hi = len;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cols[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo >= len || cols[lo] != j) set_err(sc, FE_ERR_DEVICE);
                map[(int64_t)t * n_loc + c] = (MT)lo;
            }
        }
        __syncwarp();
    }
}

// CRAC slot map: for every incidence t = e*n_loc + r and every run k of
// element e's DOFs, the value position of the run's first DOF in row
// i = D_e(r), relative to the row's first value position.  The position is
// found by the linear block search of Listing 1 over the row's pairs, read
// with the row's own bound (the last block of the row is taken when no
// later block starts at or before the column).
template <typename MT>
__global__ void k_map_crac(const int32_t *__restrict__ D, int32_t n_loc, int64_t n_dofs, int mask_words,
                           const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
                           const int64_t *__restrict__ crac_ptr, const int32_t *__restrict__ col_align,
                           const uint32_t *__restrict__ run_mask, const int64_t *__restrict__ run_ptr, int cap,
                           MT *__restrict__ mapc, int64_t *sc)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31;
    int32_t *ca_s = sbuf + (size_t)(threadIdx.x >> 5) * cap;
    for (int64_t i = warp_id_global(); i < n_dofs; i += warps_total()) {
        const int64_t pb = crac_ptr[i];
        const int np = (int)(crac_ptr[i + 1] - pb);  // ints of this row's pairs
        if (np == 0) continue;
        const bool in_smem = np + 2 <= cap;
        const int32_t *ca = in_smem ? ca_s : col_align + pb;
        if (in_smem) {
            for (int k = lane; k < np + 2; k += 32) ca_s[k] = col_align[pb + k];
            __syncwarp();
        }
        const int32_t row_base = ca[1];
        for (int64_t s = adj_ptr[i]; s < adj_ptr[i + 1]; ++s) {
            const uint32_t t = adj[s];
            const int64_t e = t / (uint32_t)n_loc;
            const int r = (int)(t - (uint32_t)(e * n_loc));
            const int32_t *De = D + e * n_loc;
            const int64_t rp = run_ptr[e];
            const int nr = (int)(run_ptr[e + 1] - rp);
            int before = 0;  // runs that start in earlier 32-column chunks
            for (int c0 = 0; c0 < n_loc; c0 += 32) {
                const uint32_t m = run_mask[e * mask_words + (c0 >> 5)];
                const int c = c0 + lane;
                if (c < n_loc && ((m >> lane) & 1u)) {
                    const int k = before + __popc(m & ((1u << lane) - 1u));
                    const int32_t j = De[c];
                    int p = 0;
                    while (p + 2 < np) {
                        if (ca[p + 2] > j) break;
                        p += 2;
                    }
                    const int32_t col_start = ca[p];
                    const int32_t val_start = ca[p + 1];
                    const int32_t col_end = col_start + (ca[p + 3] - val_start);
                    int32_t rel = 0;
                    if (j >= col_start && j < col_end) rel = val_start + (j - col_start) - row_base;
                    else set_err(sc, FE_ERR_DEVICE);
                    mapc[rp * n_loc + (int64_t)r * nr + k] = (MT)rel;
                }
                before += __popc(m);
            }
        }
        __syncwarp();
    }
}

struct Scratch {
    cudaStream_t s;
    void *p[8] = {};
    int n = 0;
    void add(void *x) { p[n++] = x; }
    ~Scratch()
    {
        for (int k = 0; k < n; ++k) fe_free_async(p[k], s);
    }
};

void pattern_release(fe_pattern *p, cudaStream_t s)
{
    void *ptrs[] = {p->elem_dofs, p->row_ptr, p->col_idx, p->crac_ptr, p->col_align,
                    p->adj_ptr,  p->adj,     p->map_csr, p->run_mask, p->run_ptr, p->map_crac};
    for (void *x : ptrs) fe_free_async(x, s);
    delete p;
}

int alloc_into(fe_pattern *p, void **dst, size_t bytes, cudaStream_t s)
{
    int rc = fe_alloc(p->ctx, dst, bytes, s);
    if (rc == FE_OK) p->device_bytes += (int64_t)bytes;
    return rc;
}

template <typename KernelT>
int configure_smem(KernelT kernel, size_t bytes)
{
    if (bytes > 48 * 1024) FE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return FE_OK;
}

int build_impl(fe_pattern *p, const int32_t *elem_dofs_in, cudaStream_t s)
{
    fe_ctx *ctx = p->ctx;
    const int64_t n_e = p->n_e, n_dofs = p->n_dofs;
    const int32_t n_loc = p->n_loc;
    const int64_t n_inc = n_e * n_loc;
    const int sms = ctx->num_sms;
    Scratch tmp;
    tmp.s = s;

    int64_t *sc = nullptr;
    int32_t *deg = nullptr, *runs = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&sc, sizeof(int64_t) * S_COUNT, s));
    tmp.add(sc);
    FE_TRY(fe_alloc(ctx, (void **)&deg, sizeof(int32_t) * (size_t)(n_dofs + 1), s));
    tmp.add(deg);
    FE_TRY(fe_alloc(ctx, (void **)&runs, sizeof(int32_t) * (size_t)(n_e + 1), s));
    tmp.add(runs);
    FE_CUDA(cudaMemsetAsync(sc, 0, sizeof(int64_t) * S_COUNT, s));
    FE_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n_dofs + 1), s));

    p->mask_words = (n_loc + 31) / 32;
    FE_TRY(alloc_into(p, (void **)&p->elem_dofs, sizeof(int32_t) * (size_t)n_inc, s));
    FE_TRY(alloc_into(p, (void **)&p->run_mask, sizeof(uint32_t) * (size_t)(n_e * p->mask_words), s));
    FE_TRY(alloc_into(p, (void **)&p->run_ptr, sizeof(int64_t) * (size_t)(n_e + 1), s));
    if (n_inc > 0)
        FE_CUDA(cudaMemcpyAsync(p->elem_dofs, elem_dofs_in, sizeof(int32_t) * (size_t)n_inc,
                                cudaMemcpyDeviceToDevice, s));

    // A1 + A2 counting
    if (n_e > 0) {
        k_elements<<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(p->elem_dofs, n_e, n_loc, n_dofs,
                                                                       p->mask_words, p->run_mask, runs, sc); fe_note_launch();
        k_count_deg<<<fe_grid_for(n_inc, 256, sms, 16), 256, 0, s>>>(p->elem_dofs, n_inc, n_dofs, deg); fe_note_launch();
        k_max_i32<<<fe_grid_for(n_dofs, 256, sms, 8), 256, 0, s>>>(deg, n_dofs, sc + S_MAX_DEG); fe_note_launch();
        FE_CUDA(cudaGetLastError());
    }
    FE_TRY(fe_scan_i32_to_i64(ctx, runs, p->run_ptr, n_e, s));

    int64_t h1[S_COUNT + 1];
    FE_CUDA(cudaMemcpyAsync(h1, sc, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(h1 + S_COUNT, p->run_ptr + n_e, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));  // sync 1: validation result and sizes
    if (h1[S_ERR] != 0) return (int)h1[S_ERR];
    p->max_deg = (int32_t)h1[S_MAX_DEG];
    p->n_runs = h1[S_COUNT];
    p->uniform_runs = (h1[S_NONUNIFORM] == 0) && n_e > 0;
    p->runs_per_elem = n_e > 0 ? (int32_t)(p->n_runs / n_e) : 0;

    const int64_t cand = (int64_t)p->max_deg * n_loc;
    int P = 32;
    while (P < cand) P <<= 1;
    if ((int64_t)P * 4 > 128 * 1024) return FE_ERR_UNSUPPORTED;

    // A2: adjacency
    FE_TRY(alloc_into(p, (void **)&p->adj_ptr, sizeof(int64_t) * (size_t)(n_dofs + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->adj, sizeof(uint32_t) * (size_t)(n_inc + 1), s));
    FE_TRY(fe_scan_i32_to_i64(ctx, deg, p->adj_ptr, n_dofs, s));
    FE_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n_dofs + 1), s));
    if (n_inc > 0) {
        k_fill_adj<<<fe_grid_for(n_inc, 256, sms, 16), 256, 0, s>>>(p->elem_dofs, n_inc, p->adj_ptr, deg, p->adj); fe_note_launch();
        k_sort_adj<<<fe_grid_for(n_dofs, 128, sms, 16), 128, 0, s>>>(p->adj_ptr, n_dofs, p->adj); fe_note_launch();
        FE_CUDA(cudaGetLastError());
    }

    // A3 pass 1: row lengths and runs
    int32_t *row_len = nullptr, *row_runs2 = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&row_len, sizeof(int32_t) * (size_t)(n_dofs + 1), s));
    tmp.add(row_len);
    FE_TRY(fe_alloc(ctx, (void **)&row_runs2, sizeof(int32_t) * (size_t)(n_dofs + 1), s));
    tmp.add(row_runs2);
    const int W = (int)std::max<int64_t>(1, std::min<int64_t>(8, (48 * 1024) / ((int64_t)P * 4)));
    const size_t smem_rows = (size_t)W * P * 4;
    FE_TRY(configure_smem(k_rows<1>, smem_rows));
    FE_TRY(configure_smem(k_rows<2>, smem_rows));
    const int grid_rows = fe_grid_for(n_dofs * 32, W * 32, sms, 64 / W > 0 ? 64 / W : 1);
    if (n_dofs > 0) {
        k_rows<1><<<grid_rows, W * 32, smem_rows, s>>>(p->elem_dofs, n_loc, n_dofs, p->adj_ptr, p->adj, P, row_len,
                                                       row_runs2, sc, nullptr, nullptr, nullptr, nullptr); fe_note_launch();
        FE_CUDA(cudaGetLastError());
    }
    FE_TRY(alloc_into(p, (void **)&p->row_ptr, sizeof(int64_t) * (size_t)(n_dofs + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->crac_ptr, sizeof(int64_t) * (size_t)(n_dofs + 1), s));
    FE_TRY(fe_scan_i32_to_i64(ctx, row_len, p->row_ptr, n_dofs, s));
    FE_TRY(fe_scan_i32_to_i64(ctx, row_runs2, p->crac_ptr, n_dofs, s));

    int64_t h2[3];
    FE_CUDA(cudaMemcpyAsync(&h2[0], p->row_ptr + n_dofs, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(&h2[1], p->crac_ptr + n_dofs, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(&h2[2], sc + S_MAX_ROW, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));  // sync 2: nnz, n_ca, longest row
    p->nnz = h2[0];
    p->n_ca = h2[1] + 2;
    p->max_row_len = (int32_t)h2[2];
    if (p->nnz >= INT32_MAX || p->n_ca >= INT32_MAX) return FE_ERR_OVERFLOW;
    p->map_bytes = p->max_row_len <= 256 ? 1 : 2;
    if (p->max_row_len > 65536 && (p->flags & (FE_PATTERN_MAP_CSR | FE_PATTERN_MAP_CRAC))) return FE_ERR_UNSUPPORTED;

    // A3 pass 2 + A4: col_idx and CRAC pairs
    FE_TRY(alloc_into(p, (void **)&p->col_idx, sizeof(int32_t) * (size_t)(p->nnz + 1), s));
    const bool want_crac = (p->flags & (FE_PATTERN_CRAC | FE_PATTERN_MAP_CRAC)) != 0;
    if (want_crac) FE_TRY(alloc_into(p, (void **)&p->col_align, sizeof(int32_t) * (size_t)p->n_ca, s));
    if (n_dofs > 0) {
        k_rows<2><<<grid_rows, W * 32, smem_rows, s>>>(p->elem_dofs, n_loc, n_dofs, p->adj_ptr, p->adj, P, nullptr,
                                                       nullptr, sc, p->row_ptr, p->crac_ptr, p->col_idx,
                                                       want_crac ? p->col_align : nullptr); fe_note_launch();
        FE_CUDA(cudaGetLastError());
    }
    if (want_crac) {
        k_final_pair<<<1, 1, 0, s>>>(p->col_align, p->n_ca, n_dofs, p->nnz); fe_note_launch();
        FE_CUDA(cudaGetLastError());
    }

    // A5: slot maps
    const int WM = 8;
    if (p->flags & FE_PATTERN_MAP_CSR) {
        const size_t bytes = (size_t)n_inc * n_loc * p->map_bytes;
        FE_TRY(alloc_into(p, &p->map_csr, bytes, s));
        int cap = std::min<int>(p->max_row_len, 4096);
        if (cap < 1) cap = 1;
        const size_t smem = (size_t)WM * cap * 4;
        if (n_dofs > 0) {
            if (p->map_bytes == 1) {
                FE_TRY(configure_smem(k_map_csr<uint8_t>, smem));
                k_map_csr<uint8_t><<<fe_grid_for(n_dofs * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->elem_dofs, n_loc, n_dofs, p->adj_ptr, p->adj, p->row_ptr, p->col_idx, cap,
                    (uint8_t *)p->map_csr, sc); fe_note_launch();
            } else {
                FE_TRY(configure_smem(k_map_csr<uint16_t>, smem));
                k_map_csr<uint16_t><<<fe_grid_for(n_dofs * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->elem_dofs, n_loc, n_dofs, p->adj_ptr, p->adj, p->row_ptr, p->col_idx, cap,
                    (uint16_t *)p->map_csr, sc); fe_note_launch();
            }
            FE_CUDA(cudaGetLastError());
        }
    }
    if (p->flags & FE_PATTERN_MAP_CRAC) {
        const size_t bytes = (size_t)p->n_runs * n_loc * p->map_bytes;
        FE_TRY(alloc_into(p, &p->map_crac, bytes, s));
        int cap = std::min<int>(2 * p->max_row_len + 2, 8192);
        const size_t smem = (size_t)WM * cap * 4;
        if (n_dofs > 0) {
            if (p->map_bytes == 1) {
                FE_TRY(configure_smem(k_map_crac<uint8_t>, smem));
                k_map_crac<uint8_t><<<fe_grid_for(n_dofs * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->elem_dofs, n_loc, n_dofs, p->mask_words, p->adj_ptr, p->adj, p->crac_ptr, p->col_align,
                    p->run_mask, p->run_ptr, cap, (uint8_t *)p->map_crac, sc); fe_note_launch();
            } else {
                FE_TRY(configure_smem(k_map_crac<uint16_t>, smem));
                k_map_crac<uint16_t><<<fe_grid_for(n_dofs * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->elem_dofs, n_loc, n_dofs, p->mask_words, p->adj_ptr, p->adj, p->crac_ptr, p->col_align,
                    p->run_mask, p->run_ptr, cap, (uint16_t *)p->map_crac, sc); fe_note_launch();
            }
            FE_CUDA(cudaGetLastError());
        }
    }
    if (!(p->flags & FE_PATTERN_ADJ)) {
        fe_free_async(p->adj, s);
        fe_free_async(p->adj_ptr, s);
        p->device_bytes -= (int64_t)(sizeof(uint32_t) * (size_t)(n_inc + 1) + sizeof(int64_t) * (size_t)(n_dofs + 1));
        p->adj = nullptr;
        p->adj_ptr = nullptr;
    }
    return FE_OK;
}

}  // namespace

extern "C" {

int fe_pattern_build(fe_ctx *ctx, int64_t n_elem, int32_t dofs_per_elem, int64_t n_dofs, const int32_t *elem_dofs,
                     uint32_t flags, void *stream, fe_pattern **out)
{
    if (!ctx || !out) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_elem < 0 || dofs_per_elem <= 0 || n_dofs < 0) return FE_ERR_INVALID_ARG;
    if (n_elem > 0 && !elem_dofs) return FE_ERR_INVALID_ARG;
    if (flags & ~FE_PATTERN_ALL) return FE_ERR_INVALID_ARG;
    if (dofs_per_elem > FE_MAX_NLOC) return FE_ERR_UNSUPPORTED;
    if (n_dofs >= INT32_MAX) return FE_ERR_OVERFLOW;
    if (n_elem * (int64_t)dofs_per_elem >= (int64_t)UINT32_MAX) return FE_ERR_OVERFLOW;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe_pattern *p = new fe_pattern();
    p->ctx = ctx;
    p->n_e = n_elem;
    p->n_loc = dofs_per_elem;
    p->n_dofs = n_dofs;
    p->flags = flags | FE_PATTERN_CSR;
    if (p->flags & FE_PATTERN_MAP_CRAC) p->flags |= FE_PATTERN_CRAC;
    int rc = build_impl(p, elem_dofs, s);
    if (rc != FE_OK) {
        cudaStreamSynchronize(s);
        pattern_release(p, s);
    } else {
        *out = p;
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

int fe_pattern_free(fe_pattern *p)
{
    if (!p) return FE_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->ctx->device) cudaSetDevice(p->ctx->device);
    const int dev = p->ctx->device;
    cudaDeviceSynchronize();
    pattern_release(p, 0);
    cudaStreamSynchronize(0);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return FE_OK;
}

int fe_pattern_csr(const fe_pattern *p, const int64_t **row_ptr, const int32_t **col_idx, int64_t *nnz)
{
    if (!p) return FE_ERR_INVALID_ARG;
    if (row_ptr) *row_ptr = p->row_ptr;
    if (col_idx) *col_idx = p->col_idx;
    if (nnz) *nnz = p->nnz;
    return FE_OK;
}

int fe_pattern_crac(const fe_pattern *p, const int64_t **row_ptr, const int32_t **col_align, int64_t *n_ca)
{
    if (!p) return FE_ERR_INVALID_ARG;
    if (!(p->flags & FE_PATTERN_CRAC) || !p->col_align) return FE_ERR_NOT_BUILT;
    if (row_ptr) *row_ptr = p->crac_ptr;
    if (col_align) *col_align = p->col_align;
    if (n_ca) *n_ca = p->n_ca;
    return FE_OK;
}

int fe_pattern_adjacency(const fe_pattern *p, const int64_t **adj_ptr, const uint32_t **adj)
{
    if (!p) return FE_ERR_INVALID_ARG;
    if (!p->adj) return FE_ERR_NOT_BUILT;
    if (adj_ptr) *adj_ptr = p->adj_ptr;
    if (adj) *adj = p->adj;
    return FE_OK;
}

int fe_pattern_info_get(const fe_pattern *p, fe_pattern_info *out)
{
    if (!p || !out) return FE_ERR_INVALID_ARG;
    out->n_elem = p->n_e;
    out->n_loc = p->n_loc;
    out->map_bytes = p->map_bytes;
    out->n_dofs = p->n_dofs;
    out->nnz = p->nnz;
    out->n_ca = (p->flags & FE_PATTERN_CRAC) ? p->n_ca : 0;
    out->n_elem_runs = p->n_runs;
    out->max_row_len = p->max_row_len;
    out->max_degree = p->max_deg;
    out->flags = p->flags;
    out->reserved = p->uniform_runs ? 1u : 0u;
    out->device_bytes = p->device_bytes;
    return FE_OK;
}

}  // extern "C"

// Symbolic phase: the sparsity pattern (CSR and CRAC) and the slot maps that
// the numeric kernels use.  The paper builds the pattern once in
// preprocessing and gives no algorithm for it (§3); the steps here are:
//   A1 validate the element_dofs_array (range, repeats) and find the largest
//      DOF block size B such that every element lists whole blocks
//      (dof = B*node + comp, the layout of the d-benchmark, §4);
//   A2 block ("node") connectivity, the maximal runs of consecutive blocks of
//      every element (the compressed form of §2.1), and the node -> (element,
//      local node) adjacency by counting sort;
//   A3 per node row: the union of the element node lists, sorted and
//      de-duplicated by one warp (register bitonic network for up to 256
//      candidates, shared memory beyond), scanned into row_ptr, then expanded
//      to the B rows and B columns per node of col_idx and of the CRAC pairs
//      (§2.2, Fig. 1c/1d);
//   A5 slot maps: per (element, local node, local node) the position of the
//      column node in the row node's row (binary search), and per (element,
//      local node, run) the position of the run's first node, found by the
//      linear block search of Listing 1 over the row's CRAC pairs.
#include <climits>
#include <mutex>
#include <utility>

#include "assemble_body.cuh"
#include "internal.cuh"

namespace {

enum { S_ERR = 0, S_MAX_DEG = 1, S_MAX_NODE = 2, S_NONUNIFORM = 3, S_BLOCKS = 4, S_SPREAD = 5, S_COUNT = 6 };

constexpr int32_t PAD = INT32_MAX;
constexpr int REG_SORT_MAX = 256;  // candidates sorted in registers (8 per lane)

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

// Combine one value per warp into one atomic per block (same-address
// atomics from every warp serialise in L2).
__device__ __forceinline__ void block_and_atomic(uint32_t v, unsigned long long *dst)
{
    __shared__ uint32_t red[32];
    v = __reduce_and_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t x = 0xffffffffu;
        for (int k = 0; k < nw; ++k) x &= red[k];
        if (x != 0xffffffffu) atomicAnd(dst, (unsigned long long)x);
    }
}

__device__ __forceinline__ void block_max_atomic(int v, int64_t *dst)
{
    __shared__ int red[32];
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int x = 0;
        for (int k = 0; k < nw; ++k) x = max(x, red[k]);
        if (x > 0) atomicMax((long long *)dst, (long long)x);
    }
}

// ---------------------------------------------------------------- A1 ---
// Block-size test for one compile-time b: every aligned group of b local
// DOFs must be b consecutive indices starting at a multiple of b.
template <int b>
__device__ __forceinline__ void block_test(uint32_t cand, int c, int32_t d, bool is_start, bool valid, uint32_t &ok)
{
    if (cand & (1u << (b - 1))) {
        const bool good = (c % b == 0) ? ((uint32_t)d % b == 0) : !is_start;
        if (valid && !good) ok &= ~(1u << (b - 1));
    }
}

// Any other block size (runtime b, kept out of line).
__device__ __noinline__ uint32_t block_test_rt(int b, int c, int32_t d, bool is_start, bool valid)
{
    const bool good = (c % b == 0) ? ((uint32_t)d % (uint32_t)b == 0) : !is_start;
    return (valid && !good) ? ~(1u << (b - 1)) : 0xffffffffu;
}

// One warp per element: DOF range, repeated DOFs (by warp shuffles), and the
// candidate block sizes b (bit b-1 of `cand`, the divisors of n_loc) for
// which the element lists whole aligned blocks.
template <int MAXW>
__global__ void __launch_bounds__(256) k_validate(const int32_t *__restrict__ D, int64_t n_e, int32_t n_loc,
                                                  int64_t n_dofs, uint32_t cand, int64_t *sc)
{
    const int lane = threadIdx.x & 31;
    uint32_t blocks_all = 0xffffffffu;
    bool bad_range = false, dup = false;
    const int nw = (n_loc + 31) / 32;
    // the next element's DOFs are loaded one element ahead
    int32_t nx[MAXW];
    {
        const int64_t e = fe_warp_id();
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            const int c = 32 * w + lane;
            nx[w] = (e < n_e && w < nw && c < n_loc) ? D[e * n_loc + c] : INT32_MIN + w;
        }
    }
    for (int64_t e = fe_warp_id(); e < n_e; e += fe_warps()) {
        int32_t dv[MAXW];
#pragma unroll
        for (int w = 0; w < MAXW; ++w) dv[w] = nx[w];
        const int64_t en = e + fe_warps();
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            const int c = 32 * w + lane;
            nx[w] = (en < n_e && w < nw && c < n_loc) ? D[en * n_loc + c] : INT32_MIN + w;
        }
        uint32_t ok = 0xffffffffu;
#pragma unroll
        for (int w = 0; w < MAXW; ++w) {
            if (w >= nw) break;
            const int c = 32 * w + lane;
            const bool valid = c < n_loc;
            const int32_t d = dv[w];
            if (valid && (d < 0 || (int64_t)d >= n_dofs)) bad_range = true;
            // repeats: lanes holding the same DOF (one word), else compare
            // with every earlier local DOF
            if (nw == 1) {
                const unsigned same = __match_any_sync(0xffffffffu, d);
                if (valid && __popc(same) > 1) dup = true;
            } else {
#pragma unroll
                for (int w2 = 0; w2 <= w; ++w2) {
                    for (int k = 0; k < 32; ++k) {
                        const int32_t o = __shfl_sync(0xffffffffu, dv[w2], k);
                        if (valid && 32 * w2 + k < c && o == d) dup = true;
                    }
                }
            }
            int32_t prev = __shfl_up_sync(0xffffffffu, d, 1);
            const int32_t last_prev_word = w > 0 ? __shfl_sync(0xffffffffu, dv[w > 0 ? w - 1 : 0], 31) : 0;
            if (lane == 0) prev = last_prev_word;
            const bool is_start = c == 0 || (int64_t)d != (int64_t)prev + 1;
            for (uint32_t m = cand; m; m &= m - 1) {  // only the candidate sizes
                switch (__ffs(m)) {
                case 2: block_test<2>(cand, c, d, is_start, valid, ok); break;
                case 3: block_test<3>(cand, c, d, is_start, valid, ok); break;
                case 4: block_test<4>(cand, c, d, is_start, valid, ok); break;
                case 5: block_test<5>(cand, c, d, is_start, valid, ok); break;
                case 6: block_test<6>(cand, c, d, is_start, valid, ok); break;
                case 8: block_test<8>(cand, c, d, is_start, valid, ok); break;
                default: ok &= block_test_rt(__ffs(m), c, d, is_start, valid);
                }
            }
        }
        blocks_all &= ok;
    }
    block_and_atomic(blocks_all, (unsigned long long *)&sc[S_BLOCKS]);
    if (bad_range) set_err(sc, FE_ERR_DOF_RANGE);
    if (dup) set_err(sc, FE_ERR_DUP_DOF);
}

// ---------------------------------------------------------------- A2 ---
// One warp per element: block ids, run-start bits over the element's blocks
// (bit k set when block k does not continue block k-1), runs per element,
// whether all elements share element 0's bits, block degrees, and the sum
// over elements of (largest - smallest block id), a measure of how local the
// numbering is.
__global__ void k_node_conn(const int32_t *__restrict__ D, int64_t n_e, int32_t n_loc, int32_t B, int32_t nln,
                            int mask_words, int32_t *__restrict__ N, uint32_t *__restrict__ run_mask,
                            int32_t *__restrict__ runs, int32_t *deg, int64_t *sc)
{
    const int lane = threadIdx.x & 31;
    int64_t spread = 0;
    if (nln <= 16) {
        // small elements: 32 / P elements per warp, P = nln rounded up to a
        // power of two lanes each (one mask word per element)
        int P = 1;
        while (P < nln) P <<= 1;
        const int G = 32 / P, grp = lane / P, k = lane - grp * P;
        const unsigned gmask = P == 32 ? 0xffffffffu : ((1u << P) - 1u);
        // element 0's run starts, the reference of the uniform-layout test
        const bool v0 = n_e > 0 && k < nln;
        const int32_t nd0 = v0 ? D[(int64_t)B * k] / B : 0;
        const int32_t pv0 = (v0 && k > 0) ? D[(int64_t)B * (k - 1)] / B : 0;
        const bool start0 = v0 && (k == 0 || nd0 != pv0 + 1);
        const unsigned m0 = (__ballot_sync(0xffffffffu, start0) >> (grp * P)) & gmask;
        bool differs = false;
        for (int64_t e0 = fe_warp_id() * G; e0 < n_e; e0 += fe_warps() * G) {
            const int64_t e = e0 + grp;
            const bool valid = e < n_e && k < nln;
            const int32_t nd = valid ? D[e * n_loc + (int64_t)B * k] / B : 0;
            const int32_t pv = (valid && k > 0) ? D[e * n_loc + (int64_t)B * (k - 1)] / B : 0;
            const bool start = valid && (k == 0 || nd != pv + 1);
            const unsigned m = (__ballot_sync(0xffffffffu, start) >> (grp * P)) & gmask;
            int32_t lo = valid ? nd : INT32_MAX, hi = valid ? nd : 0;
            if (valid) {
                N[e * nln + k] = nd;
                atomicAdd(&deg[nd], 1);
            }
            for (int o = P >> 1; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (k == 0 && e < n_e) {
                run_mask[e * mask_words] = m;
                runs[e] = __popc(m);
                spread += hi - lo;
                if (m != m0) differs = true;
            }
        }
        if (__any_sync(0xffffffffu, differs) && lane == 0) sc[S_NONUNIFORM] = 1;
        for (int o = 16; o > 0; o >>= 1) spread += __shfl_xor_sync(0xffffffffu, spread, o);
        if (lane == 0 && spread) atomicAdd((unsigned long long *)&sc[S_SPREAD], (unsigned long long)spread);
        return;
    }
    for (int64_t e = fe_warp_id(); e < n_e; e += fe_warps()) {
        int nr = 0;
        bool differs = false;
        int32_t lo = INT32_MAX, hi = 0;
        for (int k0 = 0; k0 < nln; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < nln;
            const int32_t nd = valid ? D[e * n_loc + (int64_t)B * k] / B : 0;
            const int32_t pv = (valid && k > 0) ? D[e * n_loc + (int64_t)B * (k - 1)] / B : 0;
            const bool start = valid && (k == 0 || nd != pv + 1);
            const int32_t nd0 = valid ? D[(int64_t)B * k] / B : 0;
            const int32_t pv0 = (valid && k > 0) ? D[(int64_t)B * (k - 1)] / B : 0;
            const bool start0 = valid && (k == 0 || nd0 != pv0 + 1);
            const unsigned m = __ballot_sync(0xffffffffu, start);
            const unsigned m0 = __ballot_sync(0xffffffffu, start0);
            if (m != m0) differs = true;
            if (valid) {
                N[e * nln + k] = nd;
                atomicAdd(&deg[nd], 1);
                lo = min(lo, nd);
                hi = max(hi, nd);
            }
            if (lane == 0) run_mask[e * mask_words + (k0 >> 5)] = m;
            nr += __popc(m);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        spread += hi - lo;
        if (lane == 0) {
            runs[e] = nr;
            if (differs) sc[S_NONUNIFORM] = 1;
        }
    }
    if (lane == 0 && spread) atomicAdd((unsigned long long *)&sc[S_SPREAD], (unsigned long long)spread);
}

__global__ void k_max_i32(const int32_t *__restrict__ x, int64_t n, int64_t *out)
{
    int32_t m = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        m = max(m, x[t]);
    block_max_atomic(m, out);
}

__global__ void k_fill_adj(const int32_t *__restrict__ N, int64_t n_inc, int64_t n_nodes,
                           const int64_t *__restrict__ adj_ptr, int32_t *cursor, uint32_t *__restrict__ adj)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_inc; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t nd = N[t];
        if (nd < 0 || (int64_t)nd >= n_nodes) continue;
        const int64_t pos = adj_ptr[nd] + atomicAdd(&cursor[nd], 1);
        adj[pos] = (uint32_t)t;
    }
}

// Each block's incidence list, ascending (element-major, since the id is
// e*nln + k).  Lists are short (the elements around one node).
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
// Bitonic sort of 32*V keys held V per lane (key g = lane*V + v), ascending.
template <int V>
__device__ __forceinline__ void warp_sort_regs(int32_t (&a)[V], int lane)
{
#pragma unroll
    for (int size = 2; size <= 32 * V; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= V) {
                const int lm = stride / V;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int g = lane * V + v;
                    const int32_t y = __shfl_xor_sync(0xffffffffu, a[v], lm);
                    const bool lower = (g & stride) == 0;
                    const bool asc = (g & size) == 0;
                    a[v] = (lower == asc) ? min(a[v], y) : max(a[v], y);
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    if ((v & stride) == 0) {
                        const int w = v | stride;
                        const int g = lane * V + v;
                        const bool asc = (g & size) == 0;
                        const int32_t x = a[v], y = a[w];
                        a[v] = asc ? min(x, y) : max(x, y);
                        a[w] = asc ? max(x, y) : min(x, y);
                    }
                }
            }
        }
    }
}

__device__ void warp_sort_smem(int32_t *buf, int n, int lane)
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

// One warp per node row v: gather the block ids of every element touching
// v, sort (V keys per lane), keep the distinct ones.  Writes the row's
// length L_v, 2 * (its runs of consecutive blocks) and the sorted distinct
// blocks at keys + adj_ptr[v]*nln (the row's candidate range, an upper bound).
template <int V>
__global__ void __launch_bounds__(256) k_row_keys(const int32_t *__restrict__ N, int32_t nln, int64_t n_nodes,
                                                  const int64_t *__restrict__ adj_ptr,
                                                  const uint32_t *__restrict__ adj, int32_t *__restrict__ node_len,
                                                  int32_t *__restrict__ node_runs2, int32_t *__restrict__ keys,
                                                  int64_t *sc)
{
    const int lane = threadIdx.x & 31;
    int row_max = 0;
    // the next row's adjacency range and incidences are loaded one row ahead
    const int64_t W = fe_warps();
    int64_t an = 0;
    int nn = 0;
    uint32_t tn[V];
    auto fetch = [&](int64_t v) {
        an = 0;
        nn = 0;
        if (v < n_nodes) {
            an = adj_ptr[v];
            nn = (int)(adj_ptr[v + 1] - an) * nln;
        }
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int g = lane * V + q;
            tn[q] = g < nn ? adj[an + g / nln] : 0u;
        }
    };
    fetch(fe_warp_id());
    for (int64_t v = fe_warp_id(); v < n_nodes; v += W) {
        const int64_t a = an;
        const int n = nn;
        uint32_t tc[V];
#pragma unroll
        for (int q = 0; q < V; ++q) tc[q] = tn[q];
        fetch(v + W);
        int32_t x[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int g = lane * V + q;
            x[q] = PAD;
            if (g < n) {
                const int c = g - (g / nln) * nln;
                x[q] = N[(int64_t)(tc[q] / (uint32_t)nln) * nln + c];
            }
        }
        warp_sort_regs<V>(x, lane);
        const int32_t up = __shfl_up_sync(0xffffffffu, x[V - 1], 1);
        bool keep[V];
        int nk = 0, nrs = 0;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int g = lane * V + q;
            const int32_t pv = q > 0 ? x[q - 1] : up;
            keep[q] = g < n && (g == 0 || x[q] != pv);
            nk += keep[q];
            nrs += keep[q] && (g == 0 || (int64_t)pv != (int64_t)x[q] - 1);
        }
        int ik = nk, ir = nrs;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int tk = __shfl_up_sync(0xffffffffu, ik, off);
            const int tr = __shfl_up_sync(0xffffffffu, ir, off);
            if (lane >= off) {
                ik += tk;
                ir += tr;
            }
        }
        int rho = ik - nk;
        int32_t *kv = keys + a * nln;
#pragma unroll
        for (int q = 0; q < V; ++q)
            if (keep[q]) kv[rho++] = x[q];
        if (lane == 31) {
            node_len[v] = ik;
            node_runs2[v] = 2 * ir;
        }
        row_max = max(row_max, __shfl_sync(0xffffffffu, ik, 31));
    }
    block_max_atomic(row_max, &sc[S_MAX_NODE]);
}

// Rows with more than 256 candidates: the same with a bitonic sort in shared
// memory (P keys per warp).
__global__ void k_row_keys_smem(const int32_t *__restrict__ N, int32_t nln, int64_t n_nodes,
                                const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj, int P,
                                int32_t *__restrict__ node_len, int32_t *__restrict__ node_runs2,
                                int32_t *__restrict__ keys, int64_t *sc)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31;
    int32_t *buf = sbuf + (size_t)(threadIdx.x >> 5) * P;
    int row_max = 0;
    for (int64_t v = fe_warp_id(); v < n_nodes; v += fe_warps()) {
        const int64_t a = adj_ptr[v];
        const int n = (int)(adj_ptr[v + 1] - a) * nln;
        int Pn = 32;
        while (Pn < n) Pn <<= 1;
        for (int k = lane; k < Pn; k += 32) {
            int32_t x = PAD;
            if (k < n) {
                const int s = k / nln;
                const int c = k - s * nln;
                const uint32_t t = adj[a + s];
                x = N[(int64_t)(t / (uint32_t)nln) * nln + c];
            }
            buf[k] = x;
        }
        __syncwarp();
        warp_sort_smem(buf, Pn, lane);
        int L = 0, R = 0;
        int32_t *kv = keys + a * nln;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const int32_t x = k < n ? buf[k] : PAD;
            const int32_t pv = (k > 0 && k < n) ? buf[k - 1] : PAD;
            const bool keep = k < n && (k == 0 || x != pv);
            const bool rs = keep && (k == 0 || (int64_t)pv != (int64_t)x - 1);
            const unsigned mk = __ballot_sync(0xffffffffu, keep);
            const unsigned mr = __ballot_sync(0xffffffffu, rs);
            if (keep) kv[L + __popc(mk & lanemask_lt())] = x;
            L += __popc(mk);
            R += __popc(mr);
        }
        if (lane == 0) {
            node_len[v] = L;
            node_runs2[v] = 2 * R;
        }
        row_max = max(row_max, L);
        __syncwarp();
    }
    block_max_atomic(row_max, &sc[S_MAX_NODE]);
}

// One warp per node row v: the B DOF rows B*v+j get
//   row_ptr  = B^2 * nrp[v] + j*B*L_v,   col_idx = B*key + comp (coalesced),
//   crac_ptr = B * ncp[v] + j*2*R_v,     pairs (B*first key of a run, value position)
// where nrp / ncp are the node-level scans of L and 2R.
template <int BT>
__global__ void __launch_bounds__(256) k_expand(int64_t n_nodes, int32_t B_rt, int32_t nln,
                                                const int64_t *__restrict__ adj_ptr,
                                                const int32_t *__restrict__ keys, const int32_t *__restrict__ node_len,
                                                const int32_t *__restrict__ node_runs2,
                                                const int64_t *__restrict__ nrp, const int64_t *__restrict__ ncp,
                                                int64_t *__restrict__ row_ptr, int64_t *__restrict__ crac_ptr,
                                                int32_t *__restrict__ col_idx, int32_t *__restrict__ col_align, int cap)
{
    extern __shared__ int32_t kbuf[];
    const int B = BT > 0 ? BT : B_rt;  // compile-time block size for the common cases
    const int lane = threadIdx.x & 31;
    int32_t *ks = kbuf + (size_t)(threadIdx.x >> 5) * cap;
    for (int64_t v = fe_warp_id(); v < n_nodes; v += fe_warps()) {
        const int L = node_len[v];
        const int R2 = node_runs2[v];
        const int32_t *kv_g = keys + adj_ptr[v] * nln;
        const bool in_smem = L <= cap;
        if (in_smem) {
            for (int k = lane; k < L; k += 32) ks[k] = kv_g[k];
            __syncwarp();
        }
        const int32_t *kv = in_smem ? ks : kv_g;
        const int64_t rb0 = (int64_t)B * B * nrp[v];
        const int64_t cb0 = (int64_t)B * ncp[v];
        for (int j = lane; j < B; j += 32) {
            row_ptr[(int64_t)B * v + j] = rb0 + (int64_t)j * B * L;
            crac_ptr[(int64_t)B * v + j] = cb0 + (int64_t)j * R2;
        }
        for (int j = 0; j < B; ++j) {
            const int64_t rb = rb0 + (int64_t)j * B * L;
            for (int idx = lane; idx < B * L; idx += 32) {
                const int rho = idx / B;
                col_idx[rb + idx] = B * kv[rho] + (idx - rho * B);
            }
        }
        if (col_align) {
            // the block row's runs, found once and written for each of its B rows
            int rr = 0;
            for (int k0 = 0; k0 < L; k0 += 32) {
                const int k = k0 + lane;
                const int32_t x = k < L ? kv[k] : 0;
                const int32_t pv = (k > 0 && k < L) ? kv[k - 1] : 0;
                const bool rs = k < L && (k == 0 || (int64_t)pv != (int64_t)x - 1);
                const unsigned mr = __ballot_sync(0xffffffffu, rs);
                if (rs) {
                    const int r = rr + __popc(mr & lanemask_lt());
                    for (int j = 0; j < B; ++j) {
                        const int64_t cb = cb0 + (int64_t)j * R2;
                        col_align[cb + 2 * r] = B * x;
                        col_align[cb + 2 * r + 1] = (int32_t)(rb0 + (int64_t)j * B * L + (int64_t)B * k);
                    }
                }
                rr += __popc(mr);
            }
        }
        __syncwarp();
    }
}

// A3-A5 in one pass over the block rows, for rows of at most `cap` blocks:
// the expansion of k_expand (CSR row pointers and columns, the CRAC pairs,
// the row's runs found once) followed, with the row's sorted blocks and its
// runs still in shared memory, by the row's slot maps: for every incidence
// (element e, local block k) of the row, the position of each block of e in
// the row (binary search, the CSR map) and the position of the first block
// of each run of e (the CRAC block search of Listing 1 over the row's runs:
// walk to the last run starting at or before the block, then check that the
// block lies in it; the CRAC map).  A block missing from its row (a bad
// pattern) records FE_ERR_DEVICE.
template <int BT, typename MT>
__global__ void __launch_bounds__(256) k_expand_maps(
    int64_t n_nodes, int32_t B_rt, int32_t nln, const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
    const int32_t *__restrict__ N, const int32_t *__restrict__ keys, const int32_t *__restrict__ node_len,
    const int32_t *__restrict__ node_runs2, const int64_t *__restrict__ nrp, const int64_t *__restrict__ ncp,
    int64_t *__restrict__ row_ptr, int64_t *__restrict__ crac_ptr, int32_t *__restrict__ col_idx,
    int32_t *__restrict__ col_align, MT *__restrict__ map, MT *__restrict__ mapc,
    const uint32_t *__restrict__ run_mask, const int64_t *__restrict__ run_ptr, int mask_words, int rmax,
    int uniform_R, int cap, int64_t *sc)
{
    extern __shared__ int32_t kbuf[];
    const int B = BT > 0 ? BT : B_rt;
    const int lane = threadIdx.x & 31;
    int32_t *ks = kbuf + (size_t)(threadIdx.x >> 5) * 3 * cap;  // the row's blocks
    int32_t *rf = ks + cap;                                      // first block of each run
    int32_t *rk = rf + cap;                                      // its position in the row
    // The next row's sizes and offsets are loaded one row ahead, and a row's
    // keys and its first 32 incidences are loaded together as soon as the
    // row starts, so that a row waits for two rounds of loads (these, then
    // the elements' blocks of its maps) instead of a chain of five.
    const int64_t W = fe_warps();
    int64_t v = fe_warp_id();
    int L_n = 0, R2_n = 0;
    int64_t a_n = 0, b_n = 0, nrp_n = 0, ncp_n = 0;
    if (v < n_nodes) {
        L_n = node_len[v];
        R2_n = node_runs2[v];
        a_n = adj_ptr[v];
        b_n = adj_ptr[v + 1];
        nrp_n = nrp[v];
        ncp_n = ncp[v];
    }
    for (; v < n_nodes; v += W) {
        const int L = L_n;
        const int R2 = R2_n;
        const int64_t a = a_n, b = b_n;
        const int64_t rb0 = (int64_t)B * B * nrp_n;
        const int64_t cb0 = (int64_t)B * ncp_n;
        const int32_t *kv_g = keys + a * nln;
        for (int k = lane; k < L; k += 32) ks[k] = kv_g[k];
        const uint32_t t_l = lane < b - a ? adj[a + lane] : 0u;  // incidence a + lane
        if (v + W < n_nodes) {
            const int64_t u = v + W;
            L_n = node_len[u];
            R2_n = node_runs2[u];
            a_n = adj_ptr[u];
            b_n = adj_ptr[u + 1];
            nrp_n = nrp[u];
            ncp_n = ncp[u];
        }
        __syncwarp();
        for (int j = lane; j < B; j += 32) {
            row_ptr[(int64_t)B * v + j] = rb0 + (int64_t)j * B * L;
            crac_ptr[(int64_t)B * v + j] = cb0 + (int64_t)j * R2;
        }
        for (int j = 0; j < B; ++j) {
            const int64_t rb = rb0 + (int64_t)j * B * L;
            for (int idx = lane; idx < B * L; idx += 32) {
                const int rho = idx / B;
                col_idx[rb + idx] = B * ks[rho] + (idx - rho * B);
            }
        }
        int nruns = 0;
        for (int k0 = 0; k0 < L; k0 += 32) {
            const int k = k0 + lane;
            const int32_t x = k < L ? ks[k] : 0;
            const int32_t pv = (k > 0 && k < L) ? ks[k - 1] : 0;
            const bool st = k < L && (k == 0 || (int64_t)pv != (int64_t)x - 1);
            const unsigned mr = __ballot_sync(0xffffffffu, st);
            if (st) {
                const int r = nruns + __popc(mr & lanemask_lt());
                rf[r] = x;
                rk[r] = k;
                for (int j = 0; j < B; ++j) {
                    const int64_t cb = cb0 + (int64_t)j * R2;
                    col_align[cb + 2 * r] = B * x;
                    col_align[cb + 2 * r + 1] = (int32_t)(rb0 + (int64_t)j * B * L + (int64_t)B * k);
                }
            }
            nruns += __popc(mr);
        }
        __syncwarp();
        if (map) {
            const int total = (int)(b - a) * nln;
            for (int q0 = 0; q0 < total; q0 += 32) {  // uniform trip count: the shuffle takes every lane
                const int q = q0 + lane;
                const int s_ = q / nln;
                const int kc = q - s_ * nln;
                uint32_t t = __shfl_sync(0xffffffffu, t_l, s_ & 31);
                if (q >= total) continue;
                if (s_ >= 32) t = adj[a + s_];
                const int32_t j = N[(int64_t)(t / (uint32_t)nln) * nln + kc];
                int lo = 0, hi = L;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (ks[mid] < j) lo = mid + 1; else hi = mid;
                }
                if (lo >= L || ks[lo] != j) set_err(sc, FE_ERR_DEVICE);
                map[(int64_t)t * nln + kc] = (MT)lo;
            }
        }
        if (mapc) {
            const int total = (int)(b - a) * rmax;
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                const int s_ = q / rmax;
                const int ri = q - s_ * rmax;
                uint32_t t = __shfl_sync(0xffffffffu, t_l, s_ & 31);
                if (q >= total) continue;
                if (s_ >= 32) t = adj[a + s_];
                const int64_t e = t / (uint32_t)nln;
                const int k = (int)(t - (uint32_t)(e * nln));
                const uint32_t *m = uniform_R ? run_mask : run_mask + e * mask_words;
                // local block starting the element's ri-th run (ri-th set bit of its mask)
                int kc = -1, seen = 0;
                for (int w = 0; w < mask_words && kc < 0; ++w) {
                    uint32_t x = m[w];
                    const int cnt = __popc(x);
                    if (ri < seen + cnt) {
                        for (int i = 0; i < ri - seen; ++i) x &= x - 1;
                        kc = 32 * w + __ffs(x) - 1;
                    }
                    seen += cnt;
                }
                if (kc < 0) continue;  // the element has fewer runs
                int64_t rp;
                int nr;
                if (uniform_R) {
                    nr = uniform_R;
                    rp = e * uniform_R;
                } else {
                    rp = run_ptr[e];
                    nr = (int)(run_ptr[e + 1] - rp);
                }
                const int32_t j = N[e * nln + kc];
                int pr = 0;
                while (pr + 1 < nruns && rf[pr + 1] <= j) ++pr;
                const int len = (pr + 1 < nruns ? rk[pr + 1] : L) - rk[pr];
                int32_t rel = 0;
                if (j >= rf[pr] && j < rf[pr] + len) rel = rk[pr] + (j - rf[pr]);
                else set_err(sc, FE_ERR_DEVICE);
                mapc[rp * nln + (int64_t)k * nr + ri] = (MT)rel;
            }
        }
        __syncwarp();
    }
}

__global__ void k_tail(int64_t *row_ptr, int64_t *crac_ptr, const int64_t *nrp, const int64_t *ncp, int64_t n_nodes,
                       int64_t n_dofs, int32_t B)
{
    row_ptr[n_dofs] = (int64_t)B * B * nrp[n_nodes];
    crac_ptr[n_dofs] = (int64_t)B * ncp[n_nodes];
}

__global__ void k_final_pair(int32_t *col_align, int64_t n_ca, int64_t n_dofs, int64_t nnz)
{
    col_align[n_ca - 2] = (int32_t)n_dofs;
    col_align[n_ca - 1] = (int32_t)nnz;
}

// ---------------------------------------------------------------- A5 ---
// Node slot map: for every node incidence t = e*nln + k of node row v and
// every local node kc of element e, the position of N_e(kc) in row v.
// Warp-cooperative: the row's nodes are staged in shared memory and each
// lane binary-searches its own node.
template <typename MT>
__global__ void k_map_node(const int32_t *__restrict__ N, int32_t nln, int64_t n_nodes,
                           const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
                           const int32_t *__restrict__ node_len, const int32_t *__restrict__ keys, int cap,
                           MT *__restrict__ map, int64_t *sc)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31;
    int32_t *cols_s = sbuf + (size_t)(threadIdx.x >> 5) * cap;
    for (int64_t v = fe_warp_id(); v < n_nodes; v += fe_warps()) {
        const int64_t a = adj_ptr[v], b = adj_ptr[v + 1];
        const int len = node_len[v];
        const int32_t *row = keys + a * nln;
        const bool in_smem = len <= cap;
        const int32_t *cols = in_smem ? cols_s : row;
        if (in_smem) {
            for (int k = lane; k < len; k += 32) cols_s[k] = row[k];
            __syncwarp();
        }
        // (incidence, local node) pairs of this row, spread over the lanes
        const int total = (int)(b - a) * nln;
        for (int q = lane; q < total; q += 32) {
            const int s = q / nln;
            const int kc = q - s * nln;
            const uint32_t t = adj[a + s];
            const int32_t j = N[(int64_t)(t / (uint32_t)nln) * nln + kc];
            int lo = 0, hi = len;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cols[mid] < j) lo = mid + 1; else hi = mid;
            }
            if (lo >= len || cols[lo] != j) set_err(sc, FE_ERR_DEVICE);
            map[(int64_t)t * nln + kc] = (MT)lo;
        }
        __syncwarp();
    }
}

// Run slot map: for every node incidence t = e*nln + k of node row v and
// every run of element e's blocks, the position (in blocks) of the run's
// first block in row v, found by Listing 1's block search over the CRAC
// pairs of DOF row B*v, read with the row's own bound: the last block of
// the row is taken when no later block starts at or before the column.
// uniform_R > 0: every element has element 0's runs (uniform_R of them), so
// the run starts come from element 0's mask (cache-resident, independent of
// the adjacency) and the element's map offset is e * uniform_R.
template <typename MT>
__global__ void k_map_runs(const int32_t *__restrict__ N, int32_t nln, int64_t n_nodes, int32_t B, int mask_words,
                           const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
                           const int64_t *__restrict__ crac_ptr, const int32_t *__restrict__ col_align,
                           const uint32_t *__restrict__ run_mask, const int64_t *__restrict__ run_ptr, int cap,
                           int rmax, int uniform_R, MT *__restrict__ mapc, int64_t *sc)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31;
    int32_t *ca_s = sbuf + (size_t)(threadIdx.x >> 5) * cap;
    for (int64_t v = fe_warp_id(); v < n_nodes; v += fe_warps()) {
        const int64_t i0 = (int64_t)B * v;
        const int64_t pb = crac_ptr[i0];
        const int np = (int)(crac_ptr[i0 + 1] - pb);  // ints of this row's pairs
        if (np == 0) continue;
        const bool in_smem = np + 2 <= cap;
        const int32_t *ca = in_smem ? ca_s : col_align + pb;
        if (in_smem) {
            for (int k = lane; k < np + 2; k += 32) ca_s[k] = col_align[pb + k];
            __syncwarp();
        }
        const int32_t row_base = ca[1];
        const int64_t a = adj_ptr[v], b = adj_ptr[v + 1];
        // (incidence, run) pairs over the lanes; rmax bounds the runs per element
        const int total = (int)(b - a) * rmax;
        for (int q = lane; q < total; q += 32) {
            const int s = q / rmax;
            const int ri = q - s * rmax;
            const uint32_t t = adj[a + s];
            const int64_t e = t / (uint32_t)nln;
            const int k = (int)(t - (uint32_t)(e * nln));
            const uint32_t *m = uniform_R ? run_mask : run_mask + e * mask_words;
            // position of the ri-th set bit of the element's run-start mask
            int kc = -1, seen = 0;
            for (int w = 0; w < mask_words && kc < 0; ++w) {
                uint32_t x = m[w];
                const int cnt = __popc(x);
                if (ri < seen + cnt) {
                    for (int i = 0; i < ri - seen; ++i) x &= x - 1;  // drop the lower set bits
                    kc = 32 * w + __ffs(x) - 1;
                }
                seen += cnt;
            }
            if (kc < 0) continue;  // the element has fewer runs
            int64_t rp;
            int nr;
            if (uniform_R) {
                nr = uniform_R;
                rp = e * uniform_R;
            } else {
                rp = run_ptr[e];
                nr = (int)(run_ptr[e + 1] - rp);
            }
            const int32_t j = B * N[e * nln + kc];
            int p = 0;
            while (p + 2 < np) {
                if (ca[p + 2] > j) break;
                p += 2;
            }
            const int32_t col_start = ca[p];
            const int32_t val_start = ca[p + 1];
            const int32_t col_end = col_start + (ca[p + 3] - val_start);
            int32_t rel = 0;
            if (j >= col_start && j < col_end) rel = (val_start + (j - col_start) - row_base) / B;
            else set_err(sc, FE_ERR_DEVICE);
            mapc[rp * nln + (int64_t)k * nr + ri] = (MT)rel;
        }
        __syncwarp();
    }
}

// The CRAC run map expanded to one entry per column block: entry
// (e, kr, kc) = run_start(e, kr, run of kc) + offset of kc in its run, i.e.
// the position of block kc of element e in block row D_e(kr), located once
// per run by the CRAC block search (§2.2) when the run map was built.  Uniform
// runs: every element has element 0's mask and R runs.
template <typename MT>
__global__ void k_expand_run_map(int64_t n_e, int32_t nln, int32_t mask_words, const uint32_t *__restrict__ run_mask,
                                 const int64_t *__restrict__ run_ptr, int32_t uniform_R, const MT *__restrict__ map_crac,
                                 MT *__restrict__ blk)
{
    const int64_t n = n_e * nln * nln;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = x / nln;  // e * nln + kr
        const int kc = (int)(x - t * nln);
        const int64_t e = t / nln;
        const int64_t kr = t - e * nln;
        int64_t rp, nr;
        const uint32_t *m;
        if (uniform_R) {
            rp = e * uniform_R;
            nr = uniform_R;
            m = run_mask;
        } else {
            rp = run_ptr[e];
            nr = run_ptr[e + 1] - rp;
            m = run_mask + e * mask_words;
        }
        int k, off;
        fe_dev::run_of_multi(m, kc, k, off);
        blk[x] = (MT)(map_crac[rp * nln + kr * nr + k] + off);
    }
}

// ---------------------------------------------------- element order ---
// A locality order of the elements for the atomic scatter, built when the
// numbering is scattered (e.g. node ids permuted): the atomic adds of
// consecutive elements then land in rows far apart, and a row's values are
// evicted from L2 between the elements that touch it.  The block graph
// (blocks adjacent when they share an element) is split into compact
// clusters by a breadth-first search from seeds (every stride-th block), all
// grown at once level by level; a block reached from several clusters in the
// same level joins the smallest cluster id, so the clusters do not depend on
// thread timing.  Elements are then grouped by the cluster of their first
// block (counting sort): each group touches one compact region of rows, which
// stays in L2 while the group is added.  The order within a group is
// unspecified (it only changes the order of atomic adds).
constexpr int32_t ORDER_UNSET = INT32_MAX;

__global__ void k_order_seed(int64_t n_nodes, int64_t stride, int32_t *__restrict__ owner,
                             int32_t *__restrict__ level, int32_t *__restrict__ front, int32_t *n_front)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_nodes; v += (int64_t)gridDim.x * blockDim.x) {
        if (v % stride == 0) {
            owner[v] = (int32_t)(v / stride);
            level[v] = 0;
            front[atomicAdd(n_front, 1)] = (int32_t)v;
        } else {
            owner[v] = ORDER_UNSET;
            level[v] = ORDER_UNSET;
        }
    }
}

// Level L: every block adjacent to a frontier block (whose cluster is final)
// and not reached before joins the smallest adjacent frontier cluster; blocks
// reached for the first time form the next frontier.  A warp per frontier
// block, its lanes over (incidence, local block) pairs.
__global__ void k_order_expand(const int32_t *__restrict__ front, int32_t n_front, int32_t L,
                               const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
                               const int32_t *__restrict__ N, int32_t nln, int32_t *__restrict__ owner,
                               int32_t *__restrict__ level, int32_t *__restrict__ next, int32_t *n_next)
{
    const int lane = threadIdx.x & 31;
    for (int64_t f = fe_warp_id(); f < n_front; f += fe_warps()) {
        const int32_t v = front[f];
        const int32_t ov = owner[v];
        const int64_t a = adj_ptr[v];
        const int64_t cnt = (adj_ptr[v + 1] - a) * nln;
        for (int64_t x = lane; x < cnt; x += 32) {
            const uint32_t t = adj[a + x / nln];
            const uint32_t e = t / (uint32_t)nln;
            const int32_t w = N[(int64_t)e * nln + x % nln];
            const int32_t lw = level[w];
            if (lw != ORDER_UNSET && lw != L) continue;  // settled in an earlier level
            if (lw == ORDER_UNSET && atomicCAS(&level[w], ORDER_UNSET, L) == ORDER_UNSET)
                next[atomicAdd(n_next, 1)] = w;
            atomicMin(&owner[w], ov);
        }
    }
}

// Cluster of each element (its first block's; unreached blocks: the last
// group), histogrammed.
__global__ void k_order_count(const int32_t *__restrict__ N, int64_t n_e, int32_t nln,
                              const int32_t *__restrict__ owner, int32_t n_groups, int32_t *__restrict__ grp,
                              int32_t *__restrict__ hist)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_e; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = owner[N[e * nln]];
        const int32_t c = o == ORDER_UNSET ? n_groups - 1 : o;
        grp[e] = c;
        atomicAdd(&hist[c], 1);
    }
}

__global__ void k_order_place(int64_t n_e, const int32_t *__restrict__ grp, int64_t *__restrict__ cursor,
                              int32_t *__restrict__ order)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_e; e += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd((unsigned long long *)&cursor[grp[e]], 1ull)] = (int32_t)e;
}

struct Scratch {
    cudaStream_t s;
    void *p[12] = {};
    int n = 0;
    void add(void *x) { p[n++] = x; }
    ~Scratch()
    {
        for (int k = 0; k < n; ++k) fe_free_async(p[k], s);
    }
};

void pattern_release(fe_pattern *p, cudaStream_t s)
{
    fe_colouring_free(p, s);
    void *ptrs[] = {p->node_dofs, p->row_ptr, p->col_idx, p->crac_ptr, p->col_align, p->adj_ptr, p->adj,
                    p->map_csr,   p->run_mask, p->run_ptr, p->map_crac,
                    p->map_crac_blk != p->map_csr ? p->map_crac_blk : nullptr, p->elem_order};
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

#define FE_LAUNCH(...) \
    do {               \
        __VA_ARGS__;   \
        fe_note_launch(); \
    } while (0)

// A6 (see k_order_seed): clusters of about ORDER_STRIDE blocks (for 3-DOF
// blocks of about 85 columns, some 33 MB of rows: a few clusters fit in L2).
constexpr int64_t ORDER_STRIDE = 16384;

int build_elem_order(fe_pattern *p, cudaStream_t s)
{
    fe_ctx *ctx = p->ctx;
    const int sms = ctx->num_sms;
    const int64_t n_nodes = p->n_nodes, n_e = p->n_e;
    const int32_t nln = p->nln;
    if (n_nodes >= INT32_MAX || n_e >= INT32_MAX) return FE_OK;  // no order: ascending elements
    Scratch tmp;
    tmp.s = s;
    int32_t *owner = nullptr, *level = nullptr, *front = nullptr, *next = nullptr, *counts = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&owner, sizeof(int32_t) * (size_t)n_nodes, s));
    tmp.add(owner);
    FE_TRY(fe_alloc(ctx, (void **)&level, sizeof(int32_t) * (size_t)n_nodes, s));
    tmp.add(level);
    FE_TRY(fe_alloc(ctx, (void **)&front, sizeof(int32_t) * (size_t)n_nodes, s));
    tmp.add(front);
    FE_TRY(fe_alloc(ctx, (void **)&next, sizeof(int32_t) * (size_t)n_nodes, s));
    tmp.add(next);
    FE_TRY(fe_alloc(ctx, (void **)&counts, sizeof(int32_t) * 2, s));
    tmp.add(counts);
    FE_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2, s));
    FE_LAUNCH((k_order_seed<<<fe_grid_for(n_nodes, 256, sms, 16), 256, 0, s>>>(n_nodes, ORDER_STRIDE, owner, level,
                                                                                front, counts)));
    int32_t n_front = 0;
    FE_CUDA(cudaMemcpyAsync(&n_front, counts, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    // every level settles at least one more block, so the loop ends; the
    // bound only guards against a corrupted count
    for (int32_t L = 1; n_front > 0 && L <= (int32_t)std::min<int64_t>(n_nodes, INT32_MAX - 1); ++L) {
        FE_CUDA(cudaMemsetAsync(counts + 1, 0, sizeof(int32_t), s));
        FE_LAUNCH((k_order_expand<<<fe_grid_for((int64_t)n_front * 32, 256, sms, 8), 256, 0, s>>>(
            front, n_front, L, p->adj_ptr, p->adj, p->node_dofs, nln, owner, level, next, counts + 1)));
        FE_CUDA(cudaMemcpyAsync(&n_front, counts + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        FE_CUDA(cudaStreamSynchronize(s));
        std::swap(front, next);
    }
    // groups: one per seed, plus the last for blocks no seed reached
    const int32_t n_groups = (int32_t)((n_nodes + ORDER_STRIDE - 1) / ORDER_STRIDE) + 1;
    int32_t *grp = nullptr, *hist = nullptr;
    int64_t *cursor = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&grp, sizeof(int32_t) * (size_t)n_e, s));
    tmp.add(grp);
    FE_TRY(fe_alloc(ctx, (void **)&hist, sizeof(int32_t) * (size_t)n_groups, s));
    tmp.add(hist);
    FE_TRY(fe_alloc(ctx, (void **)&cursor, sizeof(int64_t) * (size_t)(n_groups + 1), s));
    tmp.add(cursor);
    FE_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * (size_t)n_groups, s));
    FE_LAUNCH((k_order_count<<<fe_grid_for(n_e, 256, sms, 16), 256, 0, s>>>(p->node_dofs, n_e, nln, owner, n_groups,
                                                                           grp, hist)));
    FE_TRY(fe_scan_i32_to_i64(ctx, hist, cursor, n_groups, s));
    FE_TRY(alloc_into(p, (void **)&p->elem_order, sizeof(int32_t) * (size_t)n_e, s));
    FE_LAUNCH((k_order_place<<<fe_grid_for(n_e, 256, sms, 16), 256, 0, s>>>(n_e, grp, cursor, p->elem_order)));
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

int build_impl(fe_pattern *p, const int32_t *elem_dofs, cudaStream_t s)
{
    fe_ctx *ctx = p->ctx;
    const int64_t n_e = p->n_e, n_dofs = p->n_dofs;
    const int32_t n_loc = p->n_loc;
    const int sms = ctx->num_sms;
    Scratch tmp;
    tmp.s = s;

    int64_t *sc = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&sc, sizeof(int64_t) * S_COUNT, s));
    tmp.add(sc);
    FE_CUDA(cudaMemsetAsync(sc, 0, sizeof(int64_t) * S_COUNT, s));
    FE_CUDA(cudaMemsetAsync(sc + S_BLOCKS, 0xff, sizeof(int64_t), s));

    // A1: validation and block size
    FePhase ph("A1 validate");
    if (n_e > 0) {
        uint32_t cand = 0;  // block sizes that divide both n_loc and n_dofs
        for (int b = 2; b <= 32; ++b)
            if (n_loc % b == 0 && n_dofs % b == 0) cand |= 1u << (b - 1);
        if (n_loc <= 32)
            FE_LAUNCH((k_validate<1><<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(elem_dofs, n_e, n_loc, n_dofs,
                                                                                      cand, sc)));
        else
            FE_LAUNCH((k_validate<FE_MAX_NLOC / 32><<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(
                elem_dofs, n_e, n_loc, n_dofs, cand, sc)));
        FE_CUDA(cudaGetLastError());
    }
    int64_t h1[S_COUNT];
    FE_CUDA(cudaMemcpyAsync(h1, sc, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));  // sync 1: validation result, block size
    if (h1[S_ERR] != 0) return (int)h1[S_ERR];
    int B = 1;
    const uint32_t bmask = (uint32_t)h1[S_BLOCKS];
    for (int b = 32; b >= 2; --b)
        if (((bmask >> (b - 1)) & 1u) && n_loc % b == 0 && n_dofs % b == 0) {
            B = b;
            break;
        }
    if (n_e == 0) B = 1;
    p->B = B;
    p->nln = n_loc / B;
    p->n_nodes = n_dofs / B;
    const int32_t nln = p->nln;
    const int64_t n_nodes = p->n_nodes;
    const int64_t n_ninc = n_e * nln;
    p->mask_words = (nln + 31) / 32;

    // A2: block connectivity, runs, degrees
    ph.next("A2 adjacency");
    int32_t *deg = nullptr, *runs = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&deg, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    tmp.add(deg);
    FE_TRY(fe_alloc(ctx, (void **)&runs, sizeof(int32_t) * (size_t)(n_e + 1), s));
    tmp.add(runs);
    FE_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->node_dofs, sizeof(int32_t) * (size_t)(n_ninc + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->run_mask, sizeof(uint32_t) * (size_t)(n_e * p->mask_words + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->run_ptr, sizeof(int64_t) * (size_t)(n_e + 1), s));
    if (n_e > 0) {
        FE_LAUNCH((k_node_conn<<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(
            elem_dofs, n_e, n_loc, B, nln, p->mask_words, p->node_dofs, p->run_mask, runs, deg, sc)));
        FE_LAUNCH((k_max_i32<<<fe_grid_for(n_nodes, 256, sms, 8), 256, 0, s>>>(deg, n_nodes, sc + S_MAX_DEG)));
        FE_CUDA(cudaGetLastError());
    }
    FE_TRY(fe_scan_i32_to_i64(ctx, runs, p->run_ptr, n_e, s));
    FE_TRY(alloc_into(p, (void **)&p->adj_ptr, sizeof(int64_t) * (size_t)(n_nodes + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->adj, sizeof(uint32_t) * (size_t)(n_ninc + 1), s));
    FE_TRY(fe_scan_i32_to_i64(ctx, deg, p->adj_ptr, n_nodes, s));
    FE_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    if (n_ninc > 0) {
        FE_LAUNCH((k_fill_adj<<<fe_grid_for(n_ninc, 256, sms, 16), 256, 0, s>>>(p->node_dofs, n_ninc, n_nodes,
                                                                                 p->adj_ptr, deg, p->adj)));
        FE_LAUNCH((k_sort_adj<<<fe_grid_for(n_nodes, 128, sms, 16), 128, 0, s>>>(p->adj_ptr, n_nodes, p->adj)));
        FE_CUDA(cudaGetLastError());
    }
    int64_t h2[S_COUNT + 1];
    FE_CUDA(cudaMemcpyAsync(h2, sc, sizeof(int64_t) * S_COUNT, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(h2 + S_COUNT, p->run_ptr + n_e, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));  // sync 2: largest degree, element runs
    p->max_deg = (int32_t)h2[S_MAX_DEG];
    p->n_runs = h2[S_COUNT];
    p->uniform_runs = (h2[S_NONUNIFORM] == 0) && n_e > 0;
    const int64_t spread_sum = h2[S_SPREAD];
    p->runs_per_elem = n_e > 0 ? (int32_t)(p->n_runs / n_e) : 0;

    ph.next("A3-A4 rows, CSR and CRAC");
    // A3: sorted distinct blocks of every node row (kept in `keys` at the
    // row's candidate offset adj_ptr[v]*nln), lengths and runs
    int32_t *node_len = nullptr, *node_runs2 = nullptr, *keys = nullptr;
    int64_t *nrp = nullptr, *ncp = nullptr;
    FE_TRY(fe_alloc(ctx, (void **)&node_len, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    tmp.add(node_len);
    FE_TRY(fe_alloc(ctx, (void **)&node_runs2, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    tmp.add(node_runs2);
    FE_TRY(fe_alloc(ctx, (void **)&keys, sizeof(int32_t) * (size_t)(n_ninc * nln + 1), s));
    tmp.add(keys);
    FE_TRY(fe_alloc(ctx, (void **)&nrp, sizeof(int64_t) * (size_t)(n_nodes + 1), s));
    tmp.add(nrp);
    FE_TRY(fe_alloc(ctx, (void **)&ncp, sizeof(int64_t) * (size_t)(n_nodes + 1), s));
    tmp.add(ncp);
    const int64_t cand = (int64_t)p->max_deg * nln;
    if (n_nodes > 0) {
        const int grid = fe_grid_for(n_nodes * 32, 256, sms, 8);
        if (cand <= 32) {
            FE_LAUNCH((k_row_keys<1><<<grid, 256, 0, s>>>(p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, node_len,
                                                           node_runs2, keys, sc)));
        } else if (cand <= 64) {
            FE_LAUNCH((k_row_keys<2><<<grid, 256, 0, s>>>(p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, node_len,
                                                           node_runs2, keys, sc)));
        } else if (cand <= 128) {
            FE_LAUNCH((k_row_keys<4><<<grid, 256, 0, s>>>(p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, node_len,
                                                           node_runs2, keys, sc)));
        } else if (cand <= REG_SORT_MAX) {
            FE_LAUNCH((k_row_keys<8><<<grid, 256, 0, s>>>(p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, node_len,
                                                           node_runs2, keys, sc)));
        } else {
            int P = 32;
            while (P < cand) P <<= 1;
            if ((int64_t)P * 4 > 128 * 1024) return FE_ERR_UNSUPPORTED;
            const int W = (int)std::max<int64_t>(1, std::min<int64_t>(8, (64 * 1024) / ((int64_t)P * 4)));
            const size_t smem = (size_t)W * P * 4;
            FE_TRY(configure_smem(k_row_keys_smem, smem));
            FE_LAUNCH((k_row_keys_smem<<<fe_grid_for(n_nodes * 32, W * 32, sms, std::max(1, 64 / W)), W * 32, smem,
                                         s>>>(p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, P, node_len, node_runs2,
                                              keys, sc)));
        }
        FE_CUDA(cudaGetLastError());
    }
    FE_TRY(fe_scan_i32_to_i64(ctx, node_len, nrp, n_nodes, s));
    FE_TRY(fe_scan_i32_to_i64(ctx, node_runs2, ncp, n_nodes, s));
    int64_t h3[3];
    FE_CUDA(cudaMemcpyAsync(&h3[0], nrp + n_nodes, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(&h3[1], ncp + n_nodes, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(&h3[2], sc + S_MAX_NODE, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));  // sync 3: nnz, n_ca, longest row
    p->nnz = (int64_t)B * B * h3[0];
    p->n_ca = (int64_t)B * h3[1] + 2;
    p->max_node_len = (int32_t)h3[2];
    p->max_row_len = B * p->max_node_len;
    if (p->nnz >= INT32_MAX || p->n_ca >= INT32_MAX) return FE_ERR_OVERFLOW;
    p->map_bytes = p->max_node_len <= 256 ? 1 : 2;
    if (p->max_node_len > 65536) return FE_ERR_UNSUPPORTED;

    // expansion to DOF rows: row_ptr, col_idx, CRAC row pointers and pairs
    FE_TRY(alloc_into(p, (void **)&p->row_ptr, sizeof(int64_t) * (size_t)(n_dofs + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->crac_ptr, sizeof(int64_t) * (size_t)(n_dofs + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->col_idx, sizeof(int32_t) * (size_t)(p->nnz + 1), s));
    FE_TRY(alloc_into(p, (void **)&p->col_align, sizeof(int32_t) * (size_t)p->n_ca, s));
    // rows of up to 1024 blocks: the slot maps are computed in the same pass
    const bool fused = n_nodes > 0 && n_e > 0 && p->max_node_len <= 1024 &&
                       (p->flags & (FE_PATTERN_MAP_CSR | FE_PATTERN_MAP_CRAC));
    if (fused) {
        ph.next("A3-A5 rows, CSR, CRAC and slot maps");
        if (p->flags & FE_PATTERN_MAP_CSR)
            FE_TRY(alloc_into(p, &p->map_csr, (size_t)(n_ninc * nln + 1) * p->map_bytes, s));
        if (p->flags & FE_PATTERN_MAP_CRAC)
            FE_TRY(alloc_into(p, &p->map_crac, (size_t)(p->n_runs * nln + 1) * p->map_bytes, s));
        const int kcap = std::max(1, p->max_node_len);
        const size_t ksm = (size_t)8 * 3 * kcap * 4;
        const int eg = fe_grid_for(n_nodes * 32, 256, sms, 8);
        const int rmax = p->uniform_runs ? p->runs_per_elem : nln;
        const int uR = p->uniform_runs ? p->runs_per_elem : 0;
        auto launch = [&](auto kern, auto *map, auto *mapc) -> int {
            FE_TRY(configure_smem(kern, ksm));
            FE_LAUNCH((kern<<<eg, 256, ksm, s>>>(n_nodes, B, nln, p->adj_ptr, p->adj, p->node_dofs, keys, node_len,
                                                  node_runs2, nrp, ncp, p->row_ptr, p->crac_ptr, p->col_idx,
                                                  p->col_align, map, mapc, p->run_mask, p->run_ptr, p->mask_words,
                                                  rmax, uR, kcap, sc)));
            return FE_OK;
        };
        if (p->map_bytes == 1) {
            uint8_t *m = (uint8_t *)p->map_csr, *mc = (uint8_t *)p->map_crac;
            if (B == 3) FE_TRY(launch(k_expand_maps<3, uint8_t>, m, mc));
            else if (B == 1) FE_TRY(launch(k_expand_maps<1, uint8_t>, m, mc));
            else FE_TRY(launch(k_expand_maps<0, uint8_t>, m, mc));
        } else {
            uint16_t *m = (uint16_t *)p->map_csr, *mc = (uint16_t *)p->map_crac;
            if (B == 3) FE_TRY(launch(k_expand_maps<3, uint16_t>, m, mc));
            else if (B == 1) FE_TRY(launch(k_expand_maps<1, uint16_t>, m, mc));
            else FE_TRY(launch(k_expand_maps<0, uint16_t>, m, mc));
        }
    } else if (n_nodes > 0) {
        const int kcap = std::max(1, std::min(p->max_node_len, 1024));
        const size_t ksm = (size_t)8 * kcap * 4;
        const int eg = fe_grid_for(n_nodes * 32, 256, sms, 8);
        if (B == 3) {
            FE_TRY(configure_smem(k_expand<3>, ksm));
            FE_LAUNCH((k_expand<3><<<eg, 256, ksm, s>>>(n_nodes, B, nln, p->adj_ptr, keys, node_len, node_runs2, nrp,
                                                        ncp, p->row_ptr, p->crac_ptr, p->col_idx, p->col_align, kcap)));
        } else if (B == 1) {
            FE_TRY(configure_smem(k_expand<1>, ksm));
            FE_LAUNCH((k_expand<1><<<eg, 256, ksm, s>>>(n_nodes, B, nln, p->adj_ptr, keys, node_len, node_runs2, nrp,
                                                        ncp, p->row_ptr, p->crac_ptr, p->col_idx, p->col_align, kcap)));
        } else {
            FE_TRY(configure_smem(k_expand<0>, ksm));
            FE_LAUNCH((k_expand<0><<<eg, 256, ksm, s>>>(n_nodes, B, nln, p->adj_ptr, keys, node_len, node_runs2, nrp,
                                                        ncp, p->row_ptr, p->crac_ptr, p->col_idx, p->col_align, kcap)));
        }
    }
    FE_LAUNCH((k_tail<<<1, 1, 0, s>>>(p->row_ptr, p->crac_ptr, nrp, ncp, n_nodes, n_dofs, B)));
    FE_LAUNCH((k_final_pair<<<1, 1, 0, s>>>(p->col_align, p->n_ca, n_dofs, p->nnz)));
    FE_CUDA(cudaGetLastError());

    // A5: slot maps
    ph.next("A5 slot maps");
    const int WM = 8;
    if ((p->flags & FE_PATTERN_MAP_CSR) && !fused) {
        FE_TRY(alloc_into(p, &p->map_csr, (size_t)(n_ninc * nln + 1) * p->map_bytes, s));
        const int cap = std::max(1, std::min(p->max_node_len, 4096));
        const size_t smem = (size_t)WM * cap * 4;
        if (n_nodes > 0) {
            if (p->map_bytes == 1) {
                FE_TRY(configure_smem(k_map_node<uint8_t>, smem));
                FE_LAUNCH((k_map_node<uint8_t><<<fe_grid_for(n_nodes * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, node_len, keys, cap, (uint8_t *)p->map_csr,
                    sc)));
            } else {
                FE_TRY(configure_smem(k_map_node<uint16_t>, smem));
                FE_LAUNCH((k_map_node<uint16_t><<<fe_grid_for(n_nodes * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->node_dofs, nln, n_nodes, p->adj_ptr, p->adj, node_len, keys, cap, (uint16_t *)p->map_csr,
                    sc)));
            }
            FE_CUDA(cudaGetLastError());
        }
    }
    if ((p->flags & FE_PATTERN_MAP_CRAC) && !fused) {
        FE_TRY(alloc_into(p, &p->map_crac, (size_t)(p->n_runs * nln + 1) * p->map_bytes, s));
        const int cap = std::max(4, std::min(2 * p->max_node_len + 2, 8192));
        const size_t smem = (size_t)WM * cap * 4;
        if (n_nodes > 0) {
            if (p->map_bytes == 1) {
                FE_TRY(configure_smem(k_map_runs<uint8_t>, smem));
                FE_LAUNCH((k_map_runs<uint8_t><<<fe_grid_for(n_nodes * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->node_dofs, nln, n_nodes, B, p->mask_words, p->adj_ptr, p->adj, p->crac_ptr, p->col_align,
                    p->run_mask, p->run_ptr, cap, p->uniform_runs ? p->runs_per_elem : nln,
                    p->uniform_runs ? p->runs_per_elem : 0, (uint8_t *)p->map_crac, sc)));
            } else {
                FE_TRY(configure_smem(k_map_runs<uint16_t>, smem));
                FE_LAUNCH((k_map_runs<uint16_t><<<fe_grid_for(n_nodes * 32, WM * 32, sms, 8), WM * 32, smem, s>>>(
                    p->node_dofs, nln, n_nodes, B, p->mask_words, p->adj_ptr, p->adj, p->crac_ptr, p->col_align,
                    p->run_mask, p->run_ptr, cap, p->uniform_runs ? p->runs_per_elem : nln,
                    p->uniform_runs ? p->runs_per_elem : 0, (uint16_t *)p->map_crac, sc)));
            }
            FE_CUDA(cudaGetLastError());
        }
    }
    // the CRAC gather's block map, expanded from the run map.  With the CSR
    // map built too the expansion would be that map byte for byte (a block's
    // position in its row does not depend on the format): it is shared
    // instead.  Patterns built with FE_PATTERN_MAP_CRAC alone expand it.
    if ((p->flags & FE_PATTERN_MAP_CRAC) && p->map_csr) {
        p->map_crac_blk = p->map_csr;
    } else if (p->flags & FE_PATTERN_MAP_CRAC) {
        FE_TRY(alloc_into(p, &p->map_crac_blk, (size_t)(n_ninc * nln + 1) * p->map_bytes, s));
        if (n_ninc > 0) {
            const int g = fe_grid_for(n_ninc * nln, 256, sms, 16);
            const int uR = p->uniform_runs ? p->runs_per_elem : 0;
            if (p->map_bytes == 1)
                FE_LAUNCH((k_expand_run_map<uint8_t><<<g, 256, 0, s>>>(n_e, nln, p->mask_words, p->run_mask, p->run_ptr,
                                                                       uR, (const uint8_t *)p->map_crac,
                                                                       (uint8_t *)p->map_crac_blk)));
            else
                FE_LAUNCH((k_expand_run_map<uint16_t><<<g, 256, 0, s>>>(n_e, nln, p->mask_words, p->run_mask,
                                                                        p->run_ptr, uR, (const uint16_t *)p->map_crac,
                                                                        (uint16_t *)p->map_crac_blk)));
            FE_CUDA(cudaGetLastError());
        }
    }
    // A6: locality order of the elements for the atomic scatter
    {
        const int want = ctx->knob[FE_KNOB_ATOMIC_ORDER];
        const bool maps = (p->flags & (FE_PATTERN_MAP_CSR | FE_PATTERN_MAP_CRAC)) != 0;
        // auto: values too large to stay in L2, and a scattered numbering (an
        // element's blocks lie on average more than n_nodes / 16 apart)
        const bool scattered = n_e > 0 && spread_sum / n_e > n_nodes / 16;
        const bool large = p->nnz * 8 > ((int64_t)256 << 20);
        if (maps && n_e > 0 && n_nodes > 0 && (want == 2 || (want == 0 && large && scattered))) {
            ph.next("A6 element order");
            FE_TRY(build_elem_order(p, s));
        }
    }
    if (!(p->flags & FE_PATTERN_CRAC) && !(p->flags & FE_PATTERN_MAP_CRAC)) {
        // CRAC was only scaffolding for this pattern
        fe_free_async(p->col_align, s);
        p->device_bytes -= (int64_t)(sizeof(int32_t) * (size_t)p->n_ca);
        p->col_align = nullptr;
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
    FeRange range("fe_pattern_build");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe_pattern *p = new fe_pattern();
    p->ctx = ctx;
    p->n_e = n_elem;
    p->n_loc = dofs_per_elem;
    p->n_dofs = n_dofs;
    p->flags = flags | FE_PATTERN_CSR | FE_PATTERN_ADJ;  // adjacency is kept: it is small
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
    const int dev = p->ctx->device;
    if (prev != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    pattern_release(p, 0);
    cudaStreamSynchronize(0);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return FE_OK;
}

int fe_pattern_free_async(fe_pattern *p, void *stream)
{
    if (!p) return FE_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    const int dev = p->ctx->device;
    if (prev != dev) cudaSetDevice(dev);
    pattern_release(p, (cudaStream_t)stream);
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        fe_set_last_cuda_error(e, "fe_pattern_free_async", __LINE__);
        return FE_ERR_DEVICE;
    }
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

int fe_pattern_adjacency(const fe_pattern *p, int32_t *block, const int64_t **adj_ptr, const uint32_t **adj)
{
    if (!p) return FE_ERR_INVALID_ARG;
    if (!p->adj) return FE_ERR_NOT_BUILT;
    if (block) *block = p->B;
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
    out->block = p->B;
    out->uniform_runs = p->uniform_runs ? 1 : 0;
    out->atomic_order = p->elem_order ? 1 : 0;
    out->device_bytes = p->device_bytes;
    return FE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// CSR pattern build that allocates nothing (fe_pattern_csr_noalloc).
//
// For callers that must not allocate device memory: a library embedded in a
// host application that owns every byte of HBM through its own allocator, a
// real-time or latency-bound loop that cannot afford cudaMalloc's implicit
// device synchronisation, or code running where an allocation is not
// permitted.  Its working memory is the fixed array below, which every GPU
// that loads this library keeps until the process exits.

#define FE_NOALLOC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char fe_noalloc_scratch[FE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NS_THREADS = 1024;
constexpr int NS_TILE = 4096;  // elements per tile; at most NS_TILE tiles

__global__ void k_ns_tile_sums(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums)
{
    __shared__ int64_t red[NS_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * NS_TILE;
    int64_t s = 0;
    for (int k = threadIdx.x; k < NS_TILE; k += blockDim.x)
        if (base + k < n) s += in[base + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < NS_THREADS / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

// One block: exclusive scan of `tiles` sums in place (serial per thread
// chunk, then across chunks).
__global__ void k_ns_scan_sums(int64_t *sums, int tiles)
{
    __shared__ int64_t part[NS_THREADS];
    const int per = (tiles + NS_THREADS - 1) / NS_THREADS;
    const int lo = threadIdx.x * per, hi = min(tiles, lo + per);
    int64_t s = 0;
    for (int k = lo; k < hi; ++k) s += sums[k];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int k = 0; k < NS_THREADS; ++k) {
            const int64_t x = part[k];
            part[k] = run;
            run += x;
        }
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int k = lo; k < hi; ++k) {
        const int64_t x = sums[k];
        sums[k] = run;
        run += x;
    }
}

// out[i] = offs[tile] + in[tile_base] + ... + in[i-1]; out[n] = total.
__global__ void k_ns_tile_scan(const int32_t *__restrict__ in, int64_t n, const int64_t *__restrict__ offs,
                               int64_t *__restrict__ out)
{
    __shared__ int64_t wsum[NS_THREADS / 32];
    constexpr int PER = NS_TILE / NS_THREADS;
    const int64_t base = (int64_t)blockIdx.x * NS_TILE + (int64_t)threadIdx.x * PER;
    int64_t x[PER], local = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        x[k] = base + k < n ? in[base + k] : 0;
        local += x[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t v = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int64_t run = offs[blockIdx.x] + incl - local + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (base + k < n) out[base + k] = run;
        run += x[k];
        if (base + k == n - 1) out[n] = run;
    }
}

// Bump allocation inside the fixed scratch array.
struct Bump {
    unsigned char *base;
    size_t used, cap;
    void *take(size_t bytes)
    {
        const size_t at = (used + 255) & ~(size_t)255;
        used = at + bytes;
        return used <= cap ? base + at : nullptr;
    }
};

int ns_scan(const int32_t *in, int64_t *out, int64_t n, int64_t *tile_sums, cudaStream_t s)
{
    const int64_t tiles = std::max<int64_t>(1, (n + NS_TILE - 1) / NS_TILE);
    if (tiles > NS_TILE) return FE_ERR_UNSUPPORTED;
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s) == cudaSuccess ? FE_OK : FE_ERR_DEVICE;
    FE_LAUNCH((k_ns_tile_sums<<<(unsigned)tiles, NS_THREADS, 0, s>>>(in, n, tile_sums)));
    FE_LAUNCH((k_ns_scan_sums<<<1, NS_THREADS, 0, s>>>(tile_sums, (int)tiles)));
    FE_LAUNCH((k_ns_tile_scan<<<(unsigned)tiles, NS_THREADS, 0, s>>>(in, n, tile_sums, out)));
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

int noalloc_impl(unsigned char *scratch, int64_t n_e, int32_t n_loc, int64_t n_dofs, const int32_t *elem_dofs,
                 int64_t *row_ptr, int32_t *col_idx, int64_t col_capacity, int64_t *nnz_out, cudaStream_t s)
{
    int dev = 0, sms = 0;
    FE_CUDA(cudaGetDevice(&dev));
    FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // Only the status words are taken before validation; the other arrays are
    // carved once the block size B (and so the node count) is known, so that
    // blocked meshes (3 DOFs per node: keys B^2 = 9 times smaller) may use the
    // whole array.  Every array that must start at zero is cleared here: the
    // array keeps the previous call's contents.
    Bump bump{scratch, 0, FE_NOALLOC_SCRATCH_BYTES};
    int64_t *sc = (int64_t *)bump.take(sizeof(int64_t) * S_COUNT);
    if (!sc) return FE_ERR_UNSUPPORTED;
    FE_CUDA(cudaMemsetAsync(sc, 0, sizeof(int64_t) * S_COUNT, s));
    FE_CUDA(cudaMemsetAsync(sc + S_BLOCKS, 0xff, sizeof(int64_t), s));

    int64_t h[S_COUNT];
    if (n_e > 0) {
        uint32_t cand = 0;
        for (int b = 2; b <= 32; ++b)
            if (n_loc % b == 0 && n_dofs % b == 0) cand |= 1u << (b - 1);
        if (n_loc <= 32)
            FE_LAUNCH((k_validate<1><<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(elem_dofs, n_e, n_loc, n_dofs,
                                                                                      cand, sc)));
        else
            FE_LAUNCH((k_validate<FE_MAX_NLOC / 32><<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(
                elem_dofs, n_e, n_loc, n_dofs, cand, sc)));
        FE_CUDA(cudaGetLastError());
    }
    FE_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    if (h[S_ERR] != 0) return (int)h[S_ERR];
    int B = 1;
    for (int b = 32; b >= 2 && n_e > 0; --b)
        if ((((uint32_t)h[S_BLOCKS] >> (b - 1)) & 1u) && n_loc % b == 0 && n_dofs % b == 0) {
            B = b;
            break;
        }
    const int32_t nln = n_loc / B;
    const int64_t n_nodes = n_dofs / B, n_ninc = n_e * nln;
    const int mw = (nln + 31) / 32;
    int32_t *deg = (int32_t *)bump.take(sizeof(int32_t) * (size_t)(n_nodes + 1));
    int32_t *runs = (int32_t *)bump.take(sizeof(int32_t) * (size_t)(n_e + 1));
    int32_t *N = (int32_t *)bump.take(sizeof(int32_t) * (size_t)(n_ninc + 1));
    uint32_t *run_mask = (uint32_t *)bump.take(sizeof(uint32_t) * (size_t)(n_e * mw + 1));
    int64_t *adj_ptr = (int64_t *)bump.take(sizeof(int64_t) * (size_t)(n_nodes + 1));
    uint32_t *adj = (uint32_t *)bump.take(sizeof(uint32_t) * (size_t)(n_ninc + 1));
    int32_t *node_len = (int32_t *)bump.take(sizeof(int32_t) * (size_t)(n_nodes + 1));
    int32_t *node_runs2 = (int32_t *)bump.take(sizeof(int32_t) * (size_t)(n_nodes + 1));
    int32_t *keys = (int32_t *)bump.take(sizeof(int32_t) * (size_t)(n_ninc * nln + 1));
    int64_t *nrp = (int64_t *)bump.take(sizeof(int64_t) * (size_t)(n_nodes + 1));
    int64_t *ncp = (int64_t *)bump.take(sizeof(int64_t) * (size_t)(n_nodes + 1));
    int64_t *crac_ptr = (int64_t *)bump.take(sizeof(int64_t) * (size_t)(n_dofs + 1));
    int64_t *tile_sums = (int64_t *)bump.take(sizeof(int64_t) * (size_t)NS_TILE);
    // the bump only grows, so the last array failing means the mesh does not fit
    if (!tile_sums) return FE_ERR_UNSUPPORTED;
    FE_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    if (n_e > 0) {
        FE_LAUNCH((k_node_conn<<<fe_grid_for(n_e * 32, 256, sms, 16), 256, 0, s>>>(elem_dofs, n_e, n_loc, B, nln, mw, N,
                                                                                run_mask, runs, deg, sc)));
        FE_LAUNCH((k_max_i32<<<fe_grid_for(n_nodes, 256, sms, 8), 256, 0, s>>>(deg, n_nodes, sc + S_MAX_DEG)));
        FE_CUDA(cudaGetLastError());
    }
    FE_TRY(ns_scan(deg, adj_ptr, n_nodes, tile_sums, s));
    FE_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n_nodes + 1), s));
    if (n_ninc > 0) {
        FE_LAUNCH((k_fill_adj<<<fe_grid_for(n_ninc, 256, sms, 16), 256, 0, s>>>(N, n_ninc, n_nodes, adj_ptr, deg, adj)));
        FE_LAUNCH((k_sort_adj<<<fe_grid_for(n_nodes, 128, sms, 16), 128, 0, s>>>(adj_ptr, n_nodes, adj)));
        FE_CUDA(cudaGetLastError());
    }
    FE_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    const int64_t cand = h[S_MAX_DEG] * nln;
    if (n_nodes > 0) {
        const int grid = fe_grid_for(n_nodes * 32, 256, sms, 8);
        if (cand <= 32) {
            FE_LAUNCH((k_row_keys<1><<<grid, 256, 0, s>>>(N, nln, n_nodes, adj_ptr, adj, node_len, node_runs2, keys, sc)));
        } else if (cand <= 64) {
            FE_LAUNCH((k_row_keys<2><<<grid, 256, 0, s>>>(N, nln, n_nodes, adj_ptr, adj, node_len, node_runs2, keys, sc)));
        } else if (cand <= 128) {
            FE_LAUNCH((k_row_keys<4><<<grid, 256, 0, s>>>(N, nln, n_nodes, adj_ptr, adj, node_len, node_runs2, keys, sc)));
        } else if (cand <= REG_SORT_MAX) {
            FE_LAUNCH((k_row_keys<8><<<grid, 256, 0, s>>>(N, nln, n_nodes, adj_ptr, adj, node_len, node_runs2, keys, sc)));
        } else {
            int P = 32;
            while (P < cand) P <<= 1;
            if ((int64_t)P * 4 > 128 * 1024) return FE_ERR_UNSUPPORTED;
            const int W = (int)std::max<int64_t>(1, std::min<int64_t>(8, (64 * 1024) / ((int64_t)P * 4)));
            const size_t smem = (size_t)W * P * 4;
            FE_TRY(configure_smem(k_row_keys_smem, smem));
            FE_LAUNCH((k_row_keys_smem<<<fe_grid_for(n_nodes * 32, W * 32, sms, std::max(1, 64 / W)), W * 32, smem,
                                         s>>>(N, nln, n_nodes, adj_ptr, adj, P, node_len, node_runs2, keys, sc)));
        }
        FE_CUDA(cudaGetLastError());
    }
    FE_TRY(ns_scan(node_len, nrp, n_nodes, tile_sums, s));
    FE_TRY(ns_scan(node_runs2, ncp, n_nodes, tile_sums, s));
    int64_t node_nnz = 0;
    FE_CUDA(cudaMemcpyAsync(&node_nnz, nrp + n_nodes, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    const int64_t nnz = (int64_t)B * B * node_nnz;
    if (nnz_out) *nnz_out = nnz;
    if (nnz >= INT32_MAX) return FE_ERR_OVERFLOW;
    if (col_capacity < nnz) return FE_ERR_INVALID_ARG;  // *nnz_out tells the caller how much to provide
    if (n_nodes > 0) {
        // rows longer than the staging capacity read their keys from global memory
        FE_LAUNCH((k_expand<0><<<fe_grid_for(n_nodes * 32, 256, sms, 8), 256, (size_t)8 * 256 * 4, s>>>(
            n_nodes, B, nln, adj_ptr, keys, node_len, node_runs2, nrp, ncp, row_ptr, crac_ptr, col_idx, nullptr, 256)));
    }
    FE_LAUNCH((k_tail<<<1, 1, 0, s>>>(row_ptr, crac_ptr, nrp, ncp, n_nodes, n_dofs, B)));
    FE_CUDA(cudaGetLastError());
    FE_CUDA(cudaStreamSynchronize(s));
    return FE_OK;
}

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {};

}  // namespace

extern "C" int fe_pattern_csr_noalloc(int64_t n_elem, int32_t dofs_per_elem, int64_t n_dofs, const int32_t *elem_dofs,
                                      int64_t *row_ptr, int32_t *col_idx, int64_t col_capacity, int64_t *nnz,
                                      void *stream)
{
    if (nnz) *nnz = 0;
    if (n_elem < 0 || dofs_per_elem <= 0 || n_dofs < 0 || !row_ptr || col_capacity < 0) return FE_ERR_INVALID_ARG;
    if (n_elem > 0 && (!elem_dofs || !col_idx)) return FE_ERR_INVALID_ARG;
    if (dofs_per_elem > FE_MAX_NLOC) return FE_ERR_UNSUPPORTED;
    if (n_dofs >= INT32_MAX || n_elem * (int64_t)dofs_per_elem >= (int64_t)UINT32_MAX) return FE_ERR_OVERFLOW;
    int dev = 0;
    FE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return FE_ERR_UNSUPPORTED;
    void *scratch = nullptr;
    {
        // first call on a device: look up the device address of the array
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) FE_CUDA(cudaGetSymbolAddress(&g_noalloc_addr[dev], fe_noalloc_scratch));
        scratch = g_noalloc_addr[dev];
    }
    return noalloc_impl((unsigned char *)scratch, n_elem, dofs_per_elem, n_dofs, elem_dofs, row_ptr, col_idx,
                        col_capacity, nnz, (cudaStream_t)stream);
}

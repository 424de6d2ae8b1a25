// Row-locked assembly with the spin_int lock of the paper (Listings 3-5):
// the row pointer array is its own lock array.  A row is locked by turning
// its row pointer v into a negative number with a compare-and-swap and
// unlocked by writing v back; the locked thread then adds the element's row
// (as contiguous slices of its DOF runs, Listing 5) with plain loads and
// stores.  The locked value is ~v (= -v - 1) rather than -v, so that the
// first row, whose pointer is 0, can be locked too.
//
// GPU form: one warp per element; lane 0 takes the row's lock with a bounded
// spin, the warp adds K_e(r, :) with L2-coherent loads and stores, lane 0
// releases it.  A warp never waits while holding a lock, so there is no
// deadlock; a spin that runs out records FE_ERR_TIMEOUT and skips the row
// (the result is then incomplete and the status says so).
#include "assemble_body.cuh"
#include "internal.cuh"

using namespace fe_dev;

namespace {

constexpr int LOCK_SPIN_LOG2_DEFAULT = 22;  // compare-and-swap attempts per lock: 2^22

template <int NLN, int BB, typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_rowlock(const double *__restrict__ K, int64_t n_e, Geo g,
                                                 const MT *__restrict__ map, const MT *__restrict__ mapc,
                                                 int64_t *locks, double *values, int *status, uint32_t spin_limit)
{
    constexpr int NLOC = NLN * BB;
    constexpr int NN = NLOC * NLOC;
    const int lane = threadIdx.x & 31;
    for (int64_t e = fe_warp_id(); e < n_e; e += fe_warps()) {
        const int32_t nd = lane < NLN ? g.N[e * NLN + lane] : 0;
        int kk = 0, koff = 0, nr = 0;
        int64_t rp = 0;
        if (CRAC) {
            const uint32_t m = g.uniform_R ? g.run_mask[0] : g.run_mask[e];
            if (lane < NLN) run_of(m, lane, kk, koff);
            if (g.uniform_R) {
                nr = g.uniform_R;
                rp = e * nr;
            } else {
                rp = g.run_ptr[e];
                nr = (int)(g.run_ptr[e + 1] - rp);
            }
        }
        // this lane's column c = lane: its block and position inside the runs
        const int c = lane < NLOC ? lane : 0;
        const int kc = c / BB;
        const int k_c = __shfl_sync(0xffffffffu, kk, kc);
        const int off_c = __shfl_sync(0xffffffffu, koff, kc);
        const double *Ke = K + e * NN;
        for (int r = 0; r < NLOC; ++r) {
            const int64_t row = (int64_t)BB * __shfl_sync(0xffffffffu, nd, r / BB) + r % BB;
            unsigned long long *lk = (unsigned long long *)(locks + row);
            int64_t v = 0;
            int got = 0;
            if (lane == 0) {
                v = (int64_t)*(volatile long long *)lk;
                if (v < 0) v = ~v;
                for (uint32_t it = 0; it < spin_limit; ++it) {
                    if (atomicCAS(lk, (unsigned long long)v, (unsigned long long)~v) == (unsigned long long)v) {
                        got = 1;
                        break;
                    }
                }
                if (got) __threadfence();
                else atomicCAS(status, 0, FE_ERR_TIMEOUT);
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            v = __shfl_sync(0xffffffffu, v, 0);
            if (!got) continue;
            // the row's start: CSR row pointer, or the first value position of the CRAC pairs
            const int64_t base = CRAC ? (int64_t)g.col_align[v + 1] : v;
            if (lane < NLOC) {
                int pos;
                if (!CRAC) pos = (int)map[(e * NLN + r / BB) * NLN + kc];
                else pos = (int)mapc[rp * NLN + (r / BB) * nr + k_c] + off_c;
                if (FE_IN_BOUNDS(base + (int64_t)BB * pos + c % BB, g.nnz, g.status)) {
                    double *dst = values + base + (int64_t)BB * pos + c % BB;
                    __stcg(dst, __ldcg(dst) + __ldcs(Ke + r * NLOC + c));
                }
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicExch(lk, (unsigned long long)v);
            }
            __syncwarp();
        }
    }
}

// Any element size (n_loc <= FE_MAX_NLOC): the same protocol, the warp
// striding over the columns of the locked row; run positions of the column
// blocks staged in shared memory per warp.
template <typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_rowlock_generic(const double *__restrict__ K, int64_t n_e, int32_t nln,
                                                         int32_t B, Geo g, const MT *__restrict__ map,
                                                         const MT *__restrict__ mapc, int64_t *locks, double *values,
                                                         int *status, uint32_t spin_limit)
{
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
            for (int kc = lane; kc < nln; kc += 32)
                run_of_multi(g.run_mask + e * g.mask_words, kc, k_s[w][kc], off_s[w][kc]);
            __syncwarp();
        }
        const double *Ke = K + e * NN;
        for (int r = 0; r < n_loc; ++r) {
            const int64_t row = (int64_t)B * g.N[e * nln + r / B] + r % B;
            unsigned long long *lk = (unsigned long long *)(locks + row);
            int64_t v = 0;
            int got = 0;
            if (lane == 0) {
                v = (int64_t)*(volatile long long *)lk;
                if (v < 0) v = ~v;
                for (uint32_t it = 0; it < spin_limit; ++it) {
                    if (atomicCAS(lk, (unsigned long long)v, (unsigned long long)~v) == (unsigned long long)v) {
                        got = 1;
                        break;
                    }
                }
                if (got) __threadfence();
                else atomicCAS(status, 0, FE_ERR_TIMEOUT);
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            v = __shfl_sync(0xffffffffu, v, 0);
            if (!got) continue;
            const int64_t base = CRAC ? (int64_t)g.col_align[v + 1] : v;
            for (int c = lane; c < n_loc; c += 32) {
                const int kc = c / B;
                int pos;
                if (!CRAC) pos = (int)map[(e * nln + r / B) * nln + kc];
                else pos = (int)mapc[rp * nln + (int64_t)(r / B) * nr + k_s[w][kc]] + off_s[w][kc];
                if (!FE_IN_BOUNDS(base + (int64_t)B * pos + c % B, g.nnz, g.status)) continue;
                double *dst = values + base + (int64_t)B * pos + c % B;
                __stcg(dst, __ldcg(dst) + __ldcs(Ke + (int64_t)r * n_loc + c));
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicExch(lk, (unsigned long long)v);
            }
            __syncwarp();
        }
    }
}

}  // namespace

int fe_assemble_rowlock(const fe_pattern *p, const double *K, double *values, int accumulate, bool crac,
                        cudaStream_t s)
{
    if (!accumulate) FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)p->nnz, s));
    if (p->n_e == 0) return FE_OK;
    const Geo g = geo_of(p);
    int64_t *locks = crac ? p->crac_ptr : p->row_ptr;  // the row pointers are the locks (restored on exit)
    const int sms = p->ctx->num_sms;
    int *st = p->ctx->d_status;
    const int lg = p->ctx->knob[FE_KNOB_LOCK_SPIN] > 0 ? p->ctx->knob[FE_KNOB_LOCK_SPIN] : LOCK_SPIN_LOG2_DEFAULT;
    const uint32_t spin = 1u << lg;
#define FE_RL(NLN_, BB_)                                                                                            \
    do {                                                                                                            \
        if (p->map_bytes == 1) {                                                                                    \
            if (crac)                                                                                               \
                k_rowlock<NLN_, BB_, uint8_t, true><<<fe_grid_resident(k_rowlock<NLN_, BB_, uint8_t, true>, p->n_e * 32, 256, sms), 256, 0, s>>>(K, p->n_e, g, (const uint8_t *)p->map_csr,  \
                                                                         (const uint8_t *)p->map_crac, locks,        \
                                                                         values, st, spin);                                \
            else                                                                                                    \
                k_rowlock<NLN_, BB_, uint8_t, false><<<fe_grid_resident(k_rowlock<NLN_, BB_, uint8_t, false>, p->n_e * 32, 256, sms), 256, 0, s>>>(K, p->n_e, g, (const uint8_t *)p->map_csr, \
                                                                          (const uint8_t *)p->map_crac, locks,       \
                                                                          values, st, spin);                               \
        } else {                                                                                                    \
            if (crac)                                                                                               \
                k_rowlock<NLN_, BB_, uint16_t, true><<<fe_grid_resident(k_rowlock<NLN_, BB_, uint16_t, true>, p->n_e * 32, 256, sms), 256, 0, s>>>(                                           \
                    K, p->n_e, g, (const uint16_t *)p->map_csr, (const uint16_t *)p->map_crac, locks, values, st, spin);   \
            else                                                                                                    \
                k_rowlock<NLN_, BB_, uint16_t, false><<<fe_grid_resident(k_rowlock<NLN_, BB_, uint16_t, false>, p->n_e * 32, 256, sms), 256, 0, s>>>(                                          \
                    K, p->n_e, g, (const uint16_t *)p->map_csr, (const uint16_t *)p->map_crac, locks, values, st, spin);   \
        }                                                                                                           \
    } while (0)
    if (p->nln == 8 && p->B == 3) FE_RL(8, 3);
    else if (p->nln == 10 && p->B == 3) FE_RL(10, 3);
    else if (p->nln == 8 && p->B == 1) FE_RL(8, 1);
    else if (p->nln == 4 && p->B == 1) FE_RL(4, 1);
    else if (p->map_bytes == 1) {
        if (crac)
            k_rowlock_generic<uint8_t, true><<<fe_grid_resident(k_rowlock_generic<uint8_t, true>, p->n_e * 32, 256, sms), 256, 0, s>>>(K, p->n_e, p->nln, p->B, g,
                                                                  (const uint8_t *)p->map_csr,
                                                                  (const uint8_t *)p->map_crac, locks, values, st, spin);
        else
            k_rowlock_generic<uint8_t, false><<<fe_grid_resident(k_rowlock_generic<uint8_t, false>, p->n_e * 32, 256, sms), 256, 0, s>>>(K, p->n_e, p->nln, p->B, g,
                                                                   (const uint8_t *)p->map_csr,
                                                                   (const uint8_t *)p->map_crac, locks, values, st, spin);
    } else {
        if (crac)
            k_rowlock_generic<uint16_t, true><<<fe_grid_resident(k_rowlock_generic<uint16_t, true>, p->n_e * 32, 256, sms), 256, 0, s>>>(K, p->n_e, p->nln, p->B, g,
                                                                   (const uint16_t *)p->map_csr,
                                                                   (const uint16_t *)p->map_crac, locks, values, st, spin);
        else
            k_rowlock_generic<uint16_t, false><<<fe_grid_resident(k_rowlock_generic<uint16_t, false>, p->n_e * 32, 256, sms), 256, 0, s>>>(K, p->n_e, p->nln, p->B, g,
                                                                    (const uint16_t *)p->map_csr,
                                                                    (const uint16_t *)p->map_crac, locks, values, st, spin);
    }
#undef FE_RL
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

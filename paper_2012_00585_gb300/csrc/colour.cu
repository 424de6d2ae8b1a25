// Greedy element colouring and colour-ordered, atomic-free assembly (the
// colouring method of Listing 6: colours one after another, the elements of
// one colour in parallel, no locks, because elements of one colour share no
// DOF).
//
// The colouring is the sequential first-fit of the greedy algorithm: elements
// in ascending order, each taking the smallest colour not used by an
// already-coloured element sharing a DOF.  On the GPU it is computed in
// dependency waves: in every pass each uncoloured element whose lower-
// numbered neighbours are all coloured takes the smallest colour they do not
// use -- exactly what the sequential loop gives it -- so the result equals
// the sequential colouring, element by element.
#include <vector>

#include "assemble_body.cuh"
#include "internal.cuh"

using namespace fe_dev;

namespace {

constexpr int MAX_COLOURS = 256;

// One pass over the elements.  colour[] holds -1 for uncoloured elements;
// writes are final, so a concurrent reader sees either -1 or the colour.
__global__ void k_colour_pass(const int32_t *__restrict__ N, int64_t n_e, int32_t nln,
                              const int64_t *__restrict__ adj_ptr, const uint32_t *__restrict__ adj,
                              int32_t *colour, int *remaining, int *overflow)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_e; e += (int64_t)gridDim.x * blockDim.x) {
        if (((volatile int32_t *)colour)[e] >= 0) continue;
        uint64_t used[MAX_COLOURS / 64] = {0, 0, 0, 0};
        bool ready = true;
        for (int k = 0; k < nln && ready; ++k) {
            const int32_t nd = N[e * nln + k];
            for (int64_t s = adj_ptr[nd]; s < adj_ptr[nd + 1]; ++s) {
                const int64_t f = adj[s] / (uint32_t)nln;
                if (f >= e) break;  // lists are ascending: the rest are higher-numbered
                const int32_t c = ((volatile int32_t *)colour)[f];
                if (c < 0) {
                    ready = false;
                    break;
                }
                used[c >> 6] |= 1ull << (c & 63);
            }
        }
        if (!ready) {
            *remaining = 1;
            continue;
        }
        int c = 0;
        while (c < MAX_COLOURS && ((used[c >> 6] >> (c & 63)) & 1ull)) ++c;
        if (c == MAX_COLOURS) {
            *overflow = 1;
            c = MAX_COLOURS - 1;
        }
        ((volatile int32_t *)colour)[e] = c;
    }
}

__global__ void k_colour_count(const int32_t *__restrict__ colour, int64_t n_e, int32_t *count)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_e; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&count[colour[e]], 1);
}

__global__ void k_colour_scatter(const int32_t *__restrict__ colour, int64_t n_e, const int64_t *__restrict__ ptr,
                                 int32_t *cursor, int32_t *elems)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_e; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = colour[e];
        elems[ptr[c] + atomicAdd(&cursor[c], 1)] = (int32_t)e;
    }
}

// The elements of one colour, a warp each, plain read-modify-write adds.
template <int NLN, int BB, typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_colour_assemble(const double *__restrict__ K,
                                                         const int32_t *__restrict__ elems, int64_t count, Geo g,
                                                         const MT *__restrict__ map, const MT *__restrict__ mapc,
                                                         double *values)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = fe_warp_id(); i < count; i += fe_warps())
        atomic_element<NLN, BB, MT, CRAC, true>(K, elems[i], g, map, mapc, values, lane);
}

template <typename MT, bool CRAC>
__global__ void __launch_bounds__(256) k_colour_assemble_generic(const double *__restrict__ K,
                                                                 const int32_t *__restrict__ elems, int64_t count,
                                                                 int32_t nln, int32_t B, Geo g,
                                                                 const MT *__restrict__ map,
                                                                 const MT *__restrict__ mapc, double *values)
{
    __shared__ int64_t base_s[8][FE_MAX_NLOC];
    __shared__ int32_t k_s[8][FE_MAX_NLOC];
    __shared__ int32_t off_s[8][FE_MAX_NLOC];
    const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) & 7;
    for (int64_t i = fe_warp_id(); i < count; i += fe_warps())
        atomic_element_generic<MT, CRAC, true>(K, elems[i], nln, B, g, map, mapc, values, base_s[w], k_s[w],
                                               off_s[w], lane);
}

template <typename MT, bool CRAC>
int launch_colour(const fe_pattern *p, const double *K, const int32_t *elems, int64_t count, double *values,
                  cudaStream_t s)
{
    const Geo g = geo_of(p);
    const int sms = p->ctx->num_sms;
    const MT *map = (const MT *)p->map_csr, *mapc = (const MT *)p->map_crac;
    if (p->nln == 8 && p->B == 3)
        k_colour_assemble<8, 3, MT, CRAC><<<fe_grid_resident(k_colour_assemble<8, 3, MT, CRAC>, count * 32, 256, sms), 256, 0, s>>>(K, elems, count, g, map, mapc, values);
    else if (p->nln == 10 && p->B == 3)
        k_colour_assemble<10, 3, MT, CRAC><<<fe_grid_resident(k_colour_assemble<10, 3, MT, CRAC>, count * 32, 256, sms), 256, 0, s>>>(K, elems, count, g, map, mapc, values);
    else if (p->nln == 8 && p->B == 1)
        k_colour_assemble<8, 1, MT, CRAC><<<fe_grid_resident(k_colour_assemble<8, 1, MT, CRAC>, count * 32, 256, sms), 256, 0, s>>>(K, elems, count, g, map, mapc, values);
    else if (p->nln == 4 && p->B == 1)
        k_colour_assemble<4, 1, MT, CRAC><<<fe_grid_resident(k_colour_assemble<4, 1, MT, CRAC>, count * 32, 256, sms), 256, 0, s>>>(K, elems, count, g, map, mapc, values);
    else
        k_colour_assemble_generic<MT, CRAC><<<fe_grid_resident(k_colour_assemble_generic<MT, CRAC>, count * 32, 256, sms), 256, 0, s>>>(K, elems, count, p->nln, p->B, g, map, mapc, values);
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

}  // namespace

// Colouring state stored with the pattern.
struct fe_colouring {
    int32_t n_colours = 0;
    int32_t *colour = nullptr;    // [n_e]
    int64_t *ptr = nullptr;       // device [n_colours + 1]
    int32_t *elems = nullptr;     // [n_e] elements grouped by colour
    std::vector<int64_t> host_ptr;
};

void fe_colouring_free(fe_pattern *p, cudaStream_t s)
{
    if (!p->colouring) return;
    fe_free_async(p->colouring->colour, s);
    fe_free_async(p->colouring->ptr, s);
    fe_free_async(p->colouring->elems, s);
    delete p->colouring;
    p->colouring = nullptr;
}

extern "C" {

int fe_pattern_colour(fe_ctx *ctx, fe_pattern *p, void *stream, int32_t *n_colours)
{
    if (!ctx || !p || p->ctx != ctx) return FE_ERR_INVALID_ARG;
    if (!p->adj) return FE_ERR_NOT_BUILT;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe_colouring_free(p, s);
    fe_colouring *cl = new fe_colouring();
    p->colouring = cl;
    const int64_t n_e = p->n_e;
    int rc = FE_OK;
    int *flags = nullptr;  // [0] remaining, [1] overflow
    int32_t *count = nullptr;
    auto fail = [&](int code) {
        fe_free_async(flags, s);
        fe_free_async(count, s);
        cudaStreamSynchronize(s);
        fe_colouring_free(p, s);
        if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
        return code;
    };
    if ((rc = fe_alloc(ctx, (void **)&cl->colour, sizeof(int32_t) * (size_t)(n_e + 1), s)) != FE_OK) return fail(rc);
    if ((rc = fe_alloc(ctx, (void **)&flags, sizeof(int) * 2, s)) != FE_OK) return fail(rc);
    if (cudaMemsetAsync(cl->colour, 0xff, sizeof(int32_t) * (size_t)(n_e + 1), s) != cudaSuccess) return fail(FE_ERR_DEVICE);
    const int grid = fe_grid_for(n_e, 256, ctx->num_sms, 8);
    int h[2] = {1, 0};
    int passes = 0;
    // waves: a few passes between host checks; at most n_e waves in total
    while (h[0] && n_e > 0) {
        if (cudaMemsetAsync(flags, 0, sizeof(int) * 2, s) != cudaSuccess) return fail(FE_ERR_DEVICE);
        for (int k = 0; k < 8; ++k) {
            k_colour_pass<<<grid, 256, 0, s>>>(p->node_dofs, n_e, p->nln, p->adj_ptr, p->adj, cl->colour, flags,
                                               flags + 1);
            fe_note_launch();
        }
        if (cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return fail(FE_ERR_DEVICE);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FE_ERR_DEVICE);
        if (h[1]) return fail(FE_ERR_UNSUPPORTED);  // more than MAX_COLOURS colours
        passes += 8;
        if (passes > n_e + 8) return fail(FE_ERR_DEVICE);
    }
    // groups: count, scan on the host (few colours), scatter
    if ((rc = fe_alloc(ctx, (void **)&count, sizeof(int32_t) * MAX_COLOURS * 2, s)) != FE_OK) return fail(rc);
    if (cudaMemsetAsync(count, 0, sizeof(int32_t) * MAX_COLOURS * 2, s) != cudaSuccess) return fail(FE_ERR_DEVICE);
    if (n_e > 0) {
        k_colour_count<<<grid, 256, 0, s>>>(cl->colour, n_e, count);
        fe_note_launch();
    }
    std::vector<int32_t> hc(MAX_COLOURS);
    if (cudaMemcpyAsync(hc.data(), count, sizeof(int32_t) * MAX_COLOURS, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(FE_ERR_DEVICE);
    int nc = 0;
    for (int c = 0; c < MAX_COLOURS; ++c)
        if (hc[c] > 0) nc = c + 1;
    cl->n_colours = nc;
    cl->host_ptr.assign(nc + 1, 0);
    for (int c = 0; c < nc; ++c) cl->host_ptr[c + 1] = cl->host_ptr[c] + hc[c];
    if ((rc = fe_alloc(ctx, (void **)&cl->ptr, sizeof(int64_t) * (size_t)(nc + 1), s)) != FE_OK) return fail(rc);
    if ((rc = fe_alloc(ctx, (void **)&cl->elems, sizeof(int32_t) * (size_t)(n_e + 1), s)) != FE_OK) return fail(rc);
    if (cudaMemcpyAsync(cl->ptr, cl->host_ptr.data(), sizeof(int64_t) * (nc + 1), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return fail(FE_ERR_DEVICE);
    if (n_e > 0) {
        k_colour_scatter<<<grid, 256, 0, s>>>(cl->colour, n_e, cl->ptr, count + MAX_COLOURS, cl->elems);
        fe_note_launch();
    }
    fe_free_async(flags, s);
    fe_free_async(count, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(FE_ERR_DEVICE);
    if (n_colours) *n_colours = nc;
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return FE_OK;
}

int fe_pattern_colours(const fe_pattern *p, int32_t *n_colours, const int32_t **colour)
{
    if (!p) return FE_ERR_INVALID_ARG;
    if (!p->colouring) return FE_ERR_NOT_BUILT;
    if (n_colours) *n_colours = p->colouring->n_colours;
    if (colour) *colour = p->colouring->colour;
    return FE_OK;
}

}  // extern "C"

// Colour-ordered assembly used by fe_assemble_csr / fe_assemble_crac with
// FE_COLOURED: values reset (unless accumulating), then one launch per colour.
int fe_assemble_coloured(const fe_pattern *p, const double *K, double *values, int accumulate, bool crac,
                         cudaStream_t s)
{
    if (!p->colouring) return FE_ERR_NOT_BUILT;
    if (!accumulate) FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)p->nnz, s));
    const fe_colouring *cl = p->colouring;
    for (int c = 0; c < cl->n_colours; ++c) {
        const int64_t a = cl->host_ptr[c], count = cl->host_ptr[c + 1] - a;
        if (count == 0) continue;
        int rc;
        if (p->map_bytes == 1)
            rc = crac ? launch_colour<uint8_t, true>(p, K, cl->elems + a, count, values, s)
                      : launch_colour<uint8_t, false>(p, K, cl->elems + a, count, values, s);
        else
            rc = crac ? launch_colour<uint16_t, true>(p, K, cl->elems + a, count, values, s)
                      : launch_colour<uint16_t, false>(p, K, cl->elems + a, count, values, s);
        if (rc != FE_OK) return rc;
    }
    return FE_OK;
}

// Serving loop: assembly requests arrive at any time; the library admits
// them by HBM footprint, keeps their patterns (and slot maps) resident in a
// cache keyed by mesh, builds missing patterns on a separate thread, and
// launches the ready requests together as batched assemblies on several
// streams, so that requests arriving while others run are admitted as memory
// frees up and their work overlaps on the GPU (continuous batching).
//
// Element values of a request are either given (device K) or generated on
// the device after admission as K_e = alpha_e * K_ref, with alpha_e = 0.5 +
// u_e and u_e the top 20 bits of splitmix64(seed + e) / 2^20 (Steele, Lea,
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the
// 64-bit finaliser of Vigna's splitmix64), one exact IEEE multiply per entry.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "internal.cuh"

namespace {

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// K_e = alpha_e * K_ref for every element; one thread per entry.
__global__ void k_generate_scaled(const double *__restrict__ k_ref, int32_t nn, int64_t n_e, uint64_t seed,
                                  double *__restrict__ K)
{
    const int64_t total = n_e * nn;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = x / nn;
        const int q = (int)(x - e * nn);
        const double alpha = 0.5 + (double)(splitmix64(seed + (uint64_t)e) >> 44) * (1.0 / 1048576.0);
        K[x] = alpha * k_ref[q];
    }
}

int launch_generate(const double *k_ref, int32_t n_loc, int64_t n_e, uint64_t seed, double *K, int sms,
                    cudaStream_t s)
{
    if (n_e == 0) return FE_OK;
    const int64_t total = n_e * n_loc * n_loc;
    k_generate_scaled<<<fe_grid_for(total, 256, sms, 16), 256, 0, s>>>(k_ref, n_loc * n_loc, n_e, seed, K);
    fe_note_launch();
    FE_CUDA(cudaGetLastError());
    return FE_OK;
}

double now_us()
{
    using namespace std::chrono;
    return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

struct Ticket {
    fe_request req{};
    int state = FE_STATE_PENDING;
    int status = FE_OK;
    int cold = 0;
    fe_pattern *pattern = nullptr;
    double *values = nullptr;  // library-owned until fe_release
    double *K = nullptr;       // generated element matrices, freed at completion
    size_t foot = 0;           // bytes charged against the budget
    size_t k_bytes = 0, v_bytes = 0, v_charged = 0;
    double t_submit = 0, t_admit = 0, t_ready = 0, t_start = 0, t_done = 0;
    int stream = -1;
};

struct CacheEntry {
    fe_pattern *p = nullptr;
    size_t bytes = 0;
    int refs = 0;
    int64_t uses = 0;  // requests admitted on this key so far
    uint64_t last_use = 0;
    bool building = false;
};

struct Group {
    std::vector<uint64_t> ids;
    cudaEvent_t t0 = nullptr;    // recorded before the group's first kernel
    cudaEvent_t done = nullptr;  // recorded after its last
    int stream = 0;
};

// A request of a group being launched: what the launch needs, copied from its
// ticket under the lock, and what the launch produces.
struct Member {
    uint64_t id;
    Ticket *t;
    fe_request req;
    const fe_pattern *pattern;
    size_t k_bytes, v_bytes;
    double *values = nullptr, *K = nullptr;
    int rc = FE_OK;
};

struct LaunchJob {
    Group g;
    std::vector<Member> mem;
    int fmt = 0, mode = 0;
    bool big = false;
    double share = 1.0;  // of the resident blocks the group's kernels take
};

// Requests of at least this many element-matrix entries are launched alone
// on a high-priority stream: they are not grouped with small requests (whose
// completion would wait for theirs), and the GPU's block scheduler serves
// their kernels first, so that their latency stays near their own device
// time while small requests fill the SMs around them.
constexpr int64_t BIG_ENTRIES = (int64_t)1 << 26;
constexpr int N_BIG_STREAMS = 2;
// Share of the GPU's resident blocks a large request's kernels take (the
// rest stays free for pattern builds and small requests), and the share
// small groups take while a large request runs (so that it keeps most of the
// memory bandwidth; small requests still progress beside it).
constexpr double BIG_SHARE = 0.75;
constexpr double SMALL_SHARE_BESIDE_BIG = 0.25;
// Tiles a warp of a small group's kernel takes before its block exits.
constexpr int SMALL_MAX_TILES = 2;

bool is_big(const fe_request &r) { return r.n_elem * (int64_t)r.dofs_per_elem * r.dofs_per_elem >= BIG_ENTRIES; }

// Keys of evicted patterns remembered to count rebuilds (bounded).
constexpr size_t EVICTED_KEYS_MAX = 1 << 20;
// Device spans kept for fe_server_timeline (bounded).
constexpr size_t TIMELINE_MAX = 1 << 21;

}  // namespace

struct fe_server {
    fe_ctx *ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv, cv_build, cv_done;
    std::deque<uint64_t> pending, to_build, ready;
    std::list<Group> inflight;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::unordered_map<uint64_t, CacheEntry> cache;
    size_t budget = 0, in_use = 0;
    size_t cache_bytes = 0;  // bytes of the built patterns in the cache (part of in_use)
    std::vector<cudaStream_t> streams;          // n_small launch streams, then n_big high-priority ones
    int n_small = 0, n_big = 0, next_big = 0;
    int inflight_big = 0;  // launched large groups not yet complete
    cudaStream_t build_stream = nullptr;       // = build_streams[0]; evicted patterns are freed on it
    std::vector<cudaStream_t> build_streams;   // one per builder thread
    int next_stream = 0, max_batch = 64;
    uint64_t next_id = 1, clock = 0;
    int active = 0;            // admitted and not finished
    bool strict_fifo = false;  // one request at a time, end to end
    bool stop = false;
    std::thread sched;
    std::vector<std::thread> builders;
    // large requests are launched by a thread of their own: their device
    // allocations (gigabytes, which can take milliseconds) then do not hold
    // up the scheduler's launches of small groups
    std::deque<LaunchJob> big_jobs;
    std::condition_variable cv_big;
    std::thread big_launcher;
    fe_server_stats stats{};
    cudaEvent_t t_ref = nullptr;               // origin of the timeline (server start)
    std::vector<fe_span> timeline;             // device spans of launched groups and builds
    std::unordered_set<uint64_t> evicted_keys; // for the rebuild count
};

namespace {

size_t pattern_estimate(const fe_request &r)
{
    // generous upper bound of a pattern built from n_e elements of n_loc DOFs
    const size_t ninc = (size_t)r.n_elem * r.dofs_per_elem;
    return ninc * r.dofs_per_elem * 6 + (size_t)r.n_dofs * 64 + ((size_t)1 << 20);
}

size_t values_estimate(const fe_request &r, const fe_pattern *p)
{
    if (p) return (size_t)p->nnz * 8;
    return (size_t)r.n_elem * r.dofs_per_elem * r.dofs_per_elem * 8;  // nnz <= entries
}

// Evict unreferenced cached patterns until `need` more bytes fit.  Victims
// are taken among patterns no request holds and no queued request will use
// (evicting one of those would only make that request rebuild it): patterns
// used by a single request so far first (one-off meshes), then the rest,
// least recently used first within each class, so that a stream of one-off
// meshes does not push out the meshes that are reassembled again and again.
// No request holds a victim, so none of its device work is in flight (a
// request drops its hold only after its completion event was seen, and the
// builder waits for each build): its memory is released stream-ordered on the
// build stream, without a host wait under the lock.  Caller holds the lock.
void evict_for(fe_server *sv, size_t need, std::unordered_set<uint64_t> &wanted, bool &wanted_ready)
{
    if (!wanted_ready) {  // keys queued requests will use, gathered once per admission pass
        for (uint64_t id : sv->pending) wanted.insert(sv->tickets[id].req.pattern_key);
        wanted_ready = true;
    }
    while (sv->in_use + need > sv->budget) {
        uint64_t victim = 0;
        bool found = false;
        std::pair<int, uint64_t> best{2, UINT64_MAX};
        for (auto &kv : sv->cache) {
            const CacheEntry &ce = kv.second;
            if (ce.refs != 0 || ce.building || wanted.count(kv.first)) continue;
            const std::pair<int, uint64_t> rank{ce.uses > 1 ? 1 : 0, ce.last_use};
            if (rank < best) {
                best = rank;
                victim = kv.first;
                found = true;
            }
        }
        if (!found) return;
        CacheEntry ce = sv->cache[victim];
        sv->cache.erase(victim);
        sv->in_use -= std::min(ce.bytes, sv->in_use);
        sv->cache_bytes -= std::min(ce.bytes, sv->cache_bytes);
        ++sv->stats.evictions;
        if (sv->evicted_keys.size() >= EVICTED_KEYS_MAX) sv->evicted_keys.clear();
        sv->evicted_keys.insert(victim);
        fe_pattern_free_async(ce.p, sv->build_stream);
    }
}

void finish(fe_server *sv, Ticket &t, int status)
{
    if (t.t_admit > 0 && sv->active > 0) --sv->active;
    t.status = status;
    t.state = status == FE_OK ? FE_STATE_DONE : FE_STATE_FAILED;
    t.t_done = now_us();
    if (status == FE_OK) ++sv->stats.completed; else ++sv->stats.failed;
    sv->cv_done.notify_all();
}

// Device span [t0, t1] of completed work, in ms after the server's start.
void record_span(fe_server *sv, cudaEvent_t t0, cudaEvent_t t1, int32_t stream, int32_t n_requests)
{
    float a = 0.f, b = 0.f;
    if (sv->timeline.size() >= TIMELINE_MAX || !t0 || !t1) return;
    if (cudaEventElapsedTime(&a, sv->t_ref, t0) != cudaSuccess || cudaEventElapsedTime(&b, sv->t_ref, t1) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    sv->timeline.push_back(fe_span{(double)a, (double)b, stream, n_requests});
}

bool expired(const Ticket &t, double now)
{
    return t.req.deadline_s > 0 && now > t.t_submit + t.req.deadline_s * 1e6;
}

// The watchdog: requests whose deadline passed before they were launched
// fail with FE_ERR_TIMEOUT; those already admitted give their memory and
// their hold on the cached pattern back.  Requests waiting for a pattern
// build are checked when the build completes.  Caller holds the lock.
bool expire_overdue(fe_server *sv)
{
    const double now = now_us();
    bool any = false;
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        Ticket &t = sv->tickets[*it];
        if (t.state == FE_STATE_PENDING && expired(t, now)) {
            ++sv->stats.expired;
            finish(sv, t, FE_ERR_TIMEOUT);
            it = sv->pending.erase(it);
            any = true;
        } else {
            ++it;
        }
    }
    for (auto it = sv->ready.begin(); it != sv->ready.end();) {
        Ticket &t = sv->tickets[*it];
        if (t.state == FE_STATE_ADMITTED && expired(t, now)) {
            sv->in_use -= std::min(t.foot, sv->in_use);
            t.foot = 0;
            auto ce = sv->cache.find(t.req.pattern_key);
            if (ce != sv->cache.end() && ce->second.refs > 0) ce->second.refs--;
            t.pattern = nullptr;
            ++sv->stats.expired;
            finish(sv, t, FE_ERR_TIMEOUT);
            it = sv->ready.erase(it);
            any = true;
        } else {
            ++it;
        }
    }
    return any;
}

// Launch one group: its requests' values and generated K, the element
// generation and the batched assembly on the group's stream, with the lock
// released (an allocation that grows the memory pool can take
// milliseconds); then the outcome is booked.  Called with the lock held;
// returns with it held.  The members are RUNNING meanwhile: no other thread
// touches a RUNNING ticket (release, cancel and the watchdog skip it).
void run_launch(fe_server *sv, LaunchJob &job, std::unique_lock<std::mutex> &lk)
{
    Group &g = job.g;
    cudaStream_t s = sv->streams[g.stream];
    lk.unlock();
    const double t_launch = now_us();
    if (cudaEventCreate(&g.t0) != cudaSuccess || cudaEventRecord(g.t0, s) != cudaSuccess) {
        cudaGetLastError();
        if (g.t0) cudaEventDestroy(g.t0);
        g.t0 = nullptr;
    }
    std::vector<fe_batch_item> items;
    double alloc_ms = 0.0;
    const int gen_sms = std::max(1, (int)(sv->ctx->num_sms * job.share));
    for (Member &m : job.mem) {
        const double a0 = now_us();
        m.rc = fe_alloc(sv->ctx, (void **)&m.values, m.v_bytes, s);
        if (m.rc == FE_OK && !m.req.elem_mats) m.rc = fe_alloc(sv->ctx, (void **)&m.K, m.k_bytes, s);
        alloc_ms += (now_us() - a0) * 1e-3;
        if (m.rc == FE_OK && !m.req.elem_mats)
            m.rc = launch_generate(m.req.k_ref, m.req.dofs_per_elem, m.req.n_elem, m.req.seed, m.K, gen_sms, s);
        if (m.rc == FE_OK && m.req.ready_event) cudaStreamWaitEvent(s, (cudaEvent_t)m.req.ready_event, 0);
        if (m.rc == FE_OK) items.push_back(fe_batch_item{m.pattern, m.K ? m.K : m.req.elem_mats, m.values});
    }
    int rc = FE_OK;
    if (!items.empty()) {
        FeRange range("serve: batched launch");
        // a large request: a persistent grid on a share of the GPU, on a
        // high-priority stream; a small group: blocks of a few tiles each,
        // so that SMs turn over often and the high-priority streams' kernels
        // (pattern builds, large requests) are not held behind it
        rc = fe_assemble_batch_share(sv->ctx, items.data(), (int32_t)items.size(), job.fmt, job.mode, 0, s,
                                     job.share, job.big ? 0 : SMALL_MAX_TILES);
        if (rc == FE_OK && cudaEventCreate(&g.done) != cudaSuccess) rc = FE_ERR_DEVICE;
        if (rc == FE_OK && cudaEventRecord(g.done, s) != cudaSuccess) rc = FE_ERR_DEVICE;
    }
    lk.lock();
    sv->stats.alloc_ms_total += alloc_ms;
    sv->stats.alloc_ms_max = std::max(sv->stats.alloc_ms_max, alloc_ms);
    for (Member &m : job.mem) {
        Ticket &t = *m.t;
        t.values = m.values;
        t.K = m.K;
        t.v_bytes = m.v_bytes;
        if (m.rc != FE_OK || rc != FE_OK) {
            finish(sv, t, m.rc != FE_OK ? m.rc : rc);
            continue;
        }
        // footprint: the values charge becomes exact
        if (t.v_charged > t.v_bytes) {
            const size_t drop = t.v_charged - t.v_bytes;
            t.foot -= std::min(drop, t.foot);
            sv->in_use -= std::min(drop, sv->in_use);
            t.v_charged = t.v_bytes;
        }
        t.t_start = t_launch;
        g.ids.push_back(m.id);
    }
    if (g.ids.empty()) {
        if (g.done) cudaEventDestroy(g.done);
        if (g.t0) cudaEventDestroy(g.t0);
        return;
    }
    ++sv->stats.launches;
    sv->stats.batched_requests += g.ids.size();
    if (g.stream >= sv->n_small) ++sv->inflight_big;
    sv->inflight.push_back(std::move(g));
    sv->cv.notify_one();
}

// The large requests' launcher thread.
void big_launch_loop(fe_server *sv)
{
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        if (sv->big_jobs.empty()) {
            sv->cv_big.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        LaunchJob job = std::move(sv->big_jobs.front());
        sv->big_jobs.pop_front();
        run_launch(sv, job, lk);
    }
}

// Admission, launches and completions; runs on the scheduler thread.
void scheduler_loop(fe_server *sv)
{
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progress = false;
        // completions
        for (auto it = sv->inflight.begin(); it != sv->inflight.end();) {
            const cudaError_t q = cudaEventQuery(it->done);
            if (q == cudaErrorNotReady) {
                ++it;
                continue;
            }
            const int st = q == cudaSuccess ? FE_OK : FE_ERR_DEVICE;
            if (st == FE_OK) record_span(sv, it->t0, it->done, it->stream, (int32_t)it->ids.size());
            for (uint64_t id : it->ids) {
                Ticket &t = sv->tickets[id];
                if (t.K) {
                    fe_free_async(t.K, sv->streams[it->stream]);
                    t.K = nullptr;
                    sv->in_use -= t.k_bytes;
                    t.foot -= t.k_bytes;
                }
                finish(sv, t, st);
            }
            if (it->stream >= sv->n_small && sv->inflight_big > 0) --sv->inflight_big;
            cudaEventDestroy(it->t0);
            cudaEventDestroy(it->done);
            it = sv->inflight.erase(it);
            progress = true;
            sv->cv_done.notify_all();
        }
        if (expire_overdue(sv)) progress = true;
        // admission, in arrival order.  A request that does not fit waits
        // for memory; requests behind it keep their order, except that small
        // ones (a footprint under 1/16 of the budget) may pass a waiting
        // large one: their memory turns over within milliseconds, so the
        // large request still gets its memory as soon as in-flight large
        // work completes, while small requests do not queue behind it.
        bool blocked = false;
        std::unordered_set<uint64_t> wanted;
        bool wanted_ready = false;
        int passed = 0;  // requests looked at behind a waiting one (bounded: the lock is held)
        for (auto it = sv->pending.begin(); it != sv->pending.end();) {
            if (blocked && ++passed > 256) break;
            const uint64_t id = *it;
            Ticket &t = sv->tickets[id];
            if (t.state == FE_STATE_CANCELLED) {
                it = sv->pending.erase(it);
                continue;
            }
            auto ce = sv->cache.find(t.req.pattern_key);
            const bool cached = ce != sv->cache.end();
            const fe_pattern *p = cached && !ce->second.building ? ce->second.p : nullptr;
            const size_t k_bytes = t.req.elem_mats ? 0 : (size_t)t.req.n_elem * t.req.dofs_per_elem * t.req.dofs_per_elem * 8;
            const size_t v_est = values_estimate(t.req, p);
            const size_t need = k_bytes + v_est + (cached ? 0 : pattern_estimate(t.req));
            if (need > sv->budget) {
                it = sv->pending.erase(it);
                finish(sv, t, FE_ERR_ADMISSION);
                progress = true;
                continue;
            }
            if (sv->strict_fifo && sv->active > 0) break;
            const bool small = need <= sv->budget / 16;
            if (blocked && (!small || sv->strict_fifo)) {
                ++it;  // behind a waiting request: only small ones pass
                continue;
            }
            if (sv->in_use + need > sv->budget) evict_for(sv, need, wanted, wanted_ready);
            if (sv->in_use + need > sv->budget) {  // wait for memory to free up
                if (!blocked) ++sv->stats.admission_waits;
                blocked = true;
                if (sv->strict_fifo) break;
                ++it;
                continue;
            }
            it = sv->pending.erase(it);
            sv->in_use += need;
            sv->stats.peak_bytes_in_use = std::max(sv->stats.peak_bytes_in_use, (int64_t)sv->in_use);
            t.foot = need;
            t.k_bytes = k_bytes;
            t.v_charged = v_est;
            t.t_admit = now_us();
            t.state = FE_STATE_ADMITTED;
            ++sv->active;
            ++sv->stats.admitted;
            progress = true;
            if (cached) {
                ce->second.refs++;
                ce->second.uses++;
                ce->second.last_use = ++sv->clock;
                if (ce->second.building) {
                    sv->to_build.push_back(id);  // the builder hands it on when the pattern exists
                } else {
                    t.pattern = ce->second.p;
                    t.t_ready = t.t_admit;
                    sv->ready.push_back(id);
                }
            } else {
                CacheEntry &ne = sv->cache[t.req.pattern_key];
                ne.building = true;
                ne.refs = 1;
                ne.uses = 1;
                ne.last_use = ++sv->clock;
                t.cold = 1;
                sv->to_build.push_back(id);
                sv->cv_build.notify_one();
            }
        }
        // launches: ready requests grouped by (format, mode), taken from
        // the ready queue under the lock and marked RUNNING.  A small group
        // is launched here (run_launch); a large request is handed to the
        // large-request launcher thread.
        while (!sv->ready.empty()) {
            const uint64_t id0 = sv->ready.front();
            const int fmt = sv->tickets[id0].req.format, mode = sv->tickets[id0].req.mode;
            // a big request goes alone on a high-priority stream; otherwise
            // the group takes small requests only
            const bool big = sv->n_big > 0 && is_big(sv->tickets[id0].req);
            Group g;
            if (big) {
                g.stream = sv->n_small + sv->next_big;
                sv->next_big = (sv->next_big + 1) % sv->n_big;
            } else {
                g.stream = sv->next_stream;
                sv->next_stream = (sv->next_stream + 1) % sv->n_small;
            }
            std::vector<Member> mem;
            const int cap = big ? 1 : sv->max_batch;
            for (auto it = sv->ready.begin(); it != sv->ready.end() && (int)mem.size() < cap;) {
                Ticket &t = sv->tickets[*it];
                if (t.req.format != fmt || t.req.mode != mode || (sv->n_big > 0 && is_big(t.req) != big)) {
                    ++it;
                    continue;
                }
                if (t.state == FE_STATE_CANCELLED) {
                    it = sv->ready.erase(it);
                    continue;
                }
                t.state = FE_STATE_RUNNING;
                t.stream = g.stream;
                mem.push_back(Member{*it, &t, t.req, t.pattern, t.k_bytes, (size_t)t.pattern->nnz * 8});
                it = sv->ready.erase(it);
            }
            if (mem.empty()) continue;
            progress = true;
            LaunchJob job;
            job.g = std::move(g);
            job.mem = std::move(mem);
            job.fmt = fmt;
            job.mode = mode;
            job.big = big;
            job.share = big ? BIG_SHARE
                            : (sv->inflight_big > 0 || !sv->big_jobs.empty() ? SMALL_SHARE_BESIDE_BIG : 1.0);
            if (big) {
                sv->big_jobs.push_back(std::move(job));
                sv->cv_big.notify_one();
            } else {
                run_launch(sv, job, lk);
            }
        }
        if (!progress) sv->cv.wait_for(lk, std::chrono::microseconds(sv->inflight.empty() ? 2000 : 20));
    }
}

// Cold requests: build the pattern, publish it in the cache, pass the
// request (and any that waited for the same key) on to the ready queue.
// Several builder threads, each on its own stream, so that the builds of
// different meshes (each waits on the host to size its arrays) overlap.
constexpr int N_BUILDERS = 2;

void builder_loop(fe_server *sv, int idx)
{
    cudaStream_t bs = sv->build_streams[idx];
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        uint64_t id = 0;
        for (auto it = sv->to_build.begin(); it != sv->to_build.end(); ++it) {
            Ticket &t = sv->tickets[*it];
            CacheEntry &ce = sv->cache[t.req.pattern_key];
            if (!ce.building) {  // built meanwhile by another request
                t.pattern = ce.p;
                t.t_ready = now_us();
                sv->ready.push_back(*it);
                sv->to_build.erase(it);
                sv->cv.notify_one();
                id = UINT64_MAX;
                break;
            }
            if (t.cold) {
                id = *it;
                sv->to_build.erase(it);
                break;
            }
        }
        if (id == UINT64_MAX) continue;
        if (id == 0) {
            sv->cv_build.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        const fe_request req = sv->tickets[id].req;
        lk.unlock();
        fe_pattern *p = nullptr;
        FeRange range("serve: pattern build");
        cudaEvent_t b0 = nullptr, b1 = nullptr;
        if (cudaEventCreate(&b0) != cudaSuccess || cudaEventCreate(&b1) != cudaSuccess) cudaGetLastError();
        if (b0) cudaEventRecord(b0, bs);
        int rc = fe_pattern_build(sv->ctx, req.n_elem, req.dofs_per_elem, req.n_dofs, req.elem_dofs, FE_PATTERN_ALL,
                                  bs, &p);
        if (b1) cudaEventRecord(b1, bs);
        if (rc == FE_OK) rc = cudaStreamSynchronize(bs) == cudaSuccess ? FE_OK : FE_ERR_DEVICE;
        lk.lock();
        if (rc == FE_OK && b0 && b1) record_span(sv, b0, b1, -1, 1);
        if (b0) cudaEventDestroy(b0);
        if (b1) cudaEventDestroy(b1);
        Ticket &t = sv->tickets[id];
        CacheEntry &ce = sv->cache[req.pattern_key];
        ++sv->stats.patterns_built;
        if (sv->evicted_keys.erase(req.pattern_key)) ++sv->stats.rebuilds;
        if (rc != FE_OK) {
            sv->in_use -= std::min(t.foot, sv->in_use);
            t.foot = 0;
            finish(sv, t, rc);
            sv->cache.erase(req.pattern_key);
            // requests that waited for this key fail with it
            for (auto it = sv->to_build.begin(); it != sv->to_build.end();) {
                Ticket &w = sv->tickets[*it];
                if (w.req.pattern_key == req.pattern_key) {
                    sv->in_use -= std::min(w.foot, sv->in_use);
                    w.foot = 0;
                    finish(sv, w, rc);
                    it = sv->to_build.erase(it);
                } else {
                    ++it;
                }
            }
            sv->cv_done.notify_all();
            continue;
        }
        ce.p = p;
        ce.bytes = (size_t)p->device_bytes;
        sv->cache_bytes += ce.bytes;
        ce.building = false;
        // the estimate charged to this request becomes the pattern's real size
        const size_t est = pattern_estimate(req);
        sv->in_use = sv->in_use - std::min(est, sv->in_use) + ce.bytes;
        t.foot = t.foot - std::min(est, t.foot);
        t.pattern = p;
        t.t_ready = now_us();
        sv->ready.push_back(id);
        sv->cv.notify_one();
    }
}

int release_ticket(fe_server *sv, uint64_t id)
{
    auto it = sv->tickets.find(id);
    if (it == sv->tickets.end()) return FE_ERR_NOT_FOUND;
    Ticket &t = it->second;
    if (t.state == FE_STATE_RUNNING || t.state == FE_STATE_ADMITTED) return FE_ERR_INVALID_ARG;
    cudaStream_t s = t.stream >= 0 ? sv->streams[t.stream] : sv->streams[0];
    if (t.values) fe_free_async(t.values, s);
    if (t.K) fe_free_async(t.K, s);
    sv->in_use -= std::min(t.foot, sv->in_use);
    if (t.pattern) {
        auto ce = sv->cache.find(t.req.pattern_key);
        if (ce != sv->cache.end() && ce->second.refs > 0) ce->second.refs--;
    }
    sv->tickets.erase(it);
    return FE_OK;
}

void fill_result(const Ticket &t, fe_result *out)
{
    out->status = t.status;
    out->state = t.state;
    out->cold = t.cold;
    out->nnz = t.pattern ? t.pattern->nnz : 0;
    out->row_ptr = t.pattern ? t.pattern->row_ptr : nullptr;
    out->col_idx = t.pattern ? t.pattern->col_idx : nullptr;
    out->values = t.state == FE_STATE_DONE ? t.values : nullptr;
    out->t_submit_us = t.t_submit;
    out->t_admit_us = t.t_admit;
    out->t_start_us = t.t_start;
    out->t_done_us = t.t_done;
    out->t_ready_us = t.t_ready;
}

}  // namespace

extern "C" {

int fe_server_start(fe_ctx *ctx, int32_t n_streams, int32_t max_batch, size_t hbm_budget_bytes, fe_server **out)
{
    if (!ctx || !out || n_streams < 1 || n_streams > 64 || max_batch < 1) return FE_ERR_INVALID_ARG;
    *out = nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    fe_server *sv = new fe_server();
    sv->ctx = ctx;
    sv->budget = hbm_budget_bytes ? hbm_budget_bytes : ctx->hbm_budget;
    sv->max_batch = max_batch;
    sv->strict_fifo = n_streams == 1 && max_batch == 1;
    int rc = FE_OK;
    for (int k = 0; k < n_streams && rc == FE_OK; ++k) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) rc = FE_ERR_DEVICE;
        else sv->streams.push_back(s);
    }
    sv->n_small = n_streams;
    if (!sv->strict_fifo) {
        int least = 0, greatest = 0;
        if (rc == FE_OK && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) rc = FE_ERR_DEVICE;
        for (int k = 0; k < N_BIG_STREAMS && rc == FE_OK; ++k) {
            cudaStream_t s;
            if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess) rc = FE_ERR_DEVICE;
            else sv->streams.push_back(s);
        }
        if (rc == FE_OK) sv->n_big = N_BIG_STREAMS;
    }
    // pattern builds are on the critical path of every cold request: their
    // streams take the highest priority, like the large requests' launches
    int least = 0, greatest = 0;
    if (rc == FE_OK && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) rc = FE_ERR_DEVICE;
    for (int k = 0; k < N_BUILDERS && rc == FE_OK; ++k) {
        cudaStream_t s;
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess) rc = FE_ERR_DEVICE;
        else sv->build_streams.push_back(s);
    }
    if (rc == FE_OK) sv->build_stream = sv->build_streams[0];
    if (rc == FE_OK && (cudaEventCreate(&sv->t_ref) != cudaSuccess || cudaEventRecord(sv->t_ref, sv->streams[0]) != cudaSuccess ||
                        cudaEventSynchronize(sv->t_ref) != cudaSuccess))
        rc = FE_ERR_DEVICE;
    if (rc != FE_OK) {
        for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
        for (cudaStream_t s : sv->build_streams) cudaStreamDestroy(s);
        if (sv->t_ref) cudaEventDestroy(sv->t_ref);
        delete sv;
        if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
        return rc;
    }
    sv->sched = std::thread(scheduler_loop, sv);
    for (int k = 0; k < N_BUILDERS; ++k) sv->builders.emplace_back(builder_loop, sv, k);
    sv->big_launcher = std::thread(big_launch_loop, sv);
    *out = sv;
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return FE_OK;
}

int fe_server_stop(fe_server *sv)
{
    if (!sv) return FE_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    sv->cv_build.notify_all();
    sv->cv_big.notify_all();
    sv->sched.join();
    for (auto &t : sv->builders) t.join();
    sv->big_launcher.join();
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != sv->ctx->device) cudaSetDevice(sv->ctx->device);
    for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
    for (cudaStream_t s : sv->build_streams) cudaStreamSynchronize(s);
    for (auto &g : sv->inflight) {
        cudaEventDestroy(g.done);
        if (g.t0) cudaEventDestroy(g.t0);
    }
    for (auto &kv : sv->tickets) {
        if (kv.second.values) cudaFreeAsync(kv.second.values, sv->streams[0]);
        if (kv.second.K) cudaFreeAsync(kv.second.K, sv->streams[0]);
    }
    cudaStreamSynchronize(sv->streams[0]);
    for (auto &kv : sv->cache)
        if (kv.second.p) fe_pattern_free(kv.second.p);
    for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
    for (cudaStream_t s : sv->build_streams) cudaStreamDestroy(s);
    cudaEventDestroy(sv->t_ref);
    const int dev = sv->ctx->device;
    delete sv;
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return FE_OK;
}

int fe_batch_submit(fe_server *sv, const fe_request *reqs, int32_t n, uint64_t *tickets)
{
    if (!sv || n < 0 || (n > 0 && (!reqs || !tickets))) return FE_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        const fe_request &r = reqs[k];
        if (r.n_elem < 0 || r.dofs_per_elem <= 0 || r.n_dofs < 0 || (!r.elem_mats && !r.k_ref) || !(r.deadline_s >= 0) ||
            (r.format != FE_FORMAT_CSR && r.format != FE_FORMAT_CRAC) ||
            (r.mode != FE_ATOMIC && r.mode != FE_DETERMINISTIC))
            return FE_ERR_INVALID_ARG;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const double t0 = now_us();
        for (int k = 0; k < n; ++k) {
            const uint64_t id = sv->next_id++;
            Ticket &t = sv->tickets[id];
            t.req = reqs[k];
            t.t_submit = t0;
            sv->pending.push_back(id);
            tickets[k] = id;
            ++sv->stats.submitted;
        }
    }
    sv->cv.notify_one();
    return FE_OK;
}

int fe_poll(fe_server *sv, uint64_t ticket, fe_result *out)
{
    if (!sv || !out) return FE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return FE_ERR_NOT_FOUND;
    fill_result(it->second, out);
    return FE_OK;
}

int fe_wait(fe_server *sv, uint64_t ticket, double timeout_s, fe_result *out)
{
    if (!sv || !out) return FE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds((int64_t)(timeout_s * 1e6));
    for (;;) {
        auto it = sv->tickets.find(ticket);
        if (it == sv->tickets.end()) return FE_ERR_NOT_FOUND;
        const int st = it->second.state;
        if (st == FE_STATE_DONE || st == FE_STATE_FAILED || st == FE_STATE_CANCELLED) {
            fill_result(it->second, out);
            return FE_OK;
        }
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto again = sv->tickets.find(ticket);
            if (again == sv->tickets.end()) return FE_ERR_NOT_FOUND;
            fill_result(again->second, out);
            const int s2 = again->second.state;
            return (s2 == FE_STATE_DONE || s2 == FE_STATE_FAILED || s2 == FE_STATE_CANCELLED) ? FE_OK : FE_ERR_TIMEOUT;
        }
    }
}

int fe_cancel(fe_server *sv, uint64_t ticket)
{
    if (!sv) return FE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return FE_ERR_NOT_FOUND;
    Ticket &t = it->second;
    if (t.state != FE_STATE_PENDING) return FE_ERR_INVALID_ARG;  // only requests not yet admitted
    t.state = FE_STATE_CANCELLED;
    t.status = FE_ERR_CANCELLED;
    t.t_done = now_us();
    ++sv->stats.cancelled;
    sv->cv_done.notify_all();
    return FE_OK;
}

int fe_release(fe_server *sv, uint64_t ticket)
{
    if (!sv) return FE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    const int rc = release_ticket(sv, ticket);
    sv->cv.notify_one();
    return rc;
}

int fe_server_stats_get(fe_server *sv, fe_server_stats *out)
{
    if (!sv || !out) return FE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->bytes_in_use = (int64_t)sv->in_use;
    out->budget_bytes = (int64_t)sv->budget;
    out->cached_patterns = (int64_t)sv->cache.size();
    out->n_pending = (int64_t)sv->pending.size();
    out->n_to_build = (int64_t)sv->to_build.size();
    out->n_ready = (int64_t)sv->ready.size();
    out->n_big_jobs = (int64_t)sv->big_jobs.size();
    int64_t running = 0;
    for (const Group &g : sv->inflight) running += (int64_t)g.ids.size();
    out->n_running = running;
    out->n_inflight_groups = (int64_t)sv->inflight.size();
    return FE_OK;
}

int fe_server_timeline(fe_server *sv, int64_t first, int64_t cap, fe_span *out, int64_t *n_total)
{
    if (!sv || first < 0 || cap < 0 || (cap > 0 && !out)) return FE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    const int64_t n = (int64_t)sv->timeline.size();
    if (n_total) *n_total = n;
    for (int64_t k = first; k < n && k - first < cap; ++k) out[k - first] = sv->timeline[k];
    return FE_OK;
}

int fe_generate_scaled(fe_ctx *ctx, const double *k_ref, int32_t n_loc, int64_t n_elem, uint64_t seed, double *out,
                       void *stream)
{
    if (!ctx || !out || (n_elem > 0 && !k_ref) || n_loc <= 0 || n_elem < 0) return FE_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    const int rc = launch_generate(k_ref, n_loc, n_elem, seed, out, ctx->num_sms, (cudaStream_t)stream);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

}  // extern "C"

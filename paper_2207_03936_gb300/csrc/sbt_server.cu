// Continuous-batching request loop.
//
// Two host threads share a set of stream slots:
//   - the launcher admits pending events in arrival order while a slot is
//     free and the device-memory budget allows, and enqueues the group on the
//     slot's stream: upload (straight from the submitter's pinned batch when
//     the events are consecutive in it), reconstruction on the slot's own
//     handle, download of the results into a pinned result block, event record;
//   - the harvester watches the slots' events and publishes finished requests
//     (no copies: a request refers to its batch's result block).
// Several slots are in flight at once, so events arriving while others run on
// the GPU are admitted as soon as a slot and memory free up, and their work
// overlaps on the device.  No device code ever waits on host state.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sbt_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// Allocations made by the servers of this process (device and pinned host),
// for the stats: in steady state a server allocates nothing.
std::atomic<int64_t> g_allocs{0};

// Device and pinned host buffers of the slots and result blocks.  They grow
// with headroom (a quarter above the request, at least half again the old
// size) and keep the buffers they outgrow until release(): cudaFree and
// cudaFreeHost synchronise the device, which would stall every other slot's
// work in flight.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    std::vector<T*> retired;
    cudaError_t reserve(size_t want)
    {
        if (want <= n) return cudaSuccess;
        want = std::max(want + want / 4, n + n / 2);
        T* q = nullptr;
        cudaError_t e = cudaMalloc(&q, sizeof(T) * std::max<size_t>(want, 1));
        if (e != cudaSuccess) return e;
        g_allocs.fetch_add(1);
        if (p) retired.push_back(p);
        p = q;
        n = want;
        return cudaSuccess;
    }
    void release()
    {
        for (T* q : retired) cudaFree(q);
        retired.clear();
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <class T>
struct HostBuf {
    T* p = nullptr;
    size_t n = 0;
    std::vector<T*> retired;
    cudaError_t reserve(size_t want)
    {
        if (want <= n) return cudaSuccess;
        want = std::max(want + want / 4, n + n / 2);
        T* q = nullptr;
        cudaError_t e = cudaMallocHost(&q, sizeof(T) * std::max<size_t>(want, 1));
        if (e != cudaSuccess) return e;
        g_allocs.fetch_add(1);
        if (p) retired.push_back(p);
        p = q;
        n = want;
        return cudaSuccess;
    }
    void release()
    {
        for (T* q : retired) cudaFreeHost(q);
        retired.clear();
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

// Pinned copy of a scheduled batch.
// Pinned host copy of a scheduled batch (x, y, z, module of `cap` hits).
// Batches are pooled by the server: the last request that refers to one
// returns it to the pool (freeing gigabytes of pinned memory takes tens of
// milliseconds, which would hold up the results being published), and the
// next schedule reuses it when it is large enough; at most kPinnedPool idle
// batches are kept (the smallest go first).
constexpr size_t kPinnedPool = 2;  // idle pinned batches a server keeps for reuse

struct PinnedBatch {
    float *x = nullptr, *y = nullptr, *z = nullptr;
    int32_t* m = nullptr;
    size_t cap = 0;
    bool alloc(size_t hits)
    {
        const size_t nb = sizeof(float) * std::max<size_t>(hits, 1);
        if (cudaMallocHost(&x, nb) != cudaSuccess || cudaMallocHost(&y, nb) != cudaSuccess ||
            cudaMallocHost(&z, nb) != cudaSuccess || cudaMallocHost(&m, nb) != cudaSuccess)
            return false;
        g_allocs.fetch_add(1);
        cap = std::max<size_t>(hits, 1);
        return true;
    }
    ~PinnedBatch()
    {
        if (x) cudaFreeHost(x);
        if (y) cudaFreeHost(y);
        if (z) cudaFreeHost(z);
        if (m) cudaFreeHost(m);
    }
};

// One event to reconstruct.  Its hits live in the request's own vectors
// (sbt_server_submit) or in a pinned batch of the open-loop feeder
// (sbt_server_submit_schedule), kept alive by `hold`.
struct Request {
    int64_t id = 0;
    std::vector<float> ox, oy, oz;
    std::vector<int32_t> om;
    const float *x = nullptr, *y = nullptr, *z = nullptr;
    const int32_t* m = nullptr;
    int32_t n = 0;
    bool pinned = false;
    std::shared_ptr<void> hold;
    double t_submit = 0.0;
};

// Pinned downloads of one batch; shared by its requests until all of them
// are drained or polled, then recycled.
struct ResultBlock {
    HostBuf<int32_t> to, ho, th, stat;
    HostBuf<float> params, chi2;
    std::vector<int32_t> first_hit;  // batch hit index of each request's first hit
    int refs = 0;
};

struct Finished {
    int64_t id = 0;
    int32_t status = 0;
    double latency = 0.0;
    ResultBlock* block = nullptr;  // null for a failed batch
    int k = 0;
};

// A polled request's results, in event-local indices.
struct Materialized {
    std::vector<int32_t> hit_offsets, track_hits;
    std::vector<float> params, chi2;
};

struct Slot {
    sbt_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t_up = nullptr, t_kern = nullptr, t_down = nullptr;  // timing: before uploads,
                                                                     // kernels, downloads
    double t_enqueued = 0.0;  // host clock when the batch was handed to the slot
    std::atomic<bool> busy{false};
    bool failed = false;
    int64_t bytes = 0;
    std::vector<Request> reqs;
    ResultBlock* block = nullptr;
    DevBuf<float> dx, dy, dz, dparams, dchi2;
    DevBuf<int32_t> dm, doff, dto, dho, dth, dndof, dstat, dcounts;
    HostBuf<float> hx, hy, hz;
    HostBuf<int32_t> hm, hoff;
};

// Device bytes one batch needs (inputs, outputs and the plain workspace):
// per hit 16 B inputs, 18 B sorted hits, about 45 B search scratch (claims,
// links, lists, tracklets, forming and final tracks), about 12 B staging and
// about 13 B outputs, rounded up.
int64_t batch_bytes(int64_t hits, int64_t events)
{
    return hits * 112 + events * 320 + (1 << 16);
}

}  // namespace

struct sbt_server {
    int device = 0;
    int64_t budget = 0;
    int32_t max_batch = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<Finished> finished;
    std::map<int64_t, Materialized> polled;
    std::vector<ResultBlock*> free_blocks;
    std::vector<std::unique_ptr<ResultBlock>> all_blocks;
    std::vector<std::unique_ptr<PinnedBatch>> pinned_pool;  // batches no request refers to
    std::atomic<bool> stop{false};
    std::atomic<bool> launcher_done{false};
    std::atomic<bool> inject{false};
    int64_t in_flight_bytes = 0;
    double st_completed = 0, st_submitted = 0, st_batches = 0, st_events_batched = 0,
           st_peak_bytes = 0, st_failed = 0, st_feed_lag = 0;
    // per-batch time sums (ms): uploads, kernels, downloads on the slot's
    // stream (CUDA events), and enqueue to harvest on the host clock
    double st_up_ms = 0, st_kern_ms = 0, st_down_ms = 0, st_wall_ms = 0, st_timed = 0;
    std::atomic<double> st_launch_s{0.0};  // launcher time spent enqueueing batches
    int64_t allocs0 = 0;                    // g_allocs when the server was created
    std::thread launcher, harvester, feeder;
};

namespace {

void unref_block(sbt_server* S, ResultBlock* b)  // S->mu held
{
    if (b && --b->refs == 0) S->free_blocks.push_back(b);
}

// Enqueue one admitted group on a slot.  Returns false on a CUDA error.
bool launch_batch(Slot& sl)
{
    const int32_t E = (int32_t)sl.reqs.size();
    int64_t H64 = 0;
    for (auto& r : sl.reqs) H64 += (int64_t)r.n;
    const int32_t H = (int32_t)H64;
    const size_t capT = (size_t)H / 3 + 1, capH = (size_t)H + 1;
    ResultBlock& B = *sl.block;
    cudaError_t e = cudaSuccess;
    auto need = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    bool direct = sl.reqs[0].pinned;
    for (int32_t k = 1; k < E && direct; k++) {
        const Request& p = sl.reqs[k - 1];
        const Request& r = sl.reqs[k];
        direct = r.pinned && r.x == p.x + p.n && r.y == p.y + p.n && r.z == p.z + p.n && r.m == p.m + p.n;
    }
    need(sl.hoff.reserve(E + 1));
    need(B.to.reserve(E + 1)); need(B.ho.reserve(capT + 1)); need(B.th.reserve(capH));
    need(B.params.reserve(4 * capT)); need(B.chi2.reserve(capT)); need(B.stat.reserve(E));
    if (!direct) {
        need(sl.hx.reserve(H)); need(sl.hy.reserve(H)); need(sl.hz.reserve(H)); need(sl.hm.reserve(H));
    }
    need(sl.dx.reserve(H)); need(sl.dy.reserve(H)); need(sl.dz.reserve(H)); need(sl.dm.reserve(H));
    need(sl.doff.reserve(E + 1)); need(sl.dto.reserve(E + 1)); need(sl.dho.reserve(capT + 1));
    need(sl.dth.reserve(capH)); need(sl.dparams.reserve(4 * capT)); need(sl.dchi2.reserve(capT));
    need(sl.dndof.reserve(capT)); need(sl.dstat.reserve(E)); need(sl.dcounts.reserve(4));
    if (e != cudaSuccess) return false;
    B.first_hit.resize(E);
    int32_t o = 0;
    for (int32_t k = 0; k < E; k++) {
        const Request& r = sl.reqs[k];
        const size_t n = (size_t)r.n;
        sl.hoff.p[k] = o;
        B.first_hit[k] = o;
        if (!direct && n) {
            std::memcpy(sl.hx.p + o, r.x, 4 * n);
            std::memcpy(sl.hy.p + o, r.y, 4 * n);
            std::memcpy(sl.hz.p + o, r.z, 4 * n);
            std::memcpy(sl.hm.p + o, r.m, 4 * n);
        }
        o += (int32_t)n;
    }
    sl.hoff.p[E] = o;
    cudaStream_t s = sl.stream;
    need(cudaEventRecord(sl.t_up, s));
    if (H) {
        need(cudaMemcpyAsync(sl.dx.p, direct ? sl.reqs[0].x : sl.hx.p, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        need(cudaMemcpyAsync(sl.dy.p, direct ? sl.reqs[0].y : sl.hy.p, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        need(cudaMemcpyAsync(sl.dz.p, direct ? sl.reqs[0].z : sl.hz.p, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        need(cudaMemcpyAsync(sl.dm.p, direct ? sl.reqs[0].m : sl.hm.p, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
    }
    need(cudaMemcpyAsync(sl.doff.p, sl.hoff.p, 4 * (size_t)(E + 1), cudaMemcpyHostToDevice, s));
    if (e != cudaSuccess) return false;
    sbt_tracks out;
    out.track_offsets = sl.dto.p;
    out.hit_offsets = sl.dho.p;
    out.track_hits = sl.dth.p;
    out.params = sl.dparams.p;
    out.chi2 = sl.dchi2.p;
    out.ndof = sl.dndof.p;
    out.event_status = sl.dstat.p;
    out.counts = sl.dcounts.p;
    out.cap_tracks = (int32_t)capT;
    out.cap_hits = (int32_t)capH;
    need(cudaEventRecord(sl.t_kern, s));
    if (sbt_reconstruct(sl.h, sl.dx.p, sl.dy.p, sl.dz.p, sl.dm.p, sl.doff.p, E, H, &out, s) != SBT_OK)
        return false;
    need(cudaEventRecord(sl.t_down, s));
    need(cudaMemcpyAsync(B.to.p, sl.dto.p, 4 * (size_t)(E + 1), cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(B.stat.p, sl.dstat.p, 4 * (size_t)E, cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(B.ho.p, sl.dho.p, 4 * (capT + 1), cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(B.th.p, sl.dth.p, 4 * capH, cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(B.params.p, sl.dparams.p, 16 * capT, cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(B.chi2.p, sl.dchi2.p, 4 * capT, cudaMemcpyDeviceToHost, s));
    need(cudaEventRecord(sl.done, s));
    return e == cudaSuccess;
}

void launcher_loop(sbt_server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        Slot* free_slot = nullptr;
        for (auto& up : S->slots)
            if (!up->busy.load(std::memory_order_acquire)) {
                free_slot = up.get();
                break;
            }
        std::vector<Request> take;
        int64_t bytes = 0;
        ResultBlock* block = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (free_slot) {
                int64_t hits = 0;
                while (!S->pending.empty() && (int32_t)take.size() < S->max_batch) {
                    const Request& r = S->pending.front();
                    const int64_t b = batch_bytes(hits + (int64_t)r.n, (int64_t)take.size() + 1);
                    if (S->in_flight_bytes + b > S->budget && (!take.empty() || S->in_flight_bytes > 0))
                        break;
                    hits += (int64_t)r.n;
                    bytes = b;
                    take.push_back(std::move(S->pending.front()));
                    S->pending.pop_front();
                }
            }
            if (take.empty()) {
                if (S->stop.load() && S->pending.empty()) break;
                S->cv_work.wait_for(lk, std::chrono::microseconds(50));
                continue;
            }
            S->in_flight_bytes += bytes;
            S->st_peak_bytes = std::max(S->st_peak_bytes, (double)S->in_flight_bytes);
            S->st_batches += 1;
            S->st_events_batched += (double)take.size();
            if (S->free_blocks.empty()) {
                S->all_blocks.push_back(std::make_unique<ResultBlock>());
                block = S->all_blocks.back().get();
            } else {
                // the free block whose track-hit buffer is largest: blocks that
                // already hold a batch of this size are not grown again
                auto best = std::max_element(S->free_blocks.begin(), S->free_blocks.end(),
                                             [](const ResultBlock* a, const ResultBlock* b) {
                                                 return a->th.n < b->th.n;
                                             });
                block = *best;
                S->free_blocks.erase(best);
            }
        }
        Slot& sl = *free_slot;
        sl.reqs = std::move(take);
        sl.bytes = bytes;
        sl.block = block;
        sl.failed = false;
        const double tl = now_s();
        sl.t_enqueued = tl;
        if (S->inject.exchange(false)) {
            sl.failed = true;  // host-side failure: nothing was enqueued
        } else if (!launch_batch(sl)) {
            cudaStreamSynchronize(sl.stream);  // drain what was enqueued before reuse
            sl.failed = true;
        }
        S->st_launch_s.store(S->st_launch_s.load(std::memory_order_relaxed) + (now_s() - tl),
                             std::memory_order_relaxed);
        sl.busy.store(true, std::memory_order_release);
    }
    S->launcher_done.store(true);
}

void harvest(sbt_server* S, Slot& sl)
{
    const double t_done = now_s();
    float up = 0.0f, kern = 0.0f, down = 0.0f;
    const bool timed = !sl.failed && cudaEventElapsedTime(&up, sl.t_up, sl.t_kern) == cudaSuccess &&
                       cudaEventElapsedTime(&kern, sl.t_kern, sl.t_down) == cudaSuccess &&
                       cudaEventElapsedTime(&down, sl.t_down, sl.done) == cudaSuccess;
    std::vector<Finished> out(sl.reqs.size());
    ResultBlock* B = sl.block;
    for (size_t k = 0; k < sl.reqs.size(); k++) {
        Finished& f = out[k];
        f.id = sl.reqs[k].id;
        f.latency = t_done - sl.reqs[k].t_submit;
        f.k = (int)k;
        if (sl.failed) {
            f.status = SBT_ERR_CUDA;
            f.block = nullptr;
        } else {
            f.status = B->stat.p[k];
            f.block = B;
        }
    }
    sl.reqs.clear();  // releases the pinned batches the uploads read from
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (sl.failed) {
            S->free_blocks.push_back(B);
            S->st_failed += 1;
        } else {
            B->refs = (int)out.size();
            if (out.empty()) S->free_blocks.push_back(B);
        }
        for (auto& f : out) S->finished.push_back(f);
        S->st_completed += (double)out.size();
        if (timed) {
            S->st_up_ms += up;
            S->st_kern_ms += kern;
            S->st_down_ms += down;
            S->st_wall_ms += (t_done - sl.t_enqueued) * 1e3;
            S->st_timed += 1;
        }
        S->in_flight_bytes -= sl.bytes;
    }
    sl.block = nullptr;
    sl.busy.store(false, std::memory_order_release);
    S->cv_done.notify_all();
    S->cv_work.notify_one();
}

void harvester_loop(sbt_server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        bool did = false, any_busy = false;
        for (auto& up : S->slots) {
            Slot& sl = *up;
            if (!sl.busy.load(std::memory_order_acquire)) continue;
            any_busy = true;
            if (sl.failed || cudaEventQuery(sl.done) == cudaSuccess) {
                harvest(S, sl);
                did = true;
            }
        }
        if (!any_busy && S->launcher_done.load()) break;
        if (!did) std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
}

}  // namespace

extern "C" {

sbt_status sbt_server_create(sbt_handle* h, int64_t memory_budget_bytes, int32_t max_streams,
                             int32_t max_batch_events, sbt_server** out)
{
    if (!h || !out || memory_budget_bytes <= 0 || max_streams < 1 || max_streams > 16 ||
        max_batch_events < 1)
        return SBT_ERR_ARG;
    *out = nullptr;
    auto* S = new sbt_server();
    S->budget = memory_budget_bytes;
    S->max_batch = max_batch_events;
    cudaError_t e = cudaGetDevice(&S->device);
    const sbt::DevConfig& C = sbt::handle_device_config(h);
    std::vector<float> mz(C.module_z, C.module_z + C.M), mz2(C.module_z2, C.module_z2 + C.M);
    sbt_geometry g;
    g.n_modules = C.M;
    g.module_z = mz.data();
    g.r_min = 0.0f;
    g.r_max = 0.0f;
    g.module_z2 = C.pairs ? mz2.data() : nullptr;
    sbt_config cfg;
    sbt_default_config(&cfg);
    cfg.k_doublets = C.K;
    cfg.max_scatter_seed = C.S_seed;
    cfg.max_scatter_follow = C.S_follow;
    cfg.max_chi2_tracklet = C.C3;
    cfg.hit_sigma = C.sigma;
    cfg.max_hits_per_event = C.nmax;
    cfg.max_forming_tracks = C.fcap;
    cfg.threads_per_block = sbt::handle_plain_threads(h);
    cfg.gec_max_hits = C.gec;
    cfg.fp16_hits = C.h16;
    for (int i = 0; i < max_streams && e == cudaSuccess; i++) {
        auto sl = std::make_unique<Slot>();
        if (sbt_create(&g, &cfg, &sl->h) != SBT_OK) {
            e = cudaErrorUnknown;
            break;
        }
        e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&sl->done);
        if (e == cudaSuccess) e = cudaEventCreate(&sl->t_up);
        if (e == cudaSuccess) e = cudaEventCreate(&sl->t_kern);
        if (e == cudaSuccess) e = cudaEventCreate(&sl->t_down);
        S->slots.push_back(std::move(sl));
    }
    if (e != cudaSuccess) {
        for (auto& sl : S->slots) {
            if (sl->h) sbt_destroy(sl->h);
            if (sl->stream) cudaStreamDestroy(sl->stream);
            if (sl->done) cudaEventDestroy(sl->done);
            if (sl->t_up) cudaEventDestroy(sl->t_up);
            if (sl->t_kern) cudaEventDestroy(sl->t_kern);
            if (sl->t_down) cudaEventDestroy(sl->t_down);
        }
        delete S;
        return SBT_ERR_CUDA;
    }
    for (auto& sl : S->slots) sbt::handle_defer_frees(sl->h);
    S->allocs0 = g_allocs.load();
    S->launcher = std::thread(launcher_loop, S);
    S->harvester = std::thread(harvester_loop, S);
    *out = S;
    return SBT_OK;
}

sbt_status sbt_server_submit(sbt_server* S, int64_t request_id, const float* x, const float* y,
                             const float* z, const int32_t* module, int32_t n)
{
    if (!S || n < 0 || (n > 0 && (!x || !y || !z || !module))) return SBT_ERR_ARG;
    if (S->stop.load()) return SBT_ERR_STATE;
    Request r;
    r.id = request_id;
    r.ox.assign(x, x + n);
    r.oy.assign(y, y + n);
    r.oz.assign(z, z + n);
    r.om.assign(module, module + n);
    r.x = r.ox.data();
    r.y = r.oy.data();
    r.z = r.oz.data();
    r.m = r.om.data();
    r.n = n;
    r.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->pending.push_back(std::move(r));
        S->st_submitted += 1;
    }
    S->cv_work.notify_one();
    return SBT_OK;
}

sbt_status sbt_server_submit_schedule(sbt_server* S, const float* x, const float* y, const float* z,
                                      const int32_t* module, const int32_t* event_offsets,
                                      int32_t n_events, const double* arrival_s, int64_t first_id)
{
    if (!S || n_events < 0 || !event_offsets || !arrival_s) return SBT_ERR_ARG;
    if (event_offsets[0] < 0) return SBT_ERR_ARG;
    for (int32_t e = 0; e < n_events; e++)
        if (event_offsets[e] > event_offsets[e + 1]) return SBT_ERR_ARG;
    if (event_offsets[n_events] > 0 && (!x || !y || !z || !module)) return SBT_ERR_ARG;
    if (S->stop.load()) return SBT_ERR_STATE;
    if (S->feeder.joinable()) S->feeder.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->st_feed_lag = 0.0;
    }
    const int32_t H = event_offsets[n_events];
    std::unique_ptr<PinnedBatch> pb;
    std::vector<std::unique_ptr<PinnedBatch>> drop;  // idle batches beyond kPinnedPool, freed unlocked
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto& pool = S->pinned_pool;
        for (auto it = pool.begin(); it != pool.end(); ++it)
            if ((*it)->cap >= (size_t)std::max(H, 1)) {
                pb = std::move(*it);
                pool.erase(it);
                break;
            }
        while (pool.size() > kPinnedPool) {
            auto smallest = std::min_element(pool.begin(), pool.end(),
                                             [](const auto& a, const auto& b) { return a->cap < b->cap; });
            drop.push_back(std::move(*smallest));
            pool.erase(smallest);
        }
    }
    drop.clear();
    if (!pb) {
        pb.reset(new PinnedBatch());
        if (!pb->alloc((size_t)H)) return SBT_ERR_CUDA;
    }
    // the last request holding the batch hands it back to the pool (never
    // under the server lock: requests are released outside it)
    std::shared_ptr<PinnedBatch> batch(pb.release(), [S](PinnedBatch* b) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->pinned_pool.emplace_back(b);
    });
    if (H) {
        std::memcpy(batch->x, x, sizeof(float) * H);
        std::memcpy(batch->y, y, sizeof(float) * H);
        std::memcpy(batch->z, z, sizeof(float) * H);
        std::memcpy(batch->m, module, sizeof(int32_t) * H);
    }
    std::vector<int32_t> vo(event_offsets, event_offsets + n_events + 1);
    std::vector<double> at(arrival_s, arrival_s + n_events);
    S->feeder = std::thread([S, batch, vo = std::move(vo), at = std::move(at), first_id, n_events]() {
        const auto t0 = Clock::now();
        const double t0_s = std::chrono::duration<double>(t0.time_since_epoch()).count();
        double lag = 0.0;
        auto due_at = [&](int32_t e) {
            return t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(at[e]));
        };
        int32_t e = 0;
        while (e < n_events && !S->stop.load()) {
            auto now = Clock::now();
            if (now < due_at(e)) {
                auto left = due_at(e) - now;
                if (left > std::chrono::microseconds(200))
                    std::this_thread::sleep_for(left - std::chrono::microseconds(100));
                continue;
            }
            std::vector<Request> due;
            const double ts = now_s();
            while (e < n_events && due_at(e) <= now) {
                // latency counts from the scheduled arrival, so a feeder
                // running late shows in it rather than hiding a backlog
                lag = std::max(lag, ts - (t0_s + at[e]));
                Request r;
                r.id = first_id + e;
                const int32_t lo = vo[e];
                r.x = batch->x + lo;
                r.y = batch->y + lo;
                r.z = batch->z + lo;
                r.m = batch->m + lo;
                r.n = vo[e + 1] - lo;
                r.pinned = true;
                r.hold = batch;
                r.t_submit = t0_s + at[e];
                due.push_back(std::move(r));
                e++;
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto& r : due) S->pending.push_back(std::move(r));
                S->st_submitted += (double)due.size();
                S->st_feed_lag = lag;
            }
            S->cv_work.notify_one();
        }
    });
    return SBT_OK;
}

sbt_status sbt_server_drain(sbt_server* S, int64_t* ids, int32_t* status, double* latency_s,
                            int32_t max_results, int32_t* n_out, double timeout_s)
{
    if (!S || !n_out || max_results < 0 || (max_results > 0 && (!ids || !status || !latency_s)))
        return SBT_ERR_ARG;
    *n_out = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->finished.empty() && timeout_s > 0)
        S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                            [&] { return !S->finished.empty(); });
    if (S->finished.empty()) return timeout_s > 0 ? SBT_ERR_TIMEOUT : SBT_OK;
    int32_t k = 0;
    while (k < max_results && !S->finished.empty()) {
        const Finished& f = S->finished.front();
        ids[k] = f.id;
        status[k] = f.status;
        latency_s[k] = f.latency;
        unref_block(S, f.block);
        S->finished.pop_front();
        k++;
    }
    *n_out = k;
    return SBT_OK;
}

sbt_status sbt_server_poll(sbt_server* S, sbt_result* results, int32_t max_results, int32_t* n_out,
                           double timeout_s)
{
    if (!S || !n_out || max_results < 0 || (max_results > 0 && !results)) return SBT_ERR_ARG;
    *n_out = 0;
    std::vector<Finished> got;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->finished.empty() && timeout_s > 0)
            S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                [&] { return !S->finished.empty(); });
        if (S->finished.empty()) return timeout_s > 0 ? SBT_ERR_TIMEOUT : SBT_OK;
        while ((int32_t)got.size() < max_results && !S->finished.empty()) {
            got.push_back(S->finished.front());
            S->finished.pop_front();
        }
    }
    // event-local copies of each request's tracks, made outside the lock (the
    // result block stays referenced until then)
    std::vector<Materialized> mats(got.size());
    for (size_t i = 0; i < got.size(); i++) {
        const Finished& f = got[i];
        Materialized& m = mats[i];
        if (!f.block) {
            m.hit_offsets.assign(1, 0);
            continue;
        }
        const ResultBlock& B = *f.block;
        const int32_t t0 = B.to.p[f.k], t1 = B.to.p[f.k + 1];
        const int32_t h0 = B.ho.p[t0];
        m.hit_offsets.resize(t1 - t0 + 1);
        for (int32_t t = t0; t <= t1; t++) m.hit_offsets[t - t0] = B.ho.p[t] - h0;
        const int32_t nh = B.ho.p[t1] - h0;
        const int32_t base = B.first_hit[f.k];
        m.track_hits.resize(nh);
        for (int32_t j = 0; j < nh; j++) m.track_hits[j] = B.th.p[h0 + j] - base;
        m.params.assign(B.params.p + 4 * (size_t)t0, B.params.p + 4 * (size_t)t1);
        m.chi2.assign(B.chi2.p + t0, B.chi2.p + t1);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < got.size(); i++) {
        const Finished& f = got[i];
        unref_block(S, f.block);
        Materialized& g = S->polled[f.id] = std::move(mats[i]);
        sbt_result& r = results[i];
        r.request_id = f.id;
        r.status = f.status;
        r.n_tracks = (int32_t)g.hit_offsets.size() - 1;
        r.hit_offsets = g.hit_offsets.data();
        r.track_hits = g.track_hits.data();
        r.params = g.params.data();
        r.chi2 = g.chi2.data();
        r.latency_s = f.latency;
    }
    *n_out = (int32_t)got.size();
    return SBT_OK;
}

sbt_status sbt_server_release(sbt_server* S, int64_t request_id)
{
    if (!S) return SBT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    return S->polled.erase(request_id) ? SBT_OK : SBT_ERR_ARG;
}

sbt_status sbt_server_stats(sbt_server* S, double* stats)
{
    if (!S || !stats) return SBT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    stats[0] = S->st_completed;
    stats[1] = S->st_submitted;
    stats[2] = S->st_batches;
    stats[3] = S->st_batches > 0 ? S->st_events_batched / S->st_batches : 0.0;
    stats[4] = S->st_peak_bytes;
    stats[5] = S->st_failed;
    stats[6] = S->st_feed_lag;
    stats[7] = S->st_launch_s.load(std::memory_order_relaxed);
    stats[8] = S->st_up_ms;
    stats[9] = S->st_kern_ms;
    stats[10] = S->st_down_ms;
    stats[11] = S->st_wall_ms;
    stats[12] = S->st_timed;
    stats[13] = (double)(g_allocs.load() - S->allocs0);
    return SBT_OK;
}

sbt_status sbt_server_inject_failure(sbt_server* S)
{
    if (!S) return SBT_ERR_ARG;
    S->inject.store(true);
    return SBT_OK;
}

sbt_status sbt_server_destroy(sbt_server* S)
{
    if (!S) return SBT_ERR_ARG;
    if (S->feeder.joinable()) S->feeder.join();
    S->stop.store(true);
    S->cv_work.notify_all();
    if (S->launcher.joinable()) S->launcher.join();
    if (S->harvester.joinable()) S->harvester.join();
    // every request is gone before the pinned batches they refer to
    S->pending.clear();
    for (auto& up : S->slots) up->reqs.clear();
    S->pinned_pool.clear();
    for (auto& up : S->slots) {
        Slot& sl = *up;
        cudaStreamSynchronize(sl.stream);
        sl.dx.release(); sl.dy.release(); sl.dz.release(); sl.dm.release(); sl.doff.release();
        sl.dto.release(); sl.dho.release(); sl.dth.release(); sl.dparams.release();
        sl.dchi2.release(); sl.dndof.release(); sl.dstat.release(); sl.dcounts.release();
        sl.hx.release(); sl.hy.release(); sl.hz.release(); sl.hm.release(); sl.hoff.release();
        cudaEventDestroy(sl.done);
        cudaEventDestroy(sl.t_up);
        cudaEventDestroy(sl.t_kern);
        cudaEventDestroy(sl.t_down);
        cudaStreamDestroy(sl.stream);
        sbt_destroy(sl.h);
    }
    for (auto& b : S->all_blocks) {
        b->to.release(); b->ho.release(); b->th.release(); b->stat.release();
        b->params.release(); b->chi2.release();
    }
    delete S;
    return SBT_OK;
}

}  // extern "C"

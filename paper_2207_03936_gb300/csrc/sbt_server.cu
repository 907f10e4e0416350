// Continuous-batching request loop.
//
// A background host thread repeatedly (1) harvests finished batches (CUDA
// event queries; no blocking synchronisation), (2) admits pending events in
// arrival order while a free stream slot exists and the device-memory budget
// allows, packing them into one batch: pinned staging copy, H2D on the slot's
// stream, reconstruction on the slot's own handle, D2H of the results and an
// event record.  Several slots are in flight at once, so events that arrive
// while others run on the GPU are admitted and overlap them.  No device-side
// wait exists anywhere: the GPU never spins on host state.
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

// One event to reconstruct.  Its hits either live in the request's own
// vectors (sbt_server_submit) or in a pinned batch owned by the open-loop
// feeder (sbt_server_submit_schedule), kept alive by `hold`.
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

// Pinned copy of a scheduled batch.
struct PinnedBatch {
    float *x = nullptr, *y = nullptr, *z = nullptr;
    int32_t* m = nullptr;
    ~PinnedBatch()
    {
        if (x) cudaFreeHost(x);
        if (y) cudaFreeHost(y);
        if (z) cudaFreeHost(z);
        if (m) cudaFreeHost(m);
    }
};

struct Finished {
    int64_t id = 0;
    int32_t status = 0;
    std::vector<int32_t> hit_offsets, track_hits;
    std::vector<float> params, chi2;
    double latency = 0.0;
};

// Device bytes one batch needs (inputs, outputs and the plain workspace).
int64_t batch_bytes(int64_t hits, int64_t events)
{
    return hits * 96 + events * 64 + (1 << 16);
}

template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t reserve(size_t want)
    {
        if (want <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, sizeof(T) * std::max<size_t>(want, 1));
        if (e == cudaSuccess) n = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

template <class T>
struct HostBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t reserve(size_t want)
    {
        if (want <= n) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMallocHost(&p, sizeof(T) * std::max<size_t>(want, 1));
        if (e == cudaSuccess) n = want;
        return e;
    }
    void release()
    {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

struct Slot {
    sbt_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool failed = false;
    int64_t bytes = 0;
    std::vector<Request> reqs;
    int32_t n_events = 0, n_hits = 0;
    DevBuf<float> dx, dy, dz, dparams, dchi2;
    DevBuf<int32_t> dm, doff, dto, dho, dth, dndof, dstat, dcounts;
    HostBuf<float> hx, hy, hz, hparams, hchi2;
    HostBuf<int32_t> hm, hoff, hto, hho, hth, hstat, hcounts;
};

}  // namespace

struct sbt_server {
    sbt_handle* parent = nullptr;
    int device = 0;
    int64_t budget = 0;
    int32_t max_batch = 0;
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::deque<Finished> finished;
    std::map<int64_t, Finished> polled;
    std::atomic<bool> stop{false};
    std::atomic<bool> inject{false};
    int64_t in_flight_bytes = 0;
    double st_completed = 0, st_submitted = 0, st_batches = 0, st_events_batched = 0,
           st_peak_bytes = 0, st_failed = 0;
    std::string err;
    std::thread worker;
    std::thread feeder;
};

namespace {

void finish_batch(sbt_server* S, Slot& sl, double t_done)
{
    std::vector<Finished> out;
    out.reserve(sl.reqs.size());
    int32_t off = 0;
    for (size_t k = 0; k < sl.reqs.size(); k++) {
        Finished f;
        f.id = sl.reqs[k].id;
        f.latency = t_done - sl.reqs[k].t_submit;
        const int32_t n = sl.reqs[k].n;
        if (sl.failed) {
            f.status = SBT_ERR_CUDA;
            f.hit_offsets.assign(1, 0);
        } else {
            f.status = sl.hstat.p[k];
            const int32_t t0 = sl.hto.p[k], t1 = sl.hto.p[k + 1];
            f.hit_offsets.resize(t1 - t0 + 1);
            const int32_t h0 = sl.hho.p[t0];
            for (int32_t t = t0; t <= t1; t++) f.hit_offsets[t - t0] = sl.hho.p[t] - h0;
            const int32_t nh = sl.hho.p[t1] - h0;
            f.track_hits.resize(nh);
            for (int32_t j = 0; j < nh; j++) f.track_hits[j] = sl.hth.p[h0 + j] - off;
            f.params.assign(sl.hparams.p + 4 * (size_t)t0, sl.hparams.p + 4 * (size_t)t1);
            f.chi2.assign(sl.hchi2.p + t0, sl.hchi2.p + t1);
        }
        off += n;
        out.push_back(std::move(f));
    }
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& f : out) S->finished.push_back(std::move(f));
    S->st_completed += (double)out.size();
    if (sl.failed) S->st_failed += 1;
    S->in_flight_bytes -= sl.bytes;
    sl.busy = false;
    sl.failed = false;
    sl.reqs.clear();
    S->cv_done.notify_all();
}

// Launch one admitted group on a slot.  Returns false on a CUDA error (the
// group is then completed with an error status).
bool launch_batch(sbt_server* S, Slot& sl)
{
    const int32_t E = (int32_t)sl.reqs.size();
    int64_t H64 = 0;
    for (auto& r : sl.reqs) H64 += (int64_t)r.n;
    const int32_t H = (int32_t)H64;
    const size_t capT = (size_t)H / 3 + 1, capH = (size_t)H + 1;
    cudaError_t e = cudaSuccess;
    auto need = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    // a group of scheduled events that are consecutive in one pinned batch is
    // uploaded directly; anything else is packed into the slot's staging
    bool direct = sl.reqs[0].pinned;
    for (int32_t k = 1; k < E && direct; k++) {
        const Request& p = sl.reqs[k - 1];
        const Request& r = sl.reqs[k];
        direct = r.pinned && r.x == p.x + p.n && r.y == p.y + p.n && r.z == p.z + p.n && r.m == p.m + p.n;
    }
    need(sl.hoff.reserve(E + 1)); need(sl.hto.reserve(E + 1)); need(sl.hho.reserve(capT + 1));
    need(sl.hth.reserve(capH)); need(sl.hparams.reserve(4 * capT)); need(sl.hchi2.reserve(capT));
    need(sl.hstat.reserve(E)); need(sl.hcounts.reserve(4));
    if (!direct) {
        need(sl.hx.reserve(H)); need(sl.hy.reserve(H)); need(sl.hz.reserve(H)); need(sl.hm.reserve(H));
    }
    need(sl.dx.reserve(H)); need(sl.dy.reserve(H)); need(sl.dz.reserve(H)); need(sl.dm.reserve(H));
    need(sl.doff.reserve(E + 1)); need(sl.dto.reserve(E + 1)); need(sl.dho.reserve(capT + 1));
    need(sl.dth.reserve(capH)); need(sl.dparams.reserve(4 * capT)); need(sl.dchi2.reserve(capT));
    need(sl.dndof.reserve(capT)); need(sl.dstat.reserve(E)); need(sl.dcounts.reserve(4));
    if (e != cudaSuccess) return false;
    int32_t o = 0;
    for (int32_t k = 0; k < E; k++) {
        const Request& r = sl.reqs[k];
        const size_t n = (size_t)r.n;
        sl.hoff.p[k] = o;
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
    const float* sx = direct ? sl.reqs[0].x : sl.hx.p;
    const float* sy = direct ? sl.reqs[0].y : sl.hy.p;
    const float* sz = direct ? sl.reqs[0].z : sl.hz.p;
    const int32_t* sm = direct ? sl.reqs[0].m : sl.hm.p;
    if (H) {
        need(cudaMemcpyAsync(sl.dx.p, sx, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        need(cudaMemcpyAsync(sl.dy.p, sy, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        need(cudaMemcpyAsync(sl.dz.p, sz, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
        need(cudaMemcpyAsync(sl.dm.p, sm, 4 * (size_t)H, cudaMemcpyHostToDevice, s));
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
    if (sbt_reconstruct(sl.h, sl.dx.p, sl.dy.p, sl.dz.p, sl.dm.p, sl.doff.p, E, H, &out, s) != SBT_OK)
        return false;
    need(cudaMemcpyAsync(sl.hto.p, sl.dto.p, 4 * (size_t)(E + 1), cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(sl.hstat.p, sl.dstat.p, 4 * (size_t)E, cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(sl.hho.p, sl.dho.p, 4 * (capT + 1), cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(sl.hth.p, sl.dth.p, 4 * capH, cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(sl.hparams.p, sl.dparams.p, 16 * capT, cudaMemcpyDeviceToHost, s));
    need(cudaMemcpyAsync(sl.hchi2.p, sl.dchi2.p, 4 * capT, cudaMemcpyDeviceToHost, s));
    need(cudaEventRecord(sl.done, s));
    return e == cudaSuccess;
}

void worker_loop(sbt_server* S)
{
    cudaSetDevice(S->device);
    while (true) {
        bool did = false;
        // harvest
        for (auto& up : S->slots) {
            Slot& sl = *up;
            if (!sl.busy) continue;
            if (sl.failed || cudaEventQuery(sl.done) == cudaSuccess) {
                finish_batch(S, sl, now_s());
                did = true;
            }
        }
        // admit
        for (auto& up : S->slots) {
            Slot& sl = *up;
            if (sl.busy) continue;
            std::vector<Request> take;
            int64_t bytes = 0, hits = 0;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                while (!S->pending.empty() && (int32_t)take.size() < S->max_batch) {
                    const Request& r = S->pending.front();
                    int64_t b = batch_bytes(hits + (int64_t)r.n, (int64_t)take.size() + 1);
                    if (S->in_flight_bytes + b > S->budget && !take.empty()) break;
                    if (S->in_flight_bytes + b > S->budget && S->in_flight_bytes > 0) break;
                    hits += (int64_t)r.n;
                    bytes = b;
                    take.push_back(std::move(S->pending.front()));
                    S->pending.pop_front();
                }
                if (take.empty()) break;
                S->in_flight_bytes += bytes;
                S->st_peak_bytes = std::max(S->st_peak_bytes, (double)S->in_flight_bytes);
                S->st_batches += 1;
                S->st_events_batched += (double)take.size();
            }
            sl.reqs = std::move(take);
            sl.bytes = bytes;
            sl.busy = true;
            if (S->inject.exchange(false)) {
                sl.failed = true;  // host-side failure: nothing was enqueued
            } else if (!launch_batch(S, sl)) {
                // drain whatever part of the batch was enqueued before the
                // slot's buffers are reused
                cudaStreamSynchronize(sl.stream);
                sl.failed = true;
            }
            did = true;
        }
        if (S->stop.load()) {
            bool idle = true;
            for (auto& up : S->slots) idle = idle && !up->busy;
            std::lock_guard<std::mutex> lk(S->mu);
            if (idle && S->pending.empty()) break;
        }
        if (!did) {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
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
    S->parent = h;
    S->budget = memory_budget_bytes;
    S->max_batch = max_batch_events;
    cudaError_t e = cudaGetDevice(&S->device);
    const sbt::DevConfig& C = sbt::handle_device_config(h);
    std::vector<float> mz(C.module_z, C.module_z + C.M);
    sbt_geometry g;
    g.n_modules = C.M;
    g.module_z = mz.data();
    g.r_min = 0.0f;
    g.r_max = 0.0f;
    sbt_config cfg;
    sbt_default_config(&cfg);
    cfg.k_doublets = C.K;
    cfg.max_scatter_seed = C.S_seed;
    cfg.max_scatter_follow = C.S_follow;
    cfg.max_chi2_tracklet = C.C3;
    cfg.hit_sigma = C.sigma;
    cfg.max_hits_per_event = C.nmax;
    cfg.max_forming_tracks = C.fcap;
    for (int i = 0; i < max_streams && e == cudaSuccess; i++) {
        auto sl = std::make_unique<Slot>();
        if (sbt_create(&g, &cfg, &sl->h) != SBT_OK) {
            e = cudaErrorUnknown;
            break;
        }
        e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming);
        S->slots.push_back(std::move(sl));
    }
    if (e != cudaSuccess) {
        for (auto& sl : S->slots) {
            if (sl->h) sbt_destroy(sl->h);
            if (sl->stream) cudaStreamDestroy(sl->stream);
            if (sl->done) cudaEventDestroy(sl->done);
        }
        delete S;
        return SBT_ERR_CUDA;
    }
    S->worker = std::thread(worker_loop, S);
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

/*
 * Open-loop load: a native thread submits event e of the host batch (x, y, z,
 * module [event_offsets[e] .. event_offsets[e+1])) at arrival_s[e] seconds
 * after this call, with request id first_id + e.  Returns at once.
 */
sbt_status sbt_server_submit_schedule(sbt_server* S, const float* x, const float* y, const float* z,
                                      const int32_t* module, const int32_t* event_offsets,
                                      int32_t n_events, const double* arrival_s, int64_t first_id)
{
    if (!S || n_events < 0 || !event_offsets || !arrival_s) return SBT_ERR_ARG;
    if (S->feeder.joinable()) S->feeder.join();
    const int32_t H = event_offsets[n_events];
    auto batch = std::make_shared<PinnedBatch>();
    const size_t nb = sizeof(float) * (size_t)std::max(H, 1);
    if (cudaMallocHost(&batch->x, nb) != cudaSuccess || cudaMallocHost(&batch->y, nb) != cudaSuccess ||
        cudaMallocHost(&batch->z, nb) != cudaSuccess || cudaMallocHost(&batch->m, nb) != cudaSuccess)
        return SBT_ERR_CUDA;
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
        int32_t e = 0;
        while (e < n_events && !S->stop.load()) {
            const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                                      std::chrono::duration<double>(at[e]));
            auto now = Clock::now();
            if (now < due) {
                auto left = due - now;
                if (left > std::chrono::microseconds(200))
                    std::this_thread::sleep_for(left - std::chrono::microseconds(100));
                continue;
            }
            // submit every event that is due
            std::vector<Request> due_reqs;
            const double ts = now_s();
            while (e < n_events && t0 + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(at[e])) <= now) {
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
                r.t_submit = ts;
                due_reqs.push_back(std::move(r));
                e++;
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (auto& r : due_reqs) S->pending.push_back(std::move(r));
                S->st_submitted += (double)due_reqs.size();
            }
            S->cv_work.notify_one();
        }
    });
    return SBT_OK;
}

/*
 * Finished requests for consumers that only need their completion: up to
 * max_results (request id, status, latency) triples; the results are released
 * at once.  Waits at most timeout_s for the first one.
 */
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
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->finished.empty() && timeout_s > 0)
        S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                            [&] { return !S->finished.empty(); });
    if (S->finished.empty()) return timeout_s > 0 ? SBT_ERR_TIMEOUT : SBT_OK;
    int32_t k = 0;
    while (k < max_results && !S->finished.empty()) {
        Finished f = std::move(S->finished.front());
        S->finished.pop_front();
        auto it = S->polled.emplace(f.id, std::move(f)).first;
        Finished& g = it->second;
        sbt_result& r = results[k++];
        r.request_id = g.id;
        r.status = g.status;
        r.n_tracks = (int32_t)g.hit_offsets.size() - 1;
        r.hit_offsets = g.hit_offsets.data();
        r.track_hits = g.track_hits.data();
        r.params = g.params.data();
        r.chi2 = g.chi2.data();
        r.latency_s = g.latency;
    }
    *n_out = k;
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
    stats[6] = 0.0;
    stats[7] = 0.0;
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
    if (S->worker.joinable()) S->worker.join();
    for (auto& up : S->slots) {
        Slot& sl = *up;
        cudaStreamSynchronize(sl.stream);
        sl.dx.release(); sl.dy.release(); sl.dz.release(); sl.dm.release(); sl.doff.release();
        sl.dto.release(); sl.dho.release(); sl.dth.release(); sl.dparams.release();
        sl.dchi2.release(); sl.dndof.release(); sl.dstat.release(); sl.dcounts.release();
        sl.hx.release(); sl.hy.release(); sl.hz.release(); sl.hm.release(); sl.hoff.release();
        sl.hto.release(); sl.hho.release(); sl.hth.release(); sl.hparams.release();
        sl.hchi2.release(); sl.hstat.release(); sl.hcounts.release();
        cudaEventDestroy(sl.done);
        cudaStreamDestroy(sl.stream);
        sbt_destroy(sl.h);
    }
    delete S;
    return SBT_OK;
}

}  // extern "C"

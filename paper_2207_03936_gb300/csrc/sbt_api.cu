// C ABI of the library: handles, workspaces, launch sequences, the CUDA-graph
// cache of the batched launch, the block-size autotuner and the end-to-end
// host entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sbt_internal.h"

using namespace sbt;

namespace {

std::string g_create_error;

// Host pipeline: events per chunk and the most chunks per call.
// Host pipeline: batches above kChunkEvents events are cut into chunks of
// relative sizes kChunkWeights (small first chunk: short start-up; sizes
// growing by at most 1.6x; smaller last chunks: short download at the end).
// From kLargeBatchEvents on, kChunkWeightsLarge: uploads (about 0.5 us per
// event while downloads share the link) and reconstruction (about 0.47 us
// per event, plus about 0.7 ms per chunk for the tail of its search and its
// short kernels) run at nearly the same rate, so after a short ramp the
// chunks stay level at about 11k events and only the last one is small.
constexpr int64_t kChunkEvents = 12500;
constexpr int64_t kLargeBatchEvents = 60000;
constexpr int kMaxChunks = 16;
constexpr double kChunkWeights[] = {1.0, 1.6, 2.6, 4.1, 6.6, 10.5, 16.8, 8.0, 3.0};
constexpr double kChunkWeightsLarge[] = {1.96, 2.31, 2.71, 3.19, 3.75, 4.41, 5.19,
                                         6.01, 6.01, 6.01, 6.01, 6.01, 2.21};
constexpr int kWeightedChunks = sizeof(kChunkWeights) / sizeof(kChunkWeights[0]);
constexpr int kWeightedChunksLarge = sizeof(kChunkWeightsLarge) / sizeof(kChunkWeightsLarge[0]);
static_assert(kWeightedChunks <= kMaxChunks && kWeightedChunksLarge <= kMaxChunks, "chunk tables");

// One device allocation carved into aligned sub-arrays.
struct Arena {
    void* base = nullptr;
    size_t bytes = 0;
    bool defer = false;          // keep outgrown allocations until release()
    std::vector<void*> retired;
    // Grows geometrically: freeing device memory synchronises the device, so
    // workspaces must not be reallocated for every slightly larger batch.
    cudaError_t reserve(size_t need)
    {
        if (need <= bytes) return cudaSuccess;
        if (bytes) need = std::max(need, bytes + bytes / 2);
        if (base && !defer) {
            cudaError_t e = cudaFree(base);
            base = nullptr;
            bytes = 0;
            if (e != cudaSuccess) return e;
        }
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, need);
        if (e != cudaSuccess) return e;
        if (base) retired.push_back(base);
        base = p;
        bytes = need;
        return cudaSuccess;
    }
    void release()
    {
        for (void* p : retired) cudaFree(p);
        retired.clear();
        if (base) cudaFree(base);
        base = nullptr;
        bytes = 0;
    }
};

struct Carver {
    char* p;
    size_t off = 0;
    explicit Carver(void* base) : p((char*)base) {}
    template <class T>
    T* take(int64_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* r = (T*)(p ? p + off : nullptr);
        off += sizeof(T) * (size_t)std::max<int64_t>(count, 1);
        return r;
    }
};

// Scratch layout for `hits` hit slots over `regions` regions (see Work).
size_t carve_work(void* base, int64_t hits, int64_t regions, Work* W)
{
    Carver c(base);
    Work w;
    w.list = c.take<uint32_t>(hits);
    w.prev = c.take<uint16_t>(hits);
    w.claim = c.take<unsigned long long>(hits);
    w.ft = c.take<FTrack>(forming_entries(hits, regions));
    w.tracklets = c.take<unsigned long long>(tracklet_entries(hits, regions));
    w.tl_q = c.take<uint32_t>(tracklet_entries(hits, regions));
    w.finals = c.take<uint32_t>(final_entries(hits, regions));
    if (W) *W = w;
    return c.off + 256;
}

// Sorted hits of a batch (see Sorted).
size_t carve_sorted(void* base, int64_t n_hits, int64_t n_events, int M, Sorted* O)
{
    Carver c(base);
    Sorted o;
    o.coords = c.take<float4>(n_hits);
    o.phi = c.take<uint16_t>(n_hits);
    o.modoff = c.take<int32_t>(n_events * (M + 1));
    o.status = c.take<int32_t>(n_events);
    if (O) *O = o;
    return c.off + 256;
}

size_t carve_staging(void* base, int64_t n_hits, int64_t n_events, Staging* S)
{
    Carver c(base);
    Staging s;
    s.hits = c.take<float4>(n_hits);
    s.tkey = c.take<int32_t>(n_hits / 3 + n_events + 1);
    s.tinfo = c.take<uint32_t>(n_hits / 3 + n_events + 1);
    s.rinfo = c.take<uint32_t>(n_hits / 3 + n_events + 1);
    s.tfit = c.take<uint2>(n_hits / 3 + n_events + 1);
    s.ev_ntracks = c.take<int32_t>(n_events);
    s.ev_nhits = c.take<int32_t>(n_events);
    s.track_base = c.take<int32_t>(n_events);
    s.hit_base = c.take<int32_t>(n_events);
    s.order = c.take<int32_t>(n_events);
    s.queue = c.take<int32_t>(4 * kMaxChunks);  // one work-queue head per host-pipeline chunk
    if (S) *S = s;
    return c.off + 256;
}

struct GraphKey {
    const void* ptrs[13];
    int64_t vals[6];
    bool operator==(const GraphKey& o) const
    {
        return std::memcmp(ptrs, o.ptrs, sizeof(ptrs)) == 0 && std::memcmp(vals, o.vals, sizeof(vals)) == 0;
    }
};

}  // namespace

struct sbt_handle {
    sbt_config cfg;
    DevConfig C;
    int device = 0;
    int sm_count = 0;
    std::string err;
    Arena plain_arena, pers_arena, stage_arena, host_arena, misc_arena, sorted_arena;
    int tuned_threads = 0;
    int tuned_blocks_per_sm = 0;  // resident blocks per SM of the persistent launch (0: occupancy limit)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t copy_in = nullptr, copy_out = nullptr, sort_stream = nullptr;
    int32_t* host_counts = nullptr;  // pinned, 4 per chunk of the host pipeline
    cudaGraphExec_t exec = nullptr;
    GraphKey key{};
    bool have_key = false;
    int launches_last = 0;
};

namespace {

sbt_status fail(sbt_handle* h, sbt_status st, const std::string& msg)
{
    if (h) h->err = msg;
    return st;
}

sbt_status cuda_fail(sbt_handle* h, cudaError_t e, const char* where)
{
    return fail(h, SBT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int default_threads(const sbt_handle* h, bool batched)
{
    if (h->cfg.threads_per_block) return h->cfg.threads_per_block;
    if (batched && h->tuned_threads) return h->tuned_threads;
    return 128;
}

sbt_status check_inputs(sbt_handle* h, const float* x, const float* y, const float* z,
                        const int32_t* module, const int32_t* offsets, int32_t n_events,
                        int32_t n_hits, const sbt_tracks* out)
{
    if (!h) return SBT_ERR_ARG;
    if (n_events < 0 || n_hits < 0) return fail(h, SBT_ERR_ARG, "negative size");
    if (!offsets) return fail(h, SBT_ERR_ARG, "event_offsets is NULL");
    if (n_hits > 0 && (!x || !y || !z || !module)) return fail(h, SBT_ERR_ARG, "hit array is NULL");
    if (out) {
        if (!out->track_offsets || !out->hit_offsets || !out->counts ||
            (n_events > 0 && !out->event_status))
            return fail(h, SBT_ERR_ARG, "output array is NULL");
        if (out->cap_tracks < 0 || out->cap_hits < 0) return fail(h, SBT_ERR_ARG, "negative capacity");
        if ((out->cap_tracks > 0 && (!out->params || !out->chi2 || !out->ndof)) ||
            (out->cap_hits > 0 && !out->track_hits))
            return fail(h, SBT_ERR_ARG, "output array is NULL");
    }
    return SBT_OK;
}

// Host-visible event offsets: non-decreasing, from 0 or more up to n_hits.
bool host_offsets_valid(const int32_t* offsets, int32_t n_events, int64_t n_hits)
{
    if (offsets[0] < 0 || offsets[n_events] > n_hits) return false;
    for (int32_t e = 0; e < n_events; e++)
        if (offsets[e] > offsets[e + 1]) return false;
    return true;
}

Inputs make_inputs(const float* x, const float* y, const float* z, const int32_t* module,
                   const int32_t* offsets, int32_t n_events, int32_t n_hits)
{
    Inputs in;
    in.x = x;
    in.y = y;
    in.z = z;
    in.module = module;
    in.offsets = offsets;
    in.n_events = n_events;
    in.n_hits = n_hits;
    return in;
}

sbt_status ensure_sorted(sbt_handle* h, int64_t n_hits, int64_t n_events, Sorted* O)
{
    size_t need = carve_sorted(nullptr, n_hits, n_events, h->C.M, nullptr);
    cudaError_t e = h->sorted_arena.reserve(need);
    if (e != cudaSuccess) return cuda_fail(h, e, "sorted-hit allocation");
    carve_sorted(h->sorted_arena.base, n_hits, n_events, h->C.M, O);
    return SBT_OK;
}

sbt_status ensure_staging(sbt_handle* h, int64_t n_hits, int64_t n_events, Staging* S)
{
    size_t need = carve_staging(nullptr, n_hits, n_events, nullptr);
    cudaError_t e = h->stage_arena.reserve(need);
    if (e != cudaSuccess) return cuda_fail(h, e, "staging allocation");
    carve_staging(h->stage_arena.base, n_hits, n_events, S);
    return SBT_OK;
}

// Grid of the persistent launch: resident blocks per SM (the autotuned count
// when it was tuned for this block size, else the occupancy limit) times SMs.
int persistent_blocks(sbt_handle* h, int threads, int per_sm_wanted = 0)
{
    int per_sm = persistent_blocks_per_sm(h->C, threads);
    if (per_sm_wanted > 0)
        per_sm = std::min(per_sm, per_sm_wanted);
    else if (threads == h->tuned_threads && h->tuned_blocks_per_sm > 0)
        per_sm = std::min(per_sm, h->tuned_blocks_per_sm);
    return std::max(per_sm, 1) * h->sm_count;
}

sbt_status ensure_persistent(sbt_handle* h, int blocks, Work* W)
{
    int64_t hits = (int64_t)blocks * h->C.nmax;
    size_t need = carve_work(nullptr, hits, blocks, nullptr);
    cudaError_t e = h->pers_arena.reserve(need);
    if (e != cudaSuccess) return cuda_fail(h, e, "persistent workspace allocation");
    carve_work(h->pers_arena.base, hits, blocks, W);
    return SBT_OK;
}

// Enqueue the batched sequence (order, sort, persistent search, scan, output).
sbt_status enqueue_batched(sbt_handle* h, const Inputs& in, const Sorted& O, const Staging& S,
                           const Work& W, const sbt_tracks& out, int threads, int blocks,
                           cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(S.queue, 0, 4 * sizeof(int32_t), st);
    if (e == cudaSuccess && in.n_events > 0) e = launch_order(in, S, st);
    if (e == cudaSuccess && in.n_events > 0) e = launch_sort(h->C, in, O, st);
    if (e == cudaSuccess && in.n_events > 0)
        e = launch_persistent(h->C, in, O, W, S, out, threads, std::min(blocks, in.n_events), st);
    if (e == cudaSuccess) e = launch_finish(h->C, in, S, out, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "batched launch");
    return SBT_OK;
}

}  // namespace

namespace sbt {

const DevConfig& handle_device_config(const sbt_handle* h) { return h->C; }

int handle_plain_threads(const sbt_handle* h) { return default_threads(h, false); }

void handle_set_error(sbt_handle* h, const std::string& msg) { h->err = msg; }

void handle_set_launches(sbt_handle* h, int launches) { h->launches_last = launches; }

void handle_defer_frees(sbt_handle* h)
{
    for (Arena* a : {&h->plain_arena, &h->pers_arena, &h->stage_arena, &h->host_arena, &h->misc_arena,
                     &h->sorted_arena})
        a->defer = true;
}

}  // namespace sbt

extern "C" {

sbt_status sbt_default_config(sbt_config* out)
{
    if (!out) return SBT_ERR_ARG;
    out->k_doublets = 4;
    out->max_scatter_seed = 0.04f;
    out->max_scatter_follow = 0.04f;
    out->max_chi2_tracklet = 20.0f;
    out->hit_sigma = 0.012f;
    out->max_hits_per_event = 16384;
    out->max_forming_tracks = 0;
    out->threads_per_block = 0;
    out->gec_max_hits = 0;
    out->fp16_hits = 0;
    return SBT_OK;
}

sbt_status sbt_create(const sbt_geometry* geometry, const sbt_config* cfg, sbt_handle** out)
{
    if (!out || !geometry || !geometry->module_z) {
        g_create_error = "NULL argument";
        return SBT_ERR_ARG;
    }
    *out = nullptr;
    if (geometry->n_modules < 3 || geometry->n_modules > kMaxModules) {
        g_create_error = "n_modules must be in [3, 64]";
        return SBT_ERR_ARG;
    }
    for (int m = 0; m < geometry->n_modules; m++)
        if (!std::isfinite(geometry->module_z[m]) ||
            (geometry->module_z2 && !std::isfinite(geometry->module_z2[m]))) {
            g_create_error = "plane positions must be finite";
            return SBT_ERR_ARG;
        }
    sbt_config c;
    if (cfg)
        c = *cfg;
    else
        sbt_default_config(&c);
    if (c.k_doublets < 1 || c.max_hits_per_event < 1 || c.max_hits_per_event > kMaxHitsPerEvent ||
        c.max_forming_tracks < 0 || c.gec_max_hits < 0 || !(c.hit_sigma > 0.0f) ||
        (c.threads_per_block != 0 && c.threads_per_block != 64 && c.threads_per_block != 128 &&
         c.threads_per_block != 256)) {
        g_create_error = "invalid configuration";
        return SBT_ERR_ARG;
    }
    sbt_handle* h = new sbt_handle();
    h->cfg = c;
    std::memset(&h->C, 0, sizeof(h->C));
    h->C.M = geometry->n_modules;
    for (int m = 0; m < h->C.M; m++) h->C.module_z[m] = geometry->module_z[m];
    h->C.pairs = geometry->module_z2 ? 1 : 0;
    for (int m = 0; m < h->C.M; m++)
        h->C.module_z2[m] = geometry->module_z2 ? geometry->module_z2[m] : geometry->module_z[m];
    h->C.K = c.k_doublets;
    h->C.S_seed = c.max_scatter_seed;
    h->C.S_follow = c.max_scatter_follow;
    h->C.C3 = c.max_chi2_tracklet;
    h->C.sigma = c.hit_sigma;
    h->C.nmax = c.max_hits_per_event;
    h->C.fcap = c.max_forming_tracks;
    h->C.gec = c.gec_max_hits;
    h->C.h16 = c.fp16_hits ? 1 : 0;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    int max_optin = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (e != cudaSuccess) {
        g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
        delete h;
        return SBT_ERR_CUDA;
    }
    if (sort_smem_bytes(h->C.nmax) > (size_t)max_optin || smem_bytes(h->C.nmax, 256, h->C.M) > (size_t)max_optin) {
        g_create_error = "max_hits_per_event exceeds shared memory";
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        delete h;
        return SBT_ERR_ARG;
    }
    *out = h;
    return SBT_OK;
}

sbt_status sbt_destroy(sbt_handle* h)
{
    if (!h) return SBT_ERR_ARG;
    cudaDeviceSynchronize();
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->copy_in) cudaStreamDestroy(h->copy_in);
    if (h->copy_out) cudaStreamDestroy(h->copy_out);
    if (h->sort_stream) cudaStreamDestroy(h->sort_stream);
    if (h->host_counts) cudaFreeHost(h->host_counts);
    h->plain_arena.release();
    h->sorted_arena.release();
    h->pers_arena.release();
    h->stage_arena.release();
    h->host_arena.release();
    h->misc_arena.release();
    delete h;
    return SBT_OK;
}

const char* sbt_last_error(const sbt_handle* h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

sbt_status sbt_reconstruct(sbt_handle* h, const float* x, const float* y, const float* z,
                           const int32_t* module, const int32_t* event_offsets, int32_t n_events,
                           int32_t n_hits, const sbt_tracks* out, void* stream)
{
    sbt_status st = check_inputs(h, x, y, z, module, event_offsets, n_events, n_hits, out);
    if (st != SBT_OK || !out) return st != SBT_OK ? st : SBT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Staging S;
    Sorted O;
    if ((st = ensure_staging(h, n_hits, n_events, &S)) != SBT_OK) return st;
    if ((st = ensure_sorted(h, n_hits, n_events, &O)) != SBT_OK) return st;
    size_t need = carve_work(nullptr, n_hits, n_events, nullptr);
    cudaError_t e = h->plain_arena.reserve(need);
    if (e != cudaSuccess) return cuda_fail(h, e, "workspace allocation");
    Work W;
    carve_work(h->plain_arena.base, n_hits, n_events, &W);
    Inputs in = make_inputs(x, y, z, module, event_offsets, n_events, n_hits);
    e = launch_sort(h->C, in, O, s);
    if (e == cudaSuccess) e = launch_plain(h->C, in, O, W, S, *out, default_threads(h, false), s);
    if (e == cudaSuccess) e = launch_finish(h->C, in, S, *out, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "plain launch");
    h->launches_last = n_events > 0 ? 5 : 2;
    return SBT_OK;
}

sbt_status sbt_reconstruct_batched(sbt_handle* h, const float* x, const float* y, const float* z,
                                   const int32_t* module, const int32_t* event_offsets,
                                   int32_t n_events, int32_t n_hits, const sbt_tracks* out,
                                   void* stream)
{
    sbt_status st = check_inputs(h, x, y, z, module, event_offsets, n_events, n_hits, out);
    if (st != SBT_OK || !out) return st != SBT_OK ? st : SBT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = default_threads(h, true);
    const int blocks = persistent_blocks(h, threads);
    Staging S;
    Work W;
    Sorted O;
    const void* old_stage = h->stage_arena.base;
    const void* old_pers = h->pers_arena.base;
    const void* old_sorted = h->sorted_arena.base;
    if ((st = ensure_staging(h, n_hits, n_events, &S)) != SBT_OK) return st;
    if ((st = ensure_persistent(h, blocks, &W)) != SBT_OK) return st;
    if ((st = ensure_sorted(h, n_hits, n_events, &O)) != SBT_OK) return st;
    GraphKey k{};
    const void* ptrs[13] = {x, y, z, module, event_offsets, out->track_offsets, out->hit_offsets,
                            out->track_hits, out->params, out->chi2, out->ndof, out->event_status,
                            out->counts};
    std::memcpy(k.ptrs, ptrs, sizeof(ptrs));
    k.vals[0] = n_events;
    k.vals[1] = n_hits;
    k.vals[2] = out->cap_tracks;
    k.vals[3] = out->cap_hits;
    k.vals[4] = threads;
    k.vals[5] = blocks;
    const bool moved = old_stage != h->stage_arena.base || old_pers != h->pers_arena.base ||
                       old_sorted != h->sorted_arena.base;
    if (!h->exec || !h->have_key || moved || !(k == h->key)) {
        if (h->exec) {
            cudaGraphExecDestroy(h->exec);
            h->exec = nullptr;
        }
        h->have_key = false;
        Inputs in = make_inputs(x, y, z, module, event_offsets, n_events, n_hits);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture begin");
        st = enqueue_batched(h, in, O, S, W, *out, threads, blocks, h->cap_stream);
        e = cudaStreamEndCapture(h->cap_stream, &g);
        if (st != SBT_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "graph capture end");
        e = cudaGraphInstantiate(&h->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->exec = nullptr;
            return cuda_fail(h, e, "graph instantiate");
        }
        h->key = k;
        h->have_key = true;
    }
    cudaError_t e = cudaGraphLaunch(h->exec, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    h->launches_last = n_events > 0 ? 6 : 2;
    return SBT_OK;
}

sbt_status sbt_reconstruct_host(sbt_handle* h, const float* x, const float* y, const float* z,
                                const int32_t* module, const int32_t* event_offsets,
                                int32_t n_events, int32_t n_hits, const sbt_tracks* oh,
                                void* stream)
{
    sbt_status st = check_inputs(h, x, y, z, module, event_offsets, n_events, n_hits, oh);
    if (st != SBT_OK || !oh) return st != SBT_OK ? st : SBT_ERR_ARG;
    if (!host_offsets_valid(event_offsets, n_events, n_hits))
        return fail(h, SBT_ERR_ARG, "event_offsets must be non-decreasing, from >= 0 to <= n_hits");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!h->copy_in) e = cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->copy_out) e = cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->sort_stream) e = cudaStreamCreateWithFlags(&h->sort_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->host_counts) e = cudaMallocHost(&h->host_counts, sizeof(int32_t) * 4 * kMaxChunks);
    if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline set-up");
    // chunks of whole events: inputs of chunk c+1 upload while chunk c
    // computes, results of chunk c download while chunk c+1 computes
    const int64_t H = n_hits, E = n_events;
    const bool large = E >= kLargeBatchEvents;
    const double* weights = large ? kChunkWeightsLarge : kChunkWeights;
    const int C = E > kChunkEvents ? (large ? kWeightedChunksLarge : kWeightedChunks) : 1;
    std::vector<int32_t> e0(C + 1);
    {
        double wsum = 0.0, acc = 0.0;
        for (int c = 0; c < C; c++) wsum += C > 1 ? weights[c] : 1.0;
        e0[0] = 0;
        for (int c = 0; c < C; c++) {
            acc += C > 1 ? weights[c] : 1.0;
            e0[c + 1] = c + 1 == C ? (int32_t)E : (int32_t)((double)E * acc / wsum);
        }
    }
    auto layout = [&](Carver& cv, float** dx, float** dy, float** dz, int32_t** dm, int32_t** doff,
                      int32_t** dto, int32_t** dho, int32_t** dth, float** dpar, float** dchi,
                      int32_t** dndof, int32_t** dstat, int32_t** dcnt, int64_t** drun) {
        *dx = cv.take<float>(H);
        *dy = cv.take<float>(H);
        *dz = cv.take<float>(H);
        *dm = cv.take<int32_t>(H);
        *doff = cv.take<int32_t>(E + 1);
        *dto = cv.take<int32_t>(E + C);
        *dho = cv.take<int32_t>(H / 3 + 2 * C + 1);
        *dth = cv.take<int32_t>(H + C);
        *dpar = cv.take<float>(4 * (H / 3 + 2 * C));
        *dchi = cv.take<float>(H / 3 + 2 * C);
        *dndof = cv.take<int32_t>(H / 3 + 2 * C);
        *dstat = cv.take<int32_t>(E);
        *dcnt = cv.take<int32_t>(4 * C);
        *drun = cv.take<int64_t>(2 * (C + 1));
    };
    float *dx, *dy, *dz, *dpar, *dchi;
    int32_t *dm, *doff, *dto, *dho, *dth, *dndof, *dstat, *dcnt;
    int64_t* drun;
    Carver c0(nullptr);
    layout(c0, &dx, &dy, &dz, &dm, &doff, &dto, &dho, &dth, &dpar, &dchi, &dndof, &dstat, &dcnt, &drun);
    e = h->host_arena.reserve(c0.off + 256);
    if (e != cudaSuccess) return cuda_fail(h, e, "host-path allocation");
    Carver c1(h->host_arena.base);
    layout(c1, &dx, &dy, &dz, &dm, &doff, &dto, &dho, &dth, &dpar, &dchi, &dndof, &dstat, &dcnt, &drun);
    const int threads = default_threads(h, true);
    const int blocks = persistent_blocks(h, threads);
    Staging S;
    Work W;
    Sorted O;
    if ((st = ensure_staging(h, n_hits, n_events, &S)) != SBT_OK) return st;
    if ((st = ensure_persistent(h, blocks, &W)) != SBT_OK) return st;
    if ((st = ensure_sorted(h, n_hits, n_events, &O)) != SBT_OK) return st;
    std::vector<cudaEvent_t> in_ev(C), sort_ev(C), comp_ev(C);
    for (int c = 0; c < C; c++) {
        cudaEventCreateWithFlags(&in_ev[c], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&sort_ev[c], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&comp_ev[c], cudaEventDisableTiming);
    }
    auto cleanup = [&]() {
        for (int c = 0; c < C; c++) {
            cudaEventDestroy(in_ev[c]);
            cudaEventDestroy(sort_ev[c]);
            cudaEventDestroy(comp_ev[c]);
        }
    };
    // uploads
    e = cudaMemcpyAsync(doff, event_offsets, sizeof(int32_t) * (E + 1), cudaMemcpyHostToDevice, h->copy_in);
    for (int c = 0; c < C && e == cudaSuccess; c++) {
        const int64_t a = event_offsets[e0[c]], b = event_offsets[e0[c + 1]];
        const size_t nb = sizeof(float) * (size_t)(b - a);
        if (nb) {
            e = cudaMemcpyAsync(dx + a, x + a, nb, cudaMemcpyHostToDevice, h->copy_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dy + a, y + a, nb, cudaMemcpyHostToDevice, h->copy_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dz + a, z + a, nb, cudaMemcpyHostToDevice, h->copy_in);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dm + a, module + a, nb, cudaMemcpyHostToDevice, h->copy_in);
        }
        if (e == cudaSuccess) e = cudaEventRecord(in_ev[c], h->copy_in);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(drun, 0, 2 * sizeof(int64_t), s);  // totals before chunk 0
    // per-chunk reconstruction; chunk c's outputs start at event e0[c] + c,
    // track slot hits/3 + 2c and hit slot hits + c of the device buffers.
    // Every chunk has its own slice of the per-event sorted and staged arrays
    // (the hit-indexed ones are disjoint already), so a chunk's order and
    // sort run on the sort stream as soon as its inputs are up, in the tail
    // of the previous chunk's search; the searches, which share the
    // persistent scratch, stay in order on the compute stream.
    std::vector<sbt_tracks> dc(C);
    auto chunk_views = [&](int c, Sorted& Oc, Staging& Sc) {
        const int64_t ev0 = e0[c];
        Oc = O;
        Oc.modoff = O.modoff + ev0 * (h->C.M + 1);
        Oc.status = O.status + ev0;
        Sc = S;
        Sc.tkey = S.tkey + ev0;  // slot off/3 + event: the chunk-local event index plus e0[c]
        Sc.tinfo = S.tinfo + ev0;
        Sc.rinfo = S.rinfo + ev0;
        Sc.ev_ntracks = S.ev_ntracks + ev0;
        Sc.ev_nhits = S.ev_nhits + ev0;
        Sc.track_base = S.track_base + ev0;
        Sc.hit_base = S.hit_base + ev0;
        Sc.order = S.order + ev0;
        Sc.queue = S.queue + 4 * c;
        // Sc.tfit is indexed by the chunk's own track numbers: the chunks'
        // output and fit kernels run one after the other on one stream
    };
    for (int c = 0; c < C && e == cudaSuccess; c++) {
        const int32_t Ec = e0[c + 1] - e0[c];
        const int64_t a = event_offsets[e0[c]], b = event_offsets[e0[c + 1]];
        sbt_tracks& d = dc[c];
        const int64_t tslot = a / 3 + 2 * c;
        d.track_offsets = dto + e0[c] + c;
        d.hit_offsets = dho + tslot;
        d.track_hits = dth + a + c;
        d.params = dpar + 4 * tslot;
        d.chi2 = dchi + tslot;
        d.ndof = dndof + tslot;
        d.event_status = dstat + e0[c];
        d.counts = dcnt + 4 * c;
        d.cap_tracks = (int32_t)((b - a) / 3 + 1);
        d.cap_hits = (int32_t)(b - a + 1);
        Inputs in = make_inputs(dx, dy, dz, dm, doff + e0[c], Ec, (int32_t)b);
        Sorted Oc;
        Staging Sc;
        chunk_views(c, Oc, Sc);
        cudaStream_t so = h->sort_stream;
        e = cudaStreamWaitEvent(so, in_ev[c], 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(Sc.queue, 0, 4 * sizeof(int32_t), so);
        if (e == cudaSuccess && Ec > 0) e = launch_order(in, Sc, so);
        if (e == cudaSuccess && Ec > 0) e = launch_sort(h->C, in, Oc, so);
        if (e == cudaSuccess) e = cudaEventRecord(sort_ev[c], so);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, sort_ev[c], 0);
        if (e == cudaSuccess && Ec > 0) e = launch_persistent(h->C, in, Oc, W, Sc, d, threads, std::min(blocks, Ec), s);
        if (e == cudaSuccess) e = launch_finish(h->C, in, Sc, d, s);
        if (e == cudaSuccess)
            e = launch_offset_fixup(d.track_offsets, Ec, d.hit_offsets, d.counts, drun + 2 * c, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->host_counts + 4 * c, d.counts, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(comp_ev[c], s);
    }
    // downloads as chunks finish
    int64_t T = 0, HH = 0, failed = 0;
    bool cap_ok = true;
    for (int c = 0; c < C && e == cudaSuccess; c++) {
        e = cudaEventSynchronize(comp_ev[c]);
        if (e != cudaSuccess) break;
        const int32_t* cn = h->host_counts + 4 * c;
        const int32_t Ec = e0[c + 1] - e0[c];
        const int64_t Tc = cn[0], Hc = cn[1];
        failed += cn[3];
        const sbt_tracks& d = dc[c];
        cudaStream_t o = h->copy_out;
        e = cudaMemcpyAsync(oh->track_offsets + e0[c], d.track_offsets, sizeof(int32_t) * (Ec + (c == C - 1)),
                            cudaMemcpyDeviceToHost, o);
        if (e == cudaSuccess && Ec)
            e = cudaMemcpyAsync(oh->event_status + e0[c], d.event_status, sizeof(int32_t) * Ec,
                                cudaMemcpyDeviceToHost, o);
        if (cn[2] != SBT_OK || T + Tc > oh->cap_tracks || HH + Hc > oh->cap_hits) cap_ok = false;
        if (e == cudaSuccess && cap_ok) {
            e = cudaMemcpyAsync(oh->hit_offsets + T, d.hit_offsets, sizeof(int32_t) * (Tc + 1),
                                cudaMemcpyDeviceToHost, o);
            if (e == cudaSuccess && Hc)
                e = cudaMemcpyAsync(oh->track_hits + HH, d.track_hits, sizeof(int32_t) * Hc,
                                    cudaMemcpyDeviceToHost, o);
            if (e == cudaSuccess && Tc) {
                e = cudaMemcpyAsync(oh->params + 4 * T, d.params, 16 * Tc, cudaMemcpyDeviceToHost, o);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(oh->chi2 + T, d.chi2, 4 * Tc, cudaMemcpyDeviceToHost, o);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(oh->ndof + T, d.ndof, 4 * Tc, cudaMemcpyDeviceToHost, o);
            }
        }
        T += Tc;
        HH += Hc;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_out);
    if (e != cudaSuccess) {
        // nothing already queued may write into the caller's buffers after
        // the call returns: let every stream of the pipeline drain first
        cudaStreamSynchronize(h->copy_in);
        cudaStreamSynchronize(h->sort_stream);
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(h->copy_out);
    }
    cleanup();
    if (e != cudaSuccess) return cuda_fail(h, e, "host pipeline");
    if (E == 0) oh->track_offsets[0] = 0;
    oh->counts[0] = (int32_t)T;
    oh->counts[1] = (int32_t)HH;
    oh->counts[2] = cap_ok ? SBT_OK : SBT_ERR_CAPACITY;
    oh->counts[3] = (int32_t)failed;
    h->launches_last = C * 7;
    return SBT_OK;
}

sbt_status sbt_autotune(sbt_handle* h, const float* x, const float* y, const float* z,
                        const int32_t* module, const int32_t* event_offsets, int32_t n_events,
                        int32_t n_hits, int32_t* chosen, int32_t* chosen_blocks_per_sm, void* stream)
{
    sbt_status st = check_inputs(h, x, y, z, module, event_offsets, n_events, n_hits, nullptr);
    if (st != SBT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Staging S;
    Sorted O;
    if ((st = ensure_staging(h, n_hits, n_events, &S)) != SBT_OK) return st;
    if ((st = ensure_sorted(h, n_hits, n_events, &O)) != SBT_OK) return st;
    cudaError_t e = h->misc_arena.reserve(std::max(sizeof(int32_t) * ((size_t)n_events + 8), h->misc_arena.bytes));
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune allocation");
    sbt_tracks scratch_out;
    std::memset(&scratch_out, 0, sizeof(scratch_out));
    scratch_out.event_status = (int32_t*)h->misc_arena.base;
    Inputs in = make_inputs(x, y, z, module, event_offsets, n_events, n_hits);
    e = launch_order(in, S, s);
    if (e == cudaSuccess) e = launch_sort(h->C, in, O, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best_ms = 1e30f;
    int best = 128, best_per_sm = 0;
    // block sizes, and for each the occupancy limit of resident blocks per SM
    // and three quarters and half of it (the search waits on load latency:
    // more resident events hide more of it, but also share L1 and L2)
    const int cands[3] = {64, 128, 256};
    for (int threads : cands) {
        const int limit = std::max(persistent_blocks_per_sm(h->C, threads), 1);
        int per_sms[3] = {limit, std::max(1, (3 * limit) / 4), std::max(1, limit / 2)};
        for (int ci = 0; ci < 3 && e == cudaSuccess && st == SBT_OK; ci++) {
            const int per_sm = per_sms[ci];
            if (ci > 0 && per_sm == per_sms[ci - 1]) continue;
            const int blocks = persistent_blocks(h, threads, per_sm);
            Work W;
            if ((st = ensure_persistent(h, blocks, &W)) != SBT_OK) break;
            float tot = 0.0f;
            for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {
                e = cudaMemsetAsync(S.queue, 0, 16, s);
                if (e == cudaSuccess) e = cudaEventRecord(a, s);
                if (e == cudaSuccess)
                    e = launch_persistent(h->C, in, O, W, S, scratch_out, threads,
                                          std::min(blocks, std::max(n_events, 1)), s);
                if (e == cudaSuccess) e = cudaEventRecord(b, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0.0f;
                if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) tot += ms;  // first repetition is warm-up
            }
            if (e == cudaSuccess && tot < best_ms) {
                best_ms = tot;
                best = threads;
                best_per_sm = per_sm;
            }
        }
        if (e != cudaSuccess || st != SBT_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != SBT_OK) return st;
    if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
    h->tuned_threads = best;
    h->tuned_blocks_per_sm = best_per_sm;
    if (chosen) *chosen = best;
    if (chosen_blocks_per_sm) *chosen_blocks_per_sm = best_per_sm;
    if (h->exec) {  // the workspace may have moved
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
        h->have_key = false;
    }
    return SBT_OK;
}

/* Sets the launch shape of the persistent search (as sbt_autotune would). */
sbt_status sbt_set_launch_shape(sbt_handle* h, int32_t threads, int32_t blocks_per_sm)
{
    if (!h) return SBT_ERR_ARG;
    if ((threads != 64 && threads != 128 && threads != 256) || blocks_per_sm < 0)
        return fail(h, SBT_ERR_ARG, "threads must be 64, 128 or 256 and blocks_per_sm >= 0");
    h->tuned_threads = threads;
    h->tuned_blocks_per_sm = blocks_per_sm;
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
        h->have_key = false;
    }
    return SBT_OK;
}

/* Tuned launch shape of the handle (0, 0 before sbt_autotune). */
sbt_status sbt_tuned_shape(const sbt_handle* h, int32_t* threads, int32_t* blocks_per_sm)
{
    if (!h || !threads || !blocks_per_sm) return SBT_ERR_ARG;
    *threads = h->tuned_threads;
    *blocks_per_sm = h->tuned_blocks_per_sm;
    return SBT_OK;
}

sbt_status sbt_fit_adjoint(sbt_handle* h, const float* x, const float* y, const float* z,
                           const int32_t* module, int32_t n_hits, const int32_t* hit_offsets,
                           const int32_t* track_hits, int32_t n_tracks, const double* align,
                           double* chi2_sum, double* grad, int32_t* skipped, void* stream)
{
    if (!h) return SBT_ERR_ARG;
    if (h->C.pairs) return fail(h, SBT_ERR_ARG, "the alignment adjoint takes single-plane modules");
    if (n_hits < 0 || n_tracks < 0) return fail(h, SBT_ERR_ARG, "negative size");
    if (!hit_offsets || !align || !chi2_sum || (n_tracks > 0 && (!track_hits || !x || !y || !z || !module)))
        return fail(h, SBT_ERR_ARG, "NULL argument");
    AdjointWork W;
    W.blocks = adjoint_blocks(h->sm_count);
    size_t need = sizeof(double) * adjoint_partial_entries(h->C.M, W.blocks);
    cudaError_t e = h->misc_arena.reserve(std::max(need, h->misc_arena.bytes));
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint allocation");
    W.partial = (double*)h->misc_arena.base;
    Inputs in = make_inputs(x, y, z, module, nullptr, 0, n_hits);
    e = launch_adjoint(h->C, in, hit_offsets, track_hits, n_tracks, align, chi2_sum, grad, skipped, W,
                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint launch");
    return SBT_OK;
}

sbt_status sbt_debug_sort(sbt_handle* h, const float* x, const float* y, const int32_t* module,
                          const int32_t* event_offsets, int32_t n_events, int32_t n_hits,
                          uint16_t* phi16, int32_t* perm, int32_t* module_offsets, void* stream)
{
    sbt_status st = check_inputs(h, x, y, x, module, event_offsets, n_events, n_hits, nullptr);
    if (st != SBT_OK) return st;
    if (!phi16 || !perm || !module_offsets) return fail(h, SBT_ERR_ARG, "NULL output");
    Sorted O;
    if ((st = ensure_sorted(h, n_hits, n_events, &O)) != SBT_OK) return st;
    Inputs in = make_inputs(x, y, x, module, event_offsets, n_events, n_hits);
    cudaError_t e = launch_sort(h->C, in, O, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = launch_debug_sort_copy(h->C, in, O, phi16, perm, module_offsets, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "debug sort launch");
    return SBT_OK;
}

sbt_status sbt_debug_phi16(const float* x, const float* y, int32_t n, uint16_t* out, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !y || !out))) return SBT_ERR_ARG;
    cudaError_t e = launch_debug_phi16(x, y, n, out, (cudaStream_t)stream);
    return e == cudaSuccess ? SBT_OK : SBT_ERR_CUDA;
}

sbt_status sbt_profile_batched(sbt_handle* h, const float* x, const float* y, const float* z,
                               const int32_t* module, const int32_t* event_offsets,
                               int32_t n_events, int32_t n_hits, const sbt_tracks* out, int32_t reps,
                               float* ms, void* stream)
{
    sbt_status st = check_inputs(h, x, y, z, module, event_offsets, n_events, n_hits, out);
    if (st != SBT_OK || !out || !ms || reps < 1) return st != SBT_OK ? st : fail(h, SBT_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = default_threads(h, true);
    const int blocks = persistent_blocks(h, threads);
    Staging S;
    Work W;
    Sorted O;
    if ((st = ensure_staging(h, n_hits, n_events, &S)) != SBT_OK) return st;
    if ((st = ensure_persistent(h, blocks, &W)) != SBT_OK) return st;
    if ((st = ensure_sorted(h, n_hits, n_events, &O)) != SBT_OK) return st;
    if (h->exec) {  // the workspace may have moved
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
        h->have_key = false;
    }
    Inputs in = make_inputs(x, y, z, module, event_offsets, n_events, n_hits);
    cudaEvent_t ev[6];
    for (int i = 0; i < 6; i++) cudaEventCreate(&ev[i]);
    double acc[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; r++) {
        e = cudaMemsetAsync(S.queue, 0, 16, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
        if (e == cudaSuccess && n_events > 0) e = launch_order(in, S, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
        if (e == cudaSuccess && n_events > 0) e = launch_sort(h->C, in, O, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
        if (e == cudaSuccess && n_events > 0)
            e = launch_persistent(h->C, in, O, W, S, *out, threads, std::min(blocks, n_events), s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);
        if (e == cudaSuccess) e = launch_scan(in, S, *out, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[4], s);
        if (e == cudaSuccess) e = launch_output(h->C, in, S, *out, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[5], s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[5]);
        for (int k = 0; k < 5 && e == cudaSuccess; k++) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (int i = 0; i < 6; i++) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return cuda_fail(h, e, "profile");
    for (int k = 0; k < 5; k++) ms[k] = (float)(acc[k] / reps);
    return SBT_OK;
}

/* Number of kernels the last reconstruction call enqueued (for launch accounting). */
int32_t sbt_last_launch_count(const sbt_handle* h) { return h ? h->launches_last : 0; }

}  // extern "C"

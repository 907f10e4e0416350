// Reconstruction entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a trigger or serving process that
// reserves all of its device memory when it starts and forbids allocation
// afterwards (cudaMalloc and cudaFree synchronise the device and may fail once
// the memory is taken), or a plug-in running inside an application that owns
// the device's memory pool.  For them sbt_reconstruct_noalloc runs the same
// one-block-per-event reconstruction as sbt_reconstruct, but its workspace is
// the fixed array below, which is part of the library's device image: every
// GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sbt_internal.h"

using namespace sbt;

namespace {

// Limits of one call: the workspace is sized for these.
constexpr int64_t kNoAllocMaxHits = int64_t(1) << 19;   // 524288 hits
constexpr int64_t kNoAllocMaxEvents = int64_t(1) << 12; // 4096 events

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Offsets of the workspace arrays (the Sorted, Work and Staging layouts for
// kNoAllocMaxHits hits and kNoAllocMaxEvents events), each 256-byte aligned.
struct Layout {
    size_t coords, phi, modoff, status;
    size_t list, prev, claim, ft, tracklets, tl_q, finals;
    size_t hits, tkey, tinfo, rinfo, tfit, ntracks, nhits, track_base, hit_base, order, queue, total;
};

constexpr Layout make_layout()
{
    Layout L{};
    const int64_t H = kNoAllocMaxHits, E = kNoAllocMaxEvents;
    const int64_t TL = H + E + 1, FN = H / 3 + E + 1;
    size_t o = 0;
    L.coords = o;     o = align256(o + 16 * (size_t)H);
    L.phi = o;        o = align256(o + 2 * (size_t)H);
    L.modoff = o;     o = align256(o + 4 * (size_t)E * (kMaxModules + 1));
    L.status = o;     o = align256(o + 4 * (size_t)E);
    L.list = o;       o = align256(o + 4 * (size_t)H);
    L.prev = o;       o = align256(o + 2 * (size_t)H);
    L.claim = o;      o = align256(o + 8 * (size_t)H);
    L.ft = o;         o = align256(o + 16 * (size_t)(2 * (H / 12 + 72 * E) + 2));
    L.tracklets = o;  o = align256(o + 8 * (size_t)TL);
    L.tl_q = o;       o = align256(o + 4 * (size_t)TL);
    L.finals = o;     o = align256(o + 4 * (size_t)FN);
    L.hits = o;       o = align256(o + 16 * (size_t)H);
    L.tkey = o;       o = align256(o + 4 * (size_t)(H / 3 + E + 1));
    L.tinfo = o;      o = align256(o + 4 * (size_t)(H / 3 + E + 1));
    L.rinfo = o;      o = align256(o + 4 * (size_t)(H / 3 + E + 1));
    L.tfit = o;       o = align256(o + 8 * (size_t)(H / 3 + E + 1));
    L.ntracks = o;    o = align256(o + 4 * (size_t)E);
    L.nhits = o;      o = align256(o + 4 * (size_t)E);
    L.track_base = o; o = align256(o + 4 * (size_t)E);
    L.hit_base = o;   o = align256(o + 4 * (size_t)E);
    L.order = o;      o = align256(o + 4 * (size_t)E);
    L.queue = o;      o = align256(o + 16);
    L.total = o;
    return L;
}

constexpr Layout kLayout = make_layout();

// The workspace (about 48 MB).  In host code this name is only a host-side
// stand-in: its device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_noalloc_workspace[kLayout.total];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
unsigned char* g_device_ptr[kMaxDevices] = {};

// Device address of the workspace on the current device, looked up once per
// device (the first call on each device does this) and kept for the life of
// the process: a cudaDeviceReset unloads the library's device image, after
// which the kept address is no longer valid.
cudaError_t workspace_address(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_device_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_workspace);
        if (e != cudaSuccess) return e;
        g_device_ptr[dev] = (unsigned char*)p;
    }
    *out = g_device_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sbt_status sbt_reconstruct_noalloc(sbt_handle* h, const float* x, const float* y,
                                              const float* z, const int32_t* module,
                                              const int32_t* event_offsets, int32_t n_events,
                                              int32_t n_hits, const sbt_tracks* out, void* stream)
{
    if (!h) return SBT_ERR_ARG;
    if (n_events < 0 || n_hits < 0 || !event_offsets || !out) {
        handle_set_error(h, "invalid argument");
        return SBT_ERR_ARG;
    }
    if ((int64_t)n_hits > kNoAllocMaxHits || (int64_t)n_events > kNoAllocMaxEvents) {
        handle_set_error(h, "sbt_reconstruct_noalloc: batch exceeds the fixed workspace (at most " +
                                std::to_string(kNoAllocMaxHits) + " hits and " +
                                std::to_string(kNoAllocMaxEvents) + " events per call)");
        return SBT_ERR_ARG;
    }
    if (n_hits > 0 && (!x || !y || !z || !module)) {
        handle_set_error(h, "hit array is NULL");
        return SBT_ERR_ARG;
    }
    if (!out->track_offsets || !out->hit_offsets || !out->counts || (n_events > 0 && !out->event_status) ||
        out->cap_tracks < 0 || out->cap_hits < 0 ||
        (out->cap_tracks > 0 && (!out->params || !out->chi2 || !out->ndof)) ||
        (out->cap_hits > 0 && !out->track_hits)) {
        handle_set_error(h, "output array is NULL or capacity negative");
        return SBT_ERR_ARG;
    }
    unsigned char* base = nullptr;
    cudaError_t e = workspace_address(&base);
    if (e != cudaSuccess) {
        handle_set_error(h, std::string("workspace address: ") + cudaGetErrorString(e));
        return SBT_ERR_CUDA;
    }
    const Layout& L = kLayout;
    Sorted O;
    O.coords = (float4*)(base + L.coords);
    O.phi = (uint16_t*)(base + L.phi);
    O.modoff = (int32_t*)(base + L.modoff);
    O.status = (int32_t*)(base + L.status);
    Work W;
    W.list = (uint32_t*)(base + L.list);
    W.prev = (uint16_t*)(base + L.prev);
    W.claim = (unsigned long long*)(base + L.claim);
    W.ft = (FTrack*)(base + L.ft);
    W.tracklets = (unsigned long long*)(base + L.tracklets);
    W.tl_q = (uint32_t*)(base + L.tl_q);
    W.finals = (uint32_t*)(base + L.finals);
    Staging S;
    S.hits = (float4*)(base + L.hits);
    S.tkey = (int32_t*)(base + L.tkey);
    S.tinfo = (uint32_t*)(base + L.tinfo);
    S.rinfo = (uint32_t*)(base + L.rinfo);
    S.tfit = (uint2*)(base + L.tfit);
    S.ev_ntracks = (int32_t*)(base + L.ntracks);
    S.ev_nhits = (int32_t*)(base + L.nhits);
    S.track_base = (int32_t*)(base + L.track_base);
    S.hit_base = (int32_t*)(base + L.hit_base);
    S.order = (int32_t*)(base + L.order);
    S.queue = (int32_t*)(base + L.queue);
    // Every array the kernels read is written earlier in the same call (sorted
    // hits and status by the sort kernel, claims per event before they are
    // used, staged hit lists and counts per event before the scan and the
    // output kernel read them), so nothing needs clearing between calls.
    Inputs in;
    in.x = x;
    in.y = y;
    in.z = z;
    in.module = module;
    in.offsets = event_offsets;
    in.n_events = n_events;
    in.n_hits = n_hits;
    cudaStream_t s = (cudaStream_t)stream;
    const DevConfig& C = handle_device_config(h);
    e = launch_sort(C, in, O, s);
    if (e == cudaSuccess) e = launch_plain(C, in, O, W, S, *out, handle_plain_threads(h), s);
    if (e == cudaSuccess) e = launch_finish(C, in, S, *out, s);
    if (e != cudaSuccess) {
        handle_set_error(h, std::string("noalloc launch: ") + cudaGetErrorString(e));
        return SBT_ERR_CUDA;
    }
    handle_set_launches(h, n_events > 0 ? 5 : 2);
    return SBT_OK;
}

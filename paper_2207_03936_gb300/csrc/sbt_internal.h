// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "sbt.h"

namespace sbt {

constexpr int kMaxModules = 64;
constexpr int kMaxHitsPerEvent = 16384;  // the per-event sort runs in shared memory

// Method constants and per-event capacities, passed to kernels by value.
struct DevConfig {
    int M;
    float module_z[kMaxModules];
    int K;
    float S_seed, S_follow, C3, sigma;
    int nmax;  // max hits per event
    int fcap;  // upper bound on forming tracks per event (0: forming_capacity(n) only)
    int gec;   // global event cut: events above this many hits are rejected (0: none)
    int h16;   // sorted hits stored as fp16 x, y, z + 16-bit index (8 bytes) instead of float4
    int pairs; // module pairs: hits with x < 0 lie on the plane at module_z2 (0: single planes)
    float module_z2[kMaxModules];
};

struct Inputs {
    const float* x;
    const float* y;
    const float* z;
    const int32_t* module;
    const int32_t* offsets;
    int32_t n_events;
    int32_t n_hits;
};

// A forming track: its last three hits (sorted positions), key, hit count,
// consecutive misses, and this step's candidate hit and scatter.
struct __align__(16) FTrack {
    uint16_t h0, h1, h2, key;
    uint8_t nh, sk;
    uint16_t cand;
    float sc;
};

// Forming-track capacity of an event of n hits, and the slots a region of
// capacity cap reserves (two buffers).
__host__ __device__ inline int forming_capacity(int n) { return n / 12 + 64; }
__host__ __device__ inline int64_t forming_base(int64_t hb, int64_t r) { return 2 * (hb / 12 + 72 * r); }
inline int64_t forming_entries(int64_t hits, int64_t regions) { return 2 * (hits / 12 + 72 * regions) + 2; }

// Sorted hits of every event, written by the sort kernel (indexed like the
// inputs: event e owns [event_offsets[e], event_offsets[e+1])).
struct Sorted {
    float4* coords;   // (x, y, z, event-local input index as int bits) by sorted position
    uint16_t* phi;    // phi16 by sorted position
    int32_t* modoff;  // [n_events * (n_modules + 1)] event-local module offsets
    int32_t* status;  // [n_events] SBT_OK, SBT_ERR_ARG or SBT_ERR_CAPACITY after the sort
};

// Per-region scratch of the search (a region is an event in the plain launch,
// a resident block in the persistent launch).  Region r with hit base hb and
// capacity cap owns per-hit arrays [hb, hb + cap), tracklets from hb + r
// (cap + 1 entries: every seed has its own middle hit, so an event has at most
// one tracklet per hit), final-track records from hb/3 + r (cap/3 + 1
// entries: final tracks are disjoint and have three hits or more) and
// forming-track slots from forming_base(hb, r) (2 (cap/12 + 72) entries).
struct Work {
    uint32_t* list;              // seeding work lists
    uint16_t* prev;              // previous hit of a track, by sorted position
    unsigned long long* claim;   // hit claims (tagged keys), by sorted position
    FTrack* ft;                  // forming tracks, two buffers
    unsigned long long* tracklets;
    uint32_t* tl_q;
    uint32_t* finals;            // last hit | nhits << 16
};

// Per-event results of the search, consumed by the output kernel.  Track
// records of event e start at slot off/3 + e (an event has at most n/3
// tracks: they are disjoint and have three hits or more).
struct Staging {
    float4* hits;         // [n_hits]: event e from event_offsets[e], each track's hit records
                          // contiguous in traversal order, tracks in found order
                          // (x, y, z as stored, batch input index as int bits)
    int32_t* tkey;        // [n_hits / 3 + n_events + 1] smallest input index of each found track
    uint32_t* tinfo;      // same indexing: first staged hit | hits << 16, found order
    uint32_t* rinfo;      // same indexing: tinfo of the track of each rank (output kernel)
    uint2* tfit;          // same size, by batch track index: first staged hit, hits (fit kernel)
    int32_t* ev_ntracks;  // [n_events]
    int32_t* ev_nhits;    // [n_events]
    int32_t* track_base;  // [n_events]
    int32_t* hit_base;    // [n_events]
    int32_t* order;       // [n_events] processing order of the persistent launch
    int32_t* queue;       // [4]      work-queue head; [1]: tracks the output kernel writes
};

// Sizes of the scratch arrays for `hits` hit slots over `regions` regions.
inline int64_t tracklet_entries(int64_t hits, int64_t regions) { return hits + regions + 1; }
inline int64_t final_entries(int64_t hits, int64_t regions) { return hits / 3 + regions + 1; }

size_t smem_bytes(int nmax, int threads, int M);
size_t sort_smem_bytes(int nmax);

// Launchers (sbt_reco.cu).  All asynchronous on `stream`.
cudaError_t launch_sort(const DevConfig& C, const Inputs& in, const Sorted& O, cudaStream_t stream);
cudaError_t launch_plain(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                         const Staging& S, const sbt_tracks& out, int threads, cudaStream_t stream);
cudaError_t launch_order(const Inputs& in, const Staging& S, cudaStream_t stream);
cudaError_t launch_persistent(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                              const Staging& S, const sbt_tracks& out, int threads, int blocks,
                              cudaStream_t stream);
// Scan of the per-event counts, then the output kernel (CSR hit lists and fits).
cudaError_t launch_finish(const DevConfig& C, const Inputs& in, const Staging& S,
                          const sbt_tracks& out, cudaStream_t stream);
cudaError_t launch_scan(const Inputs& in, const Staging& S, const sbt_tracks& out,
                        cudaStream_t stream);
cudaError_t launch_output(const DevConfig& C, const Inputs& in, const Staging& S,
                          const sbt_tracks& out, cudaStream_t stream);
cudaError_t launch_debug_sort_copy(const DevConfig& C, const Inputs& in, const Sorted& O,
                                   uint16_t* phi16, int32_t* perm, int32_t* module_offsets,
                                   cudaStream_t stream);
cudaError_t launch_debug_phi16(const float* x, const float* y, int32_t n, uint16_t* out,
                               cudaStream_t stream);
// Adds running[0] to track_offsets[0..n_events] and running[1] to
// hit_offsets[0..counts[0]] (when counts[2] is SBT_OK), and writes the new
// totals to running[2..3].
constexpr int kFixupBlocks = 304;
cudaError_t launch_offset_fixup(int32_t* track_offsets, int32_t n_events, int32_t* hit_offsets,
                                const int32_t* counts, int64_t* running, cudaStream_t stream);
int persistent_blocks_per_sm(const DevConfig& C, int threads);

// Adjoint (sbt_adjoint.cu).
struct AdjointWork {
    double* partial;   // [adjoint_partial_entries(M, blocks)]
    int blocks;
};
cudaError_t launch_adjoint(const DevConfig& C, const Inputs& in, const int32_t* hit_offsets,
                           const int32_t* track_hits, int32_t n_tracks, const double* align,
                           double* chi2_sum, double* grad, int32_t* skipped, const AdjointWork& W,
                           cudaStream_t stream);
int adjoint_blocks(int sm_count);
size_t adjoint_partial_entries(int M, int blocks);

// Handle accessors for translation units that cannot see the handle type.
const DevConfig& handle_device_config(const sbt_handle* h);
int handle_plain_threads(const sbt_handle* h);
void handle_set_error(sbt_handle* h, const std::string& msg);
void handle_set_launches(sbt_handle* h, int launches);
// Workspaces the handle outgrows are kept until sbt_destroy instead of freed
// (cudaFree synchronises the device); for handles whose work overlaps other
// streams' work, such as the serving slots.
void handle_defer_frees(sbt_handle* h);

}  // namespace sbt

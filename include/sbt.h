/*
 * sbt.h — C ABI of the GB300 Search-by-triplet VELO track reconstruction.
 *
 * The method is the one of Cámpora Pérez, Neufeld and Riscos Núñez, "Search by
 * triplet: An efficient local track reconstruction algorithm for parallel
 * architectures" (arXiv 2207.03936), section "Search by triplet":
 *   sort of each module's hits by phi, iterative triplet seeding and track
 *   following with flagged hits, the tracklet filter, and consolidation of
 *   the tracks (section "Results", sequence item "Data consolidation") with a
 *   least-squares straight-line fit.
 * The problem statement (section 1): find disjoint sets of hits compatible
 * with straight trajectories; every hit belongs to at most one track.
 *
 * Conventions for every call:
 *   - Pointers marked "device" must be CUDA device (or managed) memory of the
 *     current device; "host" pointers are ordinary host memory.  The caller
 *     owns all memory passed in; the library never frees it.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Compute entry points are asynchronous on that stream; only
 *     argument validation is synchronous.
 *   - Every call returns an sbt_status.  SBT_ERR_ARG: invalid arguments (no
 *     work enqueued).  SBT_ERR_CUDA: a CUDA call failed (sbt_last_error has
 *     the message).  Device-side per-event problems never fail the call: they
 *     are reported in sbt_tracks.event_status and sbt_tracks.counts.
 *   - A handle may be used from one host thread at a time, and its calls must
 *     not overlap on the GPU (they share the handle's workspace): use one
 *     handle per concurrent stream.
 *   - Hit index types: the event-local hit count is at most 16384; batch hit
 *     indices and offsets are int32.
 */
#ifndef SBT_H
#define SBT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SBT_OK = 0,
    SBT_ERR_ARG = 1,      /* invalid argument; nothing enqueued */
    SBT_ERR_CAPACITY = 2, /* output or per-event capacity exceeded (device-reported) */
    SBT_ERR_CUDA = 3,     /* CUDA runtime error; see sbt_last_error */
    SBT_ERR_TIMEOUT = 4,  /* a bounded wait expired (serving) */
    SBT_ERR_STATE = 5,    /* call not valid in the object's current state */
    SBT_EVENT_CUT = 6     /* per-event only: rejected by the global event cut, no tracks */
} sbt_status;

typedef struct sbt_handle sbt_handle;

/* Detector geometry (section 1, Fig. 2: planes of pixel modules along z).
 * Module ids are given in traversal order: the reconstruction visits module
 * 0, 1, 2, ... (section "Track seeding and track following": the direction of
 * traversal is configurable, here by the order of module_z).
 *
 * Module pairs (the paper's method works on module pairs, the two sides of
 * the VELO, and calls them modules; section "Search by triplet"): with
 * module_z2 given, module i is a pair of one-sided planes, hits with x >= 0
 * on the plane at module_z[i] and hits with x < 0 on the plane at
 * module_z2[i].  Every extrapolation to a module then targets the plane of
 * the hit it is compared with.  NULL module_z2: one plane per module.  The
 * alignment adjoint (sbt_fit_adjoint) takes single planes only and returns
 * SBT_ERR_ARG on a handle made with module_z2. */
typedef struct {
    int32_t n_modules;      /* 3 .. 64 */
    const float* module_z;  /* host [n_modules]: plane z of module id i, mm (finite); copied */
    float r_min, r_max;     /* active annulus, mm (informational) */
    const float* module_z2; /* host [n_modules] or NULL: plane z of the x < 0 side of pair i; copied */
} sbt_geometry;

/* Tunable constants.  The paper states that the thresholds are configurable
 * but prints no values; the defaults below were fixed once on synthetic truth. */
typedef struct {
    int32_t k_doublets;          /* candidates per middle hit in seeding (Fig. 3: four); default 4 */
    float max_scatter_seed;      /* seeding scatter cut dx^2+dy^2, mm^2; default 0.04 */
    float max_scatter_follow;    /* following scatter cut, mm^2; default 0.04 */
    float max_chi2_tracklet;     /* tracklet filter chi2 cut; default 20 */
    float hit_sigma;             /* hit resolution for chi2, mm; default 0.012 */
    int32_t max_hits_per_event;  /* events with more hits get SBT_ERR_CAPACITY; default and maximum 16384 */
    int32_t max_forming_tracks;  /* forming tracks alive per event: n_hits/12 + 64; a positive value lowers the bound */
    int32_t threads_per_block;   /* 64, 128 or 256; 0 = 128 (batched: autotuned value if any) */
    int32_t gec_max_hits;        /* global event cut (the paper's VELO sequence, first step): events
                                    with more hits are rejected unreconstructed (event status
                                    SBT_EVENT_CUT); 0 = no cut (default) */
    int32_t fp16_hits;           /* 1: the sorted hits keep x, y, z rounded to fp16 (nearest even)
                                    and a 16-bit index, 8 bytes per hit instead of 16 (the paper's
                                    fp16 AoS hit storage); every computation stays fp32, on the
                                    rounded coordinates, phi16 included.  0 = fp32 (default) */
} sbt_config;

/* Reconstructed tracks, CSR over events and tracks.  All arrays are device
 * memory allocated by the caller.  Sizing that can never overflow:
 * cap_hits >= n_hits and cap_tracks >= n_hits / 3 (hits are disjoint and a
 * track has at least 3 hits).
 *   track_offsets [n_events + 1]   tracks of event e: [track_offsets[e], track_offsets[e+1])
 *   hit_offsets   [cap_tracks + 1] hits of track t: track_hits[hit_offsets[t] .. hit_offsets[t+1])
 *   track_hits    [cap_hits]       batch hit indices (into x/y/z), module (traversal) order
 *   params        [cap_tracks * 4] x0, y0, tx, ty of x = x0 + tx z, y = y0 + ty z
 *   chi2          [cap_tracks]     sum of squared residuals / hit_sigma^2
 *   ndof          [cap_tracks]     2 * hits - 4
 *   event_status  [n_events]       SBT_OK, SBT_ERR_ARG (module id out of range, or
 *                                  hit range [event_offsets[e], event_offsets[e+1])
 *                                  not inside [0, n_hits)),
 *                                  SBT_ERR_CAPACITY (event above max_hits_per_event
 *                                  or a per-event buffer full) or SBT_EVENT_CUT (above
 *                                  gec_max_hits); failed and cut events have no tracks
 *   counts        [4]              required tracks, required track hits, SBT_OK or
 *                                  SBT_ERR_CAPACITY when cap_* was too small (then
 *                                  nothing beyond the capacities is written), number
 *                                  of failed events (cut events not included)
 * Tracks of an event are ordered by their smallest hit index. */
typedef struct {
    int32_t* track_offsets;
    int32_t* hit_offsets;
    int32_t* track_hits;
    float* params;
    float* chi2;
    int32_t* ndof;
    int32_t* event_status;
    int32_t* counts;
    int32_t cap_tracks;
    int32_t cap_hits;
} sbt_tracks;

/* Fills *out with the defaults. */
sbt_status sbt_default_config(sbt_config* out);

/* Creates a handle: copies the geometry and configuration (cfg NULL = defaults).
 * Allocates only small device state; workspaces grow on first use.
 * SBT_ERR_ARG (checked before any CUDA call; sbt_last_error(NULL) gives the
 * reason): NULL geometry, module_z or out; n_modules outside [3, 64];
 * a non-finite plane position; an invalid configuration value. */
sbt_status sbt_create(const sbt_geometry* geometry, const sbt_config* cfg, sbt_handle** out);

/* Waits for the handle's pending work and frees everything it owns. */
sbt_status sbt_destroy(sbt_handle* h);

/* Message of the last failed call on this handle ("" if none); NULL handle
 * gives the last creation error.  The string lives until the next call. */
const char* sbt_last_error(const sbt_handle* h);

/*
 * Reconstruct a batch of events, one thread block per event (the paper's
 * mapping of events to blocks and of hits and forming tracks to threads,
 * Table 1).  Inputs (device): x, y, z [n_hits] fp32 mm, module [n_hits]
 * traversal-order module id, event_offsets [n_events + 1] (event e owns hits
 * [event_offsets[e], event_offsets[e+1])), n_hits = event_offsets[n_events].
 * The library reads event_offsets only on the device: an event whose hit
 * range is not inside [0, n_hits) gets event status SBT_ERR_ARG and nothing
 * of it is read or written beyond its offsets; x, y, z and module are read
 * at [0, n_hits) only.
 * Outputs: *out (device arrays described at sbt_tracks).
 */
sbt_status sbt_reconstruct(sbt_handle* h, const float* x, const float* y, const float* z,
                           const int32_t* module, const int32_t* event_offsets, int32_t n_events,
                           int32_t n_hits, const sbt_tracks* out, void* stream);

/*
 * Same result as sbt_reconstruct, produced by one persistent launch whose
 * blocks take events from a device work queue (sizes alternating between the
 * largest and the smallest events not yet taken); the launch
 * sequence is captured once into a CUDA graph per distinct argument set and
 * replayed.  Block size comes from sbt_autotune when it has run.
 */
sbt_status sbt_reconstruct_batched(sbt_handle* h, const float* x, const float* y, const float* z,
                                   const int32_t* module, const int32_t* event_offsets,
                                   int32_t n_events, int32_t n_hits, const sbt_tracks* out,
                                   void* stream);

/*
 * End-to-end form for callers holding host memory: copies the inputs (host)
 * to the device, reconstructs with the batched kernels and copies the tracks
 * back into host arrays of the sbt_tracks layout (out_host pointers are host
 * memory; counts is host too).  The batch is processed in chunks of whole
 * events so that uploads, kernels and downloads of different chunks overlap.
 * Synchronous: returns when the host arrays are filled.  Pinned host memory
 * gives full copy bandwidth and true overlap.  event_offsets (host here) must
 * be non-decreasing from event_offsets[0] >= 0 to event_offsets[n_events] <=
 * n_hits, else SBT_ERR_ARG and nothing is enqueued.
 */
sbt_status sbt_reconstruct_host(sbt_handle* h, const float* x, const float* y, const float* z,
                                const int32_t* module, const int32_t* event_offsets,
                                int32_t n_events, int32_t n_hits, const sbt_tracks* out_host,
                                void* stream);

/*
 * Times the batched search kernel on the given events (device inputs as in
 * sbt_reconstruct) for each block size in {64, 128, 256} and, for each, the
 * occupancy limit of resident blocks per SM, three quarters and half of it,
 * and keeps the fastest shape in the handle for the batched and host entry
 * points.  Results do not depend on the choice.  Synchronous.  *chosen and
 * *chosen_blocks_per_sm (host, each may be NULL) receive the shape.
 */
sbt_status sbt_autotune(sbt_handle* h, const float* x, const float* y, const float* z,
                        const int32_t* module, const int32_t* event_offsets, int32_t n_events,
                        int32_t n_hits, int32_t* chosen, int32_t* chosen_blocks_per_sm, void* stream);

/* The handle's tuned launch shape (host outputs): block size and resident
 * blocks per SM of the persistent launch; 0 and 0 before sbt_autotune. */
sbt_status sbt_tuned_shape(const sbt_handle* h, int32_t* threads, int32_t* blocks_per_sm);

/* Sets the launch shape of the persistent launch as sbt_autotune would (for
 * example the shape tuned on another handle for the same workload): threads
 * 64, 128 or 256 (a nonzero threads_per_block of the configuration still
 * takes precedence), blocks_per_sm > 0 caps the resident blocks per SM
 * (0 = occupancy limit).  SBT_ERR_ARG otherwise. */
sbt_status sbt_set_launch_shape(sbt_handle* h, int32_t threads, int32_t blocks_per_sm);

/*
 * Differentiation of the consolidation fit with respect to per-module
 * alignment (the fit is the least-squares line of the paper's tracklet
 * filter and data consolidation, section "Search by triplet"; the alignment
 * objective itself has no counterpart in the paper).  For a hit h on module
 * m with plane centre c = (0, 0, module_z[m]) and align[6m .. 6m+5] =
 * (dx, dy, dz, a, b, g) (mm, rad), the aligned hit is
 *     h' = Rz(g) Ry(b) Rx(a) (h - c) + c + (dx, dy, dz).
 * Every track (hit lists fixed, e.g. the output of sbt_reconstruct) is refitted
 * by least squares on its aligned hits, in fp64; *chi2_sum = sum over tracks of
 * the squared residuals / hit_sigma^2, grad = d chi2_sum / d align [n_modules*6],
 * accumulated in fp64 in a fixed order (bitwise reproducible).
 * A track may have any number of hits, several on one module included.  A
 * track contributes nothing, and is counted in *skipped, when it has no
 * straight-line fit (fewer than two hits, or all its hits on one module), when
 * one of its hit indices is outside [0, n_hits) or the module id of one of its
 * hits outside [0, n_modules), or when its range of track_hits is not inside
 * [0, hit_offsets[n_tracks]).
 * Inputs (device): x, y, z, module [n_hits]; hit_offsets [n_tracks + 1];
 * track_hits [hit_offsets[n_tracks]]; align [n_modules * 6] fp64.  Outputs
 * (device): chi2_sum [1], grad [n_modules * 6] fp64 (NULL for the value
 * alone), skipped [1] int32 (may be NULL).
 */
sbt_status sbt_fit_adjoint(sbt_handle* h, const float* x, const float* y, const float* z,
                           const int32_t* module, int32_t n_hits, const int32_t* hit_offsets,
                           const int32_t* track_hits, int32_t n_tracks, const double* align,
                           double* chi2_sum, double* grad, int32_t* skipped, void* stream);

/*
 * Stage output of the phi sort (section "Sort by phi"), for checking it in
 * isolation.  Outputs (device): phi16 [n_hits] in sorted order within each
 * event, perm [n_hits] event-local input index of the hit at each sorted
 * position, module_offsets [n_events * (n_modules + 1)] event-local.
 */
sbt_status sbt_debug_sort(sbt_handle* h, const float* x, const float* y, const int32_t* module,
                          const int32_t* event_offsets, int32_t n_events, int32_t n_hits,
                          uint16_t* phi16, int32_t* perm, int32_t* module_offsets, void* stream);

/* phi16 of n points (device x, y in; device out): the mapping of [-pi, pi]
 * onto the unsigned 16-bit range used by the sort (section "Sort by phi"). */
sbt_status sbt_debug_phi16(const float* x, const float* y, int32_t n, uint16_t* out, void* stream);

/*
 * Measurement helper: runs the batched sequence `reps` times without a graph,
 * timing each kernel with CUDA events on `stream`, and writes the mean
 * milliseconds per launch to ms[5] (host): ordering kernel, sort kernel,
 * persistent search kernel, scan, output (the output kernel's canonical
 * order and CSR starts, then the fit kernel's hit lists and fits).
 * Synchronous.
 */
sbt_status sbt_profile_batched(sbt_handle* h, const float* x, const float* y, const float* z,
                               const int32_t* module, const int32_t* event_offsets,
                               int32_t n_events, int32_t n_hits, const sbt_tracks* out, int32_t reps,
                               float* ms, void* stream);

/*
 * Reconstruction for callers that cannot allocate device memory: for example
 * a trigger or serving process that reserves all its device memory at start-up
 * and forbids allocation afterwards (cudaMalloc and cudaFree synchronise the
 * device and can fail once the memory is taken), or a plug-in inside an
 * application that owns the device memory pool.  The paper has no
 * counterpart; it computes exactly what sbt_reconstruct computes.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.  Its
 *     workspace is a fixed array of about 48 MB inside the library's device
 *     image, held by every GPU that loads the library until the process exits.
 *   - At most 524288 hits and 4096 events per call; larger batches return
 *     SBT_ERR_ARG with a message from sbt_last_error (split the batch).
 *   - The first call on each device looks up the workspace address on that
 *     device; make that first call before any stream capture.  The address
 *     is kept until the process exits: do not call this entry point on a
 *     device after cudaDeviceReset on it (the reset unloads the workspace).
 *   - Every call on a device shares the one workspace: calls whose work
 *     overlaps on the GPU (other streams, other handles, other threads) race
 *     and corrupt each other's results; serialise them.
 * Arguments, layouts and results are those of sbt_reconstruct; sbt_create
 * allocates no device memory, so a handle can be made by such callers too.
 */
sbt_status sbt_reconstruct_noalloc(sbt_handle* h, const float* x, const float* y, const float* z,
                                   const int32_t* module, const int32_t* event_offsets,
                                   int32_t n_events, int32_t n_hits, const sbt_tracks* out,
                                   void* stream);

/* Number of kernels the last reconstruction call on h enqueued (launch
 * accounting for benchmarks); 0 before any call. */
int32_t sbt_last_launch_count(const sbt_handle* h);

/* ------------------------------------------------------------ serving --- */

/*
 * Continuous-batching request loop (no counterpart in the paper, which runs
 * fixed bunches of events per stream; Results, "n events per bunch").  A
 * background host thread admits submitted events into device slots while the
 * device-memory budget allows, launches every admitted group at once on one
 * of several streams (so newly admitted work overlaps work still running),
 * copies results back and marks requests done.  Latency is measured from
 * submission to completion on the host clock.
 */
typedef struct sbt_server sbt_server;

/* Result of one request (host memory owned by the server until the request
 * is released with sbt_server_release). */
typedef struct {
    int64_t request_id;
    int32_t status;          /* event status (sbt_status) */
    int32_t n_tracks;
    const int32_t* hit_offsets;  /* [n_tracks + 1], hit indices are event-local */
    const int32_t* track_hits;
    const float* params;     /* [n_tracks * 4] */
    const float* chi2;
    double latency_s;        /* submit (scheduled arrival for sbt_server_submit_schedule) -> done */
} sbt_result;

/* memory_budget_bytes bounds the device memory of in-flight events (inputs,
 * outputs, workspace); max_streams (1..16) bounds concurrent batches;
 * max_batch_events bounds one launch. */
sbt_status sbt_server_create(sbt_handle* h, int64_t memory_budget_bytes, int32_t max_streams,
                             int32_t max_batch_events, sbt_server** out);

/* Copies one event (host arrays of n hits) into the server's queue. */
sbt_status sbt_server_submit(sbt_server* s, int64_t request_id, const float* x, const float* y,
                             const float* z, const int32_t* module, int32_t n);

/* Open-loop load generator: a native thread submits event e of the host batch
 * (x, y, z, module [event_offsets[e] .. event_offsets[e+1])) arrival_s[e]
 * seconds after this call, with request id first_id + e; its latency counts
 * from that scheduled time.  The call copies the
 * batch into pinned host memory (uploads of consecutive events then need no
 * further copy) and returns at once; results arrive through
 * sbt_server_poll or sbt_server_drain.  event_offsets must be non-decreasing
 * from event_offsets[0] >= 0 (else SBT_ERR_ARG); the hit arrays hold at least
 * event_offsets[n_events] entries. */
sbt_status sbt_server_submit_schedule(sbt_server* s, const float* x, const float* y,
                                      const float* z, const int32_t* module,
                                      const int32_t* event_offsets, int32_t n_events,
                                      const double* arrival_s, int64_t first_id);

/* Up to max_results finished requests into results[] (host); *n_out receives
 * the count.  Waits at most timeout_s for the first one (0 = do not wait);
 * returns SBT_ERR_TIMEOUT when none finished in time. */
sbt_status sbt_server_poll(sbt_server* s, sbt_result* results, int32_t max_results,
                           int32_t* n_out, double timeout_s);

/* For consumers that only need completions: up to max_results finished
 * requests as (ids, status, latency_s) host arrays; their results are freed
 * at once.  Waits at most timeout_s for the first (0 = do not wait); returns
 * SBT_ERR_TIMEOUT when none finished in time. */
sbt_status sbt_server_drain(sbt_server* s, int64_t* ids, int32_t* status, double* latency_s,
                            int32_t max_results, int32_t* n_out, double timeout_s);

/* Frees the host memory of a polled result. */
sbt_status sbt_server_release(sbt_server* s, int64_t request_id);

/* stats (host, 14 doubles): completed, submitted, batches launched, mean
 * events per batch, peak device bytes in flight, failed batches, the largest
 * delay (seconds) of the latest open-loop schedule's generator behind that
 * schedule, the launcher thread's total time (seconds) spent enqueueing
 * batches (copies, kernels, downloads); then, summed over the batches that
 * finished, the milliseconds spent in uploads, in reconstruction kernels and
 * in downloads (CUDA events on each slot's stream) and from enqueueing to
 * harvesting (host clock), and the number of batches these sums cover; last,
 * the device and pinned host allocations the servers of this process made
 * since this one was created (slots and result blocks grow to the largest
 * batch they meet and then allocate nothing; buffers they outgrow are kept
 * until sbt_server_destroy, since freeing would stall the device). */
sbt_status sbt_server_stats(sbt_server* s, double* stats);

/* Makes the next launched batch fail on the host side (test hook for the
 * failure path: the batch's requests complete with SBT_ERR_CUDA status and
 * the loop continues). */
sbt_status sbt_server_inject_failure(sbt_server* s);

/* Stops the loop after finishing admitted work and frees the server. */
sbt_status sbt_server_destroy(sbt_server* s);

#ifdef __cplusplus
}
#endif

#endif /* SBT_H */

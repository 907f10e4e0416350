// Search-by-triplet reconstruction kernels for sm_103a.
//
// Events map to thread blocks, hits and forming tracks to threads (Table 1
// of the paper).  Two kernels per event:
//   1. k_sort: phi16 of every hit and its order by (module, phi16, input
//      index) from one counting pass into (module, coarse phi) buckets and a
//      sort inside each bucket, in shared memory (section "Sort by phi"); the
//      sorted hits are written as AoS records (x, y, z, input index: float4,
//      or fp16 x, y, z and a 16-bit index) + phi16;
//   2. k_search_*: for every module triplet (s, s+1, s+2): seeding over the unflagged
//      middle hits, then following of every forming track to module s+3 with
//      one-round claims on the hits, flags, and termination after two misses
//      (section "Track seeding and track following"); barriers separate the
//      stages as the paper's flagged-hits dependency requires;
//      then the tracklet filter (section "Tracklet filter") and staging of
//      every track's hit records with its smallest input hit index.
// A device-wide scan and the output kernel then build the CSR output (section
// "Results", data consolidation): canonical ordering of each event's tracks
// by smallest input hit index, their hit lists and the least-squares fit of
// every track, outside the latency-bound search blocks.
//
// Decision arithmetic is fp32 with every operation rounded as written
// (explicit _rn intrinsics, no contraction), so that the result is the
// exact track set of the plain definition.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "sbt_internal.h"

namespace sbt {

constexpr uint16_t kNone = 0xFFFFu;
constexpr uint16_t kDead = 0xFFFEu;

// ------------------------------------------------------------------ phi ---

// 2-argument arctangent: octant reduction and the degree-9 odd polynomial of
// the Hastings form (Abramowitz & Stegun 4.4.49), every operation rounded.
__device__ __forceinline__ float atan2_sbt(float y, float x)
{
    const float a1 = 0.9998660f, a3 = -0.3302995f, a5 = 0.1801410f;
    const float a7 = -0.0851330f, a9 = 0.0208351f;
    float ax = fabsf(x);
    float ay = fabsf(y);
    float mx = ax > ay ? ax : ay;
    float mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float t = __fdiv_rn(mn, mx);
    float t2 = __fmul_rn(t, t);
    float p = a9;
    p = __fadd_rn(__fmul_rn(p, t2), a7);
    p = __fadd_rn(__fmul_rn(p, t2), a5);
    p = __fadd_rn(__fmul_rn(p, t2), a3);
    p = __fadd_rn(__fmul_rn(p, t2), a1);
    p = __fmul_rn(p, t);
    if (ay > ax) p = __fsub_rn(1.5707963267948966f, p);
    if (x < 0.0f) p = __fsub_rn(3.14159265358979323846f, p);
    if (y < 0.0f) p = -p;
    return p;
}

// [-pi, pi] onto the unsigned 16-bit range, modulo 2^16.
__device__ __forceinline__ uint32_t phi16_of(float x, float y)
{
    float a = atan2_sbt(y, x);
    int q = __float2int_rn(__fmul_rn(a, 10430.378350470453f));
    return (uint32_t)q & 0xFFFFu;
}

__device__ __forceinline__ int phi_dist(uint32_t u, uint32_t v)
{
    int d1 = (int)((u - v) & 0xFFFFu);
    int d2 = (int)((v - u) & 0xFFFFu);
    return d1 < d2 ? d1 : d2;
}

// First position in phi[0, n) with phi >= v.
__device__ __forceinline__ int lower_bound16(const uint16_t* phi, int n, uint32_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((uint32_t)phi[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Straight-line extrapolation of (a, c) to the plane z = zt.
__device__ __forceinline__ void extrapolate(float4 A, float4 Cc, float zt, float& xp, float& yp)
{
    float dz = __fsub_rn(Cc.z, A.z);
    float tz = __fdiv_rn(__fsub_rn(zt, Cc.z), dz);
    xp = __fadd_rn(Cc.x, __fmul_rn(__fsub_rn(Cc.x, A.x), tz));
    yp = __fadd_rn(Cc.y, __fmul_rn(__fsub_rn(Cc.y, A.y), tz));
}

__device__ __forceinline__ float scatter_of(float4 B, float xp, float yp)
{
    float dx = __fsub_rn(B.x, xp);
    float dy = __fsub_rn(B.y, yp);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// Least-squares straight line through n hits (get(i) -> float3 in hit
// order): params (x0, y0, tx, ty) at z = 0 and chi2 = residual sum / sigma^2.
template <class Get>
__device__ __forceinline__ void fit_line(int n, Get get, float sigma, float* params, float* chi2)
{
    float nf = (float)n;
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int i = 0; i < n; i++) {
        float3 h = get(i);
        sx = __fadd_rn(sx, h.x);
        sy = __fadd_rn(sy, h.y);
        sz = __fadd_rn(sz, h.z);
    }
    float xm = __fdiv_rn(sx, nf), ym = __fdiv_rn(sy, nf), zm = __fdiv_rn(sz, nf);
    float szz = 0.0f, szx = 0.0f, szy = 0.0f;
    for (int i = 0; i < n; i++) {
        float3 h = get(i);
        float dz = __fsub_rn(h.z, zm);
        szz = __fadd_rn(szz, __fmul_rn(dz, dz));
        szx = __fadd_rn(szx, __fmul_rn(dz, __fsub_rn(h.x, xm)));
        szy = __fadd_rn(szy, __fmul_rn(dz, __fsub_rn(h.y, ym)));
    }
    float tx = __fdiv_rn(szx, szz);
    float ty = __fdiv_rn(szy, szz);
    float s = 0.0f;
    for (int i = 0; i < n; i++) {
        float3 h = get(i);
        float dz = __fsub_rn(h.z, zm);
        float rx = __fsub_rn(__fsub_rn(h.x, xm), __fmul_rn(tx, dz));
        float ry = __fsub_rn(__fsub_rn(h.y, ym), __fmul_rn(ty, dz));
        s = __fadd_rn(s, __fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)));
    }
    if (params) {
        params[0] = __fsub_rn(xm, __fmul_rn(tx, zm));
        params[1] = __fsub_rn(ym, __fmul_rn(ty, zm));
        params[2] = tx;
        params[3] = ty;
    }
    *chi2 = __fdiv_rn(s, __fmul_rn(sigma, sigma));
}

// ------------------------------------------------------- shared layout ---

enum Misc {
    kErr = 0, kCnt0 = 1, kCnt1 = 2, kNFin = 3, kNTl = 4, kEvent = 5, kList = 6, kNOuter = 7,
    kNew = 8, kWork = 9, kCMask = 10, kMiscN = 12
};

// Per-block shared memory of the search: flag bits, module offsets, counters,
// each sized to what the configuration needs.  Everything sized by the event
// lives in global scratch (L1-resident): shared memory and L1 share one array
// per SM, so every byte a block holds here comes out of the L1 of 32 resident
// events (about n / 8 + 4 M bytes a block).
struct Smem {
    uint32_t* flag;     // one bit per sorted position
    int* modoff;
    int* misc;
    int* wsum;          // [33]
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

struct Plan {
    size_t flag, modoff, misc, wsum, total;
};

__host__ __device__ inline Plan make_plan(int nmax, int threads, int M)
{
    Plan p;
    size_t o = 0;
    p.flag = o;     o = align16(o + 4 * (((size_t)nmax + 31) / 32));
    p.modoff = o;   o = align16(o + 4 * ((size_t)M + 1));
    p.misc = o;     o = align16(o + 4 * kMiscN);
    p.wsum = o;     o = align16(o + 4 * ((size_t)threads / 32 + 1));
    p.total = o;
    return p;
}

size_t smem_bytes(int nmax, int threads, int M) { return make_plan(nmax, threads, M).total; }

__device__ inline Smem carve(unsigned char* raw, int nmax, int threads, int M)
{
    Plan p = make_plan(nmax, threads, M);
    Smem S;
    S.flag = (uint32_t*)(raw + p.flag);
    S.modoff = (int*)(raw + p.modoff);
    S.misc = (int*)(raw + p.misc);
    S.wsum = (int*)(raw + p.wsum);
    return S;
}

__device__ __forceinline__ bool flagged(const Smem& S, int p) { return (S.flag[p >> 5] >> (p & 31)) & 1u; }
__device__ __forceinline__ void set_flag(const Smem& S, int p) { atomicOr(&S.flag[p >> 5], 1u << (p & 31)); }

// Storage of the sorted hits.  HitsF32: float4 (x, y, z, input index as
// int bits), 16 bytes.  HitsF16: x, y, z rounded to fp16 (nearest even) and
// the input index in 16 bits, 8 bytes (the paper's fp16 AoS storage of hit
// coordinates); every computation still runs in fp32, on the rounded values.
struct HitsF32 {
    using T = float4;
    __device__ __forceinline__ static float round(float v) { return v; }
    __device__ __forceinline__ static float4 load(const T* p, int i) { return p[i]; }
    __device__ __forceinline__ static void store(T* p, int64_t i, float4 c) { p[i] = c; }
};

struct HitsF16 {
    using T = ushort4;
    __device__ __forceinline__ static float round(float v) { return __half2float(__float2half_rn(v)); }
    __device__ __forceinline__ static float4 load(const T* p, int i)
    {
        const ushort4 u = p[i];
        return make_float4(__half2float(__ushort_as_half(u.x)), __half2float(__ushort_as_half(u.y)),
                           __half2float(__ushort_as_half(u.z)), __int_as_float((int)u.w));
    }
    __device__ __forceinline__ static void store(T* p, int64_t i, float4 c)
    {
        p[i] = make_ushort4(__half_as_ushort(__float2half_rn(c.x)), __half_as_ushort(__float2half_rn(c.y)),
                            __half_as_ushort(__float2half_rn(c.z)), (unsigned short)__float_as_int(c.w));
    }
};

// Sorted hits of one event, hit p as float4 (x, y, z, input index bits).
template <class HS>
struct HitArr {
    const typename HS::T* p;
    __device__ __forceinline__ float4 operator[](int i) const { return HS::load(p, i); }
};

// What one event's search sees: its sorted hits (read-only) and its scratch.
template <class HS>
struct Region {
    HitArr<HS> coords;
    const uint16_t* phi;
    uint32_t* list;
    uint16_t* prev;
    unsigned long long* claim;  // the search's claim of sorted position p is claim[p & cmask]
    unsigned cmask;
    unsigned long long* tracklets;
    uint32_t* tl_q;
    int lcap;
    uint32_t* finals;
    FTrack* ft;         // buffer b starts at ft + b * fstride
    int fstride;
};

template <class HS>
__device__ inline Region<HS> region_of(const Sorted& O, int off, const Work& W, int64_t hb, int64_t r,
                                      int cap)
{
    Region<HS> R;
    R.coords = HitArr<HS>{(const typename HS::T*)O.coords + off};
    R.phi = O.phi + off;
    R.list = W.list + hb;
    R.prev = W.prev + hb;
    R.claim = W.claim + hb;
    R.cmask = ~0u;
    R.tracklets = W.tracklets + hb + r;
    R.tl_q = W.tl_q + hb + r;
    R.lcap = cap + 1;
    R.finals = W.finals + hb / 3 + r;
    R.ft = W.ft + forming_base(hb, r);
    R.fstride = cap / 12 + 72;
    return R;
}

// Exclusive block scan of one int per thread; returns the prefix, *total the
// sum.  wsum needs NT / 32 + 1 entries.
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int* wsum, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NT / 32) wsum[lane] = wi - w;
        if (lane == NT / 32 - 1) wsum[NT / 32] = wi;
    }
    __syncthreads();
    int res = wsum[warp] + incl - v;
    *total = wsum[NT / 32];
    __syncthreads();
    return res;
}

// ------------------------------------------------------------- sorting ---

constexpr int kSortThreads = 1024;
constexpr int kSortBuckets = 4096;  // (module, top six bits of phi16)
constexpr int kShortBucket = 32;    // buckets up to this size are sorted by one thread

// Shared memory of the sort kernel: the bucketed entries phi16 << 14 | input
// index (4 B per hit), phi16 by input order (2 B per hit; later the list of
// long buckets) and the bucket counters.
__host__ __device__ inline size_t sort_layout(int nmax, size_t* off_phi, size_t* off_cnt)
{
    size_t o = align16(4 * (size_t)nmax);
    *off_phi = o;  o = align16(o + 2 * (size_t)nmax);
    *off_cnt = o;  o = align16(o + 4 * (size_t)kSortBuckets);
    return o;
}

size_t sort_smem_bytes(int nmax)
{
    size_t a, b;
    return sort_layout(nmax, &a, &b);
}

// Ascending sort of a[0, s) by one warp, in place: a bitonic network in the
// form whose comparators all put the smaller key first (a mirrored merge
// step, then half-cleaners), so positions past s behave as +infinity and are
// never touched.
__device__ void warp_bitonic(uint32_t* a, int s)
{
    const int lane = threadIdx.x & 31;
    int P = 1;
    while (P < s) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) {
        const int h = k >> 1;
        for (int i = lane; i < P / 2; i += 32) {
            const int lo = (i / h) * k + (i % h), hi = (i / h) * k + k - 1 - (i % h);
            if (hi < s) {
                const uint32_t u = a[lo], v = a[hi];
                if (u > v) {
                    a[lo] = v;
                    a[hi] = u;
                }
            }
        }
        __syncwarp();
        for (int j = k >> 2; j >= 1; j >>= 1) {
            for (int i = lane; i < P / 2; i += 32) {
                const int lo = (i / j) * 2 * j + (i % j), hi = lo + j;
                if (hi < s) {
                    const uint32_t u = a[lo], v = a[hi];
                    if (u > v) {
                        a[lo] = v;
                        a[hi] = u;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// One block per event: phi16, stable sort by (module, phi16) in shared
// memory, gather of the sorted hits.  A counting pass puts every hit into its
// (module, top six bits of phi16) bucket; each bucket is then sorted by
// phi16 << 14 | input index, a unique key, so the order is the one of a
// stable sort by (module, phi16).  Status SBT_ERR_ARG for a module id out of
// range or a hit range [offsets[e], offsets[e+1]) that is not inside
// [0, n_hits) (no later kernel reads or writes anything of such an event),
// SBT_ERR_CAPACITY above the configured hit limit.
template <class HS>
__global__ void __launch_bounds__(kSortThreads, 2) k_sort(DevConfig C, Inputs in, Sorted O)
{
    constexpr int NT = kSortThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t ophi, ocnt;
    sort_layout(C.nmax, &ophi, &ocnt);
    uint32_t* ent = (uint32_t*)smem_raw;
    uint16_t* phi = (uint16_t*)(smem_raw + ophi);
    int* cnt = (int*)(smem_raw + ocnt);
    __shared__ int wsum[40];
    __shared__ int err, nlong;
    const int tid = threadIdx.x;
    const int e = blockIdx.x;
    const int off = in.offsets[e];
    const int64_t n64 = (int64_t)in.offsets[e + 1] - off;
    const bool range_bad = off < 0 || n64 < 0 || off + n64 > in.n_hits;
    if (range_bad || n64 > C.nmax || (C.gec > 0 && n64 > C.gec)) {
        if (tid == 0)
            O.status[e] = range_bad ? SBT_ERR_ARG : (C.gec > 0 && n64 > C.gec) ? SBT_EVENT_CUT : SBT_ERR_CAPACITY;
        return;
    }
    const int n = (int)n64;
    for (int b = tid; b < kSortBuckets; b += NT) cnt[b] = 0;
    if (tid == 0) {
        err = 0;
        nlong = 0;
    }
    __syncthreads();
    // phi16 and bucket counts, two hits per thread per round (loads first)
    for (int i0 = tid; i0 < n; i0 += 2 * NT) {
        float xs[2], ys[2];
        int ms[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int i = i0 + u * NT;
            const bool v = i < n;
            xs[u] = v ? in.x[off + i] : 1.0f;
            ys[u] = v ? in.y[off + i] : 0.0f;
            ms[u] = v ? in.module[off + i] : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int i = i0 + u * NT;
            if (i >= n) continue;
            int m = ms[u];
            if (m < 0 || m >= C.M) {
                err = SBT_ERR_ARG;
                m = 0;
            }
            const uint32_t ph = phi16_of(HS::round(xs[u]), HS::round(ys[u]));
            phi[i] = (uint16_t)ph;
            atomicAdd(&cnt[(m << 6) | (int)(ph >> 10)], 1);
        }
    }
    __syncthreads();
    if (err) {
        if (tid == 0) O.status[e] = SBT_ERR_ARG;
        return;
    }
    // bucket starts: exclusive scan, kSortBuckets / NT consecutive buckets per thread
    {
        constexpr int per = kSortBuckets / NT;
        int v[per];
        int s = 0;
#pragma unroll
        for (int k = 0; k < per; k++) {
            v[k] = cnt[tid * per + k];
            s += v[k];
        }
        int total;
        int st = block_exclusive_scan<NT>(s, wsum, &total);
#pragma unroll
        for (int k = 0; k < per; k++) {
            cnt[tid * per + k] = st;
            st += v[k];
        }
    }
    __syncthreads();
    // scatter into the buckets (order inside a bucket arbitrary); afterwards
    // cnt[b] is the end of bucket b
    for (int i = tid; i < n; i += NT) {
        const uint32_t ph = phi[i];
        const int m = in.module[off + i];
        const int p = atomicAdd(&cnt[(m << 6) | (int)(ph >> 10)], 1);
        ent[p] = (ph << 14) | (uint32_t)i;
    }
    __syncthreads();
    // short buckets: insertion sort by one thread; long ones listed for a warp
    uint16_t* longb = phi;  // phi16 by input order is no longer needed
    for (int b = tid; b < kSortBuckets; b += NT) {
        const int lo = b > 0 ? cnt[b - 1] : 0, hi = cnt[b];
        if (hi - lo > kShortBucket) {
            longb[atomicAdd(&nlong, 1)] = (uint16_t)b;
            continue;
        }
        for (int k = lo + 1; k < hi; k++) {
            const uint32_t v = ent[k];
            int j = k - 1;
            while (j >= lo && ent[j] > v) {
                ent[j + 1] = ent[j];
                j--;
            }
            ent[j + 1] = v;
        }
    }
    __syncthreads();
    for (int q = tid >> 5; q < nlong; q += NT / 32) {
        const int b = longb[q];
        const int lo = b > 0 ? cnt[b - 1] : 0;
        warp_bitonic(ent + lo, cnt[b] - lo);
    }
    for (int m = tid; m <= C.M; m += NT)
        O.modoff[(int64_t)e * (C.M + 1) + m] = m == 0 ? 0 : (m < C.M ? cnt[(m << 6) - 1] : n);
    __syncthreads();
    // phi16 by sorted position, and the sorted position of every input hit
    // (in the space of phi16 by input order, free now)
    uint16_t* rank = phi;
    for (int p = tid; p < n; p += NT) {
        const uint32_t en = ent[p];
        O.phi[off + p] = (uint16_t)(en >> 14);
        rank[en & 0x3FFFu] = (uint16_t)p;
    }
    __syncthreads();
    // the hits in input order (coalesced loads), each stored at its sorted
    // position; two per thread per round
    for (int i0 = tid; i0 < n; i0 += 2 * NT) {
        float4 c[2];
        int q[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int i = i0 + u * NT;
            if (i < n) {
                c[u] = make_float4(in.x[off + i], in.y[off + i], in.z[off + i], __int_as_float(i));
                q[u] = rank[i];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; u++)
            if (i0 + u * NT < n) HS::store((typename HS::T*)O.coords, (int64_t)off + q[u], c[u]);
    }
    if (tid == 0) O.status[e] = SBT_OK;
}

// ------------------------------------------------------ seeding, following ---

// phi16 of a window centre.  Only the window bounds use it, and they carry a
// margin of 16 units, so a fast division is enough here.
__device__ __forceinline__ uint32_t phi16_window(float x, float y)
{
    const float a1 = 0.9998660f, a3 = -0.3302995f, a5 = 0.1801410f;
    const float a7 = -0.0851330f, a9 = 0.0208351f;
    float ax = fabsf(x), ay = fabsf(y);
    float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    float t2 = t * t;
    float p = ((((a9 * t2 + a7) * t2 + a5) * t2 + a3) * t2 + a1) * t;
    if (ay > ax) p = 1.5707963f - p;
    if (x < 0.0f) p = 3.1415927f - p;
    if (y < 0.0f) p = -p;
    return (uint32_t)__float2int_rn(p * 10430.378f) & 0xFFFFu;
}

// Phi window of a prediction (xp, yp) for a scatter cut: hits outside it
// cannot pass the cut.  A hit within d = sqrt(cut) of the prediction differs
// from it in angle by at most asin(d / r) <= d / sqrt(r^2 - d^2); the
// half-width adds 1/16 of that plus 16 phi16 units for the rounding and
// arctangent error of both phi values and for the approximate arithmetic of
// the bound itself.  Predictions near the axis (r <= 2 d) get no window (the
// whole module is scanned).
__device__ __forceinline__ bool window_of(float xp, float yp, float cut, float sqrt_cut, uint32_t& lo,
                                          uint32_t& width)
{
    const float rp2 = xp * xp + yp * yp;
    if (rp2 < 1.0e30f && rp2 > 4.0f * cut) {
        const float wf = sqrt_cut * rsqrtf(rp2 - cut) * (10430.378f * 1.0625f);
        if (wf < 16000.0f) {
            const uint32_t W = (uint32_t)wf + 16u;
            lo = (phi16_window(xp, yp) - W) & 0xFFFFu;
            width = 2u * W;
            return true;
        }
    }
    lo = 0;
    width = 0xFFFFu;
    return false;
}

// Geometry of the module an extrapolation targets.  PlaneGeo: one plane at
// module_z[m].  PairGeo: a module pair of one-sided planes (the paper's
// method works on module pairs, the two sides of the VELO), hits with
// x >= 0 on the plane at module_z[m] and hits with x < 0 on the plane at
// module_z2[m]; a search visits each plane's hits with the prediction at
// that plane's z, so every candidate is compared at its own plane.
struct PlaneGeo {
    static constexpr int kPlanes = 1;
    __device__ __forceinline__ static float z(const DevConfig& C, int m, int) { return C.module_z[m]; }
    __device__ __forceinline__ static bool on(int, float) { return true; }
};

struct PairGeo {
    static constexpr int kPlanes = 2;
    __device__ __forceinline__ static float z(const DevConfig& C, int m, int p)
    {
        return p ? C.module_z2[m] : C.module_z[m];
    }
    __device__ __forceinline__ static bool on(int p, float x) { return (x < 0.0f) == (p != 0); }
};

// Visits the unflagged hits of plane `plane` of module [b0, b0 + nb) inside
// the window that starts at sorted index lo_idx (all hits when not
// windowed); the scatter of every visited hit is computed exactly (rounded
// operations) and `better(sc, b)` orders candidates under the cut.
template <class G, class Better, class Take, class HS>
__device__ __forceinline__ void scan_from(const Smem& S, const Region<HS>& R, int b0, int nb, float xp,
                                          float yp, float cut, bool windowed, int lo_idx,
                                          uint32_t lo, uint32_t width, int plane, Better better,
                                          Take take)
{
    for (int k = 0; k < nb; k++) {
        int e = lo_idx + k;
        if (e >= nb) e -= nb;
        const int b = b0 + e;
        // both loads issued together (b is inside the module either way)
        const uint32_t ph = R.phi[b];
        const float4 c = R.coords[b];
        if (windowed && ((ph - lo) & 0xFFFFu) > width) break;
        if (flagged(S, b)) continue;
        if (!G::on(plane, c.x)) continue;
        const float sc = scatter_of(c, xp, yp);
        if (sc < cut && better(sc, b)) take(sc, b);
    }
}

template <class G, class Better, class Take, class HS>
__device__ __forceinline__ void scan_window(const Smem& S, const Region<HS>& R, int b0, int nb, float xp,
                                            float yp, float cut, float sqrt_cut, int plane,
                                            Better better, Take take)
{
    if (nb <= 0) return;
    uint32_t lo, width;
    const bool windowed = window_of(xp, yp, cut, sqrt_cut, lo, width);
    const int lo_idx = windowed ? lower_bound16(R.phi + b0, nb, lo) : 0;
    scan_from<G>(S, R, b0, nb, xp, yp, cut, windowed, lo_idx, lo, width, plane, better, take);
}

// First index in keys[0, n) whose upper 16 bits are >= v.
__device__ __forceinline__ int lower_bound_hi16(const uint32_t* keys, int n, uint32_t v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((keys[mid] >> 16) < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

constexpr int kSeedBatch = 1;

// Candidates a[0, na) of one middle hit, processed together: extrapolations
// to each plane of module i, then the binary searches of their windows in
// lockstep (independent loads in flight), then the window scans.  Keeps the
// best (scatter, a, b).
template <class G, class HS>
__device__ __forceinline__ void seed_candidates(const DevConfig& C, const Smem& S, const Region<HS>& R,
                                                int i, int i0, int ni, float4 Cc, float sqrt_cut,
                                                const int* a, int na, bool& have, float& best_sc,
                                                int& best_a, int& best_b)
{
    for (int plane = 0; plane < G::kPlanes; plane++) {
        const float zi = G::z(C, i, plane);
        float xp[kSeedBatch], yp[kSeedBatch];
        uint32_t lo[kSeedBatch], width[kSeedBatch];
        int L[kSeedBatch], H[kSeedBatch];
        bool win[kSeedBatch];
#pragma unroll
        for (int u = 0; u < kSeedBatch; u++) {
            L[u] = 0;
            H[u] = 0;
            win[u] = false;
            if (u < na) {
                extrapolate(R.coords[a[u]], Cc, zi, xp[u], yp[u]);
                win[u] = window_of(xp[u], yp[u], C.S_seed, sqrt_cut, lo[u], width[u]);
                H[u] = win[u] ? ni : 0;
            }
        }
        const uint16_t* phi = R.phi + i0;
        for (int it = 0; it < 17; it++) {
            bool active = false;
#pragma unroll
            for (int u = 0; u < kSeedBatch; u++) active |= L[u] < H[u];
            if (!active) break;
#pragma unroll
            for (int u = 0; u < kSeedBatch; u++) {
                if (L[u] < H[u]) {
                    const int mid = (L[u] + H[u]) >> 1;
                    if ((uint32_t)phi[mid] < lo[u])
                        L[u] = mid + 1;
                    else
                        H[u] = mid;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kSeedBatch; u++) {
            if (u >= na) continue;
            const int au = a[u];
            scan_from<G>(
                S, R, i0, ni, xp[u], yp[u], C.S_seed, win[u], win[u] ? L[u] : 0, lo[u], width[u], plane,
                [&](float sc, int b) {
                    return !have || sc < best_sc ||
                           (sc == best_sc && (au < best_a || (au == best_a && b < best_b)));
                },
                [&](float sc, int b) {
                    have = true;
                    best_sc = sc;
                    best_a = au;
                    best_b = b;
                });
        }
    }
}

// Seeding for middle hit c on module s+1: the unflagged hits of module s
// nearest to c in phi (all hits at the K-th smallest distance included),
// each extrapolated through c to module s+2, where the unflagged hit of
// least scatter under the cut is sought; the kept triplet minimises
// (scatter, position of a, position of b).  `outer` lists the unflagged hits
// of module s in sorted order as (phi16 << 16 | position), `nu` of them, so
// the nearest-first walk visits no flagged hit.
template <class G, class HS>
__device__ bool seed_for(const DevConfig& C, const Smem& S, const Region<HS>& R, int s, int c,
                         const uint32_t* outer, int nu, float sqrt_cut, int& oa, int& ob)
{
    const int i0 = S.modoff[s + 2], ni = S.modoff[s + 3] - i0;
    if (nu <= 0 || ni <= 0) return false;
    const uint32_t phc = R.phi[c];
    const float4 Cc = R.coords[c];
    const int j = lower_bound_hi16(outer, nu, phc);
    int up = j, dn = j - 1;
    int found = 0, dK = INT_MAX;
    bool have = false;
    float best_sc = 0.0f;
    int best_a = 0, best_b = 0;
    int cand[kSeedBatch];
    int nc = 0;
    for (int visited = 0; visited < nu; visited++) {
        const int iu = up >= nu ? up - nu : up;
        const int id = dn < 0 ? dn + nu : dn;
        const uint32_t ku = outer[iu], kd = outer[id];
        const int du = phi_dist(ku >> 16, phc);
        const int dd = phi_dist(kd >> 16, phc);
        int a, d;
        if (du < dd || (du == dd && iu <= id)) {
            a = (int)(ku & 0xFFFFu);
            d = du;
            up++;
        } else {
            a = (int)(kd & 0xFFFFu);
            d = dd;
            dn--;
        }
        if (found >= C.K && d > dK) break;
        found++;
        if (found == C.K) dK = d;
        cand[nc++] = a;
        if (nc == kSeedBatch) {
            seed_candidates<G>(C, S, R, s + 2, i0, ni, Cc, sqrt_cut, cand, nc, have, best_sc, best_a, best_b);
            nc = 0;
        }
    }
    if (nc > 0)
        seed_candidates<G>(C, S, R, s + 2, i0, ni, Cc, sqrt_cut, cand, nc, have, best_sc, best_a, best_b);
    if (have) {
        oa = best_a;
        ob = best_b;
    }
    return have;
}

// Following: best unflagged hit on module t for the track's last two hits.
template <class G, class HS>
__device__ bool follow_best(const DevConfig& C, const Smem& S, const Region<HS>& R, int t, int h1, int h2,
                            float sqrt_cut, int& cand, float& csc)
{
    const int b0 = S.modoff[t], nb = S.modoff[t + 1] - b0;
    const float4 A = R.coords[h1], Cc = R.coords[h2];
    bool have = false;
    float best = 0.0f;
    int bb = 0;
    for (int plane = 0; plane < G::kPlanes; plane++) {
        float xp, yp;
        extrapolate(A, Cc, G::z(C, t, plane), xp, yp);
        scan_window<G>(
            S, R, b0, nb, xp, yp, C.S_follow, sqrt_cut, plane,
            [&](float sc, int b) { return !have || sc < best || (sc == best && b < bb); },
            [&](float sc, int b) {
                have = true;
                best = sc;
                bb = b;
            });
    }
    cand = bb;
    csc = best;
    return have;
}

__device__ __forceinline__ unsigned long long claim_key(unsigned long long tag, float score, int key)
{
    return tag | ((unsigned long long)__float_as_uint(score) << 16) | (unsigned long long)key;
}

template <class HS>
__device__ __forceinline__ void add_final(const Smem& S, const Region<HS>& R, int last, int nh)
{
    int k = atomicAdd(&S.misc[kNFin], 1);
    R.finals[k] = (uint32_t)last | ((uint32_t)nh << 16);
}

template <class HS>
__device__ __forceinline__ void add_tracklet(const Smem& S, const Region<HS>& R, int h0, int h1, int h2,
                                             int key)
{
    int k = atomicAdd(&S.misc[kNTl], 1);
    if (k < R.lcap)
        R.tracklets[k] = (unsigned long long)h0 | ((unsigned long long)h1 << 16) |
                         ((unsigned long long)h2 << 32) | ((unsigned long long)key << 48);
    else
        S.misc[kErr] = SBT_ERR_CAPACITY;
}

__device__ __forceinline__ FTrack make_track(int h0, int h1, int h2, int key, int nh, int sk)
{
    FTrack T;
    T.h0 = (uint16_t)h0;
    T.h1 = (uint16_t)h1;
    T.h2 = (uint16_t)h2;
    T.key = (uint16_t)key;
    T.nh = (uint8_t)nh;
    T.sk = (uint8_t)sk;
    T.cand = kNone;
    T.sc = 0.0f;
    return T;
}

// Following search of one forming track to module t and its claims: the new
// hit, and for a 3-hit track also its three hits.  A 3-hit track with a
// flagged hit cannot extend any more and is marked dead.
template <class G, class HS>
__device__ __forceinline__ void follow_and_claim(const DevConfig& C, const Smem& S, const Region<HS>& R,
                                                 int t, unsigned long long tag, float sqrt_cut,
                                                 FTrack& T)
{
    if (T.nh == 3 && (flagged(S, T.h0) || flagged(S, T.h1) || flagged(S, T.h2))) {
        T.cand = kDead;
        return;
    }
    int b;
    float sc;
    if (follow_best<G>(C, S, R, t, T.h1, T.h2, sqrt_cut, b, sc)) {
        T.cand = (uint16_t)b;
        T.sc = sc;
        const unsigned long long k = claim_key(tag, sc, T.key);
        atomicMin(&R.claim[b & R.cmask], k);
        if (T.nh == 3) {
            atomicMin(&R.claim[T.h0 & R.cmask], k);
            atomicMin(&R.claim[T.h1 & R.cmask], k);
            atomicMin(&R.claim[T.h2 & R.cmask], k);
        }
    } else {
        T.cand = kNone;
        T.sc = 0.0f;
    }
}

// Iterative seeding and following.  Returns false (uniformly) on overflow.
// Per module triplet (s, s+1, s+2) three phases separated by barriers:
//   P0  work lists: unflagged middle hits of s+1, unflagged hits of s in order;
//   P1  seeding and following of the forming tracks to t = s+3 with claims
//       (every new seed searches its own continuation at once); threads take
//       work items from a shared counter, seeds (the costlier items) first,
//       so the step's barrier waits on a balanced tail;
//   P2  resolution of the claims, flags, termination.
// Claims carry a tag (64 - t) << 48 above (scatter bits, track key), so a
// claim of an earlier step always compares larger than one of the current
// step and the claim words need no reset between steps.
template <int NT, class G, class HS>
__device__ bool search_stage(const DevConfig& C, const Region<HS>& R, const Smem& S, int n)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const int M = C.M;
    int* misc = S.misc;
    const int cap = C.fcap > 0 ? min(C.fcap, forming_capacity(n)) : forming_capacity(n);
    const float sq_seed = sqrtf(C.S_seed), sq_follow = sqrtf(C.S_follow);
    uint32_t* list = R.list;
    if (tid == 0) {
        misc[kCnt0] = 0;
        misc[kCnt1] = 0;
        misc[kNFin] = 0;
        misc[kNTl] = 0;
        misc[kErr] = 0;
        misc[kList] = 0;
        misc[kNew] = 0;
    }
    __syncthreads();
    int cur = 0;
    for (int s = 0; s + 2 <= M - 1; ++s) {
        const int nxt = cur ^ 1;
        FTrack* Fc = R.ft + cur * R.fstride;
        FTrack* Fn = R.ft + nxt * R.fstride;
        // P0
        if (tid == 0) {
            misc[kCnt0 + nxt] = 0;
            misc[kNew] = 0;
            misc[kWork] = 0;
        }
        if (s + 3 <= M - 1)  // claim words of the target module start empty
            for (int p = S.modoff[s + 3] + tid; p < S.modoff[s + 4]; p += NT) R.claim[p & R.cmask] = ~0ull;
        const int c0 = S.modoff[s + 1], c1 = S.modoff[s + 2];
        uint32_t* outer = list + (c1 - c0);
        for (int base = c0 + (tid & ~31); base < c1; base += NT) {
            const int c = base + lane;
            const bool ok = c < c1 && !flagged(S, c);
            const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
            int pos = 0;
            if (lane == 0 && m) pos = atomicAdd(&misc[kList], __popc(m));
            pos = __shfl_sync(0xFFFFFFFFu, pos, 0);
            if (ok) list[pos + __popc(m & ((1u << lane) - 1u))] = (uint32_t)c;
        }
        if ((tid >> 5) == NT / 32 - 1) {
            const int o0 = S.modoff[s], o1 = S.modoff[s + 1];
            int nu = 0;
            for (int base = o0; base < o1; base += 32) {
                const int a = base + lane;
                const bool ok = a < o1 && !flagged(S, a);
                const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);
                if (ok)
                    outer[nu + __popc(m & ((1u << lane) - 1u))] =
                        ((uint32_t)R.phi[a] << 16) | (uint32_t)a;
                nu += __popc(m);
            }
            if (lane == 0) misc[kNOuter] = nu;
        }
        __syncthreads();
        const int nl = misc[kList];
        const int nu = misc[kNOuter];
        const int nold = misc[kCnt0 + cur];
        const int t = s + 3;
        const bool follow = t <= M - 1;
        const unsigned long long tag = (unsigned long long)(64 - t) << 48;
        // P1
        for (;;) {
            const int i = atomicAdd(&misc[kWork], 1);
            if (i >= nold + nl) break;
            if (i >= nl) {
                if (follow) {
                    FTrack T = Fc[i - nl];
                    follow_and_claim<G>(C, S, R, t, tag, sq_follow, T);
                    Fc[i - nl] = T;
                }
            } else {
                const int c = (int)list[i];
                int a, b;
                if (seed_for<G>(C, S, R, s, c, outer, nu, sq_seed, a, b)) {
                    const int slot = nold + atomicAdd(&misc[kNew], 1);
                    if (slot < cap) {
                        FTrack T = make_track(a, c, b, c, 3, 0);
                        if (follow) follow_and_claim<G>(C, S, R, t, tag, sq_follow, T);
                        Fc[slot] = T;
                    } else {
                        misc[kErr] = SBT_ERR_CAPACITY;
                    }
                }
            }
        }
        __syncthreads();
        if (misc[kErr]) return false;
        const int nf = nold + misc[kNew];
        if (tid == 0) misc[kList] = 0;
        // P2
        if (follow) {
            for (int f = tid; f < nf; f += NT) {
                const FTrack T = Fc[f];
                if (T.cand == kDead) continue;
                bool won = false;
                if (T.cand != kNone) {
                    const unsigned long long k = claim_key(tag, T.sc, T.key);
                    // all claim words loaded at once (one round trip)
                    const unsigned long long c0 = __ldcg(&R.claim[T.cand & R.cmask]);
                    unsigned long long c1 = k, c2 = k, c3 = k;
                    if (T.nh == 3) {
                        c1 = __ldcg(&R.claim[T.h0 & R.cmask]);
                        c2 = __ldcg(&R.claim[T.h1 & R.cmask]);
                        c3 = __ldcg(&R.claim[T.h2 & R.cmask]);
                    }
                    won = c0 == k && c1 == k && c2 == k && c3 == k;
                }
                if (won) {
                    set_flag(S, T.cand);
                    if (T.nh == 3) {
                        set_flag(S, T.h0);
                        set_flag(S, T.h1);
                        set_flag(S, T.h2);
                        R.prev[T.h0] = kNone;
                        R.prev[T.h1] = T.h0;
                        R.prev[T.h2] = T.h1;
                    }
                    R.prev[T.cand] = T.h2;
                    const int slot = atomicAdd(&misc[kCnt0 + nxt], 1);
                    Fn[slot] = make_track(T.h1, T.h2, T.cand, T.key, T.nh + 1, 0);
                } else if (T.sk + 1 >= 2) {
                    if (T.nh >= 4)
                        add_final(S, R, T.h2, T.nh);
                    else
                        add_tracklet(S, R, T.h0, T.h1, T.h2, T.key);
                } else {
                    const int slot = atomicAdd(&misc[kCnt0 + nxt], 1);
                    Fn[slot] = make_track(T.h0, T.h1, T.h2, T.key, T.nh, T.sk + 1);
                }
            }
        } else {
            // last iteration: every forming track is finished
            for (int f = tid; f < nf; f += NT) {
                const FTrack T = Fc[f];
                if (T.nh >= 4)
                    add_final(S, R, T.h2, T.nh);
                else
                    add_tracklet(S, R, T.h0, T.h1, T.h2, T.key);
            }
        }
        __syncthreads();
        cur = nxt;
    }
    return misc[kErr] == 0;
}

// Tracklet filter: three unflagged hits and chi2 < C3, then one claim round
// among the survivors (tag 0, below every search tag).
template <int NT, class HS>
__device__ void tracklet_filter(const DevConfig& C, const Region<HS>& R, const Smem& S)
{
    const int tid = threadIdx.x;
    const int ntl = min(S.misc[kNTl], R.lcap);
    // the search kept its claims in a ring; the filter's claims use the whole
    // array, the tracklets' words cleared first
    for (int k = tid; k < ntl; k += NT) {
        const unsigned long long v = R.tracklets[k];
        R.claim[v & 0xFFFF] = ~0ull;
        R.claim[(v >> 16) & 0xFFFF] = ~0ull;
        R.claim[(v >> 32) & 0xFFFF] = ~0ull;
    }
    __syncthreads();
    for (int k = tid; k < ntl; k += NT) {
        unsigned long long v = R.tracklets[k];
        int h[3] = {(int)(v & 0xFFFF), (int)((v >> 16) & 0xFFFF), (int)((v >> 32) & 0xFFFF)};
        int key = (int)(v >> 48);
        uint32_t q = 0xFFFFFFFFu;
        if (!flagged(S, h[0]) && !flagged(S, h[1]) && !flagged(S, h[2])) {
            float chi2;
            fit_line(
                3,
                [&](int i) {
                    float4 c = R.coords[h[i]];
                    return make_float3(c.x, c.y, c.z);
                },
                C.sigma, nullptr, &chi2);
            if (chi2 < C.C3) {
                q = __float_as_uint(chi2);
                unsigned long long kk = claim_key(0ull, chi2, key);
                atomicMin(&R.claim[h[0]], kk);
                atomicMin(&R.claim[h[1]], kk);
                atomicMin(&R.claim[h[2]], kk);
            }
        }
        R.tl_q[k] = q;
    }
    __syncthreads();
    for (int k = tid; k < ntl; k += NT) {
        uint32_t q = R.tl_q[k];
        if (q == 0xFFFFFFFFu) continue;
        unsigned long long v = R.tracklets[k];
        int h0 = (int)(v & 0xFFFF), h1 = (int)((v >> 16) & 0xFFFF), h2 = (int)((v >> 32) & 0xFFFF);
        unsigned long long kk = claim_key(0ull, __uint_as_float(q), (int)(v >> 48));
        if (__ldcg(&R.claim[h0]) == kk && __ldcg(&R.claim[h1]) == kk && __ldcg(&R.claim[h2]) == kk) {
            R.prev[h0] = kNone;
            R.prev[h1] = (uint16_t)h0;
            R.prev[h2] = (uint16_t)h1;
            add_final(S, R, h2, 3);
        }
    }
    __syncthreads();
}

// Staging of the tracks: each track's linked hit list is walked once, its
// hit records written in traversal order at its found-order place among the
// event's staged hits, with its smallest input index.  Ordering and fits are
// left to the output kernel.
template <int NT, class HS>
__device__ void output_stage(int e, int off, const Region<HS>& R, const Smem& S, const Staging& G,
                             const sbt_tracks& out)
{
    const int tid = threadIdx.x;
    const int T = S.misc[kNFin];
    const int chunk = (T + NT - 1) / NT;
    const int beg = min(T, tid * chunk), end = min(T, beg + chunk);
    int cnt = 0;
    for (int k = beg; k < end; k++) cnt += (int)(R.finals[k] >> 16);
    int H;
    int u = block_exclusive_scan<NT>(cnt, S.wsum, &H);
    const int64_t slot0 = (int64_t)off / 3 + e;
    float4* hits = G.hits + off;
    for (int k = beg; k < end; k++) {
        const uint32_t v = R.finals[k];
        int q = (int)(v & 0xFFFF);
        const int nh = (int)(v >> 16);
        int mn = INT_MAX;
        for (int j = nh - 1; j >= 0; j--) {
            const int nq = R.prev[q];
            const float4 c = R.coords[q];
            const int i = __float_as_int(c.w);
            hits[u + j] = make_float4(c.x, c.y, c.z, __int_as_float(off + i));
            mn = i < mn ? i : mn;
            q = nq;
        }
        G.tkey[slot0 + k] = mn;
        G.tinfo[slot0 + k] = (uint32_t)u | ((uint32_t)nh << 16);
        u += nh;
    }
    if (tid == 0) {
        G.ev_ntracks[e] = T;
        G.ev_nhits[e] = H;
        out.event_status[e] = SBT_OK;
    }
}

__device__ __forceinline__ void fail_event(int e, int code, const Staging& G, const sbt_tracks& out)
{
    if (threadIdx.x == 0) {
        G.ev_ntracks[e] = 0;
        G.ev_nhits[e] = 0;
        out.event_status[e] = code;
    }
}

// Search of one sorted event by the whole block.
template <int NT, class HS, class GEO>
__device__ void run_event(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                          const Staging& G, const sbt_tracks& out, int e, int64_t hb, int64_t r,
                          int cap, const Smem& S)
{
    const int tid = threadIdx.x;
    const int off = in.offsets[e];
    const int n = in.offsets[e + 1] - off;
    const int st = O.status[e];
    if (st != SBT_OK || n > cap) {
        fail_event(e, st != SBT_OK ? st : SBT_ERR_CAPACITY, G, out);
        return;
    }
    Region<HS> R = region_of<HS>(O, off, W, hb, r, cap);
    for (int m = tid; m <= C.M; m += NT) S.modoff[m] = O.modoff[(int64_t)e * (C.M + 1) + m];
    for (int w = tid; w < (n + 31) / 32; w += NT) S.flag[w] = 0u;
    __syncthreads();
    // Claims are live only on the modules s-1 .. s+3 of step s (a 3-hit track
    // has its hits on s-1 or later, a new hit lies on s+3), so the search keeps
    // them in a ring of the smallest power of two that covers every such span:
    // live positions never share a slot, and the ring stays in cache.  Without
    // such a power of two within the region's capacity, no ring.
    if (tid == 0) {
        int w = 0;
        for (int s = 0; s + 2 <= C.M - 1; s++)
            w = max(w, S.modoff[min(s + 4, C.M)] - S.modoff[max(s - 1, 0)]);
        int p2 = 1;
        while (p2 < w && p2 <= cap) p2 <<= 1;
        S.misc[kCMask] = p2 >= w && p2 <= cap ? p2 - 1 : -1;
    }
    __syncthreads();
    R.cmask = (unsigned)S.misc[kCMask];
    // claim words of the modules that are never a following target
    for (int p = tid; p < S.modoff[min(3, C.M)]; p += NT) R.claim[p & R.cmask] = ~0ull;
    __syncthreads();
    if (!search_stage<NT, GEO>(C, R, S, n)) {
        fail_event(e, SBT_ERR_CAPACITY, G, out);
        __syncthreads();
        return;
    }
    tracklet_filter<NT>(C, R, S);
    output_stage<NT>(e, off, R, S, G, out);
    __syncthreads();
}

// ------------------------------------------------------------- kernels ---

// Residency of the search: the kernel waits on load latency, so throughput
// follows the number of resident events; the compiler is asked for a
// register count that lets 2048 threads (32 blocks of 64) share an SM.
constexpr int kSearchThreadsPerSM = 2048;

// One block per event.
template <int NT, class HS, class GEO>
__global__ void __launch_bounds__(NT, kSearchThreadsPerSM / NT) k_search_plain(DevConfig C, Inputs in, Sorted O, Work W,
                                                      Staging G, sbt_tracks out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S = carve(smem_raw, C.nmax, NT, C.M);
    const int e = blockIdx.x;
    const int off = in.offsets[e];
    const int n = in.offsets[e + 1] - off;
    run_event<NT, HS, GEO>(C, in, O, W, G, out, e, off, e, max(n, 0), S);
}

// Persistent: each resident block takes events from the work queue, sizes
// alternating from both ends of G.order (largest first), and reuses its own
// scratch region.
template <int NT, class HS, class GEO>
__global__ void __launch_bounds__(NT, kSearchThreadsPerSM / NT) k_search_persistent(DevConfig C, Inputs in, Sorted O, Work W,
                                                           Staging G, sbt_tracks out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem S = carve(smem_raw, C.nmax, NT, C.M);
    const int64_t hb = (int64_t)blockIdx.x * C.nmax;
    for (;;) {
        if (threadIdx.x == 0) S.misc[kEvent] = atomicAdd(&G.queue[0], 1);
        __syncthreads();
        const int q = S.misc[kEvent];
        __syncthreads();
        if (q >= in.n_events) break;
        // alternately the largest and the smallest event not yet taken, so
        // the resident events' hits and scratch stay near the average size
        // (the largest-first order alone fills L2 with the heaviest events at
        // the start); the last 2 x blocks events, from the middle of the size
        // order, are taken largest first, which keeps the tail short
        const int q0 = max(0, in.n_events - 2 * (int)gridDim.x) & ~1;
        const int qi = q >= q0 ? (q0 >> 1) + (q - q0) : (q & 1) ? in.n_events - 1 - (q >> 1) : (q >> 1);
        run_event<NT, HS, GEO>(C, in, O, W, G, out, G.order[qi], hb, blockIdx.x, C.nmax, S);
    }
}

// Processing order, largest events first (counting sort on size classes).
__global__ void __launch_bounds__(1024) k_order(Inputs in, Staging G)
{
    __shared__ int hist[1024];
    __shared__ int wsum[33];
    const int tid = threadIdx.x;
    const int E = in.n_events;
    hist[tid] = 0;
    __syncthreads();
    for (int e = tid; e < E; e += 1024) {
        int n = in.offsets[e + 1] - in.offsets[e];
        int b = 1023 - min(max(n, 0) >> 4, 1023);
        atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    int v = hist[tid];
    int total;
    int ex = block_exclusive_scan<1024>(v, wsum, &total);
    hist[tid] = ex;
    __syncthreads();
    for (int e = tid; e < E; e += 1024) {
        int n = in.offsets[e + 1] - in.offsets[e];
        int b = 1023 - min(max(n, 0) >> 4, 1023);
        G.order[atomicAdd(&hist[b], 1)] = e;
    }
}

// Device-wide exclusive scan of the per-event track and hit counts, with the
// capacity check.  One block; each thread owns a contiguous run of events.
__global__ void __launch_bounds__(1024) k_scan(Inputs in, Staging G, sbt_tracks out)
{
    __shared__ int wsum[33];
    __shared__ int first_over;
    const int tid = threadIdx.x;
    const int E = in.n_events;
    if (tid == 0) first_over = INT_MAX;
    const int chunk = (E + 1023) / 1024;
    const int beg = min(E, tid * chunk), end = min(E, beg + chunk);
    int t = 0, h = 0, f = 0;
    for (int e = beg; e < end; e++) {
        t += G.ev_ntracks[e];
        h += G.ev_nhits[e];
        f += out.event_status[e] != SBT_OK && out.event_status[e] != SBT_EVENT_CUT;
    }
    int T, H, F;
    int bt = block_exclusive_scan<1024>(t, wsum, &T);
    int bh = block_exclusive_scan<1024>(h, wsum, &H);
    block_exclusive_scan<1024>(f, wsum, &F);
    for (int e = beg; e < end; e++) {
        G.track_base[e] = bt;
        G.hit_base[e] = bh;
        out.track_offsets[e] = bt;
        // the output kernel skips the events past the capacities: a suffix
        if ((int64_t)bt + G.ev_ntracks[e] > out.cap_tracks || (int64_t)bh + G.ev_nhits[e] > out.cap_hits)
            atomicMin(&first_over, bt);
        bt += G.ev_ntracks[e];
        bh += G.ev_nhits[e];
    }
    __syncthreads();
    if (tid == 0) {
        G.queue[1] = min(first_over, T);
        out.track_offsets[E] = T;
        bool ok = T <= out.cap_tracks && H <= out.cap_hits;
        if (ok) out.hit_offsets[T] = H;
        out.counts[0] = T;
        out.counts[1] = H;
        out.counts[2] = ok ? SBT_OK : SBT_ERR_CAPACITY;
        out.counts[3] = F;
    }
}

// Least-squares fit of one track from its n staged hit records (src), with
// its hit list written on the way (th: batch input indices): sums in hit
// order, every operation rounded as in fit_line.  The first pass loads the
// records four at a time (independent loads in flight) and keeps the
// coordinates of the first kFitStash in shared memory (stash: this thread's
// column of a [kFitStash][kFitThreads] float3 array, conflict-free); the two
// centred passes read them there and re-read only the others.
constexpr int kFitThreads = 256;
constexpr int kFitStash = 16;

__device__ __forceinline__ void fit_staged(int n, const float4* src, int32_t* th, float3* stash, float sigma,
                                           float* params, float* chi2)
{
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int i0 = 0; i0 < n; i0 += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (i0 + u < n) v[u] = src[i0 + u];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (i0 + u < n) {
                th[i0 + u] = __float_as_int(v[u].w);
                sx = __fadd_rn(sx, v[u].x);
                sy = __fadd_rn(sy, v[u].y);
                sz = __fadd_rn(sz, v[u].z);
                if (i0 + u < kFitStash) stash[(i0 + u) * kFitThreads] = make_float3(v[u].x, v[u].y, v[u].z);
            }
    }
    const int ns = min(n, kFitStash);
    const float nf = (float)n;
    const float xm = __fdiv_rn(sx, nf), ym = __fdiv_rn(sy, nf), zm = __fdiv_rn(sz, nf);
    float szz = 0.0f, szx = 0.0f, szy = 0.0f;
    auto moments = [&](float x, float y, float z) {
        const float dz = __fsub_rn(z, zm);
        szz = __fadd_rn(szz, __fmul_rn(dz, dz));
        szx = __fadd_rn(szx, __fmul_rn(dz, __fsub_rn(x, xm)));
        szy = __fadd_rn(szy, __fmul_rn(dz, __fsub_rn(y, ym)));
    };
#pragma unroll 4
    for (int i = 0; i < ns; i++) {
        const float3 q = stash[i * kFitThreads];
        moments(q.x, q.y, q.z);
    }
    for (int i = kFitStash; i < n; i++) {
        const float4 q = src[i];
        moments(q.x, q.y, q.z);
    }
    const float tx = __fdiv_rn(szx, szz);
    const float ty = __fdiv_rn(szy, szz);
    float s = 0.0f;
    auto resid = [&](float x, float y, float z) {
        const float dz = __fsub_rn(z, zm);
        const float rx = __fsub_rn(__fsub_rn(x, xm), __fmul_rn(tx, dz));
        const float ry = __fsub_rn(__fsub_rn(y, ym), __fmul_rn(ty, dz));
        s = __fadd_rn(s, __fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)));
    };
#pragma unroll 4
    for (int i = 0; i < ns; i++) {
        const float3 q = stash[i * kFitThreads];
        resid(q.x, q.y, q.z);
    }
    for (int i = kFitStash; i < n; i++) {
        const float4 q = src[i];
        resid(q.x, q.y, q.z);
    }
    params[0] = __fsub_rn(xm, __fmul_rn(tx, zm));
    params[1] = __fsub_rn(ym, __fmul_rn(ty, zm));
    params[2] = tx;
    params[3] = ty;
    *chi2 = __fdiv_rn(s, __fmul_rn(sigma, sigma));
}

// Output (section "Results", data consolidation), one block per event: the
// canonical order of the event's tracks by smallest input hit index and
// their CSR starts; the hit lists and fits follow in k_fit.  A track's rank
// is the number of tracks with a smaller smallest index: one bit per input
// index marks the tracks' smallest indices (shared memory), and a prefix of
// the words' bit counts gives every rank.
constexpr int kOutputThreads = 256;

__global__ void __launch_bounds__(kOutputThreads) k_output(DevConfig C, Inputs in, Staging G,
                                                          sbt_tracks out)
{
    constexpr int NT = kOutputThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nwmax = (C.nmax + 31) / 32;
    uint32_t* bits = (uint32_t*)smem_raw;  // [nwmax]
    int* wpre = (int*)(bits + nwmax);      // [nwmax]
    __shared__ int wsum[40];
    const int e = blockIdx.x;
    const int tid = threadIdx.x;
    const int T = G.ev_ntracks[e];
    if (T == 0) return;
    const int H = G.ev_nhits[e];
    const int tb = G.track_base[e], hbase = G.hit_base[e];
    if ((int64_t)tb + T > out.cap_tracks || (int64_t)hbase + H > out.cap_hits) return;
    const int off = in.offsets[e];
    const int n = in.offsets[e + 1] - off;
    const int64_t slot0 = (int64_t)off / 3 + e;
    const int nw = (n + 31) / 32;
    for (int w = tid; w < nw; w += NT) bits[w] = 0u;
    __syncthreads();
    for (int k = tid; k < T; k += NT) {
        const int mn = G.tkey[slot0 + k];
        atomicOr(&bits[mn >> 5], 1u << (mn & 31));
    }
    __syncthreads();
    {
        const int wc = (nw + NT - 1) / NT;
        const int wb = min(nw, tid * wc), we = min(nw, wb + wc);
        int c = 0;
        for (int w = wb; w < we; w++) c += __popc(bits[w]);
        int tot;
        int st = block_exclusive_scan<NT>(c, wsum, &tot);
        for (int w = wb; w < we; w++) {
            wpre[w] = st;
            st += __popc(bits[w]);
        }
    }
    __syncthreads();
    for (int k = tid; k < T; k += NT) {
        const int mn = G.tkey[slot0 + k];
        const int r = wpre[mn >> 5] + __popc(bits[mn >> 5] & ((1u << (mn & 31)) - 1u));
        G.rinfo[slot0 + r] = G.tinfo[slot0 + k];
    }
    __syncthreads();
    // canonical starts: each thread takes a contiguous run of ranks
    const int chunk = (T + NT - 1) / NT;
    const int beg = min(T, tid * chunk), end = min(T, beg + chunk);
    int c = 0;
    for (int r = beg; r < end; r++) c += (int)(G.rinfo[slot0 + r] >> 16);
    int Ht;
    int cs = block_exclusive_scan<NT>(c, wsum, &Ht);
    for (int r = beg; r < end; r++) {
        const uint32_t ri = G.rinfo[slot0 + r];
        const int nh = (int)(ri >> 16);
        const int64_t g = (int64_t)tb + r;
        out.hit_offsets[g] = hbase + cs;
        G.tfit[g] = make_uint2((uint32_t)(off + (int)(ri & 0xFFFFu)), (uint32_t)nh);
        cs += nh;
    }
}

// Hit lists and least-squares fits of the canonical tracks, one thread per
// track of the batch, in canonical order (a warp's hit lists and parameters
// are contiguous in the output): the tracks of the events the output kernel
// wrote, G.queue[1] of them.
__global__ void __launch_bounds__(kFitThreads) k_fit(DevConfig C, Staging G, sbt_tracks out)
{
    __shared__ float3 stash[kFitStash * kFitThreads];
    const int T = G.queue[1];
    for (int g = blockIdx.x * kFitThreads + threadIdx.x; g < T; g += gridDim.x * kFitThreads) {
        const uint2 f = G.tfit[g];
        const int n = (int)f.y;
        float p[4], chi2;
        fit_staged(n, G.hits + f.x, out.track_hits + out.hit_offsets[g], stash + threadIdx.x, C.sigma, p, &chi2);
        out.params[4 * (int64_t)g + 0] = p[0];
        out.params[4 * (int64_t)g + 1] = p[1];
        out.params[4 * (int64_t)g + 2] = p[2];
        out.params[4 * (int64_t)g + 3] = p[3];
        out.chi2[g] = chi2;
        out.ndof[g] = 2 * n - 4;
    }
}

size_t output_smem_bytes(int nmax) { return 8 * (size_t)((nmax + 31) / 32); }

// Chunked host pipeline: adds the totals of the earlier chunks to one chunk's
// CSR offsets (track_offsets [n_events + 1], hit_offsets [counts[0] + 1]) and
// advances the running totals (running[0] tracks, running[1] hits).
// Chunk offsets made global: running[0..1] hold the tracks and track hits of
// the earlier chunks (read by every block), running[2..3] receive the totals
// including this chunk (written by block 0 only).
__global__ void __launch_bounds__(256) k_offset_fixup(int32_t* track_offsets, int32_t n_events,
                                                      int32_t* hit_offsets, const int32_t* counts,
                                                      int64_t* running)
{
    const int64_t bt = running[0], bh = running[1];
    const int T = counts[0];
    const bool ok = counts[2] == SBT_OK;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_events; i += stride)
        track_offsets[i] += (int32_t)bt;
    if (ok)
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= T; t += stride)
            hit_offsets[t] += (int32_t)bh;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        running[2] = bt + T;
        running[3] = bh + counts[1];
    }
}

// Sort stage output copied out, for stage-level checks.
template <class HS>
__global__ void k_debug_sort_copy(DevConfig C, Inputs in, Sorted O, uint16_t* phi16, int32_t* perm,
                                  int32_t* modoff)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < in.n_hits) {
        phi16[i] = O.phi[i];
        perm[i] = __float_as_int(HS::load((const typename HS::T*)O.coords, i).w);
    }
    if (i < (int64_t)in.n_events * (C.M + 1)) modoff[i] = O.modoff[i];
}

__global__ void k_debug_phi16(const float* x, const float* y, int32_t n, uint16_t* out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint16_t)phi16_of(x[i], y[i]);
}

// ------------------------------------------------------------ launchers ---

cudaError_t launch_sort(const DevConfig& C, const Inputs& in, const Sorted& O, cudaStream_t st)
{
    size_t sm = sort_smem_bytes(C.nmax);
    auto kern = C.h16 ? k_sort<HitsF16> : k_sort<HitsF32>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    if (in.n_events > 0) kern<<<in.n_events, kSortThreads, sm, st>>>(C, in, O);
    return cudaGetLastError();
}

template <int NT, class HS, class GEO>
static cudaError_t plain_ntg(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                             const Staging& G, const sbt_tracks& out, cudaStream_t st)
{
    size_t sm = smem_bytes(C.nmax, NT, C.M);
    cudaError_t err = cudaFuncSetAttribute(k_search_plain<NT, HS, GEO>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    if (in.n_events > 0) k_search_plain<NT, HS, GEO><<<in.n_events, NT, sm, st>>>(C, in, O, W, G, out);
    return cudaGetLastError();
}

template <int NT, class HS>
static cudaError_t plain_nt(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                            const Staging& G, const sbt_tracks& out, cudaStream_t st)
{
    return C.pairs ? plain_ntg<NT, HS, PairGeo>(C, in, O, W, G, out, st)
                   : plain_ntg<NT, HS, PlaneGeo>(C, in, O, W, G, out, st);
}

cudaError_t launch_plain(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                         const Staging& S, const sbt_tracks& out, int threads, cudaStream_t stream)
{
    switch (threads) {
        case 64: return C.h16 ? plain_nt<64, HitsF16>(C, in, O, W, S, out, stream) : plain_nt<64, HitsF32>(C, in, O, W, S, out, stream);
        case 128: return C.h16 ? plain_nt<128, HitsF16>(C, in, O, W, S, out, stream) : plain_nt<128, HitsF32>(C, in, O, W, S, out, stream);
        case 256: return C.h16 ? plain_nt<256, HitsF16>(C, in, O, W, S, out, stream) : plain_nt<256, HitsF32>(C, in, O, W, S, out, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_order(const Inputs& in, const Staging& S, cudaStream_t stream)
{
    k_order<<<1, 1024, 0, stream>>>(in, S);
    return cudaGetLastError();
}

template <int NT, class HS, class GEO>
static int occupancy_ntg(const DevConfig& C)
{
    size_t sm = smem_bytes(C.nmax, NT, C.M);
    if (cudaFuncSetAttribute(k_search_persistent<NT, HS, GEO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm) != cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_search_persistent<NT, HS, GEO>, NT, sm) !=
        cudaSuccess)
        return 0;
    return blocks;
}

template <int NT, class HS>
static int occupancy_nt(const DevConfig& C)
{
    return C.pairs ? occupancy_ntg<NT, HS, PairGeo>(C) : occupancy_ntg<NT, HS, PlaneGeo>(C);
}

int persistent_blocks_per_sm(const DevConfig& C, int threads)
{
    switch (threads) {
        case 64: return C.h16 ? occupancy_nt<64, HitsF16>(C) : occupancy_nt<64, HitsF32>(C);
        case 128: return C.h16 ? occupancy_nt<128, HitsF16>(C) : occupancy_nt<128, HitsF32>(C);
        case 256: return C.h16 ? occupancy_nt<256, HitsF16>(C) : occupancy_nt<256, HitsF32>(C);
        default: return 0;
    }
}

template <int NT, class HS, class GEO>
static cudaError_t persistent_ntg(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                                  const Staging& G, const sbt_tracks& out, int blocks,
                                  cudaStream_t st)
{
    size_t sm = smem_bytes(C.nmax, NT, C.M);
    cudaError_t err = cudaFuncSetAttribute(k_search_persistent<NT, HS, GEO>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    if (blocks > 0) k_search_persistent<NT, HS, GEO><<<blocks, NT, sm, st>>>(C, in, O, W, G, out);
    return cudaGetLastError();
}

template <int NT, class HS>
static cudaError_t persistent_nt(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                                 const Staging& G, const sbt_tracks& out, int blocks,
                                 cudaStream_t st)
{
    return C.pairs ? persistent_ntg<NT, HS, PairGeo>(C, in, O, W, G, out, blocks, st)
                   : persistent_ntg<NT, HS, PlaneGeo>(C, in, O, W, G, out, blocks, st);
}

cudaError_t launch_persistent(const DevConfig& C, const Inputs& in, const Sorted& O, const Work& W,
                              const Staging& S, const sbt_tracks& out, int threads, int blocks,
                              cudaStream_t stream)
{
    switch (threads) {
        case 64: return C.h16 ? persistent_nt<64, HitsF16>(C, in, O, W, S, out, blocks, stream) : persistent_nt<64, HitsF32>(C, in, O, W, S, out, blocks, stream);
        case 128: return C.h16 ? persistent_nt<128, HitsF16>(C, in, O, W, S, out, blocks, stream) : persistent_nt<128, HitsF32>(C, in, O, W, S, out, blocks, stream);
        case 256: return C.h16 ? persistent_nt<256, HitsF16>(C, in, O, W, S, out, blocks, stream) : persistent_nt<256, HitsF32>(C, in, O, W, S, out, blocks, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_scan(const Inputs& in, const Staging& S, const sbt_tracks& out,
                        cudaStream_t stream)
{
    k_scan<<<1, 1024, 0, stream>>>(in, S, out);
    return cudaGetLastError();
}

cudaError_t launch_output(const DevConfig& C, const Inputs& in, const Staging& S,
                          const sbt_tracks& out, cudaStream_t stream)
{
    const size_t sm = output_smem_bytes(C.nmax);
    cudaError_t err = cudaFuncSetAttribute(k_output, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    if (in.n_events > 0) k_output<<<in.n_events, kOutputThreads, sm, stream>>>(C, in, S, out);
    err = cudaGetLastError();
    if (err != cudaSuccess || in.n_events == 0) return err;
    // k_fit: one resident wave over the device, a grid-stride loop over the tracks
    int dev = 0, sms = 0, per_sm = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fit, kFitThreads, 0);
    if (err != cudaSuccess) return err;
    k_fit<<<sms * std::max(per_sm, 1), kFitThreads, 0, stream>>>(C, S, out);
    return cudaGetLastError();
}

cudaError_t launch_finish(const DevConfig& C, const Inputs& in, const Staging& S,
                          const sbt_tracks& out, cudaStream_t stream)
{
    cudaError_t e = launch_scan(in, S, out, stream);
    if (e == cudaSuccess) e = launch_output(C, in, S, out, stream);
    return e;
}

cudaError_t launch_debug_sort_copy(const DevConfig& C, const Inputs& in, const Sorted& O,
                                   uint16_t* phi16, int32_t* perm, int32_t* module_offsets,
                                   cudaStream_t stream)
{
    const int64_t n = std::max<int64_t>(in.n_hits, (int64_t)in.n_events * (C.M + 1));
    if (n > 0)
        (C.h16 ? k_debug_sort_copy<HitsF16> : k_debug_sort_copy<HitsF32>)<<<(unsigned)((n + 255) / 256), 256, 0,
                                                                          stream>>>(C, in, O, phi16, perm,
                                                                                    module_offsets);
    return cudaGetLastError();
}

cudaError_t launch_offset_fixup(int32_t* track_offsets, int32_t n_events, int32_t* hit_offsets,
                                const int32_t* counts, int64_t* running, cudaStream_t stream)
{
    k_offset_fixup<<<kFixupBlocks, 256, 0, stream>>>(track_offsets, n_events, hit_offsets, counts, running);
    return cudaGetLastError();
}

cudaError_t launch_debug_phi16(const float* x, const float* y, int32_t n, uint16_t* out,
                               cudaStream_t stream)
{
    if (n > 0) k_debug_phi16<<<(n + 255) / 256, 256, 0, stream>>>(x, y, n, out);
    return cudaGetLastError();
}

}  // namespace sbt

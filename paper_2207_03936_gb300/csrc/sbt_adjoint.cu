// Adjoint of the consolidation fit with respect to per-module alignment.
//
// Objective: sum over tracks of the least-squares residual sum / sigma^2 of
// the straight-line fit (section "Tracklet filter": least-squares fit; the
// same fit is applied to every consolidated track), evaluated on aligned hits
//     h' = Rz(g) Ry(b) Rx(a) (h - c_m) + c_m + (dx, dy, dz),  c_m = (0, 0, z_m).
// At the least-squares optimum the derivative with respect to a hit is the
// partial derivative at fixed line parameters (the parameters are stationary),
//     d chi2 / d h' = 2 / sigma^2 (rx, ry, -(rx tx + ry ty)) = g,
// chained through d h' / d(align_m): g itself for the translations, and
// g . (dR_m/da v) for a rotation angle a, v = h - c_m.  Summed over the hits
// of module m that is sum_ij (dR_m/da)_ij sum_h g_i v_j, so the kernel
// accumulates per module g and the outer product g v^T (9 products a hit)
// and the derivative matrices are applied once per module at the end.
//
// Layout: one warp per track, lanes over its hits in rounds of 32.  A track
// may have any number of hits and several hits on one module; a track
// without a straight-line fit (fewer than two hits or modules) or with an
// index out of range contributes nothing and is counted as skipped.  Each
// warp owns an fp64 accumulator in shared memory, updated in a fixed lane
// order; warps are summed in a fixed order per block and blocks in a fixed
// order by the final kernel, so the result is bitwise reproducible.
// Arithmetic is fp64 (the hits are fp32).
#include <cuda_runtime.h>

#include <cstdint>

#include "sbt_internal.h"

namespace sbt {

constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjBlocksPerSM = 4;

int adjoint_blocks(int sm_count) { return kAdjBlocksPerSM * (sm_count > 0 ? sm_count : 1); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ void matvec(const double* R, double x, double y, double z, double& ox,
                                       double& oy, double& oz)
{
    ox = R[0] * x + R[1] * y + R[2] * z;
    oy = R[3] * x + R[4] * y + R[5] * z;
    oz = R[6] * x + R[7] * y + R[8] * z;
}

__device__ __forceinline__ void matmul(const double* A, const double* B, double* C)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            C[3 * i + j] = A[3 * i + 0] * B[0 + j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// Per module: R = Rz Ry Rx and its derivatives with respect to a, b, g.
__device__ void module_matrices(const double* th, double* out /* 36 */)
{
    double ca = cos(th[3]), sa = sin(th[3]);
    double cb = cos(th[4]), sb = sin(th[4]);
    double cg = cos(th[5]), sg = sin(th[5]);
    double Rx[9] = {1, 0, 0, 0, ca, -sa, 0, sa, ca};
    double dRx[9] = {0, 0, 0, 0, -sa, -ca, 0, ca, -sa};
    double Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb};
    double dRy[9] = {-sb, 0, cb, 0, 0, 0, -cb, 0, -sb};
    double Rz[9] = {cg, -sg, 0, sg, cg, 0, 0, 0, 1};
    double dRz[9] = {-sg, -cg, 0, cg, -sg, 0, 0, 0, 0};
    double t1[9], t2[9];
    matmul(Ry, Rx, t1);
    matmul(Rz, t1, out + 0);        // R
    matmul(Ry, dRx, t1);
    matmul(Rz, t1, out + 9);        // dR/da
    matmul(dRy, Rx, t1);
    matmul(Rz, t1, out + 18);       // dR/db
    matmul(Ry, Rx, t1);
    matmul(dRz, t1, out + 27);      // dR/dg
    (void)t2;
}

// One aligned hit: its module, the local coordinates v = h - c_m and the
// aligned position p = R_m v + c_m + t_m.
struct AHit {
    double px, py, pz, vx, vy, vz;
    int m;
};

__device__ __forceinline__ AHit aligned_hit(const DevConfig& C, const Inputs& in, const double* mats,
                                            const double* align, int h)
{
    AHit a;
    a.m = in.module[h];
    const double* R = mats + 36 * a.m;
    const double* th = align + 6 * a.m;
    const double zc = (double)C.module_z[a.m];
    a.vx = (double)in.x[h];
    a.vy = (double)in.y[h];
    a.vz = (double)in.z[h] - zc;
    double ox, oy, oz;
    matvec(R, a.vx, a.vy, a.vz, ox, oy, oz);
    a.px = ox + th[0];
    a.py = oy + th[1];
    a.pz = oz + zc + th[2];
    return a;
}

// Per-block accumulator entries: per module g (3) and g v^T (9), then chi2
// and the skipped-track count.
constexpr int kAdjPerModule = 12;

__host__ __device__ inline int adjoint_entries(int M) { return kAdjPerModule * M + 2; }

__global__ void __launch_bounds__(kAdjThreads) k_adjoint(DevConfig C, Inputs in,
                                                          const int32_t* hit_offsets,
                                                          const int32_t* track_hits,
                                                          int32_t n_tracks, const double* align,
                                                          double* partial, int want_grad)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = C.M;
    const int P = adjoint_entries(M);
    double* mats = (double*)smem_raw;               // [M][36]: R and its derivatives (R used here)
    double* acc = mats + 36 * M;                    // [warps][P]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int m = tid; m < M; m += kAdjThreads) module_matrices(align + 6 * m, mats + 36 * m);
    for (int k = tid; k < kAdjWarps * P; k += kAdjThreads) acc[k] = 0.0;
    __syncthreads();
    double* my = acc + warp * P;
    const double s2 = (double)C.sigma * (double)C.sigma;
    const double inv_s2 = 1.0 / s2, two_inv_s2 = 2.0 * inv_s2;  // one fp64 division per launch
    const int gw = blockIdx.x * kAdjWarps + warp;
    const int nw = gridDim.x * kAdjWarps;
    const int64_t end = n_tracks > 0 ? hit_offsets[n_tracks] : 0;
    for (int t = gw; t < n_tracks; t += nw) {
        const int h0 = hit_offsets[t];
        const int n = hit_offsets[t + 1] - h0;
        // every lane reads the same offsets, so these branches are uniform
        if (n < 2 || h0 < 0 || (int64_t)h0 + n > end) {
            if (lane == 0) my[P - 1] += 1.0;
            continue;
        }
        // pass 1: validity, sums; hits 0..63 kept in registers (two per lane)
        AHit keep0, keep1;
        bool bad = false;
        int mlo = INT32_MAX, mhi = -1;
        double sx = 0, sy = 0, sz = 0;
        for (int base = 0; base < n; base += 32) {
            const int j = base + lane;
            if (j >= n) continue;
            const int h = track_hits[h0 + j];
            if (h < 0 || h >= in.n_hits || in.module[h] < 0 || in.module[h] >= M) {
                bad = true;
                continue;
            }
            const AHit a = aligned_hit(C, in, mats, align, h);
            if (base == 0)
                keep0 = a;
            else if (base == 32)
                keep1 = a;
            mlo = min(mlo, a.m);
            mhi = max(mhi, a.m);
            sx += a.px;
            sy += a.py;
            sz += a.pz;
        }
        bad = __any_sync(0xFFFFFFFFu, bad);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mlo = min(mlo, __shfl_xor_sync(0xFFFFFFFFu, mlo, o));
            mhi = max(mhi, __shfl_xor_sync(0xFFFFFFFFu, mhi, o));
        }
        if (bad || mlo == mhi) {
            if (lane == 0) my[P - 1] += 1.0;
            continue;
        }
        auto hit_at = [&](int base, int j) -> AHit {
            if (base == 0) return keep0;
            if (base == 32) return keep1;
            return aligned_hit(C, in, mats, align, track_hits[h0 + j]);
        };
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        sz = warp_sum(sz);
        const double xm = sx / n, ym = sy / n, zm = sz / n;
        // pass 2: second moments
        double szz = 0, szx = 0, szy = 0;
        for (int base = 0; base < n; base += 32) {
            const int j = base + lane;
            if (j >= n) continue;
            const AHit a = hit_at(base, j);
            const double dz = a.pz - zm;
            szz += dz * dz;
            szx += dz * (a.px - xm);
            szy += dz * (a.py - ym);
        }
        szz = warp_sum(szz);
        szx = warp_sum(szx);
        szy = warp_sum(szy);
        const double tx = szx / szz, ty = szy / szz;
        // pass 3: residuals, chi2 and the gradient per module; lanes of one
        // round that share a module add in lane order
        double c2 = 0;
        for (int base = 0; base < n; base += 32) {
            const int j = base + lane;
            const bool act = j < n;
            double g[kAdjPerModule];
            int m = -1 - lane;  // distinct for inactive lanes
            if (act) {
                const AHit a = hit_at(base, j);
                m = a.m;
                const double dz = a.pz - zm;
                const double rx = (a.px - xm) - tx * dz;
                const double ry = (a.py - ym) - ty * dz;
                c2 += (rx * rx + ry * ry) * inv_s2;
                g[0] = rx * two_inv_s2;
                g[1] = ry * two_inv_s2;
                g[2] = -(rx * tx + ry * ty) * two_inv_s2;
                const double v[3] = {a.vx, a.vy, a.vz};
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int k = 0; k < 3; k++) g[3 + 3 * i + k] = g[i] * v[k];
            }
            if (want_grad) {
                const unsigned same = __match_any_sync(0xFFFFFFFFu, m);
                if (!__any_sync(0xFFFFFFFFu, __popc(same) > 1)) {
                    if (act) {
#pragma unroll
                        for (int k = 0; k < kAdjPerModule; k++) my[kAdjPerModule * m + k] += g[k];
                    }
                } else {
                    for (int l = 0; l < 32; l++) {
                        if (lane == l && act) {
#pragma unroll
                            for (int k = 0; k < kAdjPerModule; k++) my[kAdjPerModule * m + k] += g[k];
                        }
                        __syncwarp();
                    }
                }
                __syncwarp();
            }
        }
        c2 = warp_sum(c2);
        if (lane == 0) my[P - 2] += c2;
        __syncwarp();
    }
    __syncthreads();
    for (int k = tid; k < P; k += kAdjThreads) {
        double s = 0;
        for (int w = 0; w < kAdjWarps; w++) s += acc[w * P + k];
        partial[(int64_t)blockIdx.x * P + k] = s;
    }
}

// Fixed-order sum of the blocks' entries, then per module: the translation
// gradient is the summed g, each rotation gradient sum_ij (dR/d angle)_ij
// (sum g v^T)_ij.  One block of kAdjReduceThreads >= 12 M + 2 threads.
constexpr int kAdjReduceThreads = 1024;
static_assert(kAdjReduceThreads >= kAdjPerModule * kMaxModules + 2, "one thread per accumulator entry");

__global__ void __launch_bounds__(kAdjReduceThreads) k_adjoint_reduce(int M, int blocks, const double* partial,
                                                                      const double* align, double* chi2_sum,
                                                                      double* grad, int32_t* skipped)
{
    __shared__ double s[kAdjPerModule * kMaxModules + 2];
    const int P = adjoint_entries(M);
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double v = 0;
        for (int b = 0; b < blocks; b++) v += partial[(int64_t)b * P + k];
        s[k] = v;
    }
    __syncthreads();
    if (threadIdx.x < M && grad) {
        const int m = threadIdx.x;
        double D[36];
        module_matrices(align + 6 * m, D);
        const double* a = s + kAdjPerModule * m;
        grad[6 * m + 0] = a[0];
        grad[6 * m + 1] = a[1];
        grad[6 * m + 2] = a[2];
        for (int r = 0; r < 3; r++) {
            const double* dR = D + 9 * (r + 1);
            double v = 0;
            for (int ij = 0; ij < 9; ij++) v += dR[ij] * a[3 + ij];
            grad[6 * m + 3 + r] = v;
        }
    }
    if (threadIdx.x == 0) {
        *chi2_sum = s[P - 2];
        if (skipped) *skipped = (int32_t)s[P - 1];
    }
}

size_t adjoint_partial_entries(int M, int blocks) { return (size_t)blocks * (size_t)adjoint_entries(M); }

cudaError_t launch_adjoint(const DevConfig& C, const Inputs& in, const int32_t* hit_offsets,
                           const int32_t* track_hits, int32_t n_tracks, const double* align,
                           double* chi2_sum, double* grad, int32_t* skipped, const AdjointWork& W,
                           cudaStream_t stream)
{
    const int M = C.M;
    size_t sm = sizeof(double) * (36 * (size_t)M + (size_t)kAdjWarps * adjoint_entries(M));
    cudaError_t err = cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm);
    if (err != cudaSuccess) return err;
    k_adjoint<<<W.blocks, kAdjThreads, sm, stream>>>(C, in, hit_offsets, track_hits, n_tracks,
                                                      align, W.partial, grad != nullptr);
    k_adjoint_reduce<<<1, kAdjReduceThreads, 0, stream>>>(M, W.blocks, W.partial, align, chi2_sum, grad, skipped);
    return cudaGetLastError();
}

}  // namespace sbt

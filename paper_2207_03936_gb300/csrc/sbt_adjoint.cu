// Adjoint of the consolidation fit with respect to per-module alignment.
//
// Objective: sum over tracks of the least-squares residual sum / sigma^2 of
// the straight-line fit (section "Tracklet filter": least-squares fit; the
// same fit is applied to every consolidated track), evaluated on aligned hits
//     h' = Rz(g) Ry(b) Rx(a) (h - c_m) + c_m + (dx, dy, dz),  c_m = (0, 0, z_m).
// At the least-squares optimum the derivative with respect to a hit is the
// partial derivative at fixed line parameters (the parameters are stationary),
//     d chi2 / d h' = 2 / sigma^2 (rx, ry, -(rx tx + ry ty)),
// chained through d h' / d(align_m).
//
// Layout: one warp per track, lanes over its hits (a track has at most one
// hit per module, so the lanes of a warp update distinct modules).  Each warp
// owns an fp64 accumulator in shared memory; warps are summed in a fixed
// order per block and blocks in a fixed order by the final kernel, so the
// result is bitwise reproducible.  Arithmetic is fp64 (the hits are fp32).
#include <cuda_runtime.h>

#include <cstdint>

#include "sbt_internal.h"

namespace sbt {

constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjBlocks = 152 * 4;

int adjoint_blocks() { return kAdjBlocks; }

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

__global__ void __launch_bounds__(kAdjThreads) k_adjoint(DevConfig C, Inputs in,
                                                          const int32_t* hit_offsets,
                                                          const int32_t* track_hits,
                                                          int32_t n_tracks, const double* align,
                                                          double* partial, int want_grad)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = C.M;
    const int P = 6 * M + 1;  // gradient entries + chi2
    double* mats = (double*)smem_raw;               // [M][36]
    double* acc = mats + 36 * M;                    // [warps][P]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int m = tid; m < M; m += kAdjThreads) module_matrices(align + 6 * m, mats + 36 * m);
    for (int k = tid; k < kAdjWarps * P; k += kAdjThreads) acc[k] = 0.0;
    __syncthreads();
    double* my = acc + warp * P;
    const double s2 = (double)C.sigma * (double)C.sigma;
    const int gw = blockIdx.x * kAdjWarps + warp;
    const int nw = gridDim.x * kAdjWarps;
    for (int t = gw; t < n_tracks; t += nw) {
        const int h0 = hit_offsets[t];
        const int n = hit_offsets[t + 1] - h0;
        // each lane holds up to two hits (tracks have at most 64 hits)
        double px[2] = {0, 0}, py[2] = {0, 0}, pz[2] = {0, 0};
        double vx[2] = {0, 0}, vy[2] = {0, 0}, vz[2] = {0, 0};
        int mod[2] = {-1, -1};
        double sx = 0, sy = 0, sz = 0;
        for (int r = 0; r < 2; r++) {
            int j = lane + 32 * r;
            if (j >= n) continue;
            int h = track_hits[h0 + j];
            int m = in.module[h];
            const double* R = mats + 36 * m;
            const double* th = align + 6 * m;
            double zc = (double)C.module_z[m];
            double lx = (double)in.x[h], ly = (double)in.y[h], lz = (double)in.z[h] - zc;
            double ox, oy, oz;
            matvec(R, lx, ly, lz, ox, oy, oz);
            px[r] = ox + th[0];
            py[r] = oy + th[1];
            pz[r] = oz + zc + th[2];
            vx[r] = lx;
            vy[r] = ly;
            vz[r] = lz;
            mod[r] = m;
            sx += px[r];
            sy += py[r];
            sz += pz[r];
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        sz = warp_sum(sz);
        const double xm = sx / n, ym = sy / n, zm = sz / n;
        double szz = 0, szx = 0, szy = 0;
        for (int r = 0; r < 2; r++) {
            if (mod[r] < 0) continue;
            double dz = pz[r] - zm;
            szz += dz * dz;
            szx += dz * (px[r] - xm);
            szy += dz * (py[r] - ym);
        }
        szz = warp_sum(szz);
        szx = warp_sum(szx);
        szy = warp_sum(szy);
        const double tx = szx / szz, ty = szy / szz;
        double c2 = 0;
        for (int r = 0; r < 2; r++) {
            if (mod[r] < 0) continue;
            double dz = pz[r] - zm;
            double rx = (px[r] - xm) - tx * dz;
            double ry = (py[r] - ym) - ty * dz;
            c2 += (rx * rx + ry * ry) / s2;
            if (!want_grad) continue;
            double gx = 2.0 * rx / s2, gy = 2.0 * ry / s2, gz = -(2.0 * rx * tx + 2.0 * ry * ty) / s2;
            const double* D = mats + 36 * mod[r];
            double ux, uy, uz;
            double* G = my + 6 * mod[r];
            G[0] += gx;
            G[1] += gy;
            G[2] += gz;
            matvec(D + 9, vx[r], vy[r], vz[r], ux, uy, uz);
            G[3] += gx * ux + gy * uy + gz * uz;
            matvec(D + 18, vx[r], vy[r], vz[r], ux, uy, uz);
            G[4] += gx * ux + gy * uy + gz * uz;
            matvec(D + 27, vx[r], vy[r], vz[r], ux, uy, uz);
            G[5] += gx * ux + gy * uy + gz * uz;
        }
        c2 = warp_sum(c2);
        if (lane == 0) my[6 * M] += c2;
        __syncwarp();
    }
    __syncthreads();
    for (int k = tid; k < P; k += kAdjThreads) {
        double s = 0;
        for (int w = 0; w < kAdjWarps; w++) s += acc[w * P + k];
        partial[(int64_t)blockIdx.x * P + k] = s;
    }
}

__global__ void k_adjoint_reduce(int M, int blocks, const double* partial, double* chi2_sum,
                                 double* grad)
{
    const int P = 6 * M + 1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
        double s = 0;
        for (int b = 0; b < blocks; b++) s += partial[(int64_t)b * P + k];
        if (k < 6 * M) {
            if (grad) grad[k] = s;
        } else {
            *chi2_sum = s;
        }
    }
}

cudaError_t launch_adjoint(const DevConfig& C, const Inputs& in, const int32_t* hit_offsets,
                           const int32_t* track_hits, int32_t n_tracks, const double* align,
                           double* chi2_sum, double* grad, const AdjointWork& W,
                           cudaStream_t stream)
{
    const int M = C.M;
    size_t sm = sizeof(double) * (36 * (size_t)M + (size_t)kAdjWarps * (6 * M + 1));
    cudaError_t err = cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm);
    if (err != cudaSuccess) return err;
    k_adjoint<<<W.blocks, kAdjThreads, sm, stream>>>(C, in, hit_offsets, track_hits, n_tracks,
                                                      align, W.partial, grad != nullptr);
    k_adjoint_reduce<<<2, 256, 0, stream>>>(M, W.blocks, W.partial, chi2_sum, grad);
    return cudaGetLastError();
}

}  // namespace sbt

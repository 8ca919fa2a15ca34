// Mean first-order distance of mesh points to the isosurface of an original
// field, and its gradient with respect to the points: the loss this library
// uses to attribute isosurface error to grid points (with the adjoint of the
// vertex positions in mc.cu).  For a point p, F is the trilinear interpolant
// of the original field in the cell with lower corner clamp(floor(p), 0,
// n-2), G = grad F, H its Hessian (only the mixed second derivatives of a
// trilinear function are non-zero), and
//   d(p) = |F(p) - k| / |G|,
//   dd/dp = sign(F - k) G/|G| - |F - k| H G / |G|^3.
// Points where G vanishes count as distance 0 with zero gradient.  The mean
// is reduced in a fixed order (per-thread sums over a fixed stride, a
// fixed-shape block tree, then one block over the block partials), so the
// result does not depend on scheduling.  Arithmetic in float64.
#include "common.cuh"
#include "internal.h"

namespace chr {

namespace {

constexpr int kLossThreads = 256;

struct LossParams {
    const float *f;
    int64_t nx, ny, nz;
    double k;
    const float *pts;
    uint64_t npts;
    float *grad;
    double *partial;
    double *loss;
    uint32_t nblocks;
};

__global__ void __launch_bounds__(kLossThreads) k_dist_loss(const __grid_constant__ LossParams p)
{
    __shared__ double s_w[kLossThreads / 32];
    double acc = 0.0;
    const double invn = 1.0 / (double)p.npts;
    const int64_t n[3] = {p.nx, p.ny, p.nz};
    for (uint64_t v = (uint64_t)blockIdx.x * kLossThreads + threadIdx.x; v < p.npts;
         v += (uint64_t)gridDim.x * kLossThreads) {
        double u[3];
        int64_t c[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double x = (double)p.pts[3 * v + a];
            double fl = floor(x);
            fl = fmin(fmax(fl, 0.0), (double)(n[a] - 2));
            c[a] = (int64_t)fl;
            u[a] = x - fl;
        }
        const float *base = p.f + c[0] + p.nx * (c[1] + p.ny * c[2]);
        double F = 0, G0 = 0, G1 = 0, G2 = 0, H01 = 0, H02 = 0, H12 = 0;
#pragma unroll
        for (int dz = 0; dz < 2; dz++)
#pragma unroll
            for (int dy = 0; dy < 2; dy++)
#pragma unroll
                for (int dx = 0; dx < 2; dx++) {
                    const double fv = (double)__ldg(base + dx + p.nx * (dy + p.ny * dz));
                    const double wx = dx ? u[0] : 1.0 - u[0], wy = dy ? u[1] : 1.0 - u[1], wz = dz ? u[2] : 1.0 - u[2];
                    const double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
                    F += wx * wy * wz * fv;
                    G0 += sx * wy * wz * fv;
                    G1 += wx * sy * wz * fv;
                    G2 += wx * wy * sz * fv;
                    H01 += sx * sy * wz * fv;
                    H02 += sx * wy * sz * fv;
                    H12 += wx * sy * sz * fv;
                }
        const double gn = sqrt(G0 * G0 + G1 * G1 + G2 * G2);
        const double r = F - p.k;
        double g[3] = {0.0, 0.0, 0.0};
        if (gn > 0.0) {
            acc += fabs(r) / gn;
            const double s = (r > 0.0) ? 1.0 : (r < 0.0) ? -1.0 : 0.0;
            const double hg0 = H01 * G1 + H02 * G2, hg1 = H01 * G0 + H12 * G2, hg2 = H02 * G0 + H12 * G1;
            const double a3 = fabs(r) / (gn * gn * gn);
            g[0] = (s * G0 / gn - a3 * hg0) * invn;
            g[1] = (s * G1 / gn - a3 * hg1) * invn;
            g[2] = (s * G2 / gn - a3 * hg2) * invn;
        }
        if (p.grad) {
            p.grad[3 * v + 0] = (float)g[0];
            p.grad[3 * v + 1] = (float)g[1];
            p.grad[3 * v + 2] = (float)g[2];
        }
    }
    // fixed-shape block reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(CHR_FULL_MASK, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kLossThreads / 32; w++) t += s_w[w];
        p.partial[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kLossThreads) k_loss_sum(const __grid_constant__ LossParams p)
{
    __shared__ double s_w[kLossThreads / 32];
    double acc = 0.0;
    for (uint32_t b = threadIdx.x; b < p.nblocks; b += kLossThreads) acc += p.partial[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(CHR_FULL_MASK, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kLossThreads / 32; w++) t += s_w[w];
        *p.loss = (p.npts > 0) ? t / (double)p.npts : 0.0;
    }
}

uint32_t loss_blocks(uint64_t npts)
{
    const uint64_t want = (npts + kLossThreads - 1) / kLossThreads;
    return (uint32_t)(want < 2048 ? (want > 0 ? want : 1) : 2048);  // fixed for a given npts
}

}  // namespace

size_t dist_loss_workspace_bytes(uint64_t npts) { return (size_t)loss_blocks(npts) * sizeof(double) + 256; }

cudaError_t launch_dist_loss(const float *orig, const Grid &g, float k, const float *pts, uint64_t npts, double *loss,
                             float *grad_pts, void *workspace, cudaStream_t s)
{
    LossParams p;
    p.f = orig;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.k = (double)k;
    p.pts = pts;
    p.npts = npts;
    p.grad = grad_pts;
    p.partial = reinterpret_cast<double *>(workspace);
    p.loss = loss;
    p.nblocks = loss_blocks(npts);
    k_dist_loss<<<p.nblocks, kLossThreads, 0, s>>>(p);
    k_loss_sum<<<1, kLossThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace chr

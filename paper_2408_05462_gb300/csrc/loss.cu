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
// result does not depend on scheduling.  Arithmetic in float64, the
// interpolation separable (x, then y, then z) and one reciprocal per point.
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
        // separable trilinear interpolation: along x for the four (y, z)
        // edges, then y, then z, carrying the derivatives along
        double a[2][2], b[2][2];  // [dz][dy]: value and x-derivative on the x-edge
#pragma unroll
        for (int dz = 0; dz < 2; dz++)
#pragma unroll
            for (int dy = 0; dy < 2; dy++) {
                const float *e = base + p.nx * (dy + p.ny * dz);
                const double f0 = (double)__ldg(e), f1 = (double)__ldg(e + 1);
                b[dz][dy] = f1 - f0;
                a[dz][dy] = fma(u[0], b[dz][dy], f0);
            }
        double Fz[2], Gyz[2], Gxz[2], Hxyz[2];
#pragma unroll
        for (int dz = 0; dz < 2; dz++) {
            Gyz[dz] = a[dz][1] - a[dz][0];
            Fz[dz] = fma(u[1], Gyz[dz], a[dz][0]);
            Hxyz[dz] = b[dz][1] - b[dz][0];
            Gxz[dz] = fma(u[1], Hxyz[dz], b[dz][0]);
        }
        const double G2 = Fz[1] - Fz[0];
        const double F = fma(u[2], G2, Fz[0]);
        const double H12 = Gyz[1] - Gyz[0], H02 = Gxz[1] - Gxz[0], H01d = Hxyz[1] - Hxyz[0];
        const double G1 = fma(u[2], H12, Gyz[0]);
        const double G0 = fma(u[2], H02, Gxz[0]);
        const double H01 = fma(u[2], H01d, Hxyz[0]);
        const double gn = sqrt(G0 * G0 + G1 * G1 + G2 * G2);
        const double r = F - p.k;
        double g[3] = {0.0, 0.0, 0.0};
        if (gn > 0.0) {
            const double inv = 1.0 / gn;
            const double ar = fabs(r) * inv;
            acc += ar;
            const double s = (r > 0.0) ? 1.0 : (r < 0.0) ? -1.0 : 0.0;
            const double hg0 = H01 * G1 + H02 * G2, hg1 = H01 * G0 + H12 * G2, hg2 = H02 * G0 + H12 * G1;
            const double a3 = ar * inv * inv;
            g[0] = (s * G0 * inv - a3 * hg0) * invn;
            g[1] = (s * G1 * inv - a3 * hg1) * invn;
            g[2] = (s * G2 * inv - a3 * hg2) * invn;
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

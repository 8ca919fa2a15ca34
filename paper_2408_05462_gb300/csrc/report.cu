// Two reductions over whole fields that the library's reports need, so that
// no step of them runs as host or framework arithmetic:
// * the sum of |g| over every 8^3 brick (the bricks whose refinement moves a
//   differentiable loss most, from the adjoint's gradient field);
// * the number of cells whose marching-cubes case at each isovalue is the
//   same in two fields: the topology accuracy of Sec. 2.2 (the share of
//   cells whose isosurface topology survives compression).
#include <math.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.h"

namespace chr {

namespace {

constexpr int kRepWarps = 8;

// One warp per brick (bricks x fastest), each lane two x-rows of 8 vertices
// (y = lane & 7, z = lane >> 3 and z + 4): the lane's sum in x order, then
// a butterfly over the warp, so the result does not depend on scheduling.
__global__ void __launch_bounds__(kRepWarps * 32) k_brick_abs_sum(const float *__restrict__ g, Grid G,
                                                                  float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * kRepWarps + (threadIdx.x >> 5);
    if (b >= G.nbricks) return;
    const int64_t bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
    const int64_t x0 = 8 * bx, y = 8 * by + (lane & 7);
    const int ex = (int)((G.nx - x0) < 8 ? (G.nx - x0) : 8);
    float acc = 0.0f;
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const int64_t z = 8 * bz + (lane >> 3) + 4 * s;
        if (y >= G.ny || z >= G.nz) continue;
        const float *row = g + x0 + G.nx * (y + G.ny * z);
#pragma unroll
        for (int x = 0; x < 8; x++)
            if (x < ex) acc = __fadd_rn(acc, fabsf(__ldg(row + x)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(CHR_FULL_MASK, acc, o));
    if (lane == 0) out[b] = acc;
}

constexpr int kAgreeThreads = 256;

struct AgreeIso {
    float k[CHR_MAX_ISO];
    int n;
};

// Cells (x fastest) over a grid-stride loop: a cell agrees at k when every
// corner lies on the same side of k (v < k, NaN outside) in both fields.
__global__ void __launch_bounds__(kAgreeThreads) k_case_agreement(const float *__restrict__ a,
                                                                  const float *__restrict__ b, Grid G,
                                                                  const __grid_constant__ AgreeIso K,
                                                                  unsigned long long *count)
{
    __shared__ unsigned long long s_w[kAgreeThreads / 32];
    const int64_t cx = G.nx - 1, cy = G.ny - 1, ncells = cx * cy * (G.nz - 1);
    unsigned long long n = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = c % cx, y = (c / cx) % cy, z = c / (cx * cy);
        const int64_t i0 = x + G.nx * (y + G.ny * z);
        float va[8], vb[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int64_t i = i0 + (j & 1) + G.nx * (((j >> 1) & 1) + G.ny * ((j >> 2) & 1));
            va[j] = __ldg(a + i);
            vb[j] = __ldg(b + i);
        }
        for (int t = 0; t < K.n; t++) {
            const float k = K.k[t];
            bool same = true;
#pragma unroll
            for (int j = 0; j < 8; j++) same &= ((va[j] < k) == (vb[j] < k));
            n += same ? 1u : 0u;
        }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(CHR_FULL_MASK, n, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kAgreeThreads / 32; w++) t += s_w[w];
        if (t) atomicAdd(count, t);
    }
}

}  // namespace

cudaError_t launch_brick_abs_sum(const float *g, const Grid &G, float *out, cudaStream_t s)
{
    if (G.nbricks == 0) return cudaSuccess;
    const int64_t blocks = (G.nbricks + kRepWarps - 1) / kRepWarps;
    k_brick_abs_sum<<<(unsigned)blocks, kRepWarps * 32, 0, s>>>(g, G, out);
    return cudaGetLastError();
}

cudaError_t launch_case_agreement(const float *a, const float *b, const Grid &G, const float *K, int nK,
                                  unsigned long long *count, cudaStream_t s)
{
    if (nK < 1 || nK > CHR_MAX_ISO) return cudaErrorInvalidValue;
    AgreeIso iso;
    for (int t = 0; t < CHR_MAX_ISO; t++) iso.k[t] = (t < nK) ? K[t] : 0.0f;
    iso.n = nK;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ncells = (G.nx - 1) * (G.ny - 1) * (G.nz - 1);
    const int64_t want = (ncells + kAgreeThreads - 1) / kAgreeThreads;
    const int64_t blocks = want < 8LL * sms ? want : 8LL * sms;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || blocks == 0) return e;
    k_case_agreement<<<(unsigned)blocks, kAgreeThreads, 0, s>>>(a, b, G, iso, count);
    return cudaGetLastError();
}

}  // namespace chr

namespace {

bool report_dims_ok(chr_dims d, const char *who)
{
    if (d.nx < 2 || d.ny < 2 || d.nz < 2 || d.nx > (1ll << 31) || d.ny > (1ll << 31) || d.nz > (1ll << 31) ||
        (double)d.nx * (double)d.ny * (double)d.nz >= 4294967295.0) {
        chr::fail(CHR_ERR_INVALID, std::string(who) + ": dims must be >= 2 along every axis and nx*ny*nz < 2^32");
        return false;
    }
    return true;
}

}  // namespace

extern "C" chr_status chr_brick_abs_sum(const float *d_g, chr_dims dims, float *d_out, void *stream)
{
    nvtxRangePushA("chr_brick_abs_sum");
    chr_status st = CHR_OK;
    if (!d_g || !d_out)
        st = chr::fail(CHR_ERR_INVALID, "chr_brick_abs_sum: NULL argument");
    else if ((reinterpret_cast<uintptr_t>(d_g) & 3u) || (reinterpret_cast<uintptr_t>(d_out) & 3u))
        st = chr::fail(CHR_ERR_INVALID, "chr_brick_abs_sum: misaligned pointer");
    else if (!report_dims_ok(dims, "chr_brick_abs_sum"))
        st = CHR_ERR_INVALID;
    else {
        const cudaError_t e = chr::launch_brick_abs_sum(d_g, chr::make_grid(dims), d_out, (cudaStream_t)stream);
        if (e != cudaSuccess) st = chr::cuda_fail(e, "chr_brick_abs_sum");
    }
    nvtxRangePop();
    return st;
}

extern "C" chr_status chr_case_agreement(const float *d_a, const float *d_b, chr_dims dims, const float *isovalues,
                                         uint32_t n_iso, unsigned long long *d_count, void *stream)
{
    nvtxRangePushA("chr_case_agreement");
    chr_status st = CHR_OK;
    if (!d_a || !d_b || !isovalues || !d_count)
        st = chr::fail(CHR_ERR_INVALID, "chr_case_agreement: NULL argument");
    else if (n_iso < 1 || n_iso > CHR_MAX_ISO)
        st = chr::fail(CHR_ERR_INVALID, "chr_case_agreement: n_iso must be 1..16");
    else if ((reinterpret_cast<uintptr_t>(d_a) & 3u) || (reinterpret_cast<uintptr_t>(d_b) & 3u) ||
             (reinterpret_cast<uintptr_t>(d_count) & 7u))
        st = chr::fail(CHR_ERR_INVALID, "chr_case_agreement: misaligned pointer");
    else if (!report_dims_ok(dims, "chr_case_agreement"))
        st = CHR_ERR_INVALID;
    else {
        for (uint32_t t = 0; t < n_iso; t++)
            if (isnan(isovalues[t])) {
                st = chr::fail(CHR_ERR_INVALID, "chr_case_agreement: NaN isovalue");
                break;
            }
        if (st == CHR_OK) {
            const cudaError_t e = chr::launch_case_agreement(d_a, d_b, chr::make_grid(dims), isovalues, (int)n_iso,
                                                             d_count, (cudaStream_t)stream);
            if (e != cudaSuccess) st = chr::cuda_fail(e, "chr_case_agreement");
        }
    }
    nvtxRangePop();
    return st;
}

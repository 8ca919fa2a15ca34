// Error-bound translation (paper Sec. 2.2): the multiset D of d0 = k - s0 and
// d1 = s1 - k over every grid edge with s0 < k < s1, and its smallest or n-th
// smallest element.  D is never materialised: each pass walks the edges again
// and either takes the minimum (accuracy 1) or builds a 256-bin histogram of
// the next 8 bits of the float patterns that match the prefix chosen so far
// (radix selection; non-negative floats order like their bit patterns).
#include "common.cuh"
#include "internal.h"

namespace chr {

namespace {

struct TrParams {
    const float *f;
    int64_t nx, ny, nz, N;
    int32_t nK;
    float K[CHR_MAX_ISO];
    int32_t pass;     // 0..3: histogram of bits [24-8*pass, 32-8*pass)
    uint32_t prefix;  // the top 8*pass bits already selected
    int32_t min_only;
    TranslateScratch sc;
};

__global__ void __launch_bounds__(256) k_translate(const __grid_constant__ TrParams p)
{
    __shared__ unsigned int s_hist[8 * 256];  // one histogram per warp: fewer collisions
    __shared__ unsigned long long s_cnt;
    __shared__ unsigned int s_min;
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) s_hist[i] = 0u;
    if (threadIdx.x == 0) {
        s_cnt = 0ull;
        s_min = 0xffffffffu;
    }
    __syncthreads();

    unsigned long long cnt = 0;
    unsigned int mn = 0xffffffffu;
    unsigned int *wh = s_hist + 256 * (threadIdx.x >> 5);  // this warp's histogram
    const int shift = 24 - 8 * p.pass;
    // rows (y, z) are spread over the grid, x over the threads of a block
    const int64_t nrows = p.ny * p.nz;
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        const uint32_t y = (uint32_t)row % (uint32_t)p.ny;  // rows < 2^32
        const bool has_y = (int64_t)y + 1 < p.ny, has_z = row + p.ny < nrows;
        const float *src = p.f + row * p.nx;
        for (int32_t x = threadIdx.x; x < p.nx; x += blockDim.x) {
            const float s = __ldg(src + x);
            const bool has[3] = {x + 1 < p.nx, has_y, has_z};
            const int64_t off[3] = {1, p.nx, p.nx * p.ny};
#pragma unroll
            for (int a = 0; a < 3; a++) {
                if (!has[a]) continue;
                float lo = s, hi = __ldg(src + x + off[a]);
                if (hi < lo) {
                    const float t = lo;
                    lo = hi;
                    hi = t;
                }
                for (int j = 0; j < p.nK; j++) {
                    const float k = p.K[j];
                    if (!(lo < k && k < hi)) continue;
                    const uint32_t d[2] = {__float_as_uint(__fsub_rd(k, lo)), __float_as_uint(__fsub_rd(hi, k))};
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        cnt++;
                        if (p.min_only) {
                            mn = min(mn, d[u]);
                        } else if (p.pass == 0 || (d[u] >> (shift + 8)) == p.prefix) {
                            atomicAdd(&wh[(d[u] >> shift) & 255u], 1u);
                        }
                    }
                }
            }
        }
    }
    // block reduction, then one global update per block
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(CHR_FULL_MASK, cnt, o);
        mn = min(mn, __shfl_xor_sync(CHR_FULL_MASK, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(&s_cnt, cnt);
        atomicMin(&s_min, mn);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cnt && p.pass == 0) atomicAdd(p.sc.count, s_cnt);
        if (p.min_only) atomicMin(p.sc.minbits, s_min);
    }
    if (!p.min_only) {
        unsigned long long h = 0;
        for (int w = 0; w < 8; w++) h += s_hist[256 * w + threadIdx.x];
        if (h) atomicAdd(p.sc.hist + threadIdx.x, h);
    }
}

}  // namespace

size_t translate_scratch_bytes() { return 256 * sizeof(unsigned long long) + 64; }

cudaError_t launch_translate_pass(const float *field, const Grid &g, const float *K, int nK, int pass, uint32_t prefix,
                                  bool min_only, TranslateScratch sc, cudaStream_t s)
{
    TrParams p;
    p.f = field;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.N = g.N;
    p.nK = nK;
    for (int j = 0; j < CHR_MAX_ISO; j++) p.K[j] = (j < nK) ? K[j] : 0.0f;
    p.pass = pass;
    p.prefix = prefix;
    p.min_only = min_only ? 1 : 0;
    p.sc = sc;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = g.ny * g.nz;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    k_translate<<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace chr

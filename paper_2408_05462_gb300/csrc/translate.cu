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
    __shared__ unsigned int s_hist[256];
    __shared__ unsigned long long s_cnt;
    __shared__ unsigned int s_min;
    s_hist[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        s_cnt = 0ull;
        s_min = 0xffffffffu;
    }
    __syncthreads();

    unsigned long long cnt = 0;
    unsigned int mn = 0xffffffffu;
    const int shift = 24 - 8 * p.pass;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.N; i += stride) {
        const int64_t x = i % p.nx, y = (i / p.nx) % p.ny, z = i / (p.nx * p.ny);
        const float s = __ldg(p.f + i);
        const bool has[3] = {x + 1 < p.nx, y + 1 < p.ny, z + 1 < p.nz};
        const int64_t off[3] = {1, p.nx, p.nx * p.ny};
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (!has[a]) continue;
            float lo = s, hi = __ldg(p.f + i + off[a]);
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
                        atomicAdd(&s_hist[(d[u] >> shift) & 255u], 1u);
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
    if (!p.min_only && s_hist[threadIdx.x]) atomicAdd(p.sc.hist + threadIdx.x, (unsigned long long)s_hist[threadIdx.x]);
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
    int64_t blocks = (g.N + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    k_translate<<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace chr

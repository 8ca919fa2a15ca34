// Device helpers shared by the libchr kernels (not by the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "chr.h"

#define CHR_FULL_MASK 0xffffffffu
#define CHR_QMAX 8388607.0f  // 2^23 - 1: codes stay exact in float32

// Bounded waits: a poll loop gives up after this many polls (each followed by
// a short sleep), raises CHR_ERR_TIMEOUT in the error word and moves on.
#define CHR_SPIN_LIMIT (1u << 22)

// Checked builds (-DCHR_CHECKED: libchr_checked.so, for tests): every
// CHR_IN_BOUNDS(cond) on a hot path tests an index bound; a failed test sets
// the translation unit's bounds word (declared by CHR_BOUNDS_WORD(), read
// by chr_debug_bounds_word) and the caller skips the access.  Normal builds
// compile the tests away.
#ifdef CHR_CHECKED
#define CHR_BOUNDS_WORD() __device__ unsigned int g_chr_bounds = 0u
#define CHR_IN_BOUNDS(cond) ::chr::in_bounds_checked((cond), &g_chr_bounds)
#else
#define CHR_BOUNDS_WORD() static_assert(true, "")
#define CHR_IN_BOUNDS(cond) true
#endif

namespace chr {

__device__ __forceinline__ bool in_bounds_checked(bool c, unsigned int *word)
{
    if (!c) atomicOr(word, 1u);
    return c;
}

__device__ __forceinline__ uint32_t zigzag(int32_t d) { return ((uint32_t)d << 1) ^ (uint32_t)(d >> 31); }

__device__ __forceinline__ int32_t unzigzag(uint32_t z) { return (int32_t)(z >> 1) ^ -(int32_t)(z & 1u); }

__device__ __forceinline__ int bitlen(uint32_t v) { return 32 - __clz(v); }

__device__ __forceinline__ uint32_t width_mask(int w) { return (w >= 32) ? 0xffffffffu : ((1u << w) - 1u); }

// Streaming 16-byte load that bypasses L1 allocation (data read once).
__device__ __forceinline__ uint4 ld_stream_u4(const uint4 *p)
{
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ float4 ld_stream_f4(const float4 *p)
{
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CHR_FULL_MASK, v, o);
    return v;
}

// Inclusive warp scan of a 64-bit value.
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(CHR_FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(CHR_FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// One level of the residual chain for one vertex (paper Sec. 2 accuracy
// levels; Sec. 2.2 sign preservation).  Every float operation is one IEEE
// binary32 operation rounded to nearest-even, so the result is identical on
// every device and on the host.  Returns true for a vertex stored exactly.
__device__ __forceinline__ bool level_step(float f, float Rprev, bool first, float e, float two_e, float inv2e,
                                           const float *K, int nK, bool fix, int32_t &q, float &R)
{
    float r = first ? f : __fsub_rn(f, Rprev);
    float x = __fmul_rn(r, inv2e);
    bool exc = !(fabsf(x) <= CHR_QMAX);
    q = 0;
    R = f;
    if (!exc) {
        int32_t qi = __float2int_rn(x);  // round half to even
        float P = __fmul_rn(__int2float_rn(qi), two_e);
        float Rn = first ? P : __fadd_rn(Rprev, P);
        float err = __fsub_rn(f, Rn);
        exc = !(fabsf(err) < e);
        if (!exc && fix) {
            for (int j = 0; j < nK; j++) exc |= ((Rn < K[j]) != (f < K[j]));
        }
        if (!exc) {
            q = qi;
            R = Rn;
        }
    }
    return exc;
}

}  // namespace chr

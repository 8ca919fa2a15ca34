// TMA (cp.async.bulk.tensor) and mbarrier helpers, inline PTX for sm_100+.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include "common.cuh"

namespace chr {

// Host: a 3-D tiled tensor map over a float32 field [nz][ny][nx] with box
// (bx, by, bz).  Out-of-range box elements read as zero.  Returns false when
// the field cannot be described (nx*4 not a multiple of 16, base not 16-byte
// aligned, or the driver entry point is missing); callers then fall back to
// plain loads.
// The field may be pitched: row y of plane z starts at f + sx*y + sy*z
// (sx >= nx, sy >= sx*ny, both multiples of 4 floats).
inline bool make_field_tensor_map_pitched(CUtensorMap *map, const float *f, int64_t nx, int64_t ny, int64_t nz,
                                          int64_t sx, int64_t sy, uint32_t bx, uint32_t by, uint32_t bz)
{
    if ((sx & 3) != 0 || (sy & 3) != 0 || (reinterpret_cast<uintptr_t>(f) & 15u) != 0) return false;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    }
    if (!encode) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)sx * 4, (cuuint64_t)sy * 4};
    const cuuint32_t box[3] = {bx, by, bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(f), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline bool make_field_tensor_map(CUtensorMap *map, const float *f, int64_t nx, int64_t ny, int64_t nz, uint32_t bx,
                                  uint32_t by, uint32_t bz)
{
    return make_field_tensor_map_pitched(map, f, nx, ny, nz, nx, nx * ny, bx, by, bz);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the mbarrier phase `parity` to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    const uint32_t a = smem_addr(mbar);
    for (uint32_t i = 0; i < CHR_SPIN_LIMIT; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

// One 3-D box of the tensor map at element coordinates (x, y, z) into dst
// (128-byte aligned shared memory); completion is signalled on mbar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, int32_t z,
                                            uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(mbar))
        : "memory");
}

// Bulk copy of `bytes` (a multiple of 16) from shared memory to global
// memory through the async proxy; both addresses 16-byte aligned.  The
// writing threads must have run fence_proxy_async_smem() on the data first.
__device__ __forceinline__ void bulk_store(void *gdst, const void *ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// The shared-memory sources of every committed bulk store have been read.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Every committed bulk store has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace chr

// isosurface_extract_noalloc: marching cubes for callers that cannot
// allocate device memory.
//
// Some callers are not allowed to call cudaMalloc: code that runs inside a
// host application or framework that owns all device memory through its own
// pool, plugins and callbacks that must not allocate, and latency-bound loops
// where an allocation (which may synchronise the device) is not acceptable.
// For them this entry point takes its scratch (per-tile triangle counts and
// offsets) from one fixed array that lives in this library's device image,
// so the caller provides only the field, the isovalues and the outputs.
//
// The array holds kNoallocScratchBytes bytes on every GPU that loads the
// library, for as long as the process runs.  Every call uses all of it, so
// calls whose work overlaps on a GPU (for example on two streams) race on it;
// serialise them.  Each call overwrites every scratch byte it reads before
// reading it, so nothing needs clearing between calls.
#include <string>

#include "internal.h"

namespace chr {

namespace {

constexpr size_t kNoallocScratchBytes = size_t(4) << 20;  // 4 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  The host-side
// name of a __device__ array is not a device address, so the address is
// looked up with the device current, at every call (cheap once the module
// is loaded, and right after a device reset too).
cudaError_t noalloc_scratch(void **out)
{
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = ptr;
    return cudaSuccess;
}

}  // namespace

}  // namespace chr

using namespace chr;

extern "C" chr_status isosurface_extract_noalloc(const float *d_field, chr_dims dims, const float *isovalues,
                                                 uint32_t n_iso, float *d_tris, uint64_t cap_tris,
                                                 uint64_t *d_ntris, uint32_t *d_err, void *stream)
{
    if (dims.nx >= 2 && dims.ny >= 2 && dims.nz >= 2 && dims.nx < (1ll << 31) && dims.ny < (1ll << 31) &&
        dims.nz < (1ll << 31) && (double)dims.nx * (double)dims.ny * (double)dims.nz < 4294967295.0) {
        const size_t need = mc_workspace_min_bytes(make_grid(dims), (int)n_iso);
        if (need > kNoallocScratchBytes) {
            set_error("isosurface_extract_noalloc: grid needs " + std::to_string(need) +
                      " bytes of scratch, more than the fixed " + std::to_string(kNoallocScratchBytes) +
                      "; use isosurface_extract with a caller-provided workspace");
            return CHR_ERR_INVALID;
        }
    }
    void *scratch = nullptr;
    const cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) {
        set_error(std::string("isosurface_extract_noalloc: scratch lookup failed: ") + cudaGetErrorString(e));
        return CHR_ERR_CUDA;
    }
    // the minimum workspace: every group of isovalues takes the single pass
    size_t ws = kNoallocScratchBytes;
    if (dims.nx >= 2 && dims.ny >= 2 && dims.nz >= 2) ws = mc_workspace_min_bytes(make_grid(dims), (int)n_iso);
    return isosurface_extract(d_field, dims, isovalues, n_iso, d_tris, cap_tris, d_ntris, d_err, scratch, ws,
                              stream);
}

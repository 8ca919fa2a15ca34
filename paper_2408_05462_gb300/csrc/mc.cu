// Marching cubes over a float32 field (paper Sec. 2.2; Lorensen & Cline):
// per-cell case classification for up to 4 isovalues from one read of the
// field, a block scan of triangle counts, a single-pass decoupled look-back
// (Merrill & Garland) for the global output offsets, and edge interpolation
// + triangle emission.
//
// Tile = 4 cell bricks along x = 32x8x8 cells; a block of 256 threads stages
// the tile's 33x9x9 vertices in shared memory.  Thread t owns brick t>>6 of
// the tile and the 8 cells of row (y,z) = (t&7, (t>>3)&7) of that brick, so
// thread order is the output order: bricks x-fastest, cells x-fastest.
#include "common.cuh"
#include "internal.h"
#include "mc_table.h"

namespace chr {

namespace {

__device__ const uint64_t g_mc_case[256] = CHR_MC_CASE_INIT;

constexpr int kTX = 8 * kMcBricksX;  // cells per tile along x
constexpr int kVX = kTX + 1;         // vertices per staged row
constexpr int kPlane = 9 * kVX;      // floats per staged z-plane

struct McParams {
    const float *f;
    int64_t nx, ny, nz;
    int32_t ntx, ncby, ncbz;  // tiles along x; cell bricks along y, z
    int64_t ntiles;
    float k[kMcIsoPerPass];
    float *tris[kMcIsoPerPass];
    uint64_t cap;
    uint64_t *ntris;  // [niso of this pass]
    uint32_t *err;
    uint64_t *status;            // [ntiles][4]: count << 2 | flag (1 aggregate, 2 inclusive)
    unsigned long long *counter; // dynamic tile ids, in launch order
};

// Exclusive prefix of the tiles before `tile` for one isovalue slot: a warp
// inspects 32 predecessors at a time and stops at the first one that has
// published its inclusive prefix.  Every poll loop is bounded.
__device__ uint64_t lookback(const McParams &p, int64_t tile, int slot, int lane)
{
    uint64_t excl = 0;
    int64_t base = tile - 1;
    while (true) {
        const int64_t t = base - lane;
        uint64_t v = 2ull;  // before tile 0: an inclusive prefix of 0
        uint32_t spins = 0;
        while (true) {
            if (t >= 0) v = ld_relaxed_u64(p.status + t * kMcIsoPerPass + slot);
            const bool ready = (v & 3ull) != 0;
            if (__all_sync(CHR_FULL_MASK, ready)) break;
            if (++spins > CHR_SPIN_LIMIT) {
                if (!ready) v = 2ull;
                if (lane == 0 && p.err) atomicOr(p.err, 1u << CHR_ERR_TIMEOUT);
                break;
            }
            __nanosleep(100);
        }
        const uint32_t incl = __ballot_sync(CHR_FULL_MASK, (v & 3ull) == 2ull);
        if (incl) {
            const int first = __ffs(incl) - 1;
            excl += warp_sum_u64(lane <= first ? (v >> 2) : 0ull);
            return excl;
        }
        excl += warp_sum_u64(v >> 2);
        base -= 32;
    }
}

__device__ __forceinline__ void emit_triangle(float *dst, uint64_t word, int t, const float *cell, float k, float cx,
                                              float cy, float cz)
{
    float out[9];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int e = (int)((word >> (12 * t + 4 * c)) & 15u);
        const int axis = e >> 2, m = e & 3;
        const int ox = (axis == 0) ? 0 : (m & 1);
        const int oy = (axis == 1) ? 0 : ((axis == 0) ? (m & 1) : (m >> 1));
        const int oz = (axis == 2) ? 0 : (m >> 1);
        const float *p0 = cell + ox + oy * kVX + oz * kPlane;
        const int step = (axis == 0) ? 1 : (axis == 1) ? kVX : kPlane;
        const float f0 = p0[0], f1 = p0[step];
        const float tt = __fdiv_rn(__fsub_rn(k, f0), __fsub_rn(f1, f0));
        float px = cx + (float)ox, py = cy + (float)oy, pz = cz + (float)oz;
        if (axis == 0) px = __fadd_rn(px, tt);
        if (axis == 1) py = __fadd_rn(py, tt);
        if (axis == 2) pz = __fadd_rn(pz, tt);
        out[3 * c + 0] = px;
        out[3 * c + 1] = py;
        out[3 * c + 2] = pz;
    }
#pragma unroll
    for (int i = 0; i < 9; i++) __stcs(dst + i, out[i]);
}

template <int NISO>
__global__ void __launch_bounds__(256) k_mc(const __grid_constant__ McParams p)
{
    __shared__ float s_f[9 * kPlane];
    __shared__ uint64_t s_tab[256];
    __shared__ uint64_t s_warp[9];
    __shared__ uint64_t s_prefix[kMcIsoPerPass];
    __shared__ long long s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_tab[tid] = g_mc_case[tid];
    if (tid == 0) s_tile = (long long)atomicAdd(p.counter, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    const int32_t tx = (int32_t)(tile % p.ntx);
    const int32_t by = (int32_t)((tile / p.ntx) % p.ncby);
    const int32_t bz = (int32_t)(tile / ((int64_t)p.ntx * p.ncby));
    const int64_t gx0 = (int64_t)tx * kTX, gy0 = (int64_t)by * 8, gz0 = (int64_t)bz * 8;

    // stage the tile's vertices (out-of-grid entries are never used by a valid cell)
    for (int i = tid; i < 9 * kPlane; i += 256) {
        const int lx = i % kVX, r = i / kVX, ly = r % 9, lz = r / 9;
        const int64_t gx = gx0 + lx, gy = gy0 + ly, gz = gz0 + lz;
        float v = 0.0f;
        if (gx < p.nx && gy < p.ny && gz < p.nz) v = __ldg(p.f + gx + p.nx * (gy + p.ny * gz));
        s_f[i] = v;
    }
    __syncthreads();

    // classify this thread's 8 cells for every isovalue
    const int j = tid >> 6, ly = tid & 7, lz = (tid >> 3) & 7;
    const int64_t cx0 = gx0 + 8 * j, cy = gy0 + ly, cz = gz0 + lz;
    int nvalid = 0;
    if (cy < p.ny - 1 && cz < p.nz - 1 && cx0 < p.nx - 1) nvalid = (int)((p.nx - 1 - cx0) < 8 ? (p.nx - 1 - cx0) : 8);
    const float *row = s_f + lz * kPlane + ly * kVX + 8 * j;
    uint32_t m[NISO][4];
#pragma unroll
    for (int i = 0; i < NISO; i++) m[i][0] = m[i][1] = m[i][2] = m[i][3] = 0u;
#pragma unroll
    for (int x = 0; x < 9; x++) {
        const float v0 = row[x], v1 = row[kVX + x], v2 = row[kPlane + x], v3 = row[kPlane + kVX + x];
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            const float k = p.k[i];
            m[i][0] |= (uint32_t)(v0 < k) << x;
            m[i][1] |= (uint32_t)(v1 < k) << x;
            m[i][2] |= (uint32_t)(v2 < k) << x;
            m[i][3] |= (uint32_t)(v3 < k) << x;
        }
    }
    uint64_t packed = 0;
#pragma unroll
    for (int i = 0; i < NISO; i++) {
        uint32_t cnt = 0;
        for (int x = 0; x < nvalid; x++) {
            const uint32_t cs = ((m[i][0] >> x) & 3u) | (((m[i][1] >> x) & 3u) << 2) | (((m[i][2] >> x) & 3u) << 4) |
                                (((m[i][3] >> x) & 3u) << 6);
            cnt += (uint32_t)(s_tab[cs] >> 60);
        }
        packed |= (uint64_t)cnt << (16 * i);
    }

    // block scan (4 x 16-bit lanes in one 64-bit word; a tile has < 2^16 triangles per isovalue)
    const uint64_t inc = warp_incl_scan_u64(packed, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t t = (lane < 8) ? s_warp[lane] : 0ull;
        const uint64_t ti = warp_incl_scan_u64(t, lane);
        if (lane < 8) s_warp[lane] = ti - t;
        if (lane == 7) s_warp[8] = ti;
    }
    __syncthreads();
    const uint64_t thread_excl = s_warp[warp] + inc - packed;
    const uint64_t block_total = s_warp[8];

    if (warp == 0) {
        uint64_t *st = p.status + tile * kMcIsoPerPass;
        if (lane == 0 && tile > 0)
            for (int i = 0; i < NISO; i++) st_relaxed_u64(st + i, (((block_total >> (16 * i)) & 0xffffull) << 2) | 1ull);
        for (int i = 0; i < NISO; i++) {
            const uint64_t tot = (block_total >> (16 * i)) & 0xffffull;
            const uint64_t ex = (tile > 0) ? lookback(p, tile, i, lane) : 0ull;
            if (lane == 0) {
                st_relaxed_u64(st + i, ((ex + tot) << 2) | 2ull);
                s_prefix[i] = ex;
                if (tile == p.ntiles - 1) p.ntris[i] = ex + tot;
            }
        }
    }
    __syncthreads();

    // emit
#pragma unroll
    for (int i = 0; i < NISO; i++) {
        uint64_t idx = s_prefix[i] + ((thread_excl >> (16 * i)) & 0xffffull);
        const float k = p.k[i];
        float *out = p.tris[i];
        for (int x = 0; x < nvalid; x++) {
            const uint32_t cs = ((m[i][0] >> x) & 3u) | (((m[i][1] >> x) & 3u) << 2) | (((m[i][2] >> x) & 3u) << 4) |
                                (((m[i][3] >> x) & 3u) << 6);
            const uint64_t word = s_tab[cs];
            const int nt = (int)(word >> 60);
            for (int t = 0; t < nt; t++, idx++)
                if (idx < p.cap)
                    emit_triangle(out + 9 * idx, word, t, row + x, k, (float)(cx0 + x), (float)cy, (float)cz);
        }
        if (idx > p.cap && p.err) atomicOr(p.err, 1u << CHR_ERR_OVERFLOW);
    }
}

}  // namespace

static void mc_tiles(const Grid &g, int32_t &ntx, int32_t &ncby, int32_t &ncbz, int64_t &ntiles)
{
    const int64_t ncbx = (g.nx - 1 + 7) / 8;
    ntx = (int32_t)((ncbx + kMcBricksX - 1) / kMcBricksX);
    ncby = (int32_t)((g.ny - 1 + 7) / 8);
    ncbz = (int32_t)((g.nz - 1 + 7) / 8);
    ntiles = (int64_t)ntx * ncby * ncbz;
}

size_t mc_workspace_bytes(const Grid &g, int n_iso)
{
    (void)n_iso;  // passes of 4 isovalues reuse the same status words
    int32_t ntx, ncby, ncbz;
    int64_t ntiles;
    mc_tiles(g, ntx, ncby, ncbz, ntiles);
    return 256 + (size_t)ntiles * kMcIsoPerPass * sizeof(uint64_t);
}

cudaError_t launch_mc(const float *field, const Grid &g, const float *iso, int n_iso, float *tris, uint64_t cap,
                      uint64_t *ntris, uint32_t *err, void *workspace, cudaStream_t s)
{
    McParams p;
    p.f = field;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    mc_tiles(g, p.ntx, p.ncby, p.ncbz, p.ntiles);
    p.cap = cap;
    p.err = err;
    p.counter = reinterpret_cast<unsigned long long *>(workspace);
    p.status = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(workspace) + 256);
    const size_t ws = mc_workspace_bytes(g, n_iso);
    for (int i0 = 0; i0 < n_iso; i0 += kMcIsoPerPass) {
        const int n = (n_iso - i0) < kMcIsoPerPass ? (n_iso - i0) : kMcIsoPerPass;
        for (int i = 0; i < kMcIsoPerPass; i++) {
            p.k[i] = (i < n) ? iso[i0 + i] : 0.0f;
            p.tris[i] = (i < n) ? tris + 9ull * cap * (uint64_t)(i0 + i) : nullptr;
        }
        p.ntris = ntris + i0;
        cudaError_t e = cudaMemsetAsync(workspace, 0, ws, s);
        if (e != cudaSuccess) return e;
        const dim3 grid((unsigned)p.ntiles);
        switch (n) {
            case 1: k_mc<1><<<grid, 256, 0, s>>>(p); break;
            case 2: k_mc<2><<<grid, 256, 0, s>>>(p); break;
            case 3: k_mc<3><<<grid, 256, 0, s>>>(p); break;
            default: k_mc<4><<<grid, 256, 0, s>>>(p); break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace chr

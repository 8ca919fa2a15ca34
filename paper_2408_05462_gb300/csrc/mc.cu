// Marching cubes over a float32 field (paper Sec. 2.2; Lorensen & Cline).
//
// isosurface_extract: per group of up to 4 isovalues one launch (below
// 2048 n^3 tiles for a group of n, or whenever the workspace holds only the
// tile arrays),
//   k_mc_fused  persistent blocks claim 32x8x8-cell tiles in increasing
//               order; per tile: inside masks by warp ballot, case bytes,
//               one block scan of (triangles, active cells) for every
//               isovalue, the tile's counts published and its output offset
//               found by a decoupled look-back over the tiles before it,
//               active cells compacted, triangle -> cell by a 32-triangle
//               window, edge interpolation, each chunk written by one TMA
//               bulk store
// The two-pass form serves larger grids (where the single pass's per-tile
// waits cost more than a count pass), the adjoint and the batched path,
// which keep the classification for a second walk over the same tiles:
//   k_mc_count  per tile: case bytes and triangle counts -> tile_cnt (and
//               the classification, 12 bytes per 8 cells and isovalue)
//   k_tscan_*   exclusive scan of the tile counts -> tile_off, totals
//   k_mc_emit_stored / k_mc_emit_batched / k_mc_adjoint  per tile again,
//               from the stored classification
// Every tile kernel fetches a tile's 36x9x9 vertex box with a TMA bulk
// tensor copy into one of two shared-memory buffers while another tile is
// processed; the box is zero-filled past the grid edge.  When the field
// cannot be described by a tensor map (nx*4 not a multiple of 16, or a base
// address not 16-byte aligned) the same kernels load the box with plain
// loads.
//
// Output order: 8^3-cell bricks in x-fastest order, cells of a brick
// x-fastest, triangles of a cell in table order.  A tile is 4 bricks along
// x; thread t owns brick t>>6 of the tile and the 8 cells of row
// (y, z) = (t&7, (t>>3)&7), so thread order is output order.
#include <string.h>

#include <atomic>
#include <mutex>
#include <type_traits>

#include "chr_box.cuh"
#include "common.cuh"
#include "internal.h"
#include "mc_table.h"
#include "tma.cuh"

namespace chr {

namespace {

CHR_BOUNDS_WORD();

__device__ const uint64_t g_mc_case[256] = CHR_MC_CASE_INIT;

constexpr int kTX = 8 * kMcBricksX;                    // cells per tile along x (32)
constexpr int kBoxX = kTX + 4;                         // vertices fetched per row (33 used; 144 bytes)
constexpr int kVX = kBoxX;                             // shared-memory row pitch
constexpr int kPlane = 9 * kVX;                        // floats per z-plane of the box
constexpr int kRows = 81;                              // rows of the box (9 y x 9 z)
constexpr int kTileBytes = kRows * kVX * 4;            // 11664
constexpr int kBufBytes = ((kTileBytes + 127) / 128) * 128;
constexpr int kCells = 64 * 8 * kMcBricksX;            // cells per tile (2048)
constexpr int kWarpStage = 32 * 9 + 4;                 // floats staged per warp: 32 triangles + alignment pad

// dynamic shared memory (bytes)
constexpr int kOffBuf = 0;                                       // 2 x float box
constexpr int kOffRow = 2 * kBufBytes;                           // uint64 [4][81] inside masks per row
constexpr int kOffCnt = kOffRow + kMcIsoPerPass * kRows * 8;     // uint8 [256] triangles per case
constexpr int kCountSmem = kOffCnt + 256 + 128;                  // + alignment slack
constexpr int kOffTri = kOffCnt + 256;                           // uint32 [256][5] edges of each triangle

// dynamic shared memory of the emit kernel (bytes)
// The active cells of a tile's isovalues share one pool: each isovalue's list
// is followed by 32 entries that read as "no cell here" to the chunk window.
// All lists go in together when they fit; a tile whose lists do not (more
// than about 2048 active cells over its isovalues) takes them one at a time.
constexpr int kPool = kCells + 32 * kMcIsoPerPass;                 // 2176 entries
// Chunk-table entries: at most 5 triangles per active cell, so the lists in
// the pool hold at most 10,240 triangles, plus one partial chunk per list.
constexpr int kMaxChunks = kCells * CHR_MC_MAX_TRI / 32 + 16;      // 336
constexpr int kEOffEdge = kOffTri + 256 * CHR_MC_MAX_TRI * 4;      // uint32 [16] edge words
constexpr int kEOffAct = kEOffEdge + 64;                           // uint32 [kPool] active cell | case << 11
constexpr int kEOffAPre = kEOffAct + kPool * 4;                    // uint16 [kPool] first triangle of each active cell
constexpr int kEOffChunk = kEOffAPre + kPool * 2;                  // uint16 [kMaxChunks] active cell holding triangle 32q
constexpr int kEOffStage = ((kEOffChunk + kMaxChunks * 2 + 15) / 16) * 16;  // float [8][32*9+4]
constexpr int kEmitSmem = kEOffStage + 8 * kWarpStage * 4 + 128;   // + alignment slack

struct McParams {
    const float *f;
    int64_t nx, ny, nz;
    int64_t sx, sy;           // row and plane pitch of f in floats (plain loads)
    int32_t ntx, ncby, ncbz;  // tiles along x; cell bricks along y, z
    int32_t use_tma;
    int64_t ntiles;
    float k[kMcIsoPerPass];
    float *tris[kMcIsoPerPass];
    uint64_t cap;
    uint32_t *err;
    uint4 *tile_cnt;     // [ntiles]: triangles per isovalue slot
    uint64_t *tile_off;  // [ntiles][4]: global index of the tile's first triangle
    // two-pass form (batched emit, adjoint): the count pass's classification
    // per tile, isovalue slot (cstride slots) and thread, the case bytes of
    // the thread's 8 cells and its triangles | active cells << 16
    uint2 *cases;
    uint32_t *tcnt;
    int32_t cstride;
    // single pass (k_mc_fused): per tile a status word (tile_status), its
    // inclusive prefix in tile_off once published, the tile counter blocks
    // claim tiles from, a word that a gave-up wait sets so that no other
    // block waits on it, and where the totals of the isovalue slots go
    uint64_t *tstat;
    uint32_t *tctr;
    uint32_t *tabort;
    uint64_t *ntris;
    // test only: a tile that never publishes its counts or prefix (-1: none),
    // so that the tiles after it wait out their bounded look-back
    int64_t unpublished_tile;
    // the field's value index (a CHR level's, chr_brick_index), NULL: none;
    // ibx, iby: its bricks along x and y.  A cell brick whose range does not
    // straddle an isovalue slot is not classified for it (tile_activity)
    const float2 *index;
    int32_t ibx, iby;
    // checked builds, test only: where each emitted triangle's cell index
    // (x + (nx-1)*(y + (ny-1)*z)) goes, per isovalue slot, in output order
    // (NULL: nowhere; chr_debug_tri_cells)
    uint32_t *dbg_cells[kMcIsoPerPass];
};

struct TileXYZ {
    int64_t x0, y0, z0;
};

// Tile indices fit 32 bits (a grid has < 2^32 vertices, a tile 2048 cells).
__device__ __forceinline__ TileXYZ tile_origin(const McParams &p, int64_t tile)
{
    const uint32_t t = (uint32_t)tile, ntx = (uint32_t)p.ntx, nby = (uint32_t)p.ncby;
    const uint32_t q = t / ntx, z = q / nby;
    TileXYZ o;
    o.x0 = (int64_t)(t - q * ntx) * kTX;
    o.y0 = (int64_t)(q - z * nby) * 8;
    o.z0 = (int64_t)z * 8;
    return o;
}

// Plain loads of the box (fallback when no tensor map): zero past the edges.
__device__ void load_box_plain(float *buf, const McParams &p, const TileXYZ &o)
{
    for (int i = threadIdx.x; i < kRows * kVX; i += blockDim.x) {
        const int lx = i % kVX, r = i / kVX, ly = r % 9, lz = r / 9;
        const int64_t gx = o.x0 + lx, gy = o.y0 + ly, gz = o.z0 + lz;
        buf[i] = (gx < p.nx && gy < p.ny && gz < p.nz) ? __ldg(p.f + gx + p.sx * gy + p.sy * gz) : 0.0f;
    }
}

// Thread 0 starts the box copy of `tile` into buf.
__device__ __forceinline__ void issue_box(float *buf, const CUtensorMap *map, uint64_t *mbar, const McParams &p,
                                          int64_t tile)
{
    const TileXYZ o = tile_origin(p, tile);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(mbar, (uint32_t)kTileBytes);
    tma_load_3d(buf, map, (int32_t)o.x0, (int32_t)o.y0, (int32_t)o.z0, mbar);
}

// Inside masks (v < k) of the box rows: bit x of s_row[i*81 + row], x < 33.
// Lane i (i < NISO) keeps isovalue i's ballot and writes its row mask.
// Isovalue slots whose bit in isomask is clear are not needed (no cell of
// the tile crosses them) and get no ballot.
template <int NISO>
__device__ __forceinline__ void row_masks(const float *buf, uint64_t *s_row, const McParams &p, uint32_t isomask = 0xfu)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float k[NISO];
#pragma unroll
    for (int i = 0; i < NISO; i++) k[i] = p.k[i];
    const float kl = p.k[lane < NISO ? lane : 0];
    for (int row = warp; row < kRows; row += 8) {
        const float v = buf[row * kVX + lane];
        const float vh = buf[row * kVX + kTX];
        uint32_t mine = 0;
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            if (!((isomask >> i) & 1u)) continue;  // (uniform)
            const uint32_t b = __ballot_sync(CHR_FULL_MASK, v < k[i]);
            mine = (lane == i) ? b : mine;
        }
        if (lane < NISO) s_row[lane * kRows + row] = (uint64_t)mine | ((uint64_t)(vh < kl) << 32);
    }
}

// Which (cell brick j, isovalue slot i) of the tile at o can have cells
// crossing k_i (bit 4j + i): min < k <= max in the value index, which
// bounds the brick's cell vertices; every pair without an index.  Each
// calling warp gets the same mask.
template <int NISO>
__device__ __forceinline__ uint32_t tile_activity(const McParams &p, const TileXYZ &o)
{
    if (!p.index) return 0xffffu;
    const int lane = threadIdx.x & 31;
    const int32_t bx0 = (int32_t)(o.x0 >> 3), by = (int32_t)(o.y0 >> 3), bz = (int32_t)(o.z0 >> 3);
    uint32_t bits = 0;
    if (lane < 4 && bx0 + lane < p.ibx) {
        const float2 r = __ldg(p.index + (bx0 + lane) + (int64_t)p.ibx * (by + (int64_t)p.iby * bz));
#pragma unroll
        for (int i = 0; i < NISO; i++) bits |= (uint32_t)(r.x < p.k[i] && p.k[i] <= r.y) << i;
    }
    return __reduce_or_sync(CHR_FULL_MASK, bits << (4 * (lane & 3)));
}

__device__ __forceinline__ uint32_t iso_mask(uint32_t act) { return (act | (act >> 4) | (act >> 8) | (act >> 12)) & 0xfu; }

// The index entry of cell brick `lane` (lanes 0..3) of the tile at o, or an
// empty range; loaded a tile ahead so its latency hides behind a tile.
__device__ __forceinline__ float2 tile_index_entry(const McParams &p, const TileXYZ &o, int lane)
{
    const int32_t bx0 = (int32_t)(o.x0 >> 3), by = (int32_t)(o.y0 >> 3), bz = (int32_t)(o.z0 >> 3);
    if (lane < 4 && bx0 + lane < p.ibx) return __ldg(p.index + (bx0 + lane) + (int64_t)p.ibx * (by + (int64_t)p.iby * bz));
    return make_float2(__int_as_float(0x7f800000), __int_as_float(0xff800000));
}

// tile_activity from entries loaded by tile_index_entry (by a whole warp).
template <int NISO>
__device__ __forceinline__ uint32_t activity_from(const McParams &p, float2 r)
{
    const int lane = threadIdx.x & 31;
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < NISO; i++) bits |= (uint32_t)(r.x < p.k[i] && p.k[i] <= r.y) << i;
    return __reduce_or_sync(CHR_FULL_MASK, (lane < 4) ? bits << (4 * lane) : 0u);
}

// Exchanges the bits of w at positions p and p + s for every p in m: with
// s = 2^j - 2^i and m the positions whose index bit i is set and bit j clear,
// this swaps index bits i and j of every bit position (a delta swap).
__device__ __forceinline__ uint32_t delta_swap(uint32_t w, int s, uint32_t m)
{
    const uint32_t t = ((w >> s) ^ w) & m;
    return w ^ t ^ (t << s);
}

// Case bytes of this thread's 8 cells from the inside masks of its four rows
// A = (y, z), B = (y+1, z), C = (y, z+1), D = (y+1, z+1), in the kernels'
// own bit order: corner (ox, oy, oz) is bit 4*ox + oy + 2*oz, so a cell's
// byte is the nibble (A, B, C, D) of its x column with the nibble of column
// x+1 above it.  The columns 8j..8j+7 of the four rows, one byte each, form
// a 4x8 bit matrix; transposing it (bit 8r + x to bit 4x + r: the five index
// bits rotated by two, four delta swaps) gives every column's nibble at
// once, and column 8's nibble comes from one multiply whose partial products
// do not overlap.  Byte x is then bits 4x..4x+7, picked by two byte
// permutes.  The case tables are stored in the same order (case_order).
// Cells past `nvalid` get case 0.
__device__ __forceinline__ void cases8(const uint64_t *R, int r00, int j, int nvalid, uint32_t &lo, uint32_t &hi)
{
    const int sh = 8 * j;
    const uint64_t ra = R[r00], rb = R[r00 + 1], rc = R[r00 + 9], rd = R[r00 + 10];
    const uint32_t a = __funnelshift_r((uint32_t)ra, (uint32_t)(ra >> 32), sh);
    const uint32_t b = __funnelshift_r((uint32_t)rb, (uint32_t)(rb >> 32), sh);
    const uint32_t c = __funnelshift_r((uint32_t)rc, (uint32_t)(rc >> 32), sh);
    const uint32_t d = __funnelshift_r((uint32_t)rd, (uint32_t)(rd >> 32), sh);
    const uint32_t ab = __byte_perm(a, b, 0x5140), cd = __byte_perm(c, d, 0x5140);
    uint32_t q = __byte_perm(ab, cd, 0x5410);                       // byte r: row r, columns 0..7
    const uint32_t c8 = __byte_perm(ab, cd, 0x7632) & 0x01010101u;  // bit 8r: row r, column 8
    q = delta_swap(q, 7, 0x00AA00AAu);   // index bits 0 <-> 3
    q = delta_swap(q, 14, 0x0000CCCCu);  // 1 <-> 4
    q = delta_swap(q, 4, 0x00F000F0u);   // 2 <-> 3
    q = delta_swap(q, 8, 0x0000FF00u);   // 3 <-> 4
    const uint32_t y = (q >> 4) | ((c8 * 0x10204080u) & 0xF0000000u);  // bit 8r of c8 -> bit 28 + r
    lo = __byte_perm(q, y, 0x5140);
    hi = __byte_perm(q, y, 0x7362);
    if (nvalid < 8) {
        const uint64_t keep = (nvalid <= 0) ? 0ull : ((1ull << (8 * nvalid)) - 1ull);
        lo &= (uint32_t)keep;
        hi &= (uint32_t)(keep >> 32);
    }
}

// The table's case index (corner ox + 2*oy + 4*oz is bit ox + 2*oy + 4*oz)
// of a case byte in the kernels' order (that corner is bit 4*ox + oy + 2*oz).
__device__ __forceinline__ int case_order(int c)
{
    int r = 0;
#pragma unroll
    for (int jc = 0; jc < 8; jc++) {
        const int ox = jc & 1, oy = (jc >> 1) & 1, oz = jc >> 2;
        r |= ((c >> (4 * ox + oy + 2 * oz)) & 1) << jc;
    }
    return r;
}

// Bytes of w that are neither 0 nor 0xff (active cells): bit 7 of each byte.
__device__ __forceinline__ uint32_t active_bytes(uint32_t w)
{
    const uint32_t nz = ((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w;     // bit 7: byte != 0
    const uint32_t nw = ~w;
    const uint32_t nf = ((nw & 0x7f7f7f7fu) + 0x7f7f7f7fu) | nw;   // bit 7: byte != 0xff
    return nz & nf & 0x80808080u;
}

__device__ __forceinline__ int valid_cells(const McParams &p, const TileXYZ &o)
{
    const int tid = threadIdx.x;
    const int j = tid >> 6, ly = tid & 7, lz = (tid >> 3) & 7;
    const int64_t cx0 = o.x0 + 8 * j, cy = o.y0 + ly, cz = o.z0 + lz;
    if (cy < p.ny - 1 && cz < p.nz - 1 && cx0 < p.nx - 1) return (int)((p.nx - 1 - cx0) < 8 ? (p.nx - 1 - cx0) : 8);
    return 0;
}

// Where tiles come from.  One field: tile t of p.  A batch: tile t of the
// concatenated tile list of many fields, each with its own McParams and
// tensor map (tile_start[i] = first tile of field i).
struct SrcOne {
    const McParams *p;
    const CUtensorMap *map;
    __device__ __forceinline__ int64_t ntiles() const { return p->ntiles; }
    __device__ __forceinline__ bool use_tma() const { return p->use_tma != 0; }
    __device__ __forceinline__ void at(int64_t tile, const McParams *&bp, const CUtensorMap *&m, int64_t &local) const
    {
        bp = p;
        m = map;
        local = tile;
    }
};

struct McBatch {
    const McParams *boxes;   // [nboxes]
    const CUtensorMap *maps; // [nboxes], 64-byte aligned
    const int64_t *tile_start;  // [nboxes + 1]
    int32_t nboxes;
    int64_t ntiles;
};

struct SrcMany {
    const McBatch *b;
    __device__ __forceinline__ int64_t ntiles() const { return b->ntiles; }
    __device__ __forceinline__ bool use_tma() const { return true; }
    __device__ __forceinline__ void at(int64_t tile, const McParams *&bp, const CUtensorMap *&m, int64_t &local) const
    {
        const int64_t *ts = b->tile_start;
        int lo = 0, hi = b->nboxes - 1;  // the last field whose first tile is <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(ts + mid) <= tile) lo = mid; else hi = mid - 1;
        }
        bp = b->boxes + lo;
        m = b->maps + lo;
        local = tile - __ldg(ts + lo);
    }
};

// One CHR level: tile t's box is decoded from the compressed stream.
// index: the level's value index (NULL: every brick is classified).
struct SrcChr {
    const McParams *p;
    const ChrLevels *L;
    const float2 *index;
};

// After a box copy gave up: one more bounded wait for each copy this block
// still has in flight (phase `par` of mbar[b], and of mbar[b ^ 1] when
// `other` is set), so that no copy lands in shared memory the block has
// left.  Kept out of line: it only runs on that failure path.
__device__ __noinline__ void drain_box_copies(uint64_t *mbar, int b, uint32_t par, bool other, uint32_t par_other)
{
    mbar_wait(&mbar[b], par);
    if (other) mbar_wait(&mbar[b ^ 1], par_other);
}

// Persistent tile loop shared by the tile kernels: the next box is fetched
// while `body` processes the current one.  A copy that never arrives
// (bounded wait) raises CHR_ERR_TIMEOUT and the block stops.
// body(tile, local tile, field params, box).
// IDX: warp 0 also reads the next tile's index entries when its box is
// issued and leaves the tile's activity mask (tile_activity) in act before
// body runs on it.
template <int NISO = 1, bool IDX = false, class Src, class Body>
__device__ __forceinline__ void tile_loop(const Src &src, uint32_t *err, float *bufs, uint64_t *mbar, Body body,
                                          uint32_t *act = nullptr)
{
    const int tid = threadIdx.x;
    __shared__ uint32_t s_act[2];
    const int64_t G = gridDim.x, ntiles = src.ntiles();
    const bool tma = src.use_tma();
    int64_t tile = blockIdx.x;
    if (tma) {
        if (tid == 0) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0 && tile < ntiles) {
            const McParams *bp;
            const CUtensorMap *m;
            int64_t local;
            src.at(tile, bp, m, local);
            issue_box(bufs, m, &mbar[0], *bp, local);
        }
    }
    uint32_t phase0 = 0, phase1 = 0;
    int cur = 0;
    if (IDX && tid < 32 && tile < ntiles) {
        const McParams *bp;
        const CUtensorMap *m;
        int64_t local;
        src.at(tile, bp, m, local);
        const uint32_t a = activity_from<NISO>(*bp, tile_index_entry(*bp, tile_origin(*bp, local), tid));
        if (tid == 0) s_act[0] = a;
    }
    for (; tile < ntiles; tile += G) {
        float *buf = bufs + cur * (kBufBytes / 4);
        const int64_t next = tile + G;
        const McParams *bp;
        const CUtensorMap *m;
        int64_t local;
        src.at(tile, bp, m, local);
        float2 rnext = make_float2(0.0f, 0.0f);
        if (IDX && tid < 32 && next < ntiles) {
            const McParams *nbp;
            const CUtensorMap *nm;
            int64_t nlocal;
            src.at(next, nbp, nm, nlocal);
            rnext = tile_index_entry(*nbp, tile_origin(*nbp, nlocal), tid);
        }
        bool ok = true;
        if (tma) {
            if (tid == 0 && next < ntiles) {
                const McParams *nbp;
                const CUtensorMap *nm;
                int64_t nlocal;
                src.at(next, nbp, nm, nlocal);
                issue_box(bufs + (cur ^ 1) * (kBufBytes / 4), nm, &mbar[cur ^ 1], *nbp, nlocal);
            }
            ok = mbar_wait(&mbar[cur], cur ? phase1 : phase0);
            if (cur)
                phase1 ^= 1u;
            else
                phase0 ^= 1u;
        } else {
            load_box_plain(buf, *bp, tile_origin(*bp, local));
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                if (err) atomicOr(err, 1u << CHR_ERR_TIMEOUT);
                // (the phase of mbar[cur] was flipped after its wait; mbar[cur ^ 1]'s was not)
                if (tma) drain_box_copies(mbar, cur, (cur ? phase1 : phase0) ^ 1u, next < ntiles, cur ? phase0 : phase1);
            }
            return;
        }
        if (IDX) *act = s_act[cur];
        body(tile, local, *bp, buf);
        if (IDX && tid < 32 && next < ntiles) {
            const McParams *nbp;
            const CUtensorMap *nm;
            int64_t nlocal;
            src.at(next, nbp, nm, nlocal);
            const uint32_t a = activity_from<NISO>(*nbp, rnext);
            if (tid == 0) s_act[cur ^ 1] = a;
        }
        __syncthreads();  // every read of buf is done before it is refilled
        cur ^= 1;
    }
}

template <int NISO, bool IDX, class Src>
__device__ __forceinline__ void mc_count_run(const Src &src, uint32_t *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float *bufs = reinterpret_cast<float *>(smem + kOffBuf);
    uint64_t *s_row = reinterpret_cast<uint64_t *>(smem + kOffRow);
    uint8_t *s_cnt = smem + kOffCnt;  // triangle count per case
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_sum[8][kMcIsoPerPass];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_cnt[tid] = (uint8_t)(g_mc_case[case_order(tid)] >> 60);

    uint32_t act_idx = 0xffffu;
    tile_loop<NISO, IDX>(src, err, bufs, mbar, [&](int64_t, int64_t tile, const McParams &p, const float *buf) {
        const TileXYZ o = tile_origin(p, tile);
        const uint32_t act = IDX ? act_idx : 0xffffu;
        row_masks<NISO>(buf, s_row, p, iso_mask(act));
        __syncthreads();
        const int nvalid = valid_cells(p, o);
        const int j = tid >> 6, ly = tid & 7, lz = (tid >> 3) & 7;
        const int r00 = lz * 9 + ly;
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            uint32_t lo = 0u, hi = 0u;
            if ((act >> (4 * j + i)) & 1u) cases8(s_row + i * kRows, r00, j, nvalid, lo, hi);
            // (cells that are all inside or all outside have no triangles: a
            // warp whose cells all are skips the table)
            const uint32_t al = active_bytes(lo), ah = active_bytes(hi);
            uint32_t c = 0;
            if (__any_sync(CHR_FULL_MASK, (al | ah) != 0u)) {
#pragma unroll
                for (int x = 0; x < 4; x++) c += s_cnt[(lo >> (8 * x)) & 0xffu] + s_cnt[(hi >> (8 * x)) & 0xffu];
            }
            if (p.cases) {
                const uint32_t na = __popc(al) + __popc(ah);
                const size_t at = ((size_t)tile * p.cstride + i) * 256 + tid;
                p.cases[at] = make_uint2(lo, hi);
                p.tcnt[at] = c | (na << 16);
            }
            c = __reduce_add_sync(CHR_FULL_MASK, c);
            if (lane == 0) s_sum[warp][i] = c;
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t t[kMcIsoPerPass] = {0, 0, 0, 0};
#pragma unroll
            for (int w = 0; w < 8; w++)
#pragma unroll
                for (int i = 0; i < NISO; i++) t[i] += s_sum[w][i];
            p.tile_cnt[tile] = make_uint4(t[0], t[1], t[2], t[3]);
        }
    }, &act_idx);
}

// IDX: the field has a value index (McParams.index), and cell bricks whose
// range does not straddle an isovalue are not classified for it.
template <int NISO>
__global__ void __launch_bounds__(256, 8) k_mc_count(const __grid_constant__ McParams p,
                                                 const __grid_constant__ CUtensorMap map)
{
    mc_count_run<NISO, false>(SrcOne{&p, &map}, p.err);
}

template <int NISO>
__global__ void __launch_bounds__(256, 5) k_mc_count_idx(const __grid_constant__ McParams p,
                                                        const __grid_constant__ CUtensorMap map)
{
    mc_count_run<NISO, true>(SrcOne{&p, &map}, p.err);
}

__global__ void __launch_bounds__(256) k_mc_count_batched(const __grid_constant__ McBatch b, uint32_t *err)
{
    mc_count_run<1, false>(SrcMany{&b}, err);
}

// t = (k - f0) / (f1 - f0): the edge parameter of a crossing.  f0 and f1 lie
// on opposite sides of k, so the quotient is in (0, 1]; the fast reciprocal
// quotient is within 2 ulp of the rounded one, and the IEEE quotient is used
// where the fast form does not apply (|f1 - f0| >= 2^126).  A tile whose
// values all lie below kHugeValue = 2^124 in magnitude has |f1 - f0| <= 2^125
// on every edge and takes the fast quotient throughout (FAST below): the
// same bits as this function, so which tiles take FAST never changes the
// output.
__device__ __forceinline__ float edge_t(float k, float f0, float f1)
{
    const float num = __fsub_rn(k, f0), den = __fsub_rn(f1, f0);
    return (fabsf(den) < 8.507059173023462e37f) ? __fdividef(num, den) : __fdiv_rn(num, den);
}


// Edge e of a cell as one word for the emit pass: bits 0-10 the byte offset
// of its lower corner in the box, 11-21 the byte step to its upper corner,
// 24-26 the lower corner's offsets (ox, oy, oz), 27-29 its axis, one-hot.
__device__ __forceinline__ uint32_t edge_word(int e)
{
    const int axis = e >> 2, m = e & 3;
    const int ox = (axis == 0) ? 0 : (m & 1);
    const int oy = (axis == 1) ? 0 : ((axis == 0) ? (m & 1) : (m >> 1));
    const int oz = (axis == 2) ? 0 : (m >> 1);
    const int step = (axis == 0) ? 1 : (axis == 1) ? kVX : kPlane;
    return (uint32_t)(4 * (ox + oy * kVX + oz * kPlane)) | ((uint32_t)(4 * step) << 11) | ((uint32_t)ox << 24) |
           ((uint32_t)oy << 25) | ((uint32_t)oz << 26) | (1u << (27 + axis));
}

__device__ __forceinline__ float lds_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

// Triangle `tri` (three edge numbers, one per byte) of the cell whose lower
// corner is at shared address cellB and grid position (cx, cy, cz), into
// dst[0..8].  A crossing sits at the edge's lower corner plus t along its
// axis; the corner's coordinates are integers, exact in float.  FAST: every
// value of the tile's box is below 2^125 in magnitude, so |f1 - f0| < 2^126
// and the fast quotient applies everywhere.
template <bool FAST>
__device__ __forceinline__ void make_triangle_w(float *dst, uint32_t cellB, const uint32_t *s_edgew, uint32_t tri,
                                                float k, float cx, float cy, float cz)
{
    const float cx1 = cx + 1.0f, cy1 = cy + 1.0f, cz1 = cz + 1.0f;
#pragma unroll
    for (int v = 0; v < 3; v++) {
        const uint32_t E = s_edgew[(tri >> (8 * v)) & 0xffu];
        const uint32_t a0 = cellB + (E & 0x7ffu);
        const float f0 = lds_f32(a0), f1 = lds_f32(a0 + ((E >> 11) & 0x7ffu));
        const float tv = FAST ? __fdividef(__fsub_rn(k, f0), __fsub_rn(f1, f0)) : edge_t(k, f0, f1);
        float x = (E & (1u << 24)) ? cx1 : cx;
        float y = (E & (1u << 25)) ? cy1 : cy;
        float z = (E & (1u << 26)) ? cz1 : cz;
        if (E & (1u << 27)) x = __fadd_rn(x, tv);
        if (E & (1u << 28)) y = __fadd_rn(y, tv);
        if (E & (1u << 29)) z = __fadd_rn(z, tv);
        dst[3 * v + 0] = x;
        dst[3 * v + 1] = y;
        dst[3 * v + 2] = z;
    }
}

// ---- single pass: tile offsets by decoupled look-back -------------------------
//
// Blocks claim tiles in increasing order from a counter.  A tile publishes
// its own triangle counts as soon as it has classified its cells, then adds
// up the counts of the tiles before it, walking back 32 at a time, until it
// meets a tile that has published its inclusive prefix; it then publishes its
// own.  A tile's counts never wait on anything and every claimed tile belongs
// to a running block, so every wait ends; each is bounded all the same, and
// one that gives up sets the abort word so that no block waits after it.
//
// Tile status word: bits 62-63 the state (0 nothing yet, 1 the tile's own
// counts, 2 its inclusive prefix is in tile_off), bits 14i..14i+13 the
// tile's triangles at isovalue slot i (at most 2048 cells x 5 < 2^14).
constexpr uint64_t kTileOwn = 1ull << 62, kTilePrefix = 2ull << 62;

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *a)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *a)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *a)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *a, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release_u64(uint64_t *a, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

// Triangles before tile t at each isovalue slot, by one warp; false when a
// wait gave up or another block's did.
template <int NISO>
__device__ __forceinline__ bool look_back(const McParams &p, int64_t t, uint64_t (&excl)[NISO])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NISO; i++) excl[i] = 0;
    for (int64_t pos = t - 1; pos >= 0; pos -= 32) {
        const int64_t idx = pos - lane;
        uint64_t w = kTilePrefix;  // before tile 0: a prefix of zero
        bool ok = true;
        if (idx >= 0) {
            w = ld_acquire_u64(p.tstat + idx);
            for (uint32_t it = 0; (w >> 62) == 0; it++) {
                if (it >= CHR_SPIN_LIMIT || ld_relaxed_u32(p.tabort) != 0u) {
                    ok = false;
                    break;
                }
                if (it > 16) __nanosleep(64);
                w = ld_acquire_u64(p.tstat + idx);
            }
        }
        if (!__all_sync(CHR_FULL_MASK, ok)) return false;
        const uint32_t pm = __ballot_sync(CHR_FULL_MASK, (w >> 62) == 2u);
        const int first = pm ? __ffs(pm) - 1 : 32;  // nearest tile with its prefix
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            const uint32_t c = (lane < first) ? (uint32_t)(w >> (14 * i)) & 0x3fffu : 0u;
            excl[i] += __reduce_add_sync(CHR_FULL_MASK, c);
        }
        if (pm) {
#pragma unroll
            for (int i = 0; i < NISO; i++) {
                const uint64_t v = (lane == first && idx >= 0) ? ld_relaxed_u64(p.tile_off + idx * kMcIsoPerPass + i)
                                                               : 0ull;
                excl[i] += __shfl_sync(CHR_FULL_MASK, v, first);
            }
            return true;
        }
    }
    return true;
}

// By warp 0 of the block: publish tile t's triangle counts (cnt[i] for
// isovalue slot i), find the triangles before it by the look-back, publish
// its inclusive prefix, and leave the tile's first triangle per slot in
// g0[i] (shared memory); the last tile also writes the totals and the
// overflow bit.  A wait that gave up sets the abort word and the timeout bit.
template <int NISO>
__device__ __forceinline__ void publish_tile(const McParams &p, int64_t tile, const uint32_t (&cnt)[NISO], uint64_t *g0)
{
    const int lane = threadIdx.x & 31;
    uint64_t own = 0;
#pragma unroll
    for (int i = 0; i < NISO; i++) own |= (uint64_t)(cnt[i] & 0xffffu) << (14 * i);
    uint64_t ex[NISO];
    bool ok = true;
    const bool publish = tile != p.unpublished_tile;
    if (tile == 0) {
#pragma unroll
        for (int i = 0; i < NISO; i++) ex[i] = 0;
    } else {
        if (lane == 0 && publish) st_relaxed_u64(p.tstat + tile, kTileOwn | own);
        ok = look_back<NISO>(p, tile, ex);
    }
    if (lane == 0) {
        if (!ok) {
            atomicExch(p.tabort, 1u);
            if (p.err) atomicOr(p.err, 1u << CHR_ERR_TIMEOUT);
        }
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            const uint64_t incl = ex[i] + (cnt[i] & 0xffffu);
            st_relaxed_u64(p.tile_off + tile * kMcIsoPerPass + i, incl);
            g0[i] = ex[i];
            if (tile == p.ntiles - 1) {  // the totals, and whether every triangle fitted below cap
                p.ntris[i] = incl;
                if (incl > p.cap && p.err) atomicOr(p.err, 1u << CHR_ERR_OVERFLOW);
            }
        }
        if (publish) st_release_u64(p.tstat + tile, kTilePrefix | own);
    }
}

// The single pass's tile loop: blocks claim tiles from p.tctr in increasing
// order.  A block claims its next tile only near the end of the current one
// (the first warp done with its share of the current tile's triangles calls
// claim(), else thread 0 after the body): a tile that is claimed but not
// started would hold up the look-back of every later tile until its block
// got to it.  The next box is fetched into the other buffer meanwhile.
// body(tile, tile, params, box, claim).
// IDX: the claiming thread also reads the claimed tile's index entries and
// leaves its activity mask (tile_activity) in act before body runs on it.
template <int NISO = 1, bool IDX = false, class Body>
__device__ __forceinline__ void tile_loop_claimed(const McParams &p, const CUtensorMap *map, float *bufs,
                                                  uint64_t *mbar, Body body, uint32_t *act = nullptr)
{
    __shared__ int64_t s_tile;
    __shared__ uint32_t s_claimed, s_act;
    const int tid = threadIdx.x;
    const bool tma = p.use_tma != 0;
    int cur = 0;
    // by one thread: the activity mask of tile t from its four index entries
    auto activity1 = [&](int64_t t) -> uint32_t {
        const TileXYZ o = tile_origin(p, t);
        const int32_t bx0 = (int32_t)(o.x0 >> 3), by = (int32_t)(o.y0 >> 3), bz = (int32_t)(o.z0 >> 3);
        float2 r[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            r[j] = make_float2(__int_as_float(0x7f800000), __int_as_float(0xff800000));
            if (bx0 + j < p.ibx) r[j] = __ldg(p.index + (bx0 + j) + (int64_t)p.ibx * (by + (int64_t)p.iby * bz));
        }
        uint32_t a = 0;
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int i = 0; i < NISO; i++) a |= (uint32_t)(r[j].x < p.k[i] && p.k[i] <= r[j].y) << (4 * j + i);
        return a;
    };
    auto claim = [&]() {  // one thread per tile: the next tile, and its box on its way
        if (atomicExch(&s_claimed, 1u) != 0u) return;
        const int64_t t = (int64_t)atomicAdd(p.tctr, 1u);
        s_tile = t;
        if (tma && t < p.ntiles) issue_box(bufs + (cur ^ 1) * (kBufBytes / 4), map, &mbar[cur ^ 1], p, t);
        if (IDX && t < p.ntiles) s_act = activity1(t);
    };
    if (tid == 0) {
        if (tma) {
            mbar_init(&mbar[0], 1);
            mbar_init(&mbar[1], 1);
            fence_mbar_init();
        }
        const int64_t t = (int64_t)atomicAdd(p.tctr, 1u);
        s_tile = t;
        s_claimed = 0u;
        if (tma && t < p.ntiles) issue_box(bufs, map, &mbar[0], p, t);
        if (IDX && t < p.ntiles) s_act = activity1(t);
    }
    __syncthreads();
    int64_t tile = s_tile;
    uint32_t phase0 = 0, phase1 = 0;
    while (tile < p.ntiles) {
        float *buf = bufs + cur * (kBufBytes / 4);
        bool ok = true;
        if (tma) {
            ok = mbar_wait(&mbar[cur], cur ? phase1 : phase0);
            if (cur)
                phase1 ^= 1u;
            else
                phase0 ^= 1u;
        } else {
            load_box_plain(buf, p, tile_origin(p, tile));
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) {
                atomicExch(p.tabort, 1u);
                if (p.err) atomicOr(p.err, 1u << CHR_ERR_TIMEOUT);
                if (tma) drain_box_copies(mbar, cur, (cur ? phase1 : phase0) ^ 1u, false, 0u);
            }
            return;
        }
        // (the other buffer's last reads ended at the previous barrier, so claim() may refill it)
        if (IDX) *act = s_act;
        body(tile, tile, p, buf, claim);
        if (tid == 0) claim();  // unless a warp already did
        __syncthreads();        // every read of buf is done, and s_tile holds the next tile
        tile = s_tile;          // (read before the next tile's first barrier, so before the next claim)
        if (tid == 0) s_claimed = 0u;
        cur ^= 1;
    }
}

// The one-pass decode + marching-cubes tile loop: like tile_loop_claimed,
// but each tile's box is decoded from the CHR by the block's own warps
// (warps 0-3 the tile's four vertex bricks, staged through the second box
// buffer; warps 4-7 the first planes, lines and corner of the bricks after
// them).  The first warp done with its share of a tile's triangles claims
// the next tile and reads the records of its 20 bricks (every level) and
// the index of its four cell bricks: act bit 4j + i says that brick j can
// have cells crossing isovalue slot i (min < k <= max over the brick's cell
// vertices).  A tile with none is not decoded: warp 0 publishes zero
// counts for it.  fast: no box value reaches 2^124.
// body(tile, tile, params, box, claim).
template <int NISO, class Body>
__device__ __forceinline__ void tile_loop_chr(const McParams &p, const ChrLevels &L, const float2 *index, float *bufs,
                                              uint32_t &act, bool &fast, uint64_t *g0, Body body)
{
    __shared__ int64_t s_tile[2];
    __shared__ uint32_t s_act[2];
    __shared__ uint32_t s_claimed;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *box = bufs;
    // the second box buffer: 4 staging areas of the own-brick warps, then the records
    constexpr int kRecBytes = CHR_MAX_LEVELS * kTileBricks * 16;
    constexpr int kStageWords = ((kBufBytes - kRecBytes) / 16) & ~3;  // per own-brick warp
    static_assert(4 * kStageWords * 4 + kRecBytes <= kBufBytes, "staging and records fit the second buffer");
    uint32_t *stage = reinterpret_cast<uint32_t *>(bufs + kBufBytes / 4);
    uint4(*s_rec)[kTileBricks] = reinterpret_cast<uint4(*)[kTileBricks]>(bufs + kBufBytes / 4 + 4 * kStageWords);
    int par = 0;
    // by a whole warp, the first to call it for the current tile: claim the
    // next tile, read its records and its bricks' index
    auto claim = [&]() {
        uint32_t first = 0u;
        if (lane == 0) first = atomicExch(&s_claimed, 1u);
        if (__shfl_sync(CHR_FULL_MASK, first, 0) != 0u) return;
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(p.tctr, 1u);
        t = __shfl_sync(CHR_FULL_MASK, t, 0);
        uint32_t a = 0u;
        if (t < p.ntiles) {
            const TileXYZ o = tile_origin(p, t);
            const int32_t bx0 = (int32_t)(o.x0 >> 3), by = (int32_t)(o.y0 >> 3), bz = (int32_t)(o.z0 >> 3);
            load_tile_records(s_rec, L, bx0, by, bz, lane);
            a = 0xffffu;
            if (index) {
                uint32_t bits = 0;
                if (lane < 4 && bx0 + lane < L.nbx) {
                    const float2 r = __ldg(index + (bx0 + lane) + (int64_t)L.nbx * (by + (int64_t)L.nby * bz));
#pragma unroll
                    for (int i = 0; i < NISO; i++) bits |= (uint32_t)(r.x < p.k[i] && p.k[i] <= r.y) << i;
                }
                a = __reduce_or_sync(CHR_FULL_MASK, bits << (4 * (lane & 3)));
            }
        }
        if (lane == 0) {
            s_tile[par] = t;
            s_act[par] = a;
        }
    };
    if (tid == 0) s_claimed = 0u;
    __syncthreads();
    if (warp == 0) claim();
    __syncthreads();
    int64_t tile = s_tile[par];
    uint32_t a = s_act[par];
    if (tid == 0) s_claimed = 0u;
    par ^= 1;
    while (tile < p.ntiles) {
        act = a;
        if (a == 0) {
            if (warp == 0) {
                uint32_t zero[NISO];
#pragma unroll
                for (int i = 0; i < NISO; i++) zero[i] = 0u;
                publish_tile<NISO>(p, tile, zero, g0);
            }
        } else {
            const TileXYZ o = tile_origin(p, tile);
            const int32_t bx0 = (int32_t)(o.x0 >> 3), by = (int32_t)(o.y0 >> 3), bz = (int32_t)(o.z0 >> 3);
            auto slot = [&](int dx, int dy, int dz) -> int {  // the brick's record slot, -1 outside the grid
                return (bx0 + dx < L.nbx && by + dy < L.nby && bz + dz < L.nbz) ? dx + 5 * (dy + 2 * dz) : -1;
            };
            bool huge = false;
            if (warp < 4) {
                const int id = slot(warp, 0, 0);
                if (id >= 0) {
                    huge = box_own_brick<kVX, kPlane>(box, L, s_rec, id, 8 * warp, lane, stage + warp * kStageWords,
                                                      kStageWords);
                } else {
                    float *row0 = box + 8 * warp + kVX * (lane & 7) + kPlane * (lane >> 3);
                    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    *reinterpret_cast<float4 *>(row0) = z4;
                    *reinterpret_cast<float4 *>(row0 + 4) = z4;
                    *reinterpret_cast<float4 *>(row0 + 4 * kPlane) = z4;
                    *reinterpret_cast<float4 *>(row0 + 4 * kPlane + 4) = z4;
                }
            } else if (warp < 7) {
                // warps 4-6: nine planes, three each: the y = 0 planes of the
                // bricks after the tile's along y (q 0-3), the z = 0 planes of
                // those after it along z (q 4-7), the x = 0 plane of the one
                // after it along x (q 8)
#pragma unroll 1
                for (int q = 3 * (warp - 4); q < 3 * (warp - 3); q++) {
                    HaloPiece hp;
                    hp.len = 8;
                    if (q < 4) {
                        hp.id = slot(q, 1, 0);
                        hp.axa = 0;
                        hp.axb = 2;
                        hp.base = 8 * kVX + 8 * q;
                        hp.da = 1;
                        hp.db = kPlane;
                    } else if (q < 8) {
                        hp.id = slot(q - 4, 0, 1);
                        hp.axa = 0;
                        hp.axb = 1;
                        hp.base = 8 * kPlane + 8 * (q - 4);
                        hp.da = 1;
                        hp.db = kVX;
                    } else {
                        hp.id = slot(4, 0, 0);
                        hp.axa = 1;
                        hp.axb = 2;
                        hp.base = kTX;
                        hp.da = kVX;
                        hp.db = kPlane;
                    }
                    huge |= box_halo<true, kVX, kPlane>(box, L, s_rec, hp, lane);
                }
            } else {
                // warp 7: the y = z = 0 lines of the bricks after the tile's
                // along y and z, then the lines x = y = 0 (+x+y brick), x = z = 0
                // (+x+z) and the corner (+x+y+z); lanes 8g..8g+7 take line g
                const int g = lane >> 3;
                HaloPiece hp;
                hp.axb = 0;
                hp.db = 0;
                hp.id = slot(g, 1, 1);
                hp.axa = 0;
                hp.base = 8 * kVX + 8 * kPlane + 8 * g;
                hp.da = 1;
                hp.len = 8;
                huge |= box_halo<false, kVX, kPlane>(box, L, s_rec, hp, lane);
                if (g == 0) {
                    hp.id = slot(4, 1, 0);
                    hp.axa = 2;
                    hp.base = kTX + 8 * kVX;
                    hp.da = kPlane;
                    hp.len = 8;
                } else if (g == 1) {
                    hp.id = slot(4, 0, 1);
                    hp.axa = 1;
                    hp.base = kTX + 8 * kPlane;
                    hp.da = kVX;
                    hp.len = 8;
                } else {
                    hp.id = (g == 2) ? slot(4, 1, 1) : -1;
                    hp.axa = 0;
                    hp.base = kTX + 8 * kVX + 8 * kPlane;
                    hp.da = 1;
                    hp.len = (g == 2) ? 1 : 0;
                }
                huge |= box_halo<false, kVX, kPlane>(box, L, s_rec, hp, lane);
            }
            fast = !__syncthreads_or(huge);
            body(tile, tile, p, box, claim);
        }
        if (warp == 0) claim();  // unless a warp already did
        __syncthreads();         // the box is free, and s_tile[par] holds the next tile
        tile = s_tile[par];
        a = s_act[par];
        if (tid == 0) s_claimed = 0u;
        par ^= 1;
    }
}

// A small non-negative integer as a float without the conversion unit:
// 2^23 + u has u in its low mantissa bits, and subtracting 2^23 is exact.
__device__ __forceinline__ float small_to_float(uint32_t u)
{
    return __fsub_rn(__uint_as_float(0x4B000000u | u), 8388608.0f);
}

__device__ __forceinline__ uint32_t lanemask_le()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

// Emit, per tile: case bytes of the thread's 8 cells for every isovalue, one
// block scan of (triangles, active cells) for all of them, the active cells
// of each isovalue compacted in cell order (with their first triangle) into
// the shared pool, and the first active cell of every 32-triangle chunk
// noted.  Warps then take the chunks of all the tile's isovalues
// round-robin, with no barrier between isovalues; a lane finds its
// triangle's cell from the chunk's window of 32 active cells (a cell that
// starts at window position s marks bit s; the lane's cell is the number of
// marks at or below it), builds the triangle in the warp's staging buffer,
// and the warp writes the chunk with aligned 16-byte stores.
//
// FUSED: the single pass (no count pass before it): the tiles come from the
// claimed-tile loop and the case bytes from the box, and once the block scan
// has the tile's totals, warp 0 publishes them and finds the tile's offsets
// by the look-back while the other warps compact.
template <int NISO, bool STORED, bool FUSED, class Src, bool CHR = false, bool IDX = false>
__device__ __forceinline__ void mc_emit_run(const Src &src, uint32_t *err)
{
    static_assert(!(FUSED && STORED), "the single pass classifies from the box");
    static_assert(!CHR || FUSED, "the CHR box is decoded in the single pass");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float *bufs = reinterpret_cast<float *>(smem + kOffBuf);
    uint64_t *s_row = reinterpret_cast<uint64_t *>(smem + kOffRow);
    uint8_t *s_cnt = smem + kOffCnt;
    uint32_t *s_tri = reinterpret_cast<uint32_t *>(smem + kOffTri);
    uint32_t *s_edgew = reinterpret_cast<uint32_t *>(smem + kEOffEdge);
    uint32_t *s_act = reinterpret_cast<uint32_t *>(smem + kEOffAct);
    uint16_t *s_apre = reinterpret_cast<uint16_t *>(smem + kEOffAPre);
    uint16_t *s_chunk = reinterpret_cast<uint16_t *>(smem + kEOffChunk);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_w[kMcIsoPerPass][9];  // per isovalue slot: warp offsets, then the tile total
    __shared__ uint64_t s_g0[kMcIsoPerPass];    // single pass: the tile's first triangle per slot
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t le = lanemask_le();
    float *s_stage = reinterpret_cast<float *>(smem + kEOffStage) + warp * kWarpStage;
    s_cnt[tid] = (uint8_t)(g_mc_case[case_order(tid)] >> 60);
    for (int i = tid; i < 256 * CHR_MC_MAX_TRI; i += 256) {
        const uint64_t word = g_mc_case[case_order(i / CHR_MC_MAX_TRI)];
        const int t = i % CHR_MC_MAX_TRI;
        uint32_t tri = 0;
        if (t < (int)(word >> 60))
            for (int v = 0; v < 3; v++) tri |= (uint32_t)((word >> (12 * t + 4 * v)) & 15u) << (8 * v);
        s_tri[i] = tri;
    }
    if (tid < 12) s_edgew[tid] = edge_word(tid);

    // CHR: which (cell brick j, isovalue slot i) can have triangles (bit
    // 4j + i; the others are not classified), and whether no box value
    // reaches 2^124, both set by the tile loop
    uint32_t chr_act = 0xffffu, idx_act = 0xffffu;
    bool chr_fast = true;
    auto body = [&](int64_t, int64_t tile, const McParams &p, const float *box, auto &&claim) {
        // fast quotients unless some value of the box is 2^124 or more in magnitude (or infinite)
        bool fast = chr_fast;
        if (!CHR) {
            bool huge = false;
            for (int u = tid; u < kRows * kVX / 4; u += 256) {
                const float4 v = reinterpret_cast<const float4 *>(box)[u];
                huge |= fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))) >= kHugeValue;
            }
            fast = !__syncthreads_or(huge);
        }
        const TileXYZ o = tile_origin(p, tile);
        const uint32_t act = CHR ? chr_act : ((IDX && !STORED) ? idx_act : 0xffffu);
        if (!STORED) {
            row_masks<NISO>(box, s_row, p, iso_mask(act));
            __syncthreads();
        }
        const int j = tid >> 6, ly = tid & 7, lz = (tid >> 3) & 7;
        const int r00 = lz * 9 + ly;
        const int nvalid = STORED ? 8 : valid_cells(p, o);
        const uint32_t boxB = smem_addr(box);
        const float fx0 = (float)o.x0, fy0 = (float)o.y0, fz0 = (float)o.z0;
        const size_t at0 = (size_t)tile * p.cstride * 256 + tid;

        // isovalue slot i of this thread: case bytes, triangles | active cells << 16
        auto classify = [&](int i, uint32_t &lo, uint32_t &hi) -> uint32_t {
            if (STORED) {
                const uint2 cw = __ldg(p.cases + at0 + 256 * i);
                lo = cw.x;
                hi = cw.y;
                return __ldg(p.tcnt + at0 + 256 * i);
            }
            if (!((act >> (4 * j + i)) & 1u)) {  // (uniform across the thread's two warps)
                lo = hi = 0u;
                return 0u;
            }
            cases8(s_row + i * kRows, r00, j, nvalid, lo, hi);
            const uint32_t al = active_bytes(lo), ah = active_bytes(hi);
            uint32_t cnt = 0;
            if (__any_sync(CHR_FULL_MASK, (al | ah) != 0u)) {  // (a warp without active cells skips the table)
#pragma unroll
                for (int x = 0; x < 4; x++) cnt += s_cnt[(lo >> (8 * x)) & 0xffu] + s_cnt[(hi >> (8 * x)) & 0xffu];
            }
            return cnt | ((__popc(al) + __popc(ah)) << 16);
        };
        // this thread's active cells of slot i into the pool from entry `a` on,
        // triangle prefix `pre`; chunk q of the slot is entry cq + q of the table
        auto compact = [&](uint32_t lo, uint32_t hi, uint32_t a, uint32_t pre, uint32_t cq) {
#pragma unroll
            for (int x = 0; x < 8; x++) {
                const uint32_t cb = ((x < 4 ? lo : hi) >> (8 * (x & 3))) & 0xffu;
                const uint32_t c = s_cnt[cb];
                if (c) {
                    if (CHR_IN_BOUNDS(a < (uint32_t)kPool)) {
                        s_act[a] = (uint32_t)(tid * 8 + x) | (cb << 11);
                        s_apre[a] = (uint16_t)pre;
                    }
                    const uint32_t q = (pre + 31u) >> 5;
                    if ((q << 5) < pre + c && CHR_IN_BOUNDS(cq + q < (uint32_t)kMaxChunks)) s_chunk[cq + q] = (uint16_t)a;
                    a++;
                    pre += c;
                }
            }
        };
        // the chunks of slot i (list from pool entry ab, chunk table from cq);
        // warp w takes the chunks whose index counted from the first chunk
        // of the group is w modulo 8
        auto chunks = [&](int i, uint32_t n, uint32_t cq, auto fast_tag) {
            constexpr bool FAST = decltype(fast_tag)::value;
            const uint64_t g0 = FUSED ? s_g0[i] : __ldg(p.tile_off + tile * kMcIsoPerPass + i);
            const float k = p.k[i];
            // triangles of this tile that fit below cap (the rest are counted, not written)
            const int lim = (g0 >= p.cap) ? 0 : (int)((p.cap - g0) < (uint64_t)n ? (p.cap - g0) : (uint64_t)n);
            float *tout = p.tris[i] + 9ull * g0;
            // a chunk is 288 floats, so every chunk of the tile has the same 16-byte phase
            const int pad = (int)((reinterpret_cast<uintptr_t>(tout) >> 2) & 3u);
            const int head = (4 - pad) & 3;
            float *stage = s_stage + pad;
            for (int q = (warp - (int)cq) & 7; 32 * q < lim; q += 8) {
                const int base = 32 * q;
                const int mm = (lim - base) < 32 ? (lim - base) : 32;
                // (uniform across the warp: a chunk whose table entry or output range is out of bounds is skipped)
                if (!CHR_IN_BOUNDS(cq + q < (uint32_t)kMaxChunks && g0 + (uint64_t)(base + mm) <= p.cap)) continue;
                const int a_lo = s_chunk[cq + q];
                const int s0 = CHR_IN_BOUNDS(a_lo + lane < kPool) ? (int)s_apre[a_lo + lane] - base : 32;
                const uint32_t mark = (s0 > 0 && s0 < 32) ? (1u << s0) : 0u;
                const uint32_t starts = __reduce_or_sync(CHR_FULL_MASK, mark);
                const int jj = __popc(starts & le);
                if (lane == 0) bulk_wait_read_all();  // the previous chunk's bulk store has read the staging buffer
                __syncwarp();
                if (lane < mm && CHR_IN_BOUNDS(a_lo + jj < kPool)) {
                    const int a = a_lo + jj;
                    const uint32_t e = s_act[a];
                    const int t = base + lane - (int)s_apre[a];
                    const uint32_t c = e & 2047u;
                    const uint32_t lx = (c & 7u) + ((c >> 6) & 0x18u), cly = (c >> 3) & 7u, clz = (c >> 6) & 7u;
                    // the triangle's table entry, and the cell's far corner inside the box
                    if (CHR_IN_BOUNDS(t >= 0 && t < CHR_MC_MAX_TRI &&
                                      4u * (clz * kPlane + cly * kVX + lx + 1u + kVX + kPlane) < (uint32_t)kTileBytes)) {
                        const uint32_t tri = s_tri[(e >> 11) * CHR_MC_MAX_TRI + t];
                        make_triangle_w<FAST>(stage + 9 * lane, boxB + 4u * (clz * kPlane + cly * kVX + lx), s_edgew,
                                              tri, k, fx0 + small_to_float(lx), fy0 + small_to_float(cly),
                                              fz0 + small_to_float(clz));
                    }
#ifdef CHR_CHECKED
                    if (p.dbg_cells[i])
                        p.dbg_cells[i][g0 + base + lane] =
                            (uint32_t)((o.x0 + lx) + (p.nx - 1) * ((o.y0 + cly) + (p.ny - 1) * (o.z0 + clz)));
#endif
                }
                fence_proxy_async_smem();
                __syncwarp();
                // dst[u] = stage[u]; dst + u and stage + u are 16-byte aligned when (pad + u) % 4 == 0: the
                // aligned middle goes out as one bulk store, the ragged ends as plain stores
                float *dst = tout + 9 * base;
                const int F = 9 * mm;
                const int h = min(head, F);
                if (lane < h) __stcs(dst + lane, stage[lane]);
                const int nb16 = (F - h) >> 2;
                if (lane == 0 && nb16 > 0) {
                    bulk_store(dst + h, stage + h, (uint32_t)nb16 * 16u);
                    bulk_commit();
                }
                const int tail0 = h + 4 * nb16;
                if (lane < F - tail0) __stcs(dst + tail0 + lane, stage[tail0 + lane]);
            }
        };
        auto chunks_any = [&](int i, uint32_t n, uint32_t cq) {
            if (fast)
                chunks(i, n, cq, std::true_type{});
            else
                chunks(i, n, cq, std::false_type{});
        };

        // one block scan of every slot's (triangles | active cells << 16)
        uint32_t lo[NISO], hi[NISO], excl[NISO];
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            const uint32_t packed = classify(i, lo[i], hi[i]);
            const uint32_t inc = warp_incl_scan_u32(packed, lane);
            excl[i] = inc - packed;
            if (lane == 31) s_w[i][warp] = inc;
        }
        __syncthreads();
        if (warp == 0) {  // lane 8i + w scans warp w's total of slot i over the 8 warps
            const int ii = lane >> 3, wi = lane & 7;
            const uint32_t t = (ii < NISO) ? s_w[ii][wi] : 0u;
            uint32_t ti = t;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const uint32_t u = __shfl_up_sync(CHR_FULL_MASK, ti, o, 8);
                if (wi >= o) ti += u;
            }
            if (ii < NISO) {
                s_w[ii][wi] = ti - t;
                if (wi == 7) s_w[ii][8] = ti;
            }
        }
        __syncthreads();
        if (FUSED && warp == 0) {
            // publish this tile's counts, find the triangles before it, publish its inclusive prefix
            uint32_t cnt[NISO];
#pragma unroll
            for (int i = 0; i < NISO; i++) cnt[i] = s_w[i][8];
            publish_tile<NISO>(p, tile, cnt, s_g0);
        }
        // pool entries and chunk-table entries of the slots, all lists together
        uint32_t used = 0;
#pragma unroll
        for (int i = 0; i < NISO; i++) {
            const uint32_t na = s_w[i][8] >> 16;
            used += na ? na + 32u : 0u;
        }
        if (used <= (uint32_t)kPool) {
            uint32_t ab = 0, cq = 0;
#pragma unroll
            for (int i = 0; i < NISO; i++) {
                const uint32_t tot = s_w[i][8], n = tot & 0xffffu, na = tot >> 16;
                if (n) {
                    const uint32_t ex = s_w[i][warp] + excl[i];
                    // (a warp without active cells at slot i has nothing to compact)
                    if (((warp < 7) ? s_w[i][warp + 1] : tot) != s_w[i][warp]) {
                        // without a stored classification the case bytes are made again rather than kept
                        if (!STORED) {
                            if (!((act >> (4 * j + i)) & 1u))
                                lo[i] = hi[i] = 0u;
                            else
                                cases8(s_row + i * kRows, r00, j, nvalid, lo[i], hi[i]);
                        }
                        compact(lo[i], hi[i], ab + (ex >> 16), ex & 0xffffu, cq);
                    }
                    if (tid < 32 && CHR_IN_BOUNDS(ab + na + tid < (uint32_t)kPool))
                        s_apre[ab + na + tid] = 0xffffu;  // window tail past the last active cell
                    ab += na + 32u;
                    cq += (n + 31u) >> 5;
                }
            }
            __syncthreads();
            cq = 0;
#pragma unroll 1
            for (int i = 0; i < NISO; i++) {
                const uint32_t n = s_w[i][8] & 0xffffu;
                if (n) {
                    chunks_any(i, n, cq);
                    cq += (n + 31u) >> 5;
                }
            }
            // the first warp done claims the next tile (the CHR loop claims at the tile's end)
            if (FUSED && !CHR && lane == 0) claim();
            // (the tile loop's barrier keeps the pool until every chunk is written)
        } else {
#pragma unroll 1
            for (int i = 0; i < NISO; i++) {  // one slot at a time
                const uint32_t tot = s_w[i][8], n = tot & 0xffffu, na = tot >> 16;
                if (n == 0) continue;  // uniform across the block
                uint32_t l, h;
                const uint32_t packed = classify(i, l, h);
                const uint32_t ex = s_w[i][warp] + warp_incl_scan_u32(packed, lane) - packed;
                compact(l, h, ex >> 16, ex & 0xffffu, 0u);
                if (tid < 32 && CHR_IN_BOUNDS(na + tid < (uint32_t)kPool)) s_apre[na + tid] = 0xffffu;
                __syncthreads();
                chunks_any(i, n, 0u);
                __syncthreads();  // the pool is rewritten for the next slot
            }
        }
    };
    if constexpr (CHR)
        tile_loop_chr<NISO>(*src.p, *src.L, src.index, bufs, chr_act, chr_fast, s_g0, body);
    else if constexpr (FUSED)
        tile_loop_claimed<NISO, IDX>(*src.p, src.map, bufs, mbar, body, &idx_act);
    else
        tile_loop<NISO, IDX && !STORED>(
            src, err, bufs, mbar,
            [&](int64_t g, int64_t t, const McParams &p, const float *box) { body(g, t, p, box, [] {}); }, &idx_act);
    if (lane == 0) bulk_wait_all();  // shared memory stays valid until every bulk store is done
}

// Two-pass emit from the count pass's stored classification (large grids,
// where the single pass's per-tile waits cost more than the count pass).
template <int NISO>
__global__ void __launch_bounds__(256, 4) k_mc_emit_stored(const __grid_constant__ McParams p,
                                                          const __grid_constant__ CUtensorMap map)
{
    mc_emit_run<NISO, true, false>(SrcOne{&p, &map}, p.err);
}

// Classification, tile offsets and emission in one launch (no count pass).
template <int NISO, bool IDX>
__global__ void __launch_bounds__(256, 4) k_mc_fused(const __grid_constant__ McParams p,
                                                    const __grid_constant__ CUtensorMap map)
{
    mc_emit_run<NISO, false, true, SrcOne, false, IDX>(SrcOne{&p, &map}, p.err);
}

// Decode of a CHR level, classification, tile offsets and emission in one
// launch: the field never goes to memory.
template <int NISO>
__global__ void __launch_bounds__(256, 4) k_mc_chr(const __grid_constant__ McParams p,
                                                  const __grid_constant__ ChrLevels L, const float2 *index)
{
    mc_emit_run<NISO, false, true, SrcChr, true, true>(SrcChr{&p, &L, index}, p.err);
}

__global__ void __launch_bounds__(256, 4) k_mc_emit_batched(const __grid_constant__ McBatch b, uint32_t *err)
{
    mc_emit_run<1, true, false>(SrcMany{&b}, err);
}

// ---- adjoint of the vertex positions ----------------------------------------
//
// A vertex on edge (i0, i1) along `axis` sits at p_axis = x0 + t with
// t = (k - f0)/(f1 - f0): dp_axis/df0 = (t - 1)/(f1 - f0) and
// dp_axis/df1 = -t/(f1 - f0); the other coordinates do not depend on the
// field.  The adjoint walks the triangles in exactly the emit order (same
// tiles, classification, compaction and window), reads dL/dp where the
// forward pass wrote p, and
// adds each contribution to both edge ends.  Sums are made deterministic by
// fixed-point int64 atomics: pass 0 finds the largest |contribution|, pass 1
// adds round(c * S) with S = 2^(52 - exponent of that maximum), so every
// term is an exact integer and integer addition does not depend on order.
// Non-finite contributions are skipped.

struct AdjParams {
    const float *grad[kMcIsoPerPass];  // dL/dtris per isovalue slot (the forward layout)
    unsigned long long *acc;           // [N] fixed-point sums
    unsigned int *maxbits;             // max |contribution| as float bits
    int32_t pass;
};

__device__ __forceinline__ double adj_scale(unsigned int maxbits)
{
    const float m = __uint_as_float(maxbits);
    if (!(m > 0.0f) || !isfinite(m)) return 1.0;
    return ldexp(1.0, 52 - ilogbf(m));
}

// The adjoint walks each tile and isovalue exactly like the emit pass (the
// count pass's classification, the compacted active cells, the chunk window)
// so lane m of a chunk meets triangle m of the forward output.
template <int NISO>
__global__ void __launch_bounds__(256, 4) k_mc_adjoint(const __grid_constant__ McParams p,
                                                      const __grid_constant__ AdjParams a,
                                                      const __grid_constant__ CUtensorMap map)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    float *bufs = reinterpret_cast<float *>(smem + kOffBuf);
    uint8_t *s_cnt = smem + kOffCnt;
    uint32_t *s_tri = reinterpret_cast<uint32_t *>(smem + kOffTri);
    uint32_t *s_edgew = reinterpret_cast<uint32_t *>(smem + kEOffEdge);
    uint32_t *s_act = reinterpret_cast<uint32_t *>(smem + kEOffAct);
    uint16_t *s_apre = reinterpret_cast<uint16_t *>(smem + kEOffAPre);
    uint16_t *s_chunk = reinterpret_cast<uint16_t *>(smem + kEOffChunk);
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t s_w[2][9];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_cnt[tid] = (uint8_t)(g_mc_case[case_order(tid)] >> 60);
    for (int i = tid; i < 256 * CHR_MC_MAX_TRI; i += 256) {
        const uint64_t word = g_mc_case[case_order(i / CHR_MC_MAX_TRI)];
        const int t = i % CHR_MC_MAX_TRI;
        uint32_t tri = 0;
        if (t < (int)(word >> 60))
            for (int v = 0; v < 3; v++) tri |= (uint32_t)((word >> (12 * t + 4 * v)) & 15u) << (8 * v);
        s_tri[i] = tri;
    }
    if (tid < 12) s_edgew[tid] = edge_word(tid);
    const double S = (a.pass == 1) ? adj_scale(*a.maxbits) : 1.0;
    float lane_max = 0.0f;
    const int64_t step_g[3] = {1, p.nx, p.nx * p.ny};

    tile_loop(SrcOne{&p, &map}, p.err, bufs, mbar, [&](int64_t, int64_t tile, const McParams &, const float *box) {
        const TileXYZ o = tile_origin(p, tile);
        const uint32_t boxB = smem_addr(box);
        const size_t at0 = (size_t)tile * p.cstride * 256 + tid;
        uint2 cw_next = __ldg(p.cases + at0);
        uint32_t pk_next = __ldg(p.tcnt + at0);

#pragma unroll 1
        for (int i = 0; i < NISO; i++) {
            const uint32_t lo = cw_next.x, hi = cw_next.y, packed = pk_next;
            if (i + 1 < NISO) {
                cw_next = __ldg(p.cases + at0 + 256 * (i + 1));
                pk_next = __ldg(p.tcnt + at0 + 256 * (i + 1));
            }
            const uint32_t inc = warp_incl_scan_u32(packed, lane);
            uint32_t *sw = s_w[i & 1];
            if (lane == 31) sw[warp] = inc;
            __syncthreads();
            if (warp == 0) {
                const uint32_t t = (lane < 8) ? sw[lane] : 0u;
                const uint32_t ti = warp_incl_scan_u32(t, lane);
                if (lane < 8) sw[lane] = ti - t;
                if (lane == 7) sw[8] = ti;
            }
            __syncthreads();
            const uint32_t excl = sw[warp] + inc - packed, total = sw[8];
            const int n = (int)(total & 0xffffu);
            if (n == 0) continue;  // uniform across the block
            {
                uint32_t ai = excl >> 16, pre = excl & 0xffffu;
#pragma unroll
                for (int x = 0; x < 8; x++) {
                    const uint32_t cb = ((x < 4 ? lo : hi) >> (8 * (x & 3))) & 0xffu;
                    const uint32_t c = s_cnt[cb];
                    if (c) {
                        if (CHR_IN_BOUNDS(ai < (uint32_t)kPool)) {
                            s_act[ai] = (uint32_t)(tid * 8 + x) | (cb << 11);
                            s_apre[ai] = (uint16_t)pre;
                        }
                        const uint32_t q = (pre + 31u) >> 5;
                        if ((q << 5) < pre + c && CHR_IN_BOUNDS(q < (uint32_t)kMaxChunks)) s_chunk[q] = (uint16_t)ai;
                        ai++;
                        pre += c;
                    }
                }
                if (tid < 32 && CHR_IN_BOUNDS((total >> 16) + tid < (uint32_t)kPool)) s_apre[(total >> 16) + tid] = 0xffffu;
            }
            __syncthreads();
            const uint64_t g0 = __ldg(p.tile_off + tile * kMcIsoPerPass + i);
            const float k = p.k[i];
            const int lim = (g0 >= p.cap) ? 0 : (int)((p.cap - g0) < (uint64_t)n ? (p.cap - g0) : (uint64_t)n);
            const float *gin = a.grad[i] + 9ull * g0;
            for (int q = warp; 32 * q < lim; q += 8) {
                const int base = 32 * q;
                if (!CHR_IN_BOUNDS(q < kMaxChunks)) continue;  // uniform across the warp
                const int a_lo = s_chunk[q];
                const int s0 = CHR_IN_BOUNDS(a_lo + lane < kPool) ? (int)s_apre[a_lo + lane] - base : 32;
                const uint32_t mark = (s0 > 0 && s0 < 32) ? (1u << s0) : 0u;
                const uint32_t starts = __reduce_or_sync(CHR_FULL_MASK, mark);
                const int jj = __popc(starts & (0xffffffffu >> (31 - lane)));
                const int m = base + lane;
                if (m < lim && CHR_IN_BOUNDS(a_lo + jj < kPool)) {
                    const int aa = a_lo + jj;
                    const uint32_t e = s_act[aa];
                    const int t = m - (int)s_apre[aa];
                    const uint32_t tri =
                        CHR_IN_BOUNDS(t >= 0 && t < CHR_MC_MAX_TRI) ? s_tri[(e >> 11) * CHR_MC_MAX_TRI + t] : 0u;
                    const uint32_t c = e & 2047u;
                    const uint32_t lx = c & 7u, cly = (c >> 3) & 7u, clz = (c >> 6) & 7u, jb = c >> 9;
                    const uint32_t cellB = boxB + 4u * (clz * kPlane + cly * kVX + 8u * jb + lx);
                    const int64_t gx = o.x0 + 8 * jb + lx, gy = o.y0 + cly, gz = o.z0 + clz;
                    const float *g9 = gin + 9ull * m;
#pragma unroll
                    for (int v = 0; v < 3; v++) {
                        const uint32_t E = s_edgew[(tri >> (8 * v)) & 0xffu];
                        const uint32_t a0 = cellB + (E & 0x7ffu);
                        const float f0 = lds_f32(a0), f1 = lds_f32(a0 + ((E >> 11) & 0x7ffu));
                        const float tv = edge_t(k, f0, f1);
                        const int axis = (E & (1u << 27)) ? 0 : (E & (1u << 28)) ? 1 : 2;
                        const float gax = __ldg(g9 + 3 * v + axis);
                        const float inv = 1.0f / __fsub_rn(f1, f0);
                        const float c0 = gax * (tv - 1.0f) * inv, c1 = -gax * tv * inv;
                        if (a.pass == 0) {
                            if (isfinite(c0)) lane_max = fmaxf(lane_max, fabsf(c0));
                            if (isfinite(c1)) lane_max = fmaxf(lane_max, fabsf(c1));
                        } else {
                            const int64_t i0 = (gx + (int64_t)((E >> 24) & 1u)) +
                                               p.nx * ((gy + (int64_t)((E >> 25) & 1u)) +
                                                       p.ny * (gz + (int64_t)((E >> 26) & 1u)));
                            const int64_t i1 = i0 + step_g[axis];
                            if (isfinite(c0))
                                atomicAdd(a.acc + i0, (unsigned long long)(long long)llrint((double)c0 * S));
                            if (isfinite(c1))
                                atomicAdd(a.acc + i1, (unsigned long long)(long long)llrint((double)c1 * S));
                        }
                    }
                }
            }
            __syncthreads();  // the compacted lists are rewritten for the next isovalue
        }
    });
    if (a.pass == 0) {
        const unsigned int mb = __reduce_max_sync(CHR_FULL_MASK, __float_as_uint(lane_max));
        if (lane == 0 && mb) atomicMax(a.maxbits, mb);
    }
}

__global__ void __launch_bounds__(256) k_adj_finalize(const unsigned long long *acc, const unsigned int *maxbits,
                                                      float *grad, int64_t N)
{
    const double S = adj_scale(*maxbits);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        grad[i] = (float)((double)(long long)acc[i] / S);
}

// ---- exclusive scan of the tile counts ----------------------------------

constexpr int kTScanThreads = 256, kTScanPer = 8, kTScanChunk = kTScanThreads * kTScanPer;

struct __align__(32) Sum4 {
    uint64_t x, y, z, w;
};

__device__ __forceinline__ Sum4 make_sum4(uint64_t x, uint64_t y, uint64_t z, uint64_t w)
{
    Sum4 r;
    r.x = x;
    r.y = y;
    r.z = z;
    r.w = w;
    return r;
}

struct TScanArgs {
    const uint4 *cnt;
    uint64_t *off;      // [ntiles][4]
    Sum4 *chunk;  // [nchunks]
    int64_t ntiles, nchunks;
    uint64_t *ntris;
    int niso;
    uint64_t cap;
    uint32_t *err;
};

__device__ __forceinline__ void block_excl_scan4(uint64_t (&v)[4], uint64_t (&tot)[4], uint64_t (*s_w)[4])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc[4];
#pragma unroll
    for (int i = 0; i < 4; i++) inc[i] = warp_incl_scan_u64(v[i], lane);
    if (lane == 31)
#pragma unroll
        for (int i = 0; i < 4; i++) s_w[warp][i] = inc[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint64_t t = (lane < 8) ? s_w[lane][i] : 0ull;
            const uint64_t ti = warp_incl_scan_u64(t, lane);
            if (lane < 8) s_w[lane][i] = ti - t;
            if (lane == 7) s_w[8][i] = ti;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; i++) {
        tot[i] = s_w[8][i];
        v[i] = s_w[warp][i] + inc[i] - v[i];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kTScanThreads) k_tscan_reduce(const __grid_constant__ TScanArgs a)
{
    __shared__ uint64_t s_w[9][4];
    const int64_t b0 = (int64_t)blockIdx.x * kTScanChunk + (int64_t)threadIdx.x * kTScanPer;
    uint64_t v[4] = {0, 0, 0, 0}, tot[4];
    for (int e = 0; e < kTScanPer; e++)
        if (b0 + e < a.ntiles) {
            const uint4 c = a.cnt[b0 + e];
            v[0] += c.x;
            v[1] += c.y;
            v[2] += c.z;
            v[3] += c.w;
        }
    block_excl_scan4(v, tot, s_w);
    if (threadIdx.x == 0) a.chunk[blockIdx.x] = make_sum4(tot[0], tot[1], tot[2], tot[3]);
}

__global__ void __launch_bounds__(kTScanThreads) k_tscan_chunks(const __grid_constant__ TScanArgs a)
{
    __shared__ uint64_t s_w[9][4];
    uint64_t carry[4] = {0, 0, 0, 0};
    for (int64_t c0 = 0; c0 < a.nchunks; c0 += kTScanThreads) {
        const int64_t c = c0 + threadIdx.x;
        const Sum4 s = (c < a.nchunks) ? a.chunk[c] : make_sum4(0, 0, 0, 0);
        uint64_t v[4] = {s.x, s.y, s.z, s.w}, tot[4];
        block_excl_scan4(v, tot, s_w);
        if (c < a.nchunks)
            a.chunk[c] = make_sum4(carry[0] + v[0], carry[1] + v[1], carry[2] + v[2], carry[3] + v[3]);
#pragma unroll
        for (int i = 0; i < 4; i++) carry[i] += tot[i];
    }
    if (threadIdx.x < a.niso) {
        a.ntris[threadIdx.x] = carry[threadIdx.x];
        if (carry[threadIdx.x] > a.cap && a.err) atomicOr(a.err, 1u << CHR_ERR_OVERFLOW);
    }
}

__global__ void __launch_bounds__(kTScanThreads) k_tscan_apply(const __grid_constant__ TScanArgs a)
{
    __shared__ uint64_t s_w[9][4];
    const int64_t b0 = (int64_t)blockIdx.x * kTScanChunk + (int64_t)threadIdx.x * kTScanPer;
    uint4 c[kTScanPer];
    uint64_t v[4] = {0, 0, 0, 0}, tot[4];
    for (int e = 0; e < kTScanPer; e++) {
        c[e] = (b0 + e < a.ntiles) ? a.cnt[b0 + e] : make_uint4(0, 0, 0, 0);
        v[0] += c[e].x;
        v[1] += c[e].y;
        v[2] += c[e].z;
        v[3] += c[e].w;
    }
    block_excl_scan4(v, tot, s_w);
    const Sum4 base = a.chunk[blockIdx.x];
    uint64_t run[4] = {base.x + v[0], base.y + v[1], base.z + v[2], base.w + v[3]};
    for (int e = 0; e < kTScanPer; e++) {
        if (b0 + e >= a.ntiles) break;
        uint64_t *o = a.off + (b0 + e) * kMcIsoPerPass;
        o[0] = run[0];
        o[1] = run[1];
        o[2] = run[2];
        o[3] = run[3];
        run[0] += c[e].x;
        run[1] += c[e].y;
        run[2] += c[e].z;
        run[3] += c[e].w;
    }
}

// First triangle of every field of a batch (the scan value at its first
// tile) and the total at index nboxes.
__global__ void k_box_starts(const uint64_t *off, const int64_t *tile_start, int32_t nboxes, int64_t ntiles,
                             const uint64_t *total, uint64_t *box_start)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nboxes; i += gridDim.x * blockDim.x) {
        const int64_t t = tile_start[i];
        box_start[i] = (i < nboxes && t < ntiles) ? off[t * kMcIsoPerPass] : *total;
    }
}

}  // namespace

// Test only (checked builds): the triangle-cell output of chr_debug_tri_cells.
static uint32_t *g_dbg_cells = nullptr;

#ifdef CHR_CHECKED
namespace {
// The count pass's stored case bytes of isovalue slot 0 (per tile and
// thread, 8 cells of a brick row, corner (ox, oy, oz) at bit 4 ox + oy +
// 2 oz) rewritten per cell in the grid's cell order with corner (ox, oy, oz)
// at bit ox + 2 oy + 4 oz.  One thread per (tile, thread of the tile).
__global__ void k_debug_cases(const uint2 *cases, int32_t cstride, int64_t ntiles, int32_t ntx, int32_t ncby,
                              int64_t nx, int64_t ny, int64_t nz, uint8_t *out)
{
    const int64_t u = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (u >= ntiles * 256) return;
    const int64_t tile = u >> 8;
    const int t = (int)(u & 255);
    const int64_t tq = tile / ntx, tz = tq / ncby;
    const int64_t x0 = (tile - tq * ntx) * kTX + 8 * (t >> 6), y = (tq - tz * ncby) * 8 + (t & 7),
                  z = tz * 8 + ((t >> 3) & 7);
    if (y >= ny - 1 || z >= nz - 1) return;
    const uint2 cw = cases[(tile * cstride) * 256 + t];
    for (int x = 0; x < 8; x++) {
        if (x0 + x >= nx - 1) break;
        const uint32_t cb = ((x < 4 ? cw.x : cw.y) >> (8 * (x & 3))) & 0xffu;
        out[(x0 + x) + (nx - 1) * (y + (ny - 1) * z)] = (uint8_t)case_order((int)cb);
    }
}
}  // namespace
#endif

// Checked builds: see chr_debug_tri_cells / chr_debug_cases (false in normal builds).
bool mc_debug_set_tri_cells(uint32_t *cells)
{
#ifdef CHR_CHECKED
    g_dbg_cells = cells;
    return true;
#else
    (void)cells;
    return false;
#endif
}

static void mc_tiles(const Grid &g, int32_t &ntx, int32_t &ncby, int32_t &ncbz, int64_t &ntiles)
{
    const int64_t ncbx = (g.nx - 1 + 7) / 8;
    ntx = (int32_t)((ncbx + kMcBricksX - 1) / kMcBricksX);
    ncby = (int32_t)((g.ny - 1 + 7) / 8);
    ncbz = (int32_t)((g.nz - 1 + 7) / 8);
    ntiles = (int64_t)ntx * ncby * ncbz;
}

struct McWorkspace {
    uint4 *cnt;
    uint64_t *off;
    Sum4 *chunk;
    int64_t nchunks;
    uint2 *cases;    // null in the compact layout
    uint32_t *tcnt;
};

static size_t align256(size_t n) { return ((n + 255) / 256) * 256; }

// Scratch of one marching-cubes call: tile counts, offsets and scan chunks,
// plus (stored layout) the count pass's classification for cstride isovalue
// slots per tile, 12 bytes per thread and slot.
static size_t mc_layout(const Grid &g, int cstride, void *base, McWorkspace *w)
{
    int32_t ntx, ncby, ncbz;
    int64_t ntiles;
    mc_tiles(g, ntx, ncby, ncbz, ntiles);
    const int64_t nchunks = (ntiles + kTScanChunk - 1) / kTScanChunk;
    const size_t o_cnt = 0, o_off = o_cnt + align256(ntiles * 16);
    const size_t o_chunk = o_off + align256(ntiles * 32);
    const size_t o_cases = o_chunk + align256(nchunks * 32);
    const size_t o_tcnt = o_cases + align256((size_t)ntiles * cstride * 256 * 8);
    const size_t total = o_tcnt + align256((size_t)ntiles * cstride * 256 * 4);
    if (w) {
        char *b = reinterpret_cast<char *>(base);
        w->cnt = reinterpret_cast<uint4 *>(b + o_cnt);
        w->off = reinterpret_cast<uint64_t *>(b + o_off);
        w->chunk = reinterpret_cast<Sum4 *>(b + o_chunk);
        w->nchunks = nchunks;
        w->cases = cstride ? reinterpret_cast<uint2 *>(b + o_cases) : nullptr;
        w->tcnt = cstride ? reinterpret_cast<uint32_t *>(b + o_tcnt) : nullptr;
    }
    return total;
}

static int stored_slots(int n_iso) { return n_iso < kMcIsoPerPass ? (n_iso > 0 ? n_iso : 1) : kMcIsoPerPass; }

// The full workspace holds the tile arrays and the count pass's
// classification for up to 4 isovalue slots (the groups of 4 reuse it);
// the minimum workspace the tile arrays alone, which is all the single
// pass needs (status words, counter and abort word in the tile-count
// region, inclusive prefixes in the offsets).
size_t mc_workspace_bytes(const Grid &g, int n_iso)
{
    return mc_layout(g, stored_slots(n_iso), nullptr, nullptr);
}

size_t mc_workspace_min_bytes(const Grid &g, int n_iso)
{
    (void)n_iso;
    return mc_layout(g, 0, nullptr, nullptr);
}

// Tiles from which a group of n isovalues is faster in two passes than in
// one, when the workspace allows both: the single pass saves the count
// pass and its stored classification, but each tile waits for its claim,
// its box and its look-back, which the triangle work of few isovalues or of
// a small grid cannot hide.  Measured on 128^3..1024^3 turbulence: n = 1
// from 1,024 (single faster) to 8,192 tiles (two-pass faster), n = 2 from
// 8,192 to 65,536, n = 4 from 65,536 (512^3) to 221,184 (768^3).
static int64_t two_pass_min_tiles(int n) { return (int64_t)2048 * n * n * n; }



struct McGrids {
    int count, adjoint, fused, emit;  // resident blocks of each persistent kernel
    int count_idx, fused_idx;         // (the variants that read a value index)
};

template <int NISO>
static cudaError_t mc_prepare(McGrids &out)
{
    // resident blocks, computed once per device; filled under the lock and
    // published with the flag, so a caller never sees a half-filled entry
    static McGrids Gd[kMaxDevices] = {};
    static std::atomic<bool> ready[kMaxDevices] = {};
    static std::mutex mu;
    const int dev = current_device();
    if (!ready[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready[dev].load(std::memory_order_relaxed)) {
            cudaError_t e = cudaFuncSetAttribute(k_mc_adjoint<NISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEmitSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_mc_count<NISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCountSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_mc_fused<NISO, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEmitSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_mc_count_idx<NISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCountSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_mc_fused<NISO, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEmitSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_mc_emit_stored<NISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEmitSmem);
            if (e != cudaSuccess) return e;
            int sms = 0, bc = 0, ba = 0, bu = 0, be = 0, bci = 0, bui = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bc, k_mc_count<NISO>, 256, kCountSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ba, k_mc_adjoint<NISO>, 256, kEmitSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu, k_mc_fused<NISO, false>, 256, kEmitSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&be, k_mc_emit_stored<NISO>, 256, kEmitSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bci, k_mc_count_idx<NISO>, 256, kCountSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bui, k_mc_fused<NISO, true>, 256, kEmitSmem);
            if (sms < 1) sms = 1;
            McGrids &G = Gd[dev];
            G.count_idx = sms * (bci > 0 ? bci : 1);
            G.fused_idx = sms * (bui > 0 ? bui : 1);
            G.count = sms * (bc > 0 ? bc : 1);
            G.adjoint = sms * (ba > 0 ? ba : 1);
            G.fused = sms * (bu > 0 ? bu : 1);
            G.emit = sms * (be > 0 ? be : 1);
            ready[dev].store(true, std::memory_order_release);
        }
    }
    out = Gd[dev];
    return cudaSuccess;
}

// Tile counts and their exclusive scan (tile_off, totals into ntris).
template <int NISO>
static cudaError_t launch_count_scan(const McParams &p, const CUtensorMap &map, const McWorkspace &w, uint64_t *ntris,
                                     int niso, cudaStream_t s)
{
    McGrids G;
    cudaError_t e = mc_prepare<NISO>(G);
    if (e != cudaSuccess) return e;
    if (p.index) {
        const unsigned gc = (unsigned)(p.ntiles < G.count_idx ? p.ntiles : G.count_idx);
        k_mc_count_idx<NISO><<<gc, 256, kCountSmem, s>>>(p, map);
    } else {
        const unsigned gc = (unsigned)(p.ntiles < G.count ? p.ntiles : G.count);
        k_mc_count<NISO><<<gc, 256, kCountSmem, s>>>(p, map);
    }
    TScanArgs a;
    a.cnt = w.cnt;
    a.off = w.off;
    a.chunk = w.chunk;
    a.ntiles = p.ntiles;
    a.nchunks = w.nchunks;
    a.ntris = ntris;
    a.niso = niso;
    a.cap = p.cap;
    a.err = p.err;
    k_tscan_reduce<<<(unsigned)w.nchunks, kTScanThreads, 0, s>>>(a);
    k_tscan_chunks<<<1, kTScanThreads, 0, s>>>(a);
    k_tscan_apply<<<(unsigned)w.nchunks, kTScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// Checked builds only: a tile of the single pass that publishes nothing
// (chr_debug_unpublished_tile), so the tiles after it give up their bounded
// look-back and raise CHR_ERR_TIMEOUT; -1 (none) otherwise.
#ifdef CHR_CHECKED
static std::atomic<int64_t> g_unpublished_tile{-1};
static int64_t test_unpublished_tile() { return g_unpublished_tile.load(); }
#else
static int64_t test_unpublished_tile() { return -1; }
#endif

bool mc_set_unpublished_tile(int64_t tile)
{
#ifdef CHR_CHECKED
    g_unpublished_tile.store(tile < 0 ? -1 : tile);
    return true;
#else
    (void)tile;
    return false;
#endif
}

// One group of up to 4 isovalues.  With room for the stored classification
// and at least two_pass_min_tiles tiles: count pass, tile scan, emit from
// the stored classification.  Otherwise the single pass: the tile status
// words, the tile counter and the abort word (the start of the tile-count
// region) are cleared, then k_mc_fused classifies, offsets and emits every
// tile.
template <int NISO>
static cudaError_t launch_mc_group(const McParams &p0, const CUtensorMap &map, const McWorkspace &w, uint64_t *ntris,
                                   int niso, cudaStream_t s)
{
    McGrids G;
    cudaError_t e = mc_prepare<NISO>(G);
    if (e != cudaSuccess) return e;
    if (p0.cases && p0.cstride >= NISO && p0.ntiles >= two_pass_min_tiles(NISO)) {
        e = launch_count_scan<NISO>(p0, map, w, ntris, niso, s);
        if (e != cudaSuccess) return e;
        const unsigned ge = (unsigned)(p0.ntiles < G.emit ? p0.ntiles : G.emit);
        k_mc_emit_stored<NISO><<<ge, 256, kEmitSmem, s>>>(p0, map);
        return cudaGetLastError();
    }
    McParams p = p0;
    p.unpublished_tile = test_unpublished_tile();
    p.tstat = reinterpret_cast<uint64_t *>(w.cnt);
    p.tctr = reinterpret_cast<uint32_t *>(p.tstat + p.ntiles);
    p.tabort = p.tctr + 1;
    p.ntris = ntris;
    e = cudaMemsetAsync(p.tstat, 0, (size_t)p.ntiles * 8 + 8, s);
    if (e != cudaSuccess) return e;
    if (p.index) {
        const unsigned gf = (unsigned)(p.ntiles < G.fused_idx ? p.ntiles : G.fused_idx);
        k_mc_fused<NISO, true><<<gf, 256, kEmitSmem, s>>>(p, map);
    } else {
        const unsigned gf = (unsigned)(p.ntiles < G.fused ? p.ntiles : G.fused);
        k_mc_fused<NISO, false><<<gf, 256, kEmitSmem, s>>>(p, map);
    }
    return cudaGetLastError();
}

template <int NISO>
static cudaError_t launch_adjoint_group(const McParams &p, const AdjParams &a, const CUtensorMap &map,
                                        const McWorkspace &w, uint64_t *ntris, int niso, bool recount, cudaStream_t s)
{
    if (recount) {
        cudaError_t e = launch_count_scan<NISO>(p, map, w, ntris, niso, s);
        if (e != cudaSuccess) return e;
    }
    McGrids G;
    cudaError_t e = mc_prepare<NISO>(G);
    if (e != cudaSuccess) return e;
    const unsigned ge = (unsigned)(p.ntiles < G.adjoint ? p.ntiles : G.adjoint);
    k_mc_adjoint<NISO><<<ge, 256, kEmitSmem, s>>>(p, a, map);
    return cudaGetLastError();
}

cudaError_t launch_mc(const float *field, const Grid &g, const float *iso, int n_iso, float *tris, uint64_t cap,
                      uint64_t *ntris, uint32_t *err, void *workspace, size_t workspace_bytes, cudaStream_t s,
                      const float2 *index)
{
    return launch_mc_pitched(field, g, g.nx, g.nx * g.ny, iso, n_iso, tris, cap, ntris, err, workspace,
                             workspace_bytes, s, index);
}

cudaError_t launch_mc_pitched(const float *field, const Grid &g, int64_t sx, int64_t sy, const float *iso, int n_iso,
                              float *tris, uint64_t cap, uint64_t *ntris, uint32_t *err, void *workspace,
                              size_t workspace_bytes, cudaStream_t s, const float2 *index)
{
    McParams p;
    memset(&p, 0, sizeof(p));
    p.f = field;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.sx = sx;
    p.sy = sy;
    mc_tiles(g, p.ntx, p.ncby, p.ncbz, p.ntiles);
    p.cap = cap;
    p.err = err;
    p.index = index;
    p.ibx = (int32_t)g.nbx;
    p.iby = (int32_t)g.nby;
    // the stored classification when the workspace holds it (large grids take two passes)
    const int cstride = (workspace_bytes >= mc_workspace_bytes(g, n_iso)) ? stored_slots(n_iso) : 0;
    McWorkspace w;
    mc_layout(g, cstride, workspace, &w);
    p.tile_cnt = w.cnt;
    p.tile_off = w.off;
    p.cases = w.cases;
    p.tcnt = w.tcnt;
    p.cstride = cstride;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    p.use_tma = make_field_tensor_map_pitched(&map, field, g.nx, g.ny, g.nz, sx, sy, kBoxX, 9, 9) ? 1 : 0;
    for (int i0 = 0; i0 < n_iso; i0 += kMcIsoPerPass) {
        const int n = (n_iso - i0) < kMcIsoPerPass ? (n_iso - i0) : kMcIsoPerPass;
        for (int i = 0; i < kMcIsoPerPass; i++) {
            p.k[i] = (i < n) ? iso[i0 + i] : 0.0f;
            p.tris[i] = (i < n) ? tris + 9ull * cap * (uint64_t)(i0 + i) : nullptr;
            p.dbg_cells[i] = (i < n && g_dbg_cells) ? g_dbg_cells + cap * (uint64_t)(i0 + i) : nullptr;
        }
        cudaError_t e;
        switch (n) {
            case 1: e = launch_mc_group<1>(p, map, w, ntris + i0, n, s); break;
            case 2: e = launch_mc_group<2>(p, map, w, ntris + i0, n, s); break;
            case 3: e = launch_mc_group<3>(p, map, w, ntris + i0, n, s); break;
            default: e = launch_mc_group<4>(p, map, w, ntris + i0, n, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Resident blocks of k_mc_chr<NISO>, once per device (as mc_prepare).
template <int NISO>
static cudaError_t mc_chr_prepare(int &grid)
{
    static int Gd[kMaxDevices] = {};
    static std::atomic<bool> ready[kMaxDevices] = {};
    static std::mutex mu;
    const int dev = current_device();
    if (!ready[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready[dev].load(std::memory_order_relaxed)) {
            cudaError_t e = cudaFuncSetAttribute(k_mc_chr<NISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEmitSmem);
            if (e != cudaSuccess) return e;
            int sms = 0, bu = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu, k_mc_chr<NISO>, 256, kEmitSmem);
            Gd[dev] = (sms > 0 ? sms : 1) * (bu > 0 ? bu : 1);
            ready[dev].store(true, std::memory_order_release);
        }
    }
    grid = Gd[dev];
    return cudaSuccess;
}

template <int NISO>
static cudaError_t launch_chr_group(const McParams &p0, const ChrLevels &L, const float2 *index,
                                    const McWorkspace &w, uint64_t *ntris, cudaStream_t s)
{
    int grid = 0;
    cudaError_t e = mc_chr_prepare<NISO>(grid);
    if (e != cudaSuccess) return e;
    McParams p = p0;
    p.unpublished_tile = test_unpublished_tile();
    p.tstat = reinterpret_cast<uint64_t *>(w.cnt);
    p.tctr = reinterpret_cast<uint32_t *>(p.tstat + p.ntiles);
    p.tabort = p.tctr + 1;
    p.ntris = ntris;
    e = cudaMemsetAsync(p.tstat, 0, (size_t)p.ntiles * 8 + 8, s);
    if (e != cudaSuccess) return e;
    const unsigned gf = (unsigned)(p.ntiles < grid ? p.ntiles : grid);
    k_mc_chr<NISO><<<gf, 256, kEmitSmem, s>>>(p, L, index);
    return cudaGetLastError();
}

cudaError_t launch_mc_chr(const ChrMcLevels &c, const Grid &g, const float *iso, int n_iso, float *tris, uint64_t cap,
                          uint64_t *ntris, uint32_t *err, void *workspace, size_t workspace_bytes, cudaStream_t s)
{
    if (workspace_bytes < mc_workspace_min_bytes(g, n_iso)) return cudaErrorInvalidValue;
    McParams p;
    memset(&p, 0, sizeof(p));
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    mc_tiles(g, p.ntx, p.ncby, p.ncbz, p.ntiles);
    p.cap = cap;
    p.err = err;
    McWorkspace w;
    mc_layout(g, 0, workspace, &w);
    p.tile_cnt = w.cnt;
    p.tile_off = w.off;
    ChrLevels L;
    memset(&L, 0, sizeof(L));
    for (int l = 0; l < c.nlevels; l++) {
        L.recs[l] = c.recs[l];
        L.words[l] = c.words[l];
        L.exc_idx[l] = c.exc_idx[l];
        L.exc_val[l] = c.exc_val[l];
        L.two_e[l] = c.two_e[l];
    }
    L.nlevels = c.nlevels;
    L.nbx = (int32_t)g.nbx;
    L.nby = (int32_t)g.nby;
    L.nbz = (int32_t)g.nbz;
    for (int i0 = 0; i0 < n_iso; i0 += kMcIsoPerPass) {
        const int n = (n_iso - i0) < kMcIsoPerPass ? (n_iso - i0) : kMcIsoPerPass;
        for (int i = 0; i < kMcIsoPerPass; i++) {
            p.k[i] = (i < n) ? iso[i0 + i] : 0.0f;
            p.tris[i] = (i < n) ? tris + 9ull * cap * (uint64_t)(i0 + i) : nullptr;
            p.dbg_cells[i] = (i < n && g_dbg_cells) ? g_dbg_cells + cap * (uint64_t)(i0 + i) : nullptr;
        }
        cudaError_t e;
        switch (n) {
            case 1: e = launch_chr_group<1>(p, L, c.index, w, ntris + i0, s); break;
            case 2: e = launch_chr_group<2>(p, L, c.index, w, ntris + i0, s); break;
            case 3: e = launch_chr_group<3>(p, L, c.index, w, ntris + i0, s); break;
            default: e = launch_chr_group<4>(p, L, c.index, w, ntris + i0, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t mc_adjoint_workspace_bytes(const Grid &g, int n_iso)
{
    const size_t base = ((mc_workspace_bytes(g, n_iso) + 255) / 256) * 256;
    return base + (size_t)g.N * 8 + 256;
}

cudaError_t launch_mc_adjoint(const float *field, const Grid &g, const float *iso, int n_iso, const float *grad_tris,
                              uint64_t cap, float *grad_field, void *workspace, cudaStream_t s)
{
    McParams p;
    memset(&p, 0, sizeof(p));
    p.f = field;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.sx = g.nx;
    p.sy = g.nx * g.ny;
    mc_tiles(g, p.ntx, p.ncby, p.ncbz, p.ntiles);
    p.cap = cap;
    p.err = nullptr;
    const int cstride = stored_slots(n_iso);
    McWorkspace w;
    mc_layout(g, cstride, workspace, &w);
    p.tile_cnt = w.cnt;
    p.tile_off = w.off;
    p.cases = w.cases;
    p.tcnt = w.tcnt;
    p.cstride = cstride;
    const size_t base = ((mc_workspace_bytes(g, n_iso) + 255) / 256) * 256;
    AdjParams a;
    memset(&a, 0, sizeof(a));
    a.acc = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(workspace) + base);
    a.maxbits = reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(workspace) + base + (size_t)g.N * 8);
    cudaError_t e = cudaMemsetAsync(a.acc, 0, (size_t)g.N * 8 + 256, s);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    p.use_tma = make_field_tensor_map(&map, field, g.nx, g.ny, g.nz, kBoxX, 9, 9) ? 1 : 0;
    // the tile counts are recomputed per group unless one group covers every isovalue
    uint64_t *scratch_counts = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(workspace) + base + (size_t)g.N * 8 + 64);
    const bool single = n_iso <= kMcIsoPerPass;
    for (int pass = 0; pass < 2; pass++) {
        a.pass = pass;
        for (int i0 = 0; i0 < n_iso; i0 += kMcIsoPerPass) {
            const int n = (n_iso - i0) < kMcIsoPerPass ? (n_iso - i0) : kMcIsoPerPass;
            for (int i = 0; i < kMcIsoPerPass; i++) {
                p.k[i] = (i < n) ? iso[i0 + i] : 0.0f;
                a.grad[i] = (i < n) ? grad_tris + 9ull * cap * (uint64_t)(i0 + i) : nullptr;
            }
            const bool recount = !single || pass == 0;
            switch (n) {
                case 1: e = launch_adjoint_group<1>(p, a, map, w, scratch_counts, n, recount, s); break;
                case 2: e = launch_adjoint_group<2>(p, a, map, w, scratch_counts, n, recount, s); break;
                case 3: e = launch_adjoint_group<3>(p, a, map, w, scratch_counts, n, recount, s); break;
                default: e = launch_adjoint_group<4>(p, a, map, w, scratch_counts, n, recount, s); break;
            }
            if (e != cudaSuccess) return e;
        }
    }
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_adj_finalize<<<(unsigned)(sms * 8), 256, 0, s>>>(a.acc, a.maxbits, grad_field, g.N);
    return cudaGetLastError();
}

// ---- many fields in one launch sequence ------------------------------------

size_t mc_batch_param_bytes() { return sizeof(McParams); }

int64_t mc_tile_count(int64_t nx, int64_t ny, int64_t nz)
{
    Grid g = make_grid(chr_dims{nx, ny, nz});
    int32_t ntx, ncby, ncbz;
    int64_t ntiles;
    mc_tiles(g, ntx, ncby, ncbz, ntiles);
    return ntiles;
}

// Batch scratch: tile counts, offsets, scan chunks, then the count pass's
// classification (one isovalue slot per tile).
static size_t batch_offsets(int64_t ntiles, size_t &o_off, size_t &o_chunk, size_t &o_cases, size_t &o_tcnt)
{
    const int64_t nchunks = (ntiles + kTScanChunk - 1) / kTScanChunk;
    o_off = align256(ntiles * 16);
    o_chunk = o_off + align256(ntiles * 32);
    o_cases = o_chunk + align256(nchunks * 32);
    o_tcnt = o_cases + align256((size_t)ntiles * 256 * 8);
    return o_tcnt + align256((size_t)ntiles * 256 * 4);
}

size_t mc_batch_scratch_bytes(int64_t ntiles)
{
    size_t a, b, c, d;
    return batch_offsets(ntiles, a, b, c, d);
}

bool mc_batch_fill(void *params, void *map, const float *field, int64_t nx, int64_t ny, int64_t nz, int64_t sx,
                   int64_t sy, float k, float *tris, uint64_t cap, void *scratch, int64_t total_tiles, int64_t tile0,
                   uint32_t *err)
{
    McParams &p = *reinterpret_cast<McParams *>(params);
    memset(&p, 0, sizeof(p));
    p.f = field;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.sx = sx;
    p.sy = sy;
    mc_tiles(make_grid(chr_dims{nx, ny, nz}), p.ntx, p.ncby, p.ncbz, p.ntiles);
    p.k[0] = k;
    p.tris[0] = tris;
    p.cap = cap;
    p.err = err;
    char *b = reinterpret_cast<char *>(scratch);
    size_t o_off, o_chunk, o_cases, o_tcnt;
    batch_offsets(total_tiles, o_off, o_chunk, o_cases, o_tcnt);
    p.tile_cnt = reinterpret_cast<uint4 *>(b) + tile0;
    p.tile_off = reinterpret_cast<uint64_t *>(b + o_off) + tile0 * kMcIsoPerPass;
    p.cases = reinterpret_cast<uint2 *>(b + o_cases) + tile0 * 256;
    p.tcnt = reinterpret_cast<uint32_t *>(b + o_tcnt) + tile0 * 256;
    p.cstride = 1;
    p.use_tma = make_field_tensor_map_pitched(reinterpret_cast<CUtensorMap *>(map), field, nx, ny, nz, sx, sy, kBoxX,
                                              9, 9)
                    ? 1
                    : 0;
    return p.use_tma != 0;
}

cudaError_t mc_batch_prepare(int &count_per_sm, int &emit_per_sm, int &sms)
{
    // computed once per device under the lock, published with the flag
    static int bcd[kMaxDevices] = {}, bed[kMaxDevices] = {}, nsd[kMaxDevices] = {};
    static std::atomic<bool> ready[kMaxDevices] = {};
    static std::mutex mu;
    const int dev = current_device();
    if (!ready[dev].load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(mu);
        if (!ready[dev].load(std::memory_order_relaxed)) {
            cudaError_t e = cudaFuncSetAttribute(k_mc_emit_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, kEmitSmem);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_mc_count_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, kCountSmem);
            if (e != cudaSuccess) return e;
            int ns = 0, bc = 0, be = 0;
            cudaDeviceGetAttribute(&ns, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bc, k_mc_count_batched, 256, kCountSmem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&be, k_mc_emit_batched, 256, kEmitSmem);
            bcd[dev] = bc < 1 ? 1 : bc;
            bed[dev] = be < 1 ? 1 : be;
            nsd[dev] = ns < 1 ? 1 : ns;
            ready[dev].store(true, std::memory_order_release);
        }
    }
    count_per_sm = bcd[dev];
    emit_per_sm = bed[dev];
    sms = nsd[dev];
    return cudaSuccess;
}

bool mc_debug_cases(const float *field, const Grid &g, float isovalue, uint8_t *out, void *workspace,
                    size_t workspace_bytes, cudaStream_t s, cudaError_t &err)
{
#ifdef CHR_CHECKED
    err = cudaSuccess;
    if (workspace_bytes < mc_workspace_bytes(g, 1)) {
        err = cudaErrorInvalidValue;
        return true;
    }
    McParams p;
    memset(&p, 0, sizeof(p));
    p.f = field;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.sx = g.nx;
    p.sy = g.nx * g.ny;
    mc_tiles(g, p.ntx, p.ncby, p.ncbz, p.ntiles);
    p.k[0] = isovalue;
    McWorkspace w;
    mc_layout(g, 1, workspace, &w);
    p.tile_cnt = w.cnt;
    p.tile_off = w.off;
    p.cases = w.cases;
    p.tcnt = w.tcnt;
    p.cstride = 1;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    p.use_tma = make_field_tensor_map_pitched(&map, field, g.nx, g.ny, g.nz, p.sx, p.sy, kBoxX, 9, 9) ? 1 : 0;
    McGrids G;
    if ((err = mc_prepare<1>(G)) != cudaSuccess) return true;
    const unsigned gc = (unsigned)(p.ntiles < G.count ? p.ntiles : G.count);
    k_mc_count<1><<<gc, 256, kCountSmem, s>>>(p, map);
    k_debug_cases<<<(unsigned)((p.ntiles * 256 + 255) / 256), 256, 0, s>>>(w.cases, 1, p.ntiles, p.ntx, p.ncby, g.nx,
                                                                          g.ny, g.nz, out);
    err = cudaGetLastError();
    return true;
#else
    (void)field; (void)g; (void)isovalue; (void)out; (void)workspace; (void)workspace_bytes; (void)s;
    err = cudaSuccess;
    return false;
#endif
}

uint32_t mc_bounds_word(bool reset)
{
#ifdef CHR_CHECKED
    unsigned int v = 0u, z = 0u;
    if (cudaMemcpyFromSymbol(&v, g_chr_bounds, sizeof(v)) != cudaSuccess) cudaGetLastError();
    if (reset && cudaMemcpyToSymbol(g_chr_bounds, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
    return v;
#else
    (void)reset;
    return 0u;
#endif
}

cudaError_t launch_mc_batched(const McBatchLaunch &L, cudaStream_t s)
{
    if (L.ntiles == 0) {
        cudaError_t e = cudaMemsetAsync(L.total, 0, sizeof(uint64_t), s);
        if (e != cudaSuccess) return e;
        k_box_starts<<<1, 256, 0, s>>>(nullptr, L.tile_start, L.nboxes, 0, L.total, L.box_start);
        return cudaGetLastError();
    }
    McBatch b;
    b.boxes = reinterpret_cast<const McParams *>(L.params);
    b.maps = reinterpret_cast<const CUtensorMap *>(L.maps);
    b.tile_start = L.tile_start;
    b.nboxes = L.nboxes;
    b.ntiles = L.ntiles;
    char *sc = reinterpret_cast<char *>(L.scratch);
    size_t o_off, o_chunk, o_cases, o_tcnt;
    batch_offsets(L.ntiles, o_off, o_chunk, o_cases, o_tcnt);
    TScanArgs a;
    a.cnt = reinterpret_cast<const uint4 *>(sc);
    a.off = reinterpret_cast<uint64_t *>(sc + o_off);
    a.chunk = reinterpret_cast<Sum4 *>(sc + o_chunk);
    a.ntiles = L.ntiles;
    a.nchunks = (L.ntiles + kTScanChunk - 1) / kTScanChunk;
    a.ntris = L.total;
    a.niso = 1;
    a.cap = L.cap;
    a.err = L.err;
    const unsigned gc = (unsigned)(L.ntiles < L.count_blocks ? L.ntiles : L.count_blocks);
    const unsigned ge = (unsigned)(L.ntiles < L.emit_blocks ? L.ntiles : L.emit_blocks);
    k_mc_count_batched<<<gc, 256, kCountSmem, s>>>(b, L.err);
    k_tscan_reduce<<<(unsigned)a.nchunks, kTScanThreads, 0, s>>>(a);
    k_tscan_chunks<<<1, kTScanThreads, 0, s>>>(a);
    k_tscan_apply<<<(unsigned)a.nchunks, kTScanThreads, 0, s>>>(a);
    k_mc_emit_batched<<<ge, 256, kEmitSmem, s>>>(b, L.err);
    k_box_starts<<<(unsigned)((L.nboxes + 256) / 256), 256, 0, s>>>(a.off, L.tile_start, L.nboxes, L.ntiles, L.total,
                                                                    L.box_start);
    return cudaGetLastError();
}

}  // namespace chr

// Host-side declarations shared by the libchr translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "chr.h"

namespace chr {

constexpr int kWarpsPerBlock = 8;  // codec: one warp per 8^3 brick, 8 bricks along x per block
constexpr int kMcBricksX = 4;      // marching cubes: a tile is 4 cell bricks along x (32x8x8 cells)
constexpr int kMcIsoPerPass = 4;   // isovalues classified per read of the field

struct Grid {
    int64_t nx, ny, nz, N;
    int64_t nbx, nby, nbz, nbricks;  // 8^3 vertex bricks
};

inline Grid make_grid(chr_dims d)
{
    Grid g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.N = d.nx * d.ny * d.nz;
    g.nbx = (d.nx + 7) / 8;
    g.nby = (d.ny + 7) / 8;
    g.nbz = (d.nz + 7) / 8;
    g.nbricks = g.nbx * g.nby * g.nbz;
    return g;
}

// Codec launch parameters (passed by value to the kernels).
struct CodecParams {
    const float *f;  // encode: input field
    float *out;      // decode: output field
    int64_t nx, ny, nz;
    int32_t nbx, nby, nbz, ngx;  // ngx = ceil(nbx / 8) brick groups along x
    int32_t nlevels;             // encode: levels to build; decode: levels to apply (target + 1)
    int32_t nK;
    int32_t fix;
    float e[CHR_MAX_LEVELS], two_e[CHR_MAX_LEVELS], inv2e[CHR_MAX_LEVELS];
    float K[CHR_MAX_ISO];  // the isovalues, -inf past nK
    // encoder sign check: a vertex with c candidates strictly above its value
    // keeps every sign exactly when its reconstruction lies in
    // [kdn[c], kup[c]): kup[c] the smallest of those c candidates (+inf if
    // c = 0), kdn[c] the largest of the others (-inf if there are none)
    float kup[CHR_MAX_ISO + 1], kdn[CHR_MAX_ISO + 1];
    uint4 *recs[CHR_MAX_LEVELS];
    uint32_t *words[CHR_MAX_LEVELS];
    uint16_t *exc_idx[CHR_MAX_LEVELS];
    uint32_t *exc_val[CHR_MAX_LEVELS];
    // decode output box: vertices [box_org, box_org + box_dim) of the grid,
    // written x-fastest with the box's own strides; bricks box_brick0 ..
    // box_brick0 + box_bricks cover it (the whole grid for chr_reconstruct)
    int64_t box_org[3], box_dim[3];
    int64_t out_sx, out_sy;  // output row and plane pitch in floats
    int32_t box_brick0[3], box_bricks[3];
    float2 *range;  // optional per-brick (min, max) of the decoded values
    // encode: per brick and level the value ranges of 8 vertex subsets of the
    // brick (kIdxParts float2 each, see k_encode), combined into the index by
    // k_brick_index; NULL: no index
    float2 *idx_part;
    float2 *index[CHR_MAX_LEVELS];  // the index per level (nbricks float2)
    // encode scratch: fixed per-brick slots (512 words, 512 exception entries)
    uint32_t *slot_words[CHR_MAX_LEVELS];
    uint16_t *slot_idx[CHR_MAX_LEVELS];
    uint32_t *slot_val[CHR_MAX_LEVELS];
};

// Encode scratch per level: 512 words + 512 exception entries per brick.
inline size_t encode_slot_bytes(int64_t nbricks) { return (size_t)nbricks * 512 * (4 + 2 + 4); }

cudaError_t launch_encode(const CodecParams &p, cudaStream_t s);
// The per-brick value index (min, max over the vertices of each brick's
// cells, NaN as +inf, (+inf, -inf) for a brick without cells) of every
// level, from the encoder's per-brick parts (p.idx_part -> p.index[l]).
constexpr int kIdxParts = 8;
inline size_t index_part_bytes(int64_t nbricks, int nlevels) { return (size_t)nbricks * nlevels * kIdxParts * 8; }
cudaError_t launch_brick_index(const CodecParams &p, cudaStream_t s);
cudaError_t launch_compact(const CodecParams &p, cudaStream_t s);
cudaError_t launch_decode(const CodecParams &p, cudaStream_t s);
// Decode of many CHRs in one launch (descs, brick_start [nboxes+1] on the device).
cudaError_t launch_decode_batched(const CodecParams *d_descs, const int64_t *d_brick_start, int32_t nboxes,
                                  int64_t total_bricks, int warps_per_block, cudaStream_t s);
// Exclusive scans of the widths and exception counts of each level's records;
// totals[2*l] = sum of w, totals[2*l+1] = exceptions.  scratch needs
// scan_scratch_bytes(nbricks, nlevels).
size_t scan_scratch_bytes(int64_t nbricks, int nlevels);
cudaError_t launch_scan_records(uint4 *const *recs, int nlevels, int64_t nbricks, void *scratch, uint64_t *totals,
                                cudaStream_t s);

// Checked builds: the bounds word of the marching-cubes and the codec kernels
// (non-zero once an index failed its test); 0 in normal builds.  Synchronises.
uint32_t mc_bounds_word(bool reset);
// Checked builds: the single pass's unpublished test tile (-1: none); false
// in normal builds.
bool mc_set_unpublished_tile(int64_t tile);
// Checked builds, test only: every later extraction writes each triangle's
// cell index to cells (NULL: stop); false in normal builds.
bool mc_debug_set_tri_cells(uint32_t *cells);
// Checked builds, test only: the count pass's case bytes of one isovalue,
// per cell in grid order with corner (ox, oy, oz) at bit ox + 2 oy + 4 oz;
// false in normal builds.  err: the launch status.
bool mc_debug_cases(const float *field, const Grid &g, float isovalue, uint8_t *out, void *workspace,
                    size_t workspace_bytes, cudaStream_t s, cudaError_t &err);
uint32_t codec_bounds_word(bool reset);

// Marching cubes over a plain field, per group of up to 4 isovalues one
// single-pass launch, or count + scan + emit on large grids when the
// workspace holds the classification.  mc_workspace_bytes: the tile arrays
// plus that classification; mc_workspace_min_bytes: the tile arrays alone.
size_t mc_workspace_bytes(const Grid &g, int n_iso);
size_t mc_workspace_min_bytes(const Grid &g, int n_iso);
// index: the field's value index (nbricks (min, max) over each 8^3 brick's
// cell vertices, a CHR level's), or NULL; bricks whose range does not
// straddle an isovalue are not classified for it (same output).
cudaError_t launch_mc(const float *field, const Grid &g, const float *iso, int n_iso, float *tris, uint64_t cap,
                      uint64_t *ntris, uint32_t *err, void *workspace, size_t workspace_bytes, cudaStream_t s,
                      const float2 *index = nullptr);
// The same over a pitched field: value (x, y, z) at field[x + sx*y + sy*z].
cudaError_t launch_mc_pitched(const float *field, const Grid &g, int64_t sx, int64_t sy, const float *iso, int n_iso,
                              float *tris, uint64_t cap, uint64_t *ntris, uint32_t *err, void *workspace,
                              size_t workspace_bytes, cudaStream_t s, const float2 *index = nullptr);

// Decode + marching cubes of one CHR level in one launch per group of up to
// 4 isovalues (k_mc_chr): levels 0..nlevels-1 of the stream below are
// decoded tile by tile into shared memory and meshed there; same output as
// launch_decode followed by launch_mc.  index: the level's value index, or
// NULL to classify every brick.  workspace: mc_workspace_min_bytes.
struct ChrMcLevels {
    const uint4 *recs[CHR_MAX_LEVELS];
    const uint32_t *words[CHR_MAX_LEVELS];
    const uint16_t *exc_idx[CHR_MAX_LEVELS];
    const uint32_t *exc_val[CHR_MAX_LEVELS];
    float two_e[CHR_MAX_LEVELS];
    int32_t nlevels;
    const float2 *index;
};
cudaError_t launch_mc_chr(const ChrMcLevels &c, const Grid &g, const float *iso, int n_iso, float *tris, uint64_t cap,
                          uint64_t *ntris, uint32_t *err, void *workspace, size_t workspace_bytes, cudaStream_t s);

// Marching cubes of many fields (each with its own isovalue and pitch) in one
// launch sequence: count over the concatenated tile list, one scan, emit.
// Every field's triangles land in one buffer, field i's from box_start[i];
// box_start[nboxes] = total (> cap: CHR_ERR_OVERFLOW in err).
struct McBatchLaunch {
    const void *params;      // device McParams [nboxes] (mc_batch_fill)
    const void *maps;        // device CUtensorMap [nboxes], 64-byte aligned
    const int64_t *tile_start;  // device [nboxes + 1]
    int32_t nboxes;
    int64_t ntiles;
    void *scratch;           // mc_batch_scratch_bytes(ntiles)
    uint64_t *total;         // device [1]
    uint64_t *box_start;     // device [nboxes + 1]
    uint64_t cap;
    uint32_t *err;
    int count_blocks, emit_blocks;  // grid sizes of the two tile kernels
};
size_t mc_batch_param_bytes();
int64_t mc_tile_count(int64_t nx, int64_t ny, int64_t nz);
size_t mc_batch_scratch_bytes(int64_t ntiles);
// Host: field i's parameters and tensor map (false if no tensor map can be made).
bool mc_batch_fill(void *params, void *map, const float *field, int64_t nx, int64_t ny, int64_t nz, int64_t sx,
                   int64_t sy, float k, float *tris, uint64_t cap, void *scratch, int64_t total_tiles, int64_t tile0,
                   uint32_t *err);
cudaError_t mc_batch_prepare(int &count_per_sm, int &emit_per_sm, int &sms);
cudaError_t launch_mc_batched(const McBatchLaunch &L, cudaStream_t s);

// Adjoint of the vertex positions: dL/dfield from dL/dtris (forward layout).
size_t mc_adjoint_workspace_bytes(const Grid &g, int n_iso);
cudaError_t launch_mc_adjoint(const float *field, const Grid &g, const float *iso, int n_iso, const float *grad_tris,
                              uint64_t cap, float *grad_field, void *workspace, cudaStream_t s);

// Mean distance of points to an original field's isosurface, and its gradient.
size_t dist_loss_workspace_bytes(uint64_t npts);
cudaError_t launch_dist_loss(const float *orig, const Grid &g, float k, const float *pts, uint64_t npts, double *loss,
                             float *grad_pts, void *workspace, cudaStream_t s);

// Reports (report.cu): the sum of |g| over every 8^3 brick into out
// (nbricks floats, bricks x fastest); the number of cells whose case byte
// at each of the nK host isovalues K is the same in fields a and b, summed
// over the isovalues, into *count (device).
cudaError_t launch_brick_abs_sum(const float *g, const Grid &G, float *out, cudaStream_t s);
cudaError_t launch_case_agreement(const float *a, const float *b, const Grid &G, const float *K, int nK,
                                  unsigned long long *count, cudaStream_t s);

// Error-bound translation (selection over D).  mode 0: the minimum
// (minbits) and |D| (count); mode 1: |D| and a 4096-bin histogram of the
// elements' top 12 bits (hist); mode 2: every element whose top 12 bits equal
// prefix, its low 20 bits appended to coll (at most cap; ncoll counts them).
struct TranslateScratch {
    unsigned long long *hist;  // 4096 counters
    unsigned long long *count; // |D|
    unsigned int *minbits;     // min D as float bits
    unsigned long long *ncoll; // elements appended (modes 2, 3)
    unsigned long long *count_lo;  // elements below lo_bits (mode 3)
    uint32_t *coll;            // modes 2, 3 output
    unsigned long long cap;
};
size_t translate_scratch_bytes();
// One walk over the field's edges (mode 0 minimum, 1 histogram, 2 collect
// the bucket `prefix`, 3 count below lo_bits and collect [lo_bits,
// hi_bits)); item_step > 1 walks every item_step-th item only (a sample);
// n_items (if set) receives the number of items of the whole walk.
cudaError_t launch_translate_pass(const float *field, const Grid &g, const float *K, int nK, int mode,
                                  uint32_t prefix, TranslateScratch sc, cudaStream_t s, uint32_t lo_bits = 0,
                                  uint32_t hi_bits = 0, int64_t item_step = 1, int64_t *n_items = nullptr);
// Histogram (1024 bins, hist) of bits [shift, shift+10) of the n collected
// values whose bits from shift+10 up equal `above`.
cudaError_t launch_translate_select(const uint32_t *coll, unsigned long long n, int shift, uint32_t above,
                                    unsigned long long *hist, cudaStream_t s);

void set_error(const std::string &msg);

// Per-device one-time setup (kernel attributes, occupancy): the current
// device's index, clamped to the table size used by the launchers.
constexpr int kMaxDevices = 64;
inline int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        d = 0;
    }
    return (d >= 0 && d < kMaxDevices) ? d : 0;
}

}  // namespace chr

struct chr_handle;

namespace chr {

// The library's own stream-ordered memory pool on the current device (for a
// NULL chr_allocator): freed blocks stay in the pool for the next call
// instead of going back to the driver at every synchronisation; NULL if the
// pool cannot be made.
cudaMemPool_t library_pool();

// Device memory from a caller's chr_allocator, or the library pool.
struct Alloc {
    chr_allocator a{};
    bool dflt = true;
    cudaStream_t s = nullptr;

    Alloc(const chr_allocator *al, cudaStream_t st) : s(st)
    {
        if (al) {
            a = *al;
            dflt = false;
        }
    }
    void *get(size_t n)
    {
        if (n == 0) n = 16;
        n = (n + 255) & ~size_t(255);
        void *p = nullptr;
        if (dflt) {
            cudaMemPool_t mp = library_pool();
            if (!mp || cudaMallocFromPoolAsync(&p, n, mp, s) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
        } else {
            p = a.alloc(n, s, a.ctx);
        }
        return p;
    }
    void put(void *p, size_t n)
    {
        if (!p) return;
        if (n == 0) n = 16;
        n = (n + 255) & ~size_t(255);
        if (dflt)
            cudaFreeAsync(p, s);
        else
            a.free(p, n, s, a.ctx);
    }
};

chr_status fail(chr_status st, const std::string &msg);
chr_status cuda_fail(cudaError_t e, const char *where);
// Decode parameters of a handle (every level, whole grid as the output box).
void fill_codec_params(const chr_handle *h, CodecParams &p);
void set_box(CodecParams &p, const Grid &g, int64_t x0, int64_t y0, int64_t z0, int64_t bx, int64_t by, int64_t bz);

}  // namespace chr

struct chr_handle {
    chr::Grid g;
    chr_dims dims;
    uint32_t nlevels, n_iso, topo_mode, flags;
    float topo_accuracy, eb_translated;
    uint64_t D_count;
    float eb[CHR_MAX_LEVELS], two_e[CHR_MAX_LEVELS], inv2e[CHR_MAX_LEVELS];
    float iso[CHR_MAX_ISO];
    uint64_t nwords[CHR_MAX_LEVELS], nexc[CHR_MAX_LEVELS];
    uint4 *d_recs[CHR_MAX_LEVELS];
    uint32_t *d_words[CHR_MAX_LEVELS];
    uint16_t *d_exc_idx[CHR_MAX_LEVELS];
    uint32_t *d_exc_val[CHR_MAX_LEVELS];
    // the value index per level (Sec. 2.1): nbricks (min, max) over each
    // brick's cell vertices; NULL when the handle has none (a version-1
    // byte string), and then nothing is skipped
    float2 *d_index[CHR_MAX_LEVELS];
    bool has_index;
    size_t sz_recs, sz_words[CHR_MAX_LEVELS], sz_exc_idx[CHR_MAX_LEVELS], sz_exc_val[CHR_MAX_LEVELS];
    // the arrays above live in two allocations: every level's records and
    // index in one block, every level's packed words and exception slots and
    // values in the other (each array 256-byte aligned inside its block)
    void *d_rec_block, *d_pay_block;
    size_t sz_rec_block, sz_pay_block;
    chr_allocator alloc;
    bool default_alloc;
    cudaStream_t stream;
};

/*
 * chr.h — C ABI of libchr.so: topology-preserving compression and marching
 * cubes on one GB300 GPU (arXiv 2408.05462, Li & Chen, "Accelerating
 * In-transit Isosurface Generation With Topology Preserving Compression").
 *
 * The paper's workflow (Sec. 2): the data source compresses each field into a
 * Compressed Hierarchical Representation (CHR); the visualization side asks
 * for an isovalue and an accuracy, reconstructs the field and generates the
 * isosurface.  Topology preservation (Sec. 2.2) means every marching-cubes
 * cell keeps its case after compression.
 *
 * Conventions for every call:
 *  - Fields are float32, nx*ny*nz values, x fastest: index x + nx*(y + ny*z).
 *    Grid coordinates of vertex (x,y,z) are (x,y,z) (unit spacing).
 *  - Pointers named d_* are device pointers on the current CUDA device; the
 *    caller owns them and keeps them alive until the work on `stream` ends.
 *    Host arrays are read before the call returns.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued asynchronously unless a call says it synchronises.
 *  - Every call returns a chr_status and never throws.  Argument errors are
 *    reported before any work is enqueued, as CHR_ERR_INVALID (or
 *    CHR_ERR_CORRUPT for bad serialized bytes); chr_last_error() then holds a
 *    message for the calling thread.
 *  - Device-side conditions (output overflow, a wait that gave up) are
 *    reported through a caller-provided device error word: bit
 *    (1u << CHR_ERR_OVERFLOW) or (1u << CHR_ERR_TIMEOUT) is OR-ed into it.
 */
#ifndef CHR_H
#define CHR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHR_MAX_LEVELS 8
#define CHR_MAX_ISO 16
#define CHR_BRICK 8 /* codec bricks and marching-cubes tiles are 8^3 */

typedef enum chr_status {
    CHR_OK = 0,
    CHR_ERR_INVALID = 1,  /* bad argument; nothing was enqueued            */
    CHR_ERR_OOM = 2,      /* the allocator returned NULL                   */
    CHR_ERR_CUDA = 3,     /* a CUDA runtime call failed                    */
    CHR_ERR_OVERFLOW = 4, /* device flag: an output buffer was too small   */
    CHR_ERR_TIMEOUT = 5,  /* device flag: a bounded wait gave up           */
    CHR_ERR_CORRUPT = 6   /* serialized bytes failed validation            */
} chr_status;

typedef struct chr_dims {
    int64_t nx, ny, nz; /* each >= 2; nx*ny*nz < 2^32 */
} chr_dims;

/*
 * Stream-ordered device allocator supplied by the caller.  alloc returns a
 * device pointer of at least `bytes` bytes (256-byte aligned) usable on
 * `stream`, or NULL; free releases it after the work already enqueued on
 * `stream`.  A NULL chr_allocator* selects the library's own stream-ordered
 * pool on the current device (cudaMallocFromPoolAsync / cudaFreeAsync),
 * which keeps freed memory for later calls; chr_pool_trim gives it back.
 */
typedef struct chr_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} chr_allocator;

/* How topology is preserved (Sec. 2.2). */
enum {
    CHR_TOPO_NONE = 0,     /* error bounds only                                  */
    CHR_TOPO_FIX = 1,      /* every vertex keeps the side of every candidate k:   */
                           /* vertices whose reconstruction would change side    */
                           /* are stored exactly (exceptions)                     */
    CHR_TOPO_TRANSLATE = 2 /* Sec. 2.2 error-bound translation: every level's    */
                           /* bound becomes min(e_l, the n-th smallest of D)      */
};

typedef struct chr_params {
    uint32_t nlevels;          /* 1..CHR_MAX_LEVELS accuracy levels (Sec. 2 "accuracy")      */
    const float *error_bounds; /* host [nlevels]: absolute bounds, finite, > 0, strictly      */
                               /* decreasing, < 1e37                                          */
    const float *isovalues;    /* host [n_iso]: candidate isovalues K (finite)                */
    uint32_t n_iso;            /* 0..CHR_MAX_ISO                                              */
    uint32_t topo_mode;        /* CHR_TOPO_*; FIX and TRANSLATE need n_iso >= 1               */
    float topo_accuracy;       /* TRANSLATE: fraction in (0,1]; 1 = min D, otherwise the      */
                               /* element of rank floor((1-accuracy)*|D|)                     */
    uint32_t flags;            /* reserved, must be 0                                         */
} chr_params;
/* Where chr_params departs from a block-structured compressor's options:
 * there is no block size (the paper's 64^3/128^3 domain blocks of Sec. 2.1
 * are the caller's boxes, each compressed on its own; the format's unit is
 * the 8^3 brick, with a value index per brick, chr_brick_index), and flags
 * bit 0 (the paper's differentiated error control per block) is not
 * implemented: every vertex keeps every level's bound. */

typedef struct chr_handle chr_handle; /* opaque; owns device buffers */

typedef struct chr_stats_t {
    chr_dims dims;
    uint32_t nlevels, n_iso, topo_mode, reserved;
    uint64_t nbricks;                       /* 8^3 bricks, x fastest                         */
    float eb[CHR_MAX_LEVELS];               /* bounds in effect per level                    */
    float eb_translated;                    /* TRANSLATE: the translated bound, else +inf    */
    float topo_accuracy;
    uint64_t translate_D_count;             /* TRANSLATE: |D|                                */
    uint64_t payload_words[CHR_MAX_LEVELS]; /* packed 32-bit words per level                 */
    uint64_t exceptions[CHR_MAX_LEVELS];    /* exactly stored vertices per level             */
    uint64_t level_bytes[CHR_MAX_LEVELS];   /* records + payload + exceptions of the level   */
} chr_stats_t;

/*
 * chr_compress — build a CHR of d_field (Sec. 2: "compressed into a
 * Compressed Hierarchical Representation"; Sec. 2.2 topology preservation).
 *
 * Level l holds residual codes q with step 2*e_l: level 0 quantises the
 * field, level l>0 the residual f - R_{l-1}.  R_l = R_{l-1} + q*2e_l in
 * float32, and every vertex satisfies |f - R_l| < e_l strictly (vertices that
 * would not are stored exactly).  With CHR_TOPO_FIX, (R_l < k) == (f < k) for
 * every vertex, level and k in isovalues, so every marching-cubes case of
 * every candidate isovalue is preserved at every level.  Codes are predicted
 * per 8^3 brick (3-D Lorenzo or none, whichever packs narrower), zig-zag
 * coded and bit-packed at the brick's width.
 *
 * Synchronises `stream` once (to size the packed stream).  *out receives a
 * handle whose buffers come from `alloc` (NULL: the library pool); release it
 * with chr_free.  d_field is only read.
 */
chr_status chr_compress(const float *d_field, chr_dims dims, const chr_params *params, const chr_allocator *alloc,
                        void *stream, chr_handle **out);

/*
 * chr_reconstruct — decode level `level` (0-based, < nlevels) into d_out
 * (caller-owned, nx*ny*nz floats): the visualization side's reconstruction at
 * the requested accuracy (Sec. 2).  Levels 0..level are unpacked, their
 * prediction undone, accumulated in float32 and the stored exact vertices
 * restored.  Bit-identical to the R_level the encoder checked.  Asynchronous.
 */
chr_status chr_reconstruct(const chr_handle *h, uint32_t level, float *d_out, void *stream);

/*
 * chr_reconstruct_box — chr_reconstruct restricted to the vertices
 * [x0, x0+box.nx) x [y0, y0+box.ny) x [z0, z0+box.nz) of the grid (each
 * box side >= 1 and inside the grid): only the 8^3 bricks that meet the box
 * are decoded, and d_out (caller-owned, box.nx*box.ny*box.nz floats, x
 * fastest) receives exactly the matching values of the full reconstruction.
 * The visualization side's request for a subvolume at a given accuracy
 * (Sec. 2).  Asynchronous.
 */
chr_status chr_reconstruct_box(const chr_handle *h, uint32_t level, int64_t x0, int64_t y0, int64_t z0, chr_dims box,
                               float *d_out, void *stream);

/*
 * chr_serve_request — one request of the visualization side in one call:
 * decode the box [x0, x0+box.nx) x [y0, ...) x [z0, ...) of level `level`
 * (every side >= 2 and inside the grid), run marching cubes on it at
 * `isovalue` with room for cap_tris triangles, and copy (triangle count,
 * error word) as two uint64 to h_result (host memory, pinned for a truly
 * asynchronous copy) when the stream gets there.  d_mem: caller-owned device
 * memory, 256-byte aligned, of at least chr_serve_request_bytes(box,
 * cap_tris) bytes; the triangles (box-local grid coordinates, the layout of
 * isosurface_extract with one isovalue) start at d_mem, the rest is scratch
 * (the box field, pitched to 16-byte rows, and the marching-cubes
 * workspace).  Equal, bit for bit, to chr_reconstruct_box +
 * isosurface_extract of the box.  Asynchronous.
 */
size_t chr_serve_request_bytes(chr_dims box, uint64_t cap_tris);
chr_status chr_serve_request(const chr_handle *h, uint32_t level, int64_t x0, int64_t y0, int64_t z0, chr_dims box,
                             float isovalue, void *d_mem, size_t mem_bytes, uint64_t cap_tris, uint64_t *h_result,
                             void *stream);

/*
 * chr_box_tri_bound — host-side upper bound on the triangles of the box
 * [x0, x0+box.nx) x [y0, ...) x [z0, ...) at `isovalue`, from a per-brick
 * index on the host: h_min/h_max [nbz][nby][nbx] hold each brick's value
 * range widened by its +x, +y and +z neighbours (the vertices its cells
 * touch, as from chr_brick_range).  Counts 5 triangles for every cell of
 * the box in a brick whose range straddles the isovalue (min < k <= max);
 * 0 for bad arguments.  No device work.
 */
uint64_t chr_box_tri_bound(const float *h_min, const float *h_max, int64_t nbx, int64_t nby, int64_t nbz, int64_t x0,
                           int64_t y0, int64_t z0, chr_dims box, float isovalue);

/*
 * chr_brick_range — per-brick value range of level `level`: d_range
 * (caller-owned, 2 floats per 8^3 brick, brick (bx, by, bz) at index
 * bx + nbx*(by + nby*bz), nbx = ceil(nx/8) and so on) receives the (min, max)
 * of the reconstructed values at the brick's grid vertices, NaN counted as
 * +inf.  An index of the CHR (Sec. 2: the visualization side picks the
 * blocks a request needs): a cell whose 8 corners lie in bricks whose
 * combined range does not straddle k (min < k <= max) has no triangles.
 * Decodes the level without writing the field.  d_range must be 8-byte
 * aligned.  Asynchronous.
 */
chr_status chr_brick_range(const chr_handle *h, uint32_t level, float *d_range, void *stream);

/*
 * chr_topo_translate — the error-bound translation of Sec. 2.2 on its own:
 * D holds, for every grid edge (s0,s1) with min < k < max and every k in
 * isovalues, d0 = k - min and d1 = max - k, each rounded toward -inf in
 * float32.  *eb_out = element of rank floor((1 - accuracy)*|D|) of D in
 * ascending order (min D for accuracy 1), +inf when D is empty;
 * *count_out = |D| (may be NULL).  Exact (radix selection on the float bits).
 * An edge with a NaN end adds nothing; an infinite end makes its own
 * difference +inf; an isovalue listed twice adds its elements twice.
 * Synchronises `stream`; scratch comes from `alloc` (NULL: the library pool).
 */
chr_status chr_topo_translate(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                              float accuracy, const chr_allocator *alloc, void *stream, float *eb_out,
                              uint64_t *count_out);

/*
 * isosurface_workspace_size — bytes of device scratch for isosurface_extract
 * with these dims and number of isovalues: per 32x8x8-cell tile its status
 * word, triangle counts and output offsets, and the counting pass's
 * classification (12 bytes per 8 cells and isovalue, at most 4 isovalues at
 * a time) for grids large enough to take two passes.
 */
size_t isosurface_workspace_size(chr_dims dims, uint32_t n_iso);

/*
 * isosurface_workspace_min_size — the smallest workspace isosurface_extract
 * accepts: the tile arrays alone (48 bytes per tile plus the scan chunks);
 * every group then takes the single pass (same output).
 */
size_t isosurface_workspace_min_size(chr_dims dims, uint32_t n_iso);

/*
 * isosurface_extract — marching cubes (Sec. 2.2, Lorensen & Cline) of
 * d_field for n_iso (1..CHR_MAX_ISO) isovalues in one pass per 4 isovalues.
 *
 * A vertex is inside when v < k (NaN is outside).  Each cell's triangles come
 * from the case table (gen_mc_table.py): faces with two diagonal inside
 * corners keep them apart, triangles are oriented with normals pointing away
 * from the inside, and a vertex on edge (v0,v1) (v0 the lower end) sits at
 * v0 + t*(v1 - v0), t = (k - f0)/(f1 - f0) in float32.
 *
 * Output (triangle soup): isovalue j's triangles start at
 * d_tris + 9*j*cap_tris; triangle t is 3 vertices of (x,y,z) floats.  Order:
 * 8^3-cell bricks in x-fastest brick order, cells of a brick in x-fastest
 * order, triangles of a cell in table order.  d_ntris[j] (device uint64)
 * receives isovalue j's true triangle count even when it exceeds cap_tris;
 * triangles beyond cap_tris are not written and bit CHR_ERR_OVERFLOW is set in
 * *d_err.  d_err (device uint32) is cleared by the call; may be NULL.
 * d_workspace: device scratch of workspace_bytes (at least
 * isosurface_workspace_min_size(), else CHR_ERR_INVALID), overwritten by the
 * call.  A group of n isovalues on fewer than 2048*n^3 tiles (or any group,
 * with less than isosurface_workspace_size() bytes) takes one launch
 * (k_mc_fused): blocks claim tiles in order and find each tile's output
 * offset from the counts the tiles before it publish (bounded waits; a wait
 * that gives up sets CHR_ERR_TIMEOUT).  Larger grids with the full
 * workspace take a counting pass, a scan of the tile counts and an
 * emitting pass.  Same output either way.  Asynchronous.
 */
chr_status isosurface_extract(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                              float *d_tris, uint64_t cap_tris, uint64_t *d_ntris, uint32_t *d_err, void *d_workspace,
                              size_t workspace_bytes, void *stream);

/*
 * chr_isosurface — the visualization side of Sec. 2 in one call: decode
 * level `level` of the CHR and run marching cubes on it for n_iso
 * (1..CHR_MAX_ISO) isovalues.  Equal, bit for bit, to chr_reconstruct
 * followed by isosurface_extract on the decoded field: same triangle layout,
 * order, counts (d_ntris, device, n_iso uint64, true counts even past
 * cap_tris) and error word (d_err, device uint32, cleared by the call; may be
 * NULL).  Every flag combination gives that same output.
 *
 * Default: the decoder writes the level into a field (d_field_out, or
 * scratch when NULL) and the marching cubes read it back, in the form
 * isosurface_extract takes with its full workspace.
 * CHR_ISO_INDEX: the CHR's value index (chr_brick_index) decides which 8^3
 * bricks can hold a crossing of each isovalue (min < k <= max over the
 * brick's cell vertices) and the others are not classified for it; their
 * cells have no triangles.  (On GB300 the tile classification is bound by
 * latency rather than by its instructions, and the index read costs
 * registers: this measured no faster, so it is not the default.)
 * CHR_ISO_FUSED: one launch per group of 4 isovalues, in which persistent
 * blocks claim 32x8x8-cell tiles in order, decode each tile's vertex box
 * (its 4 bricks and the first vertex planes of the bricks after them,
 * levels 0..level with their exact vertices) straight into shared memory
 * and mesh it there: the field never goes to memory; with CHR_ISO_INDEX a
 * tile none of whose bricks crosses an isovalue is not even decoded.  On
 * GB300 this form is the slower one (the per-tile decode is bound by memory
 * latency inside each block), so it is not the default; d_field_out, when
 * not NULL, is written by one more decoding launch.
 * Scratch (the field, the marching-cubes workspace; with CHR_ISO_FUSED only
 * the tile arrays, 48 bytes per tile) comes from `alloc` (NULL: the library
 * pool) and is released, stream-ordered, before the call returns;
 * CHR_ERR_OOM when the allocator returns NULL, with no kernel enqueued.
 * Asynchronous.  (chr_params has no `block` field: the paper's 64^3/128^3
 * domain blocks are the caller's boxes here, and the format's unit is the
 * 8^3 brick; chr_params.flags stays reserved, see chr_compress.)
 */
#define CHR_ISO_INDEX 1u
#define CHR_ISO_FUSED 2u
chr_status chr_isosurface(const chr_handle *h, uint32_t level, const float *isovalues, uint32_t n_iso,
                          float *d_field_out, float *d_tris, uint64_t cap_tris, uint64_t *d_ntris, uint32_t *d_err,
                          uint32_t flags, const chr_allocator *alloc, void *stream);

/*
 * chr_brick_index — the CHR's value index of level `level` (Sec. 2.1: an
 * index over the blocks so that isovalue-based pruning can skip them):
 * d_out (caller-owned, 8-byte aligned, 2 floats per 8^3 brick, brick (bx,
 * by, bz) at bx + nbx*(by + nby*bz)) receives (min, max) of the level's
 * reconstructed values over the vertices of the brick's cells, x in
 * [8bx, min(8bx+8, nx-1)] and likewise along y and z (the brick and the
 * first vertex plane of its +x, +y and +z neighbours), NaN counted as
 * +inf; (+inf, -inf) for a brick without cells.  A cell of the brick can
 * cross k only if min < k <= max.  chr_compress builds it (the encoder
 * reduces each brick's reconstruction, a small pass assembles the
 * neighbours' planes); it is stored in the byte string.  CHR_ERR_INVALID
 * for a handle read from a version-1 string (no index).  Asynchronous.
 */
chr_status chr_brick_index(const chr_handle *h, uint32_t level, float *d_out, void *stream);

/*
 * isosurface_backward — adjoint of isosurface_extract's vertex positions with
 * respect to the field (this library's reading of attributing isosurface
 * error to grid points; the paper's translation of Sec. 2.2 runs from
 * isosurface error to field error).  A vertex on edge (i0,i1) sits at
 * p_axis = x0 + t, t = (k - f0)/(f1 - f0), so dp_axis/df0 = (t-1)/(f1-f0) and
 * dp_axis/df1 = -t/(f1-f0).  d_grad_tris holds dL/dp in isosurface_extract's
 * layout (isovalue j at d_grad_tris + 9*j*cap_tris, same order); triangles
 * past cap_tris are ignored.  d_grad_field (nx*ny*nz floats) receives
 * dL/dfield, summed over every vertex and isovalue.  The sums are exact
 * integer sums of fixed-point terms scaled from the largest term, so the
 * result does not depend on scheduling; non-finite terms are skipped.
 * d_workspace: at least isosurface_backward_workspace_size() bytes.
 * Asynchronous.
 */
size_t isosurface_backward_workspace_size(chr_dims dims, uint32_t n_iso);
chr_status isosurface_backward(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                               const float *d_grad_tris, uint64_t cap_tris, float *d_grad_field, void *d_workspace,
                               size_t workspace_bytes, void *stream);

/*
 * isosurface_distance_loss — mean first-order distance of npts points
 * (x,y,z floats, e.g. a triangle soup) to the isovalue surface of an original
 * field: |F(p) - k| / |grad F(p)|, F the trilinear interpolant in the cell
 * with lower corner clamp(floor(p), 0, n-2); points where grad F vanishes
 * count as 0.  *d_loss (device double) receives the mean, d_grad_points (may
 * be NULL) its gradient with respect to every point coordinate.  Computed in
 * double, reduced in a fixed order.  d_workspace: at least
 * isosurface_distance_loss_workspace_size(npts) bytes.  Asynchronous.
 */
size_t isosurface_distance_loss_workspace_size(uint64_t npts);
chr_status isosurface_distance_loss(const float *d_orig_field, chr_dims dims, float isovalue, const float *d_points,
                                    uint64_t npts, double *d_loss, float *d_grad_points, void *d_workspace,
                                    size_t workspace_bytes, void *stream);

/*
 * chr_brick_abs_sum — for every 8^3 brick (brick (bx, by, bz) at bx + nbx*(by
 * + nby*bz)) the sum of |g| over its vertices, into d_out (caller-owned,
 * nbricks floats).  Applied to isosurface_backward's gradient field it ranks
 * the bricks whose refinement moves a loss on the mesh most (this library's
 * reading of attributing isosurface error to blocks; the paper refines whole
 * blocks, Sec. 2.1).  Each brick is summed in a fixed order (a lane's rows
 * in x order, then a butterfly over the warp), so the result does not depend
 * on scheduling.  Asynchronous.
 */
chr_status chr_brick_abs_sum(const float *d_g, chr_dims dims, float *d_out, void *stream);

/*
 * chr_case_agreement — the number of cells whose marching-cubes case byte
 * at each of the n_iso (1..16, host array, no NaN) isovalues is the same in
 * the fields d_a and d_b (same dims), summed over the isovalues, into
 * *d_count (device, 8-byte aligned; set, not added to).  Divided by
 * n_iso * (nx-1)(ny-1)(nz-1) it is the topology accuracy of Sec. 2.2, the
 * share of cells whose isosurface topology survives compression.
 * Asynchronous.
 */
chr_status chr_case_agreement(const float *d_a, const float *d_b, chr_dims dims, const float *isovalues,
                              uint32_t n_iso, unsigned long long *d_count, void *stream);

/*
 * isosurface_extract_noalloc — isosurface_extract for callers that may not
 * allocate device memory: code inside an application or framework that owns
 * all GPU memory through its own pool, plugins and callbacks that must not
 * allocate, and latency-bound loops that cannot afford an allocation (which
 * may synchronise the device).  The paper has no counterpart; this is a
 * deployment convenience of this library.
 *
 * Same arguments, outputs and results as isosurface_extract, without the
 * workspace: the scratch is one fixed 4 MiB array in the library's device
 * image, present on every GPU that loads the library until the process
 * exits.  Grids needing more scratch than that (more than about 87,000 tiles
 * of 32x8x8 cells, i.e. roughly 178 million cells; a 512^3 grid fits) are
 * rejected with CHR_ERR_INVALID before any work is enqueued.
 * Every call looks up the array's device address on the current device
 * (so a device reset needs nothing more), and runs the single pass on the
 * minimum workspace (isosurface_workspace_min_size).  Make the first call
 * on a device before any stream capture.
 * All calls share the one array, so calls whose work overlaps on a GPU race
 * on it and must be serialised by the caller.  No call clears it: every
 * scratch value is written before it is read.  Asynchronous.
 */
chr_status isosurface_extract_noalloc(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                                      float *d_tris, uint64_t cap_tris, uint64_t *d_ntris, uint32_t *d_err,
                                      void *stream);

/*
 * chr_serialize — the CHR as one little-endian byte string, the form that
 * crosses the network in the paper's in-transit setting (Sec. 3 streams it
 * over a WAN).  Writes into host_buf when cap >= the size; *need always
 * receives the size.  Synchronises `stream`.
 * Layout: "CHR1", u32 version 2, i64 nx,ny,nz, u32 nlevels, n_iso, topo_mode,
 * flags, f32 topo_accuracy, eb_translated, u64 translate_D_count,
 * f32 eb[nlevels], f32 isovalues[n_iso], then per level u64 nwords, u64 nexc,
 * then per level: records (nbricks x {u32 wsum, u32 exc_off, i32 anchor,
 * u32 w | mode<<8 | nexc<<16}), u32 words[nwords], u16 exc_idx[nexc] padded
 * to 4 bytes, u32 exc_val[nexc] (value bits); then per level the value
 * index, nbricks x {f32 min, f32 max} (see chr_brick_index).  Version 1
 * strings (no index) are still read; their handles classify every brick.
 */
chr_status chr_serialize(const chr_handle *h, void *host_buf, size_t cap, size_t *need, void *stream);

/*
 * chr_deserialize — validate a byte string from chr_serialize on the host
 * (CHR_ERR_CORRUPT on any inconsistency: sizes, widths > 32, prefix sums,
 * exception slots) and upload it into a new handle.  Synchronises `stream`.
 * The copies to the device are issued before the records are checked, so
 * that the checks run while the bytes move (from pinned memory the copies
 * are asynchronous); nothing on the device reads them before the call
 * returns, and a string that fails a check is freed after its copies end
 * (CHR_ERR_CORRUPT is reported ahead of a failed allocation).
 */
chr_status chr_deserialize(const void *host_buf, size_t n, const chr_allocator *alloc, void *stream,
                           chr_handle **out);

/*
 * ---- batches: many CHRs of uneven size in one launch sequence ----------
 *
 * The paper merges active blocks into rectangular boxes of uneven size and
 * compresses each (Sec. 2); a batch decodes level `level` of every item's
 * CHR and runs marching cubes on it at the item's own isovalue, as one
 * captured sequence of launches: one decode over the concatenated brick
 * list, one tile-count pass, one scan and one emit pass over the
 * concatenated tile list.  Item i's triangles equal, bit for bit, those of
 * chr_reconstruct + isosurface_extract of that item alone, and lie in the
 * batch's triangle buffer from box_start[i] to box_start[i+1]
 * (box_start[n] = total; total > cap sets CHR_ERR_OVERFLOW in the error
 * word and only the first cap triangles are written).
 */
typedef struct chr_batch chr_batch; /* opaque; owns device buffers and a CUDA graph */

typedef struct chr_batch_item {
    const chr_handle *h; /* must outlive the batch */
    uint32_t level;      /* accuracy level to decode */
    float isovalue;
} chr_batch_item;

typedef struct chr_batch_config {
    int32_t count_blocks_per_sm;    /* resident blocks per SM of the tile-count pass (0: the most that fit) */
    int32_t emit_blocks_per_sm;     /* the same for the emit pass */
    int32_t use_graph;              /* 1: capture the sequence once and replay it */
    int32_t decode_warps_per_block; /* bricks (one per warp) per decode block: 4 or 8 (0: 8) */
} chr_batch_config;

/*
 * chr_batch_create — plan a batch of n items (n >= 1).  Outputs are
 * caller-owned device buffers, written by every run: d_tris (cap_tris
 * triangles of 9 floats, 4-byte aligned; may be NULL when cap_tris = 0),
 * d_box_start (n+1 uint64) and d_err (one uint32 error word, reset by each
 * run).  The library allocates the pitched field buffer (rows padded to 16
 * bytes), the per-item parameters and tensor maps and the scan scratch from
 * `alloc` (NULL: the library pool) on `stream`, which it synchronises once.
 * The configuration is the one the autotuner last chose for a batch with the
 * same size-class signature, else the defaults.
 */
chr_status chr_batch_create(const chr_batch_item *items, uint32_t n, float *d_tris, uint64_t cap_tris,
                            uint64_t *d_box_start, uint32_t *d_err, const chr_allocator *alloc, void *stream,
                            chr_batch **out);

/* chr_batch_run — decode + marching cubes of every item, asynchronous on stream. */
chr_status chr_batch_run(chr_batch *b, void *stream);

/*
 * chr_batch_autotune — time every candidate configuration (tile-kernel grid
 * sizes and the decode brick-group size) on this batch, reps runs each, keep
 * the fastest and remember it for the batch's size-class signature.  Synchronises stream.  The outputs then
 * hold the last candidate's (identical) results.
 */
chr_status chr_batch_autotune(chr_batch *b, uint32_t reps, void *stream, chr_batch_config *chosen);
chr_status chr_batch_get_config(const chr_batch *b, chr_batch_config *cfg);
/* chr_batch_set_config — zero fields pick the largest grid; over-large values are clamped. */
chr_status chr_batch_set_config(chr_batch *b, const chr_batch_config *cfg);

/* chr_batch_field — item i's decoded field (library-owned): value (x, y, z) at d_field[x + sx*y + sy*z]. */
chr_status chr_batch_field(const chr_batch *b, uint32_t i, float **d_field, int64_t *sx, int64_t *sy);

/* chr_batch_field_copy — item i's decoded field into d_out (nx*ny*nz floats, x fastest), asynchronous. */
chr_status chr_batch_field_copy(const chr_batch *b, uint32_t i, float *d_out, void *stream);

/* chr_batch_free — release the batch (after its work has finished). NULL ok. */
void chr_batch_free(chr_batch *b);

/* chr_stats — sizes and bounds of a CHR (host-side, no device work). */
chr_status chr_stats(const chr_handle *h, chr_stats_t *out);

/* chr_free — release a handle's buffers (stream-ordered on its stream). NULL ok. */
void chr_free(chr_handle *h);

/*
 * chr_pool_trim — give all but `keep_bytes` of the unused memory held by the
 * library's pool on the current device (the NULL-allocator path) back to the
 * driver (cudaMemPoolTrimTo).  Memory freed by work still in flight is not
 * unused yet: synchronise its stream first.  CHR_ERR_CUDA if the pool cannot
 * be made or trimmed.
 */
chr_status chr_pool_trim(size_t keep_bytes);

/*
 * chr_checked_build — 1 if this library was built with bounds checks
 * (-DCHR_CHECKED: every data-dependent shared-memory index and output range
 * on the hot paths is tested, and an access that fails is skipped), else 0.
 */
int chr_checked_build(void);

/*
 * chr_debug_bounds_word — in a checked build, which kernel families have
 * seen an index fail its bounds test since the last reset: bit 0 marching
 * cubes (extraction, batched, adjoint), bit 1 the codec (encode, decode).
 * 0 in normal builds.  reset != 0 clears the record.  Synchronises the
 * device.  CHR_ERR_INVALID if h_word is NULL.
 */
chr_status chr_debug_bounds_word(uint32_t *h_word, int reset);

/*
 * chr_debug_unpublished_tile — in a checked build, make tile `tile` of every
 * later single-pass extraction publish nothing (-1: none), so that the
 * tiles after it give up their bounded wait and the call reports
 * CHR_ERR_TIMEOUT: the test of a wait that runs out, without a fault.
 * CHR_ERR_INVALID in normal builds, which have no such hook.
 */
chr_status chr_debug_unpublished_tile(int64_t tile);

/*
 * chr_debug_tri_cells — in a checked build, make every later marching-cubes
 * extraction (isosurface_extract, chr_isosurface, ..._noalloc) also write
 * each triangle's cell, x + (nx-1)*(y + (ny-1)*z), to d_cells (device,
 * uint32, cap_tris per isovalue, isovalue j from d_cells + j*cap_tris, in
 * the triangle order): the active cells in output order, each repeated for
 * its triangles.  NULL stops it.  Test output; CHR_ERR_INVALID in normal
 * builds.
 */
chr_status chr_debug_tri_cells(uint32_t *d_cells);

/*
 * chr_debug_cases — in a checked build, the marching-cubes case byte of
 * every cell of d_field at `isovalue` as the extraction's counting pass
 * computes it: d_cases (device, (nx-1)(ny-1)(nz-1) bytes, cell order as
 * above) with corner (ox, oy, oz) at bit ox + 2 oy + 4 oz, set when v < k.
 * d_workspace: isosurface_workspace_size(dims, 1) bytes.  Test output;
 * CHR_ERR_INVALID in normal builds.  Asynchronous.
 */
chr_status chr_debug_cases(const float *d_field, chr_dims dims, float isovalue, uint8_t *d_cases, void *d_workspace,
                           size_t workspace_bytes, void *stream);

/* chr_last_error — message for the last failing call on this thread. */
const char *chr_last_error(void);

/* chr_version — ABI version (2: chr_isosurface takes flags; chr_brick_index). */
int chr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CHR_H */

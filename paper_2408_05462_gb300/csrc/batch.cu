// Many CHRs of uneven size, each with its own level and isovalue, decoded
// and meshed by one launch sequence (Sec. 2: the blocks of a merged
// region are compressed one by one, so the visualization side receives many
// boxes of different shapes at once).
//
// One batched decode launch walks the concatenated brick list of every box
// (one warp per brick, so small boxes leave no warp idle) into one pitched
// field buffer; the marching-cubes count and emit kernels then stride over
// the concatenated tile list of every box, each tile loading its own box's
// parameters and tensor map, with one scan of the tile counts in between.
// The whole sequence is captured once into a CUDA graph and replayed.
//
// The grid sizes of the two tile kernels and the decoder's brick-group size
// (bricks per block) are picked by a small autotuner that times the
// candidates on the batch itself; the choice is remembered per size-class
// signature of the batch (how many boxes fall in each volume class), so a
// later batch of the same mix reuses it without timing.
#include <cuda.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace chr;

struct chr_batch {
    uint32_t n = 0;
    std::vector<chr_batch_item> items;
    std::vector<int64_t> dims;      // 3 per box: nx, ny, nz
    std::vector<int64_t> sx, sy;    // pitches of each box's field (floats)
    std::vector<int64_t> field_off; // offset of each box's field (floats)
    std::string key;                // size-class signature
    int64_t ntiles = 0, nbricks = 0;
    uint64_t cap = 0;
    chr_batch_config cfg{0, 0, 1, 8};
    int sms = 0, count_max = 1, emit_max = 1;
    // device buffers
    Alloc *al = nullptr;
    struct Buf {
        void *p;
        size_t n;
    };
    std::vector<Buf> bufs;
    void *d_params = nullptr, *d_maps = nullptr, *d_scratch = nullptr;
    CodecParams *d_descs = nullptr;
    int64_t *d_tile_start = nullptr, *d_brick_start = nullptr;
    float *d_fields = nullptr, *d_tris = nullptr;
    uint64_t *d_total = nullptr, *d_box_start = nullptr;
    uint32_t *d_err = nullptr;
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    void *get(size_t bytes)
    {
        void *p = al->get(bytes);
        if (p) bufs.push_back({p, bytes});
        return p;
    }
    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, chr_batch_config> g_tuned;  // size-class signature -> chosen configuration

// Volume classes (vertices): < 48^3, < 96^3, < 144^3, larger.  The signature
// holds, per class, the box count rounded to a power of two.
std::string size_signature(const std::vector<int64_t> &dims, uint32_t n)
{
    uint32_t cls[4] = {0, 0, 0, 0};
    for (uint32_t i = 0; i < n; i++) {
        const double v = (double)dims[3 * i] * (double)dims[3 * i + 1] * (double)dims[3 * i + 2];
        const int c = v < 48.0 * 48 * 48 ? 0 : v < 96.0 * 96 * 96 ? 1 : v < 144.0 * 144 * 144 ? 2 : 3;
        cls[c]++;
    }
    std::string s;
    for (int c = 0; c < 4; c++) {
        uint32_t q = 0;
        while ((1u << q) < cls[c]) q++;
        s += std::to_string(cls[c] ? q + 1 : 0) + (c < 3 ? "/" : "");
    }
    return s;
}

cudaError_t record_work(chr_batch *b, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b->d_err, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    e = launch_decode_batched(b->d_descs, b->d_brick_start, (int32_t)b->n, b->nbricks, b->cfg.decode_warps_per_block,
                              s);
    if (e != cudaSuccess) return e;
    McBatchLaunch L;
    L.params = b->d_params;
    L.maps = b->d_maps;
    L.tile_start = b->d_tile_start;
    L.nboxes = (int32_t)b->n;
    L.ntiles = b->ntiles;
    L.scratch = b->d_scratch;
    L.total = b->d_total;
    L.box_start = b->d_box_start;
    L.cap = b->cap;
    L.err = b->d_err;
    L.count_blocks = b->sms * b->cfg.count_blocks_per_sm;
    L.emit_blocks = b->sms * b->cfg.emit_blocks_per_sm;
    return launch_mc_batched(L, s);
}

chr_status clamp_config(const chr_batch *b, chr_batch_config &c)
{
    if (c.count_blocks_per_sm < 0 || c.emit_blocks_per_sm < 0)
        return fail(CHR_ERR_INVALID, "chr_batch: negative blocks per SM");
    if (c.count_blocks_per_sm == 0 || c.count_blocks_per_sm > b->count_max) c.count_blocks_per_sm = b->count_max;
    if (c.emit_blocks_per_sm == 0 || c.emit_blocks_per_sm > b->emit_max) c.emit_blocks_per_sm = b->emit_max;
    c.use_graph = c.use_graph ? 1 : 0;
    c.decode_warps_per_block = (c.decode_warps_per_block == 4) ? 4 : 8;
    return CHR_OK;
}

}  // namespace

extern "C" {

chr_status chr_batch_create(const chr_batch_item *items, uint32_t n, float *d_tris, uint64_t cap_tris,
                            uint64_t *d_box_start, uint32_t *d_err, const chr_allocator *alloc, void *stream,
                            chr_batch **out)
{
    if (!items || !out || n == 0) return fail(CHR_ERR_INVALID, "chr_batch_create: no items or NULL output");
    if ((cap_tris && !d_tris) || !d_box_start || !d_err)
        return fail(CHR_ERR_INVALID, "chr_batch_create: NULL output buffer");
    if ((reinterpret_cast<uintptr_t>(d_tris) & 3u) || (reinterpret_cast<uintptr_t>(d_box_start) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_err) & 3u))
        return fail(CHR_ERR_INVALID, "chr_batch_create: misaligned output buffer");
    if (n > (1u << 20)) return fail(CHR_ERR_INVALID, "chr_batch_create: more than 2^20 items");
    for (uint32_t i = 0; i < n; i++) {
        if (!items[i].h) return fail(CHR_ERR_INVALID, "chr_batch_create: NULL handle");
        if (items[i].level >= items[i].h->nlevels) return fail(CHR_ERR_INVALID, "chr_batch_create: level out of range");
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    chr_batch *b = new chr_batch();
    b->al = new Alloc(alloc, s);
    b->n = n;
    b->cap = cap_tris;
    b->items.assign(items, items + n);
    b->dims.resize(3 * (size_t)n);
    b->sx.resize(n);
    b->sy.resize(n);
    b->field_off.resize(n);
    std::vector<int64_t> tile_start(n + 1), brick_start(n + 1);
    int64_t floats = 0;
    for (uint32_t i = 0; i < n; i++) {
        const Grid &g = items[i].h->g;
        b->dims[3 * i] = g.nx;
        b->dims[3 * i + 1] = g.ny;
        b->dims[3 * i + 2] = g.nz;
        b->sx[i] = (g.nx + 3) & ~int64_t(3);  // rows start on 16 bytes, so every box has a tensor map
        b->sy[i] = b->sx[i] * g.ny;
        b->field_off[i] = floats;
        floats += ((b->sy[i] * g.nz + 63) / 64) * 64;  // boxes start on 256 bytes
        tile_start[i] = b->ntiles;
        b->ntiles += mc_tile_count(g.nx, g.ny, g.nz);
        brick_start[i] = b->nbricks;
        b->nbricks += g.nbricks;
    }
    tile_start[n] = b->ntiles;
    brick_start[n] = b->nbricks;
    b->key = size_signature(b->dims, n);

    int cmax = 1, emax = 1, sms = 0;
    cudaError_t e = mc_batch_prepare(cmax, emax, sms);
    if (e != cudaSuccess) {
        chr_batch_free(b);
        return cuda_fail(e, "chr_batch_create");
    }
    b->sms = sms;
    b->count_max = cmax;
    b->emit_max = emax;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(b->key);
        b->cfg = (it != g_tuned.end()) ? it->second : chr_batch_config{0, 0, 1, 8};
    }
    clamp_config(b, b->cfg);

    const size_t pbytes = mc_batch_param_bytes();
    b->d_params = b->get(pbytes * n);
    b->d_maps = b->get(sizeof(CUtensorMap) * n);
    b->d_descs = reinterpret_cast<CodecParams *>(b->get(sizeof(CodecParams) * n));
    b->d_tile_start = reinterpret_cast<int64_t *>(b->get(sizeof(int64_t) * (n + 1)));
    b->d_brick_start = reinterpret_cast<int64_t *>(b->get(sizeof(int64_t) * (n + 1)));
    b->d_fields = reinterpret_cast<float *>(b->get((size_t)floats * 4));
    b->d_tris = d_tris;
    b->d_scratch = b->get(mc_batch_scratch_bytes(b->ntiles));
    b->d_total = reinterpret_cast<uint64_t *>(b->get(sizeof(uint64_t)));
    b->d_box_start = d_box_start;
    b->d_err = d_err;
    if (!b->d_params || !b->d_maps || !b->d_descs || !b->d_tile_start || !b->d_brick_start || !b->d_fields ||
        !b->d_scratch || !b->d_total) {
        chr_batch_free(b);
        return fail(CHR_ERR_OOM, "chr_batch_create: device allocation failed");
    }

    std::vector<unsigned char> params(pbytes * n);
    std::vector<CUtensorMap> maps(n);
    std::vector<CodecParams> descs(n);
    for (uint32_t i = 0; i < n; i++) {
        const chr_handle *h = items[i].h;
        float *field = b->d_fields + b->field_off[i];
        if (!mc_batch_fill(params.data() + pbytes * i, &maps[i], field, h->g.nx, h->g.ny, h->g.nz, b->sx[i], b->sy[i],
                           items[i].isovalue, b->d_tris, b->cap, b->d_scratch, b->ntiles, tile_start[i], b->d_err)) {
            chr_batch_free(b);
            return fail(CHR_ERR_INVALID, "chr_batch_create: no tensor map for item " + std::to_string(i));
        }
        CodecParams &p = descs[i];
        fill_codec_params(h, p);
        p.nlevels = (int32_t)items[i].level + 1;
        set_box(p, h->g, 0, 0, 0, h->g.nx, h->g.ny, h->g.nz);
        p.out = field;
        p.out_sx = b->sx[i];
        p.out_sy = b->sy[i];
    }
    e = cudaMemcpyAsync(b->d_params, params.data(), params.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_descs, descs.data(), sizeof(CodecParams) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tile_start, tile_start.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_brick_start, brick_start.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host staging vectors go out of scope
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        chr_batch_free(b);
        return cuda_fail(e, "chr_batch_create");
    }
    *out = b;
    return CHR_OK;
}

static chr_status batch_run(chr_batch *b, void *stream);

chr_status chr_batch_run(chr_batch *b, void *stream)
{
    nvtxRangePushA("chr_batch_run");
    const chr_status st = batch_run(b, stream);
    nvtxRangePop();
    return st;
}

static chr_status batch_run(chr_batch *b, void *stream)
{
    if (!b) return fail(CHR_ERR_INVALID, "chr_batch_run: NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->cfg.use_graph) {
        cudaError_t e = record_work(b, s);
        return e == cudaSuccess ? CHR_OK : cuda_fail(e, "chr_batch_run");
    }
    if (!b->exec) {
        cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "chr_batch_run: begin capture");
        cudaError_t ew = record_work(b, b->cap_stream);
        e = cudaStreamEndCapture(b->cap_stream, &b->graph);
        if (ew != cudaSuccess || e != cudaSuccess) {
            b->drop_graph();
            return cuda_fail(ew != cudaSuccess ? ew : e, "chr_batch_run: capture");
        }
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            b->drop_graph();
            return cuda_fail(e, "chr_batch_run: instantiate");
        }
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? CHR_OK : cuda_fail(e, "chr_batch_run");
}

chr_status chr_batch_get_config(const chr_batch *b, chr_batch_config *cfg)
{
    if (!b || !cfg) return fail(CHR_ERR_INVALID, "chr_batch_get_config: NULL argument");
    *cfg = b->cfg;
    return CHR_OK;
}

chr_status chr_batch_set_config(chr_batch *b, const chr_batch_config *cfg)
{
    if (!b || !cfg) return fail(CHR_ERR_INVALID, "chr_batch_set_config: NULL argument");
    chr_batch_config c = *cfg;
    chr_status st = clamp_config(b, c);
    if (st != CHR_OK) return st;
    if (memcmp(&c, &b->cfg, sizeof(c)) != 0) {
        b->drop_graph();
        b->cfg = c;
    }
    return CHR_OK;
}

chr_status chr_batch_autotune(chr_batch *b, uint32_t reps, void *stream, chr_batch_config *chosen)
{
    if (!b) return fail(CHR_ERR_INVALID, "chr_batch_autotune: NULL batch");
    if (reps == 0) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<chr_batch_config> cand;
    const int cc[4] = {1, 2, 4, 8}, ec[4] = {1, 2, 3, 4}, dw[2] = {4, 8};
    for (int d = 0; d < 2; d++)
        for (int i = 0; i < 4; i++) {
            if (cc[i] > b->count_max) continue;
            for (int j = 0; j < 4; j++)
                if (ec[j] <= b->emit_max) cand.push_back(chr_batch_config{cc[i], ec[j], 1, dw[d]});
        }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "chr_batch_autotune");
    float best = 0.0f;
    chr_batch_config best_cfg = b->cfg;
    chr_status st = CHR_OK;
    for (const chr_batch_config &c : cand) {
        if ((st = chr_batch_set_config(b, &c)) != CHR_OK) break;
        if ((st = chr_batch_run(b, stream)) != CHR_OK) break;  // capture and warm up
        cudaEventRecord(e0, s);
        for (uint32_t r = 0; r < reps && st == CHR_OK; r++) st = chr_batch_run(b, stream);
        cudaEventRecord(e1, s);
        if (st != CHR_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "chr_batch_autotune");
            break;
        }
        if (best == 0.0f || ms < best) {
            best = ms;
            best_cfg = b->cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CHR_OK) return st;
    st = chr_batch_set_config(b, &best_cfg);
    if (st != CHR_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[b->key] = b->cfg;
    }
    if (chosen) *chosen = b->cfg;
    return CHR_OK;
}

chr_status chr_batch_field(const chr_batch *b, uint32_t i, float **d_field, int64_t *sx, int64_t *sy)
{
    if (!b || i >= b->n) return fail(CHR_ERR_INVALID, "chr_batch_field: NULL batch or item out of range");
    if (d_field) *d_field = b->d_fields + b->field_off[i];
    if (sx) *sx = b->sx[i];
    if (sy) *sy = b->sy[i];
    return CHR_OK;
}

chr_status chr_batch_field_copy(const chr_batch *b, uint32_t i, float *d_out, void *stream)
{
    if (!b || i >= b->n || !d_out) return fail(CHR_ERR_INVALID, "chr_batch_field_copy: NULL argument or item out of range");
    const int64_t nx = b->dims[3 * i], ny = b->dims[3 * i + 1], nz = b->dims[3 * i + 2];
    cudaError_t e = cudaMemcpy2DAsync(d_out, (size_t)nx * 4, b->d_fields + b->field_off[i], (size_t)b->sx[i] * 4,
                                      (size_t)nx * 4, (size_t)(ny * nz), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? CHR_OK : cuda_fail(e, "chr_batch_field_copy");
}

void chr_batch_free(chr_batch *b)
{
    if (!b) return;
    b->drop_graph();
    if (b->cap_stream) {
        cudaStreamSynchronize(b->cap_stream);
        cudaStreamDestroy(b->cap_stream);
    }
    if (b->al) {
        for (auto it = b->bufs.rbegin(); it != b->bufs.rend(); ++it) b->al->put(it->p, it->n);
        delete b->al;
    }
    delete b;
}

}  // extern "C"

// C ABI of libchr (include/chr.h): argument validation, CHR handles,
// serialization, and the launch sequences of the kernels in codec.cu, mc.cu
// and translate.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace chr {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

chr_status fail(chr_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

chr_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(CHR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

namespace {

// An NVTX range around each C-ABI call (visible in Nsight timelines; no
// cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

#define CHR_CUDA(call, where)                         \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool dims_ok(chr_dims d, std::string &why)
{
    if (d.nx < 2 || d.ny < 2 || d.nz < 2) {
        why = "dims must be >= 2 along every axis";
        return false;
    }
    if (d.nx > (1ll << 31) || d.ny > (1ll << 31) || d.nz > (1ll << 31) ||
        (double)d.nx * (double)d.ny * (double)d.nz >= 4294967295.0) {
        why = "nx*ny*nz must be < 2^32";
        return false;
    }
    return true;
}

void free_handle_buffers(chr_handle *h)
{
    Alloc al(h->default_alloc ? nullptr : &h->alloc, h->stream);
    al.put(h->d_rec_block, h->sz_rec_block);
    al.put(h->d_pay_block, h->sz_pay_block);
    h->d_rec_block = h->d_pay_block = nullptr;
    for (uint32_t l = 0; l < CHR_MAX_LEVELS; l++) {
        h->d_recs[l] = nullptr;
        h->d_index[l] = nullptr;
        h->d_words[l] = nullptr;
        h->d_exc_idx[l] = nullptr;
        h->d_exc_val[l] = nullptr;
    }
}

size_t up256(size_t n) { return (n + 255) & ~size_t(255); }

// Every level's records (and, with_index, its value index) in one
// allocation; false if the allocator failed.
bool alloc_records(chr_handle *h, Alloc &al, bool with_index)
{
    h->sz_recs = (size_t)h->g.nbricks * sizeof(uint4);
    const size_t per = up256(h->sz_recs), per_idx = with_index ? up256((size_t)h->g.nbricks * sizeof(float2)) : 0;
    h->sz_rec_block = (per + per_idx) * h->nlevels;
    char *b = (char *)al.get(h->sz_rec_block);
    h->d_rec_block = b;
    if (!b) return false;
    h->has_index = with_index;
    for (uint32_t l = 0; l < h->nlevels; l++) {
        h->d_recs[l] = reinterpret_cast<uint4 *>(b + per * l);
        h->d_index[l] = with_index ? reinterpret_cast<float2 *>(b + per * h->nlevels + per_idx * l) : nullptr;
    }
    return true;
}

// Every level's packed words, exception slots and exception values (sizes
// from nwords and nexc, each with 64 bytes of read-ahead room) in one
// allocation; false if the allocator failed.
bool alloc_payload(chr_handle *h, Alloc &al)
{
    size_t total = 0;
    for (uint32_t l = 0; l < h->nlevels; l++) {
        h->sz_words[l] = h->nwords[l] * 4 + 64;
        h->sz_exc_idx[l] = h->nexc[l] * 2 + 64;
        h->sz_exc_val[l] = h->nexc[l] * 4 + 64;
        total += up256(h->sz_words[l]) + up256(h->sz_exc_idx[l]) + up256(h->sz_exc_val[l]);
    }
    h->sz_pay_block = total;
    char *b = (char *)al.get(total);
    h->d_pay_block = b;
    if (!b) return false;
    size_t o = 0;
    for (uint32_t l = 0; l < h->nlevels; l++) {
        h->d_words[l] = reinterpret_cast<uint32_t *>(b + o);
        o += up256(h->sz_words[l]);
        h->d_exc_idx[l] = reinterpret_cast<uint16_t *>(b + o);
        o += up256(h->sz_exc_idx[l]);
        h->d_exc_val[l] = reinterpret_cast<uint32_t *>(b + o);
        o += up256(h->sz_exc_val[l]);
    }
    return true;
}

chr_handle *new_handle(chr_dims dims, const chr_allocator *alloc, cudaStream_t s)
{
    chr_handle *h = new chr_handle();
    memset(h, 0, sizeof(*h));
    h->dims = dims;
    h->g = make_grid(dims);
    h->default_alloc = (alloc == nullptr);
    if (alloc) h->alloc = *alloc;
    h->stream = s;
    h->eb_translated = INFINITY;
    return h;
}

}  // namespace

void fill_codec_params(const chr_handle *h, CodecParams &p)
{
    memset(&p, 0, sizeof(p));
    p.nx = h->g.nx;
    p.ny = h->g.ny;
    p.nz = h->g.nz;
    p.nbx = (int32_t)h->g.nbx;
    p.nby = (int32_t)h->g.nby;
    p.nbz = (int32_t)h->g.nbz;
    p.ngx = (int32_t)((h->g.nbx + kWarpsPerBlock - 1) / kWarpsPerBlock);
    p.nlevels = (int32_t)h->nlevels;
    for (uint32_t l = 0; l < h->nlevels; l++) {
        p.e[l] = h->eb[l];
        p.two_e[l] = h->two_e[l];
        p.inv2e[l] = h->inv2e[l];
        p.recs[l] = h->d_recs[l];
        p.index[l] = h->d_index[l];
        p.words[l] = h->d_words[l];
        p.exc_idx[l] = h->d_exc_idx[l];
        p.exc_val[l] = h->d_exc_val[l];
    }
    p.nK = (int32_t)h->n_iso;
    for (uint32_t j = 0; j < CHR_MAX_ISO; j++) p.K[j] = (j < h->n_iso) ? h->iso[j] : -INFINITY;  // (-inf: never above a value)
    p.fix = (h->topo_mode == CHR_TOPO_FIX) ? 1 : 0;
    float ks[CHR_MAX_ISO];
    const int nK = (int)h->n_iso;
    for (int j = 0; j < nK; j++) ks[j] = h->iso[j];
    std::sort(ks, ks + nK);
    for (int c = 0; c <= nK; c++) {
        p.kup[c] = (c > 0) ? ks[nK - c] : INFINITY;
        p.kdn[c] = (c < nK) ? ks[nK - c - 1] : -INFINITY;
    }
}

void set_box(CodecParams &p, const Grid &g, int64_t x0, int64_t y0, int64_t z0, int64_t bx, int64_t by, int64_t bz)
{
    const int64_t org[3] = {x0, y0, z0}, dim[3] = {bx, by, bz};
    for (int a = 0; a < 3; a++) {
        p.box_org[a] = org[a];
        p.box_dim[a] = dim[a];
        p.box_brick0[a] = (int32_t)(org[a] / 8);
        p.box_bricks[a] = (int32_t)((org[a] + dim[a] - 1) / 8 - org[a] / 8 + 1);
    }
    p.out_sx = bx;
    p.out_sy = bx * by;
    (void)g;
}

namespace {

void set_constants(chr_handle *h)
{
    for (uint32_t l = 0; l < h->nlevels; l++) {
        volatile float e = h->eb[l];
        volatile float two = 2.0f * e;
        h->two_e[l] = two;
        h->inv2e[l] = 1.0f / two;
    }
}

// The selection of chr_topo_translate; synchronises the stream.  Accuracy 1:
// one walk for min D.  Otherwise a walk for the 4096-bin histogram of the
// top 12 bits of D's elements, which names the bucket holding rank n; a walk
// that collects that bucket's elements; and two small histogram passes over
// them (bits 10..19, then 0..9 within the chosen bits 10..19).
chr_status translate_impl(const float *d_field, const Grid &g, const float *K, uint32_t nK, float accuracy, Alloc &al,
                          float *eb_out, uint64_t *count_out)
{
    constexpr int kBins = 4096;
    constexpr int64_t kSampleStep = 16;  // the sample walks every 16th item
    const size_t sb = translate_scratch_bytes();
    char *scr = (char *)al.get(sb);
    if (!scr) return fail(CHR_ERR_OOM, "chr_topo_translate: allocator returned NULL");
    TranslateScratch sc;
    memset(&sc, 0, sizeof(sc));
    sc.hist = reinterpret_cast<unsigned long long *>(scr);
    sc.count = reinterpret_cast<unsigned long long *>(scr + kBins * 8);
    sc.minbits = reinterpret_cast<unsigned int *>(scr + kBins * 8 + 8);
    sc.ncoll = reinterpret_cast<unsigned long long *>(scr + kBins * 8 + 16);
    sc.count_lo = reinterpret_cast<unsigned long long *>(scr + kBins * 8 + 24);
    chr_status st = CHR_OK;
    std::vector<unsigned long long> hist(kBins);
    unsigned long long count = 0;
    unsigned int minbits = 0xffffffffu;
    float eb = INFINITY;
    uint32_t *coll = nullptr;
    size_t coll_bytes = 0;
    auto pick = [](const std::vector<unsigned long long> &h, int nb, unsigned long long &rank) {
        unsigned long long cum = 0;
        for (int b = 0; b < nb; b++) {
            if (rank < cum + h[b]) {
                rank -= cum;
                return b;
            }
            cum += h[b];
        }
        rank = 0;
        return nb - 1;
    };
    auto rank_of = [&](unsigned long long n) {  // the rank (from 0) of the element the accuracy names
        const double r = floor((1.0 - (double)accuracy) * (double)n);
        unsigned long long k = (r < 0) ? 0ull : (unsigned long long)r;
        return (k > n - 1) ? n - 1 : k;
    };
    auto zero_scratch = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(scr, 0, kBins * 8 + 32, al.s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sc.minbits, 0xff, 4, al.s);
        return e;
    };
    // the n collected values (each below 2^30) whose digits select rank `rank`:
    // bits 20..29, then 10..19, then 0..9, one histogram pass each
    auto select3 = [&](unsigned long long n, unsigned long long rank, uint32_t &out) -> cudaError_t {
        uint32_t above = 0;
        for (int shift = 20; shift >= 0; shift -= 10) {
            cudaError_t e;
            if ((e = cudaMemsetAsync(sc.hist, 0, 1024 * 8, al.s)) != cudaSuccess ||
                (e = launch_translate_select(coll, n, shift, above, sc.hist, al.s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(hist.data(), sc.hist, 1024 * 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(al.s)) != cudaSuccess)
                return e;
            above = (above << 10) | (uint32_t)pick(hist, 1024, rank);
        }
        out = above;
        return cudaSuccess;
    };
    do {
        cudaError_t e;
        const bool min_only = (accuracy >= 1.0f);
        if (min_only) {
            if ((e = zero_scratch()) != cudaSuccess ||
                (e = launch_translate_pass(d_field, g, K, (int)nK, 0, 0u, sc, al.s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&count, sc.count, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(&minbits, sc.minbits, 4, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(al.s)) != cudaSuccess) {
                st = cuda_fail(e, "chr_topo_translate");
                break;
            }
            if (count) memcpy(&eb, &minbits, 4);
            break;
        }

        // the sampled walk and the range that should hold rank n
        int64_t items = 0;
        unsigned long long count_s = 0;
        if ((e = zero_scratch()) != cudaSuccess ||
            (e = launch_translate_pass(d_field, g, K, (int)nK, 1, 0u, sc, al.s, 0u, 0u, kSampleStep, &items)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(&count_s, sc.count, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(hist.data(), sc.hist, kBins * 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(al.s)) != cudaSuccess) {
            st = cuda_fail(e, "chr_topo_translate");
            break;
        }
        bool done = false;
        if (count_s >= 4096) {
            const double scale = (double)items / (double)((items + kSampleStep - 1) / kSampleStep);
            const double rs = floor((1.0 - (double)accuracy) * (double)count_s * scale) / scale;  // rank n in the sample
            // 3% either side of it, plus four standard deviations of a
            // binomial count (the sample misses that much only when it does
            // not represent the field, and then the exact walks follow)
            const double margin = 0.03 * rs + 4.0 * sqrt(rs + 1.0) + 32.0;
            unsigned long long r_lo = (unsigned long long)std::max(0.0, rs - margin);
            unsigned long long r_hi = (unsigned long long)std::min((double)(count_s - 1), rs + margin);
            const uint32_t b_lo = (uint32_t)pick(hist, kBins, r_lo), b_hi = (uint32_t)pick(hist, kBins, r_hi);
            // (elements are non-negative floats: bucket 2040 holds +inf, so b_hi + 1 never wraps)
            if (b_hi - b_lo < 1024) {
                unsigned long long in_s = 0;
                for (uint32_t b = b_lo; b <= b_hi; b++) in_s += hist[b];
                const unsigned long long cap = (unsigned long long)(1.5 * (double)in_s * scale) + 65536;
                coll_bytes = cap * 4;
                if (!(coll = (uint32_t *)al.get(coll_bytes))) {
                    st = fail(CHR_ERR_OOM, "chr_topo_translate: allocator returned NULL");
                    break;
                }
                sc.coll = coll;
                sc.cap = cap;
                const uint32_t lo_bits = b_lo << 20, hi_bits = (b_hi + 1) << 20;
                unsigned long long got = 0, below = 0;
                if ((e = zero_scratch()) != cudaSuccess ||
                    (e = launch_translate_pass(d_field, g, K, (int)nK, 3, 0u, sc, al.s, lo_bits, hi_bits)) !=
                        cudaSuccess ||
                    (e = cudaMemcpyAsync(&count, sc.count, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(&below, sc.count_lo, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(&got, sc.ncoll, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(al.s)) != cudaSuccess) {
                    st = cuda_fail(e, "chr_topo_translate");
                    break;
                }
                const unsigned long long rank = count ? rank_of(count) : 0ull;
                if (count && got <= cap && below <= rank && rank < below + got) {
                    uint32_t off = 0;
                    if ((e = select3(got, rank - below, off)) != cudaSuccess) {
                        st = cuda_fail(e, "chr_topo_translate");
                        break;
                    }
                    const uint32_t bits = lo_bits + off;
                    memcpy(&eb, &bits, 4);
                    done = true;
                }
                al.put(coll, coll_bytes);
                coll = nullptr;
            }
        }
        if (done) break;

        // the exact two-walk selection
        if ((e = zero_scratch()) != cudaSuccess ||
            (e = launch_translate_pass(d_field, g, K, (int)nK, 1, 0u, sc, al.s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&count, sc.count, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(hist.data(), sc.hist, kBins * 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(al.s)) != cudaSuccess) {
            st = cuda_fail(e, "chr_topo_translate");
            break;
        }
        if (count == 0) break;
        unsigned long long rank = rank_of(count);
        const uint32_t b1 = (uint32_t)pick(hist, kBins, rank);
        const unsigned long long nb = hist[b1];
        coll_bytes = nb * 4;
        if (!(coll = (uint32_t *)al.get(coll_bytes))) {
            st = fail(CHR_ERR_OOM, "chr_topo_translate: allocator returned NULL");
            break;
        }
        sc.coll = coll;
        sc.cap = nb;
        unsigned long long got = 0;
        if ((e = launch_translate_pass(d_field, g, K, (int)nK, 2, b1, sc, al.s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&got, sc.ncoll, 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(al.s)) != cudaSuccess) {
            st = cuda_fail(e, "chr_topo_translate");
            break;
        }
        if (got != nb) {
            st = fail(CHR_ERR_CUDA, "chr_topo_translate: the collecting walk found a different bucket size");
            break;
        }
        // the bucket's values are its elements' low 20 bits: digits 10..19, then 0..9
        uint32_t above = 0;
        for (int shift = 10; shift >= 0; shift -= 10) {
            if ((e = cudaMemsetAsync(sc.hist, 0, 1024 * 8, al.s)) != cudaSuccess ||
                (e = launch_translate_select(coll, nb, shift, above, sc.hist, al.s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(hist.data(), sc.hist, 1024 * 8, cudaMemcpyDeviceToHost, al.s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(al.s)) != cudaSuccess)
                break;
            above = (above << 10) | (uint32_t)pick(hist, 1024, rank);
        }
        if (e != cudaSuccess) {
            st = cuda_fail(e, "chr_topo_translate");
            break;
        }
        const uint32_t bits = (b1 << 20) | above;
        memcpy(&eb, &bits, 4);
    } while (0);
    if (coll) al.put(coll, coll_bytes);
    al.put(scr, sb);
    if (st == CHR_OK) {
        *eb_out = eb;
        if (count_out) *count_out = count;
    }
    return st;
}

// ---- serialization helpers -------------------------------------------------

struct Writer {
    std::vector<char> *buf;
    template <class T>
    void put(const T &v)
    {
        const char *p = reinterpret_cast<const char *>(&v);
        buf->insert(buf->end(), p, p + sizeof(T));
    }
};

size_t header_bytes(uint32_t nlevels, uint32_t n_iso)
{
    return 4 + 4 + 24 + 16 + 8 + 8 + 4 * (size_t)nlevels + 4 * (size_t)n_iso + 16 * (size_t)nlevels;
}

// One level's records and exception slots of a byte string, checked on the
// host: widths <= 32, modes 0/1, <= 512 exceptions per brick, every record's
// prefix sums (wsum, exc_off) equal to the sums over the bricks before it,
// exception slots ascending inside each brick and on the grid.  The bricks
// are split into chunks checked by several threads: a first sweep sums each
// chunk's widths and exception counts, the prefix over chunks gives every
// chunk its starting sums, a second sweep checks the records against them.
// wsum, esum: the level's totals.
bool validate_level(const uint32_t *rec, const uint16_t *eidx, const Grid &g, uint64_t nexc, uint64_t &wsum,
                    uint64_t &esum)
{
    const int64_t nb = g.nbricks;
    unsigned hw = std::thread::hardware_concurrency();
    const int64_t nchunks = std::max<int64_t>(1, std::min<int64_t>(hw ? hw : 1, std::min<int64_t>(64, nb / 4096)));
    const int64_t per = (nb + nchunks - 1) / nchunks;
    std::vector<uint64_t> cw(nchunks, 0), ce(nchunks, 0);
    std::vector<char> good(nchunks, 1);
    auto sweep = [&](int64_t c, bool check) {
        const int64_t b0 = c * per, b1 = std::min(nb, b0 + per);
        uint64_t w_run = check ? cw[c] : 0, e_run = check ? ce[c] : 0;
        for (int64_t b = b0; b < b1; b++) {
            uint32_t r[4];
            memcpy(r, rec + 4 * b, 16);
            const uint32_t w = r[3] & 0xffu, mode = (r[3] >> 8) & 0xffu, ne = r[3] >> 16;
            if (w > 32 || mode > 1 || ne > 512) {
                good[c] = 0;
                return;
            }
            if (check) {
                if (r[0] != w_run || r[1] != e_run || e_run + ne > nexc) {
                    good[c] = 0;
                    return;
                }
                const int64_t bx = b % g.nbx, by = (b / g.nbx) % g.nby, bz = b / (g.nbx * g.nby);
                int prev = -1;
                for (uint32_t j = 0; j < ne; j++) {
                    uint16_t sl;
                    memcpy(&sl, eidx + e_run + j, 2);
                    const int64_t x = bx * 8 + (sl & 7), y = by * 8 + ((sl >> 3) & 7), z = bz * 8 + (sl >> 6);
                    if (sl >= 512 || (int)sl <= prev || x >= g.nx || y >= g.ny || z >= g.nz) {
                        good[c] = 0;
                        return;
                    }
                    prev = sl;
                }
            }
            w_run += w;
            e_run += ne;
        }
        if (!check) {
            cw[c] = w_run;
            ce[c] = e_run;
        }
    };
    auto run = [&](bool check) {
        std::vector<std::thread> th;
        for (int64_t c = 1; c < nchunks; c++) th.emplace_back(sweep, c, check);
        sweep(0, check);
        for (auto &t : th) t.join();
    };
    run(false);
    for (int64_t c = 0; c < nchunks; c++)
        if (!good[c]) return false;
    uint64_t W = 0, E = 0;
    for (int64_t c = 0; c < nchunks; c++) {  // exclusive prefix: each chunk's starting sums
        const uint64_t w = cw[c], e = ce[c];
        cw[c] = W;
        ce[c] = E;
        W += w;
        E += e;
    }
    if (E > nexc) return false;
    run(true);
    for (int64_t c = 0; c < nchunks; c++)
        if (!good[c]) return false;
    wsum = W;
    esum = E;
    return true;
}

size_t level_bytes(const chr_handle *h, uint32_t l)
{
    size_t idx = ((size_t)h->nexc[l] * 2 + 3) & ~size_t(3);
    return (size_t)h->g.nbricks * 16 + (size_t)h->nwords[l] * 4 + idx + (size_t)h->nexc[l] * 4;
}

}  // namespace

cudaMemPool_t library_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices] = {};
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps pr;
        memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.handleTypes = cudaMemHandleTypeNone;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t mp = nullptr;
        if (cudaMemPoolCreate(&mp, &pr) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;  // freed memory stays in the pool until chr_pool_trim
        if (cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) cudaGetLastError();
        pools[dev] = mp;
    }
    return pools[dev];
}

}  // namespace chr

using namespace chr;

extern "C" {

int chr_version(void) { return 2; }

int chr_checked_build(void)
{
#ifdef CHR_CHECKED
    return 1;
#else
    return 0;
#endif
}

chr_status chr_debug_bounds_word(uint32_t *h_word, int reset)
{
    if (!h_word) return fail(CHR_ERR_INVALID, "chr_debug_bounds_word: NULL output");
    *h_word = (mc_bounds_word(reset != 0) ? 1u : 0u) | (codec_bounds_word(reset != 0) ? 2u : 0u);
    return CHR_OK;
}

chr_status chr_debug_tri_cells(uint32_t *d_cells)
{
    if (reinterpret_cast<uintptr_t>(d_cells) & 3u) return fail(CHR_ERR_INVALID, "chr_debug_tri_cells: misaligned output");
    if (!mc_debug_set_tri_cells(d_cells))
        return fail(CHR_ERR_INVALID, "chr_debug_tri_cells: only the checked build has this test output");
    return CHR_OK;
}

chr_status chr_debug_cases(const float *d_field, chr_dims dims, float isovalue, uint8_t *d_cases, void *d_workspace,
                           size_t workspace_bytes, void *stream)
{
    std::string why;
    if (!d_field || !d_cases || !d_workspace) return fail(CHR_ERR_INVALID, "chr_debug_cases: NULL pointer");
    if (!dims_ok(dims, why)) return fail(CHR_ERR_INVALID, "chr_debug_cases: " + why);
    if (!isfinite(isovalue)) return fail(CHR_ERR_INVALID, "chr_debug_cases: isovalue must be finite");
    cudaError_t e = cudaSuccess;
    if (!mc_debug_cases(d_field, make_grid(dims), isovalue, d_cases, d_workspace, workspace_bytes,
                        (cudaStream_t)stream, e))
        return fail(CHR_ERR_INVALID, "chr_debug_cases: only the checked build has this test output");
    if (e == cudaErrorInvalidValue) return fail(CHR_ERR_INVALID, "chr_debug_cases: workspace smaller than isosurface_workspace_size(dims, 1)");
    if (e != cudaSuccess) return cuda_fail(e, "chr_debug_cases");
    return CHR_OK;
}

chr_status chr_debug_unpublished_tile(int64_t tile)
{
    if (!mc_set_unpublished_tile(tile))
        return fail(CHR_ERR_INVALID, "chr_debug_unpublished_tile: only the checked build has this test hook");
    return CHR_OK;
}

chr_status chr_pool_trim(size_t keep_bytes)
{
    cudaMemPool_t mp = library_pool();
    if (!mp) return fail(CHR_ERR_CUDA, "chr_pool_trim: the library's memory pool could not be made");
    const cudaError_t e = cudaMemPoolTrimTo(mp, keep_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "chr_pool_trim");
    return CHR_OK;
}

const char *chr_last_error(void) { return g_last_error.c_str(); }

chr_status chr_compress(const float *d_field, chr_dims dims, const chr_params *prm, const chr_allocator *alloc,
                        void *stream, chr_handle **out)
{
    NvtxRange nvtx_("chr_compress");
    std::string why;
    if (!out) return fail(CHR_ERR_INVALID, "chr_compress: out is NULL");
    *out = nullptr;
    if (!d_field || !prm) return fail(CHR_ERR_INVALID, "chr_compress: NULL field or params");
    if (reinterpret_cast<uintptr_t>(d_field) & 3u) return fail(CHR_ERR_INVALID, "chr_compress: misaligned field");
    if (!dims_ok(dims, why)) return fail(CHR_ERR_INVALID, "chr_compress: " + why);
    if (prm->nlevels < 1 || prm->nlevels > CHR_MAX_LEVELS || !prm->error_bounds)
        return fail(CHR_ERR_INVALID, "chr_compress: nlevels must be 1..8 with error_bounds");
    for (uint32_t l = 0; l < prm->nlevels; l++) {
        const float e = prm->error_bounds[l];
        if (!(e > 0.0f) || !(e < 1e37f)) return fail(CHR_ERR_INVALID, "chr_compress: error bounds must be finite, > 0, < 1e37");
        if (l > 0 && !(e < prm->error_bounds[l - 1]))
            return fail(CHR_ERR_INVALID, "chr_compress: error bounds must decrease strictly");
    }
    if (prm->n_iso > CHR_MAX_ISO || (prm->n_iso > 0 && !prm->isovalues))
        return fail(CHR_ERR_INVALID, "chr_compress: n_iso must be <= 16 with isovalues");
    for (uint32_t j = 0; j < prm->n_iso; j++)
        if (!isfinite(prm->isovalues[j])) return fail(CHR_ERR_INVALID, "chr_compress: isovalues must be finite");
    if (prm->topo_mode > CHR_TOPO_TRANSLATE) return fail(CHR_ERR_INVALID, "chr_compress: bad topo_mode");
    if (prm->topo_mode != CHR_TOPO_NONE && prm->n_iso == 0)
        return fail(CHR_ERR_INVALID, "chr_compress: topology preservation needs isovalues");
    if (prm->topo_mode == CHR_TOPO_TRANSLATE && !(prm->topo_accuracy > 0.0f && prm->topo_accuracy <= 1.0f))
        return fail(CHR_ERR_INVALID, "chr_compress: topo_accuracy must be in (0, 1]");
    if (prm->flags != 0) return fail(CHR_ERR_INVALID, "chr_compress: flags must be 0");

    cudaStream_t s = (cudaStream_t)stream;
    chr_handle *h = new_handle(dims, alloc, s);
    h->nlevels = prm->nlevels;
    h->n_iso = prm->n_iso;
    h->topo_mode = prm->topo_mode;
    h->topo_accuracy = (prm->topo_mode == CHR_TOPO_TRANSLATE) ? prm->topo_accuracy : 1.0f;
    for (uint32_t j = 0; j < prm->n_iso; j++) h->iso[j] = prm->isovalues[j];
    for (uint32_t l = 0; l < prm->nlevels; l++) h->eb[l] = prm->error_bounds[l];
    Alloc al(alloc, s);
    chr_status st = CHR_OK;

    if (h->topo_mode == CHR_TOPO_TRANSLATE) {
        float ebt = INFINITY;
        uint64_t cnt = 0;
        st = translate_impl(d_field, h->g, h->iso, h->n_iso, h->topo_accuracy, al, &ebt, &cnt);
        if (st != CHR_OK) {
            delete h;
            return st;
        }
        h->eb_translated = ebt;
        h->D_count = cnt;
        for (uint32_t l = 0; l < h->nlevels; l++)
            if (ebt < h->eb[l]) h->eb[l] = ebt;
    }
    set_constants(h);

    const Grid &g = h->g;
    // scratch first (the per-brick slots of every level, then the
    // record-scan buffers), so that a pool that keeps freed memory hands the
    // same block back to the next call; then the handle's records
    const size_t slot_bytes = encode_slot_bytes(g.nbricks);
    const size_t scan_bytes = scan_scratch_bytes(g.nbricks, (int)h->nlevels);
    const size_t idx_off = up256(slot_bytes * h->nlevels + scan_bytes + 16 * CHR_MAX_LEVELS);
    const size_t scr_bytes = idx_off + index_part_bytes(g.nbricks, (int)h->nlevels);
    char *scr = (char *)al.get(scr_bytes);
    if (!scr) {
        delete h;
        return fail(CHR_ERR_OOM, "chr_compress: allocator returned NULL");
    }
    if (!alloc_records(h, al, true)) {
        al.put(scr, scr_bytes);
        free_handle_buffers(h);
        delete h;
        return fail(CHR_ERR_OOM, "chr_compress: allocator returned NULL");
    }
    CodecParams p;
    fill_codec_params(h, p);
    p.f = d_field;
    cudaError_t e = cudaSuccess;
    uint64_t totals[2 * CHR_MAX_LEVELS] = {0};
    if (st == CHR_OK) {
        const size_t nb512 = (size_t)g.nbricks * 512;
        for (uint32_t l = 0; l < h->nlevels; l++) {
            char *b = scr + slot_bytes * l;
            p.slot_words[l] = reinterpret_cast<uint32_t *>(b);
            p.slot_val[l] = reinterpret_cast<uint32_t *>(b + nb512 * 4);
            p.slot_idx[l] = reinterpret_cast<uint16_t *>(b + nb512 * 8);
        }
        char *scan_scr = scr + slot_bytes * h->nlevels;
        uint64_t *d_tot = reinterpret_cast<uint64_t *>(scan_scr + scan_bytes);
        p.idx_part = reinterpret_cast<float2 *>(scr + idx_off);
        e = launch_encode(p, s);
        if (e == cudaSuccess) e = launch_brick_index(p, s);
        if (e == cudaSuccess) e = launch_scan_records(h->d_recs, (int)h->nlevels, g.nbricks, scan_scr, d_tot, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(totals, d_tot, 16 * h->nlevels, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess && st == CHR_OK) {
        for (uint32_t l = 0; l < h->nlevels; l++) {
            h->nwords[l] = 16 * totals[2 * l];
            h->nexc[l] = totals[2 * l + 1];
        }
        if (!alloc_payload(h, al)) st = fail(CHR_ERR_OOM, "chr_compress: allocator returned NULL");
    }
    if (e == cudaSuccess && st == CHR_OK) {
        for (uint32_t l = 0; l < h->nlevels; l++) {
            p.words[l] = h->d_words[l];
            p.exc_idx[l] = h->d_exc_idx[l];
            p.exc_val[l] = h->d_exc_val[l];
        }
        e = launch_compact(p, s);
    }
    al.put(scr, scr_bytes);
    if (e != cudaSuccess) st = cuda_fail(e, "chr_compress");
    if (st != CHR_OK) {
        free_handle_buffers(h);
        delete h;
        return st;
    }
    *out = h;
    return CHR_OK;
}

chr_status chr_reconstruct(const chr_handle *h, uint32_t level, float *d_out, void *stream)
{
    NvtxRange nvtx_("chr_reconstruct");
    if (!h || !d_out) return fail(CHR_ERR_INVALID, "chr_reconstruct: NULL handle or output");
    if (level >= h->nlevels) return fail(CHR_ERR_INVALID, "chr_reconstruct: level out of range");
    if (reinterpret_cast<uintptr_t>(d_out) & 3u) return fail(CHR_ERR_INVALID, "chr_reconstruct: misaligned output");
    CodecParams p;
    fill_codec_params(h, p);
    p.out = d_out;
    p.nlevels = (int32_t)level + 1;
    set_box(p, h->g, 0, 0, 0, h->g.nx, h->g.ny, h->g.nz);
    cudaError_t e = launch_decode(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "chr_reconstruct");
    return CHR_OK;
}

chr_status chr_brick_range(const chr_handle *h, uint32_t level, float *d_range, void *stream)
{
    NvtxRange nvtx_("chr_brick_range");
    if (!h || !d_range) return fail(CHR_ERR_INVALID, "chr_brick_range: NULL handle or output");
    if (level >= h->nlevels) return fail(CHR_ERR_INVALID, "chr_brick_range: level out of range");
    if (reinterpret_cast<uintptr_t>(d_range) & 7u) return fail(CHR_ERR_INVALID, "chr_brick_range: misaligned output");
    CodecParams p;
    fill_codec_params(h, p);
    p.out = nullptr;
    p.range = reinterpret_cast<float2 *>(d_range);
    p.nlevels = (int32_t)level + 1;
    set_box(p, h->g, 0, 0, 0, h->g.nx, h->g.ny, h->g.nz);
    cudaError_t e = launch_decode(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "chr_brick_range");
    return CHR_OK;
}

chr_status chr_reconstruct_box(const chr_handle *h, uint32_t level, int64_t x0, int64_t y0, int64_t z0, chr_dims box,
                               float *d_out, void *stream)
{
    NvtxRange nvtx_("chr_reconstruct_box");
    if (!h || !d_out) return fail(CHR_ERR_INVALID, "chr_reconstruct_box: NULL handle or output");
    if (level >= h->nlevels) return fail(CHR_ERR_INVALID, "chr_reconstruct_box: level out of range");
    if (reinterpret_cast<uintptr_t>(d_out) & 3u) return fail(CHR_ERR_INVALID, "chr_reconstruct_box: misaligned output");
    if (box.nx < 1 || box.ny < 1 || box.nz < 1 || x0 < 0 || y0 < 0 || z0 < 0 || x0 + box.nx > h->g.nx ||
        y0 + box.ny > h->g.ny || z0 + box.nz > h->g.nz)
        return fail(CHR_ERR_INVALID, "chr_reconstruct_box: box outside the grid");
    CodecParams p;
    fill_codec_params(h, p);
    p.out = d_out;
    p.nlevels = (int32_t)level + 1;
    set_box(p, h->g, x0, y0, z0, box.nx, box.ny, box.nz);
    cudaError_t e = launch_decode(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "chr_reconstruct_box");
    return CHR_OK;
}

namespace {

struct ServeLayout {
    size_t tris, field, ws, result, total;  // byte offsets of each part, total size
    int64_t sx, sy;
};

ServeLayout serve_layout(chr_dims box, uint64_t cap_tris)
{
    ServeLayout L;
    L.sx = (box.nx + 3) & ~int64_t(3);  // rows start on 16 bytes: the marching cubes always have a tensor map
    L.sy = L.sx * box.ny;
    auto up = [](size_t n) { return (n + 255) & ~size_t(255); };
    L.tris = 0;
    L.field = up((size_t)cap_tris * 36);
    L.ws = L.field + up((size_t)L.sy * box.nz * 4);
    L.result = L.ws + up(mc_workspace_bytes(make_grid(box), 1));
    L.total = L.result + 256;
    return L;
}

}  // namespace

uint64_t chr_box_tri_bound(const float *h_min, const float *h_max, int64_t nbx, int64_t nby, int64_t nbz, int64_t x0,
                           int64_t y0, int64_t z0, chr_dims box, float isovalue)
{
    if (!h_min || !h_max || nbx < 1 || nby < 1 || nbz < 1 || box.nx < 2 || box.ny < 2 || box.nz < 2 || x0 < 0 ||
        y0 < 0 || z0 < 0)
        return 0;
    // cells [o, o + n - 1) along each axis; brick b holds cells [8b, 8b + 8)
    const int64_t o[3] = {x0, y0, z0}, n[3] = {box.nx, box.ny, box.nz}, nb[3] = {nbx, nby, nbz};
    int64_t b0[3], b1[3];
    for (int a = 0; a < 3; a++) {
        b0[a] = o[a] / 8;
        b1[a] = (o[a] + n[a] - 2) / 8 + 1;
        if (b1[a] > nb[a]) b1[a] = nb[a];
        if (b0[a] >= b1[a]) return 0;
    }
    auto cells = [&](int a, int64_t b) {
        const int64_t lo = (8 * b > o[a]) ? 8 * b : o[a];
        const int64_t hi = (8 * b + 8 < o[a] + n[a] - 1) ? 8 * b + 8 : o[a] + n[a] - 1;
        return hi - lo;
    };
    uint64_t total = 0;
    for (int64_t bz = b0[2]; bz < b1[2]; bz++) {
        const int64_t cz = cells(2, bz);
        for (int64_t by = b0[1]; by < b1[1]; by++) {
            const int64_t cyz = cz * cells(1, by);
            const float *mn = h_min + nbx * (by + nby * bz), *mx = h_max + nbx * (by + nby * bz);
            uint64_t row = 0;
            for (int64_t bx = b0[0]; bx < b1[0]; bx++)
                if (mn[bx] < isovalue && mx[bx] >= isovalue) row += (uint64_t)cells(0, bx);
            total += row * (uint64_t)cyz;
        }
    }
    return 5 * total;
}

size_t chr_serve_request_bytes(chr_dims box, uint64_t cap_tris)
{
    std::string why;
    if (!dims_ok(box, why) || cap_tris > (1ull << 58)) return 0;
    return serve_layout(box, cap_tris).total;
}

chr_status chr_serve_request(const chr_handle *h, uint32_t level, int64_t x0, int64_t y0, int64_t z0, chr_dims box,
                             float isovalue, void *d_mem, size_t mem_bytes, uint64_t cap_tris, uint64_t *h_result,
                             void *stream)
{
    NvtxRange nvtx_("chr_serve_request");
    std::string why;
    if (!h || !d_mem || !h_result) return fail(CHR_ERR_INVALID, "chr_serve_request: NULL handle, memory or result");
    if (level >= h->nlevels) return fail(CHR_ERR_INVALID, "chr_serve_request: level out of range");
    if (!dims_ok(box, why)) return fail(CHR_ERR_INVALID, "chr_serve_request: " + why);
    if (x0 < 0 || y0 < 0 || z0 < 0 || x0 + box.nx > h->g.nx || y0 + box.ny > h->g.ny || z0 + box.nz > h->g.nz)
        return fail(CHR_ERR_INVALID, "chr_serve_request: box outside the grid");
    if (!isfinite(isovalue)) return fail(CHR_ERR_INVALID, "chr_serve_request: isovalue must be finite");
    if (reinterpret_cast<uintptr_t>(d_mem) & 255u) return fail(CHR_ERR_INVALID, "chr_serve_request: misaligned memory");
    if (cap_tris > (1ull << 58)) return fail(CHR_ERR_INVALID, "chr_serve_request: cap_tris too large");
    const ServeLayout L = serve_layout(box, cap_tris);
    if (mem_bytes < L.total) return fail(CHR_ERR_INVALID, "chr_serve_request: memory smaller than chr_serve_request_bytes()");
    cudaStream_t s = (cudaStream_t)stream;
    char *base = reinterpret_cast<char *>(d_mem);
    float *field = reinterpret_cast<float *>(base + L.field);
    uint64_t *res = reinterpret_cast<uint64_t *>(base + L.result);
    CodecParams p;
    fill_codec_params(h, p);
    p.out = field;
    p.nlevels = (int32_t)level + 1;
    set_box(p, h->g, x0, y0, z0, box.nx, box.ny, box.nz);
    p.out_sx = L.sx;
    p.out_sy = L.sy;
    CHR_CUDA(cudaMemsetAsync(res, 0, 16, s), "chr_serve_request");
    CHR_CUDA(launch_decode(p, s), "chr_serve_request");
    CHR_CUDA(launch_mc_pitched(field, make_grid(box), L.sx, L.sy, &isovalue, 1,
                               cap_tris ? reinterpret_cast<float *>(base + L.tris) : nullptr, cap_tris, res,
                               reinterpret_cast<uint32_t *>(res + 1), base + L.ws, L.result - L.ws, s),
             "chr_serve_request");
    CHR_CUDA(cudaMemcpyAsync(h_result, res, 16, cudaMemcpyDeviceToHost, s), "chr_serve_request");
    return CHR_OK;
}

chr_status chr_topo_translate(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                              float accuracy, const chr_allocator *alloc, void *stream, float *eb_out,
                              uint64_t *count_out)
{
    NvtxRange nvtx_("chr_topo_translate");
    std::string why;
    if (!d_field || !eb_out) return fail(CHR_ERR_INVALID, "chr_topo_translate: NULL field or output");
    if (reinterpret_cast<uintptr_t>(d_field) & 3u) return fail(CHR_ERR_INVALID, "chr_topo_translate: misaligned field");
    if (!dims_ok(dims, why)) return fail(CHR_ERR_INVALID, "chr_topo_translate: " + why);
    if (n_iso < 1 || n_iso > CHR_MAX_ISO || !isovalues)
        return fail(CHR_ERR_INVALID, "chr_topo_translate: n_iso must be 1..16 with isovalues");
    for (uint32_t j = 0; j < n_iso; j++)
        if (!isfinite(isovalues[j])) return fail(CHR_ERR_INVALID, "chr_topo_translate: isovalues must be finite");
    if (!(accuracy > 0.0f && accuracy <= 1.0f)) return fail(CHR_ERR_INVALID, "chr_topo_translate: accuracy must be in (0, 1]");
    Alloc al(alloc, (cudaStream_t)stream);
    return translate_impl(d_field, make_grid(dims), isovalues, n_iso, accuracy, al, eb_out, count_out);
}

size_t isosurface_workspace_size(chr_dims dims, uint32_t n_iso)
{
    std::string why;
    if (!dims_ok(dims, why)) return 0;
    return mc_workspace_bytes(make_grid(dims), (int)n_iso);
}

size_t isosurface_workspace_min_size(chr_dims dims, uint32_t n_iso)
{
    std::string why;
    if (!dims_ok(dims, why)) return 0;
    return mc_workspace_min_bytes(make_grid(dims), (int)n_iso);
}

chr_status isosurface_extract(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                              float *d_tris, uint64_t cap_tris, uint64_t *d_ntris, uint32_t *d_err, void *d_workspace,
                              size_t workspace_bytes, void *stream)
{
    NvtxRange nvtx_("isosurface_extract");
    std::string why;
    if (!d_field || !d_ntris || !isovalues) return fail(CHR_ERR_INVALID, "isosurface_extract: NULL field, counts or isovalues");
    if (!dims_ok(dims, why)) return fail(CHR_ERR_INVALID, "isosurface_extract: " + why);
    if (n_iso < 1 || n_iso > CHR_MAX_ISO) return fail(CHR_ERR_INVALID, "isosurface_extract: n_iso must be 1..16");
    for (uint32_t j = 0; j < n_iso; j++)
        if (!isfinite(isovalues[j])) return fail(CHR_ERR_INVALID, "isosurface_extract: isovalues must be finite");
    if (cap_tris > 0 && !d_tris) return fail(CHR_ERR_INVALID, "isosurface_extract: NULL triangle buffer");
    if ((reinterpret_cast<uintptr_t>(d_field) & 3u) || (reinterpret_cast<uintptr_t>(d_tris) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_ntris) & 7u) || (reinterpret_cast<uintptr_t>(d_err) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_workspace) & 7u))
        return fail(CHR_ERR_INVALID, "isosurface_extract: misaligned pointer");
    if (cap_tris > (1ull << 58)) return fail(CHR_ERR_INVALID, "isosurface_extract: cap_tris too large");
    const Grid g = make_grid(dims);
    if (!d_workspace || workspace_bytes < mc_workspace_min_bytes(g, (int)n_iso))
        return fail(CHR_ERR_INVALID, "isosurface_extract: workspace smaller than the minimum (see isosurface_workspace_size)");
    cudaStream_t s = (cudaStream_t)stream;
    CHR_CUDA(cudaMemsetAsync(d_ntris, 0, sizeof(uint64_t) * n_iso, s), "isosurface_extract");
    if (d_err) CHR_CUDA(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s), "isosurface_extract");
    CHR_CUDA(launch_mc(d_field, g, isovalues, (int)n_iso, d_tris, cap_tris, d_ntris, d_err, d_workspace,
                       workspace_bytes, s),
             "isosurface_extract");
    return CHR_OK;
}

chr_status chr_isosurface(const chr_handle *h, uint32_t level, const float *isovalues, uint32_t n_iso,
                          float *d_field_out, float *d_tris, uint64_t cap_tris, uint64_t *d_ntris, uint32_t *d_err,
                          uint32_t flags, const chr_allocator *alloc, void *stream)
{
    NvtxRange nvtx_("chr_isosurface");
    if (!h || !d_ntris || !isovalues) return fail(CHR_ERR_INVALID, "chr_isosurface: NULL handle, counts or isovalues");
    if (level >= h->nlevels) return fail(CHR_ERR_INVALID, "chr_isosurface: level out of range");
    if (n_iso < 1 || n_iso > CHR_MAX_ISO) return fail(CHR_ERR_INVALID, "chr_isosurface: n_iso must be 1..16");
    for (uint32_t j = 0; j < n_iso; j++)
        if (!isfinite(isovalues[j])) return fail(CHR_ERR_INVALID, "chr_isosurface: isovalues must be finite");
    if (flags & ~(uint32_t)(CHR_ISO_INDEX | CHR_ISO_FUSED)) return fail(CHR_ERR_INVALID, "chr_isosurface: unknown flags");
    if (cap_tris > 0 && !d_tris) return fail(CHR_ERR_INVALID, "chr_isosurface: NULL triangle buffer");
    if (cap_tris > (1ull << 58)) return fail(CHR_ERR_INVALID, "chr_isosurface: cap_tris too large");
    if ((reinterpret_cast<uintptr_t>(d_field_out) & 3u) || (reinterpret_cast<uintptr_t>(d_tris) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_ntris) & 7u) || (reinterpret_cast<uintptr_t>(d_err) & 3u))
        return fail(CHR_ERR_INVALID, "chr_isosurface: misaligned pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Alloc al(alloc, s);
    const Grid &g = h->g;
    const float2 *index = (h->has_index && (flags & CHR_ISO_INDEX)) ? h->d_index[level] : nullptr;
    CodecParams p;
    fill_codec_params(h, p);
    p.nlevels = (int32_t)level + 1;
    set_box(p, g, 0, 0, 0, g.nx, g.ny, g.nz);
    chr_status st = CHR_OK;
    cudaError_t e = cudaSuccess;
    if (!(flags & CHR_ISO_FUSED)) {
        // decode into a field (scratch when d_field_out is NULL), then
        // marching cubes on it with the index
        const size_t field_bytes = d_field_out ? 0 : (size_t)g.N * sizeof(float);
        const size_t ws_bytes = mc_workspace_bytes(g, (int)n_iso);
        void *field_scratch = nullptr;
        if (!d_field_out && !(field_scratch = al.get(field_bytes)))
            return fail(CHR_ERR_OOM, "chr_isosurface: allocator returned NULL");
        void *ws = al.get(ws_bytes);
        if (!ws) {
            al.put(field_scratch, field_bytes);
            return fail(CHR_ERR_OOM, "chr_isosurface: allocator returned NULL");
        }
        float *field = d_field_out ? d_field_out : reinterpret_cast<float *>(field_scratch);
        p.out = field;
        if ((e = launch_decode(p, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_ntris, 0, sizeof(uint64_t) * n_iso, s)) != cudaSuccess ||
            (d_err && (e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s)) != cudaSuccess) ||
            (e = launch_mc(field, g, isovalues, (int)n_iso, d_tris, cap_tris, d_ntris, d_err, ws, ws_bytes, s,
                           index)) != cudaSuccess)
            st = cuda_fail(e, "chr_isosurface");
        al.put(ws, ws_bytes);
        al.put(field_scratch, field_bytes);
        return st;
    }
    // one launch per 4 isovalues: each tile's box is decoded in shared memory
    const size_t ws_bytes = mc_workspace_min_bytes(g, (int)n_iso);
    void *ws = al.get(ws_bytes);
    if (!ws) return fail(CHR_ERR_OOM, "chr_isosurface: allocator returned NULL");
    ChrMcLevels c;
    memset(&c, 0, sizeof(c));
    for (uint32_t l = 0; l <= level; l++) {
        c.recs[l] = h->d_recs[l];
        c.words[l] = h->d_words[l];
        c.exc_idx[l] = h->d_exc_idx[l];
        c.exc_val[l] = h->d_exc_val[l];
        c.two_e[l] = h->two_e[l];
    }
    c.nlevels = (int32_t)level + 1;
    c.index = index;
    if (d_field_out) {
        p.out = d_field_out;
        e = launch_decode(p, s);
    }
    if (e != cudaSuccess || (e = cudaMemsetAsync(d_ntris, 0, sizeof(uint64_t) * n_iso, s)) != cudaSuccess ||
        (d_err && (e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s)) != cudaSuccess) ||
        (e = launch_mc_chr(c, g, isovalues, (int)n_iso, d_tris, cap_tris, d_ntris, d_err, ws, ws_bytes, s)) !=
            cudaSuccess)
        st = cuda_fail(e, "chr_isosurface");
    al.put(ws, ws_bytes);
    return st;
}

chr_status chr_brick_index(const chr_handle *h, uint32_t level, float *d_out, void *stream)
{
    NvtxRange nvtx_("chr_brick_index");
    if (!h || !d_out) return fail(CHR_ERR_INVALID, "chr_brick_index: NULL handle or output");
    if (level >= h->nlevels) return fail(CHR_ERR_INVALID, "chr_brick_index: level out of range");
    if (!h->has_index) return fail(CHR_ERR_INVALID, "chr_brick_index: the handle has no value index (a version-1 byte string)");
    if (reinterpret_cast<uintptr_t>(d_out) & 7u) return fail(CHR_ERR_INVALID, "chr_brick_index: misaligned output");
    CHR_CUDA(cudaMemcpyAsync(d_out, h->d_index[level], (size_t)h->g.nbricks * sizeof(float2), cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream),
             "chr_brick_index");
    return CHR_OK;
}

size_t isosurface_backward_workspace_size(chr_dims dims, uint32_t n_iso)
{
    std::string why;
    if (!dims_ok(dims, why)) return 0;
    return mc_adjoint_workspace_bytes(make_grid(dims), (int)n_iso);
}

chr_status isosurface_backward(const float *d_field, chr_dims dims, const float *isovalues, uint32_t n_iso,
                               const float *d_grad_tris, uint64_t cap_tris, float *d_grad_field, void *d_workspace,
                               size_t workspace_bytes, void *stream)
{
    NvtxRange nvtx_("isosurface_backward");
    std::string why;
    if (!d_field || !isovalues || !d_grad_field) return fail(CHR_ERR_INVALID, "isosurface_backward: NULL argument");
    if (!dims_ok(dims, why)) return fail(CHR_ERR_INVALID, "isosurface_backward: " + why);
    if (n_iso < 1 || n_iso > CHR_MAX_ISO) return fail(CHR_ERR_INVALID, "isosurface_backward: n_iso must be 1..16");
    for (uint32_t j = 0; j < n_iso; j++)
        if (!isfinite(isovalues[j])) return fail(CHR_ERR_INVALID, "isosurface_backward: isovalues must be finite");
    if (cap_tris > 0 && !d_grad_tris) return fail(CHR_ERR_INVALID, "isosurface_backward: NULL gradient buffer");
    if (cap_tris > (1ull << 58)) return fail(CHR_ERR_INVALID, "isosurface_backward: cap_tris too large");
    if ((reinterpret_cast<uintptr_t>(d_field) & 3u) || (reinterpret_cast<uintptr_t>(d_grad_tris) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_grad_field) & 3u) || (reinterpret_cast<uintptr_t>(d_workspace) & 7u))
        return fail(CHR_ERR_INVALID, "isosurface_backward: misaligned pointer");
    const Grid g = make_grid(dims);
    if (!d_workspace || workspace_bytes < mc_adjoint_workspace_bytes(g, (int)n_iso))
        return fail(CHR_ERR_INVALID, "isosurface_backward: workspace smaller than isosurface_backward_workspace_size()");
    CHR_CUDA(launch_mc_adjoint(d_field, g, isovalues, (int)n_iso, d_grad_tris, cap_tris, d_grad_field, d_workspace,
                               (cudaStream_t)stream),
             "isosurface_backward");
    return CHR_OK;
}

size_t isosurface_distance_loss_workspace_size(uint64_t npts) { return dist_loss_workspace_bytes(npts); }

chr_status isosurface_distance_loss(const float *d_orig_field, chr_dims dims, float isovalue, const float *d_points,
                                    uint64_t npts, double *d_loss, float *d_grad_points, void *d_workspace,
                                    size_t workspace_bytes, void *stream)
{
    NvtxRange nvtx_("isosurface_distance_loss");
    std::string why;
    if (!d_orig_field || !d_loss || (npts > 0 && !d_points))
        return fail(CHR_ERR_INVALID, "isosurface_distance_loss: NULL argument");
    if (!dims_ok(dims, why)) return fail(CHR_ERR_INVALID, "isosurface_distance_loss: " + why);
    if (!isfinite(isovalue)) return fail(CHR_ERR_INVALID, "isosurface_distance_loss: isovalue must be finite");
    if ((reinterpret_cast<uintptr_t>(d_orig_field) & 3u) || (reinterpret_cast<uintptr_t>(d_points) & 3u) ||
        (reinterpret_cast<uintptr_t>(d_grad_points) & 3u) || (reinterpret_cast<uintptr_t>(d_loss) & 7u) ||
        (reinterpret_cast<uintptr_t>(d_workspace) & 7u))
        return fail(CHR_ERR_INVALID, "isosurface_distance_loss: misaligned pointer");
    if (!d_workspace || workspace_bytes < dist_loss_workspace_bytes(npts))
        return fail(CHR_ERR_INVALID, "isosurface_distance_loss: workspace too small");
    CHR_CUDA(launch_dist_loss(d_orig_field, make_grid(dims), isovalue, d_points, npts, d_loss, d_grad_points,
                              d_workspace, (cudaStream_t)stream),
             "isosurface_distance_loss");
    return CHR_OK;
}

chr_status chr_stats(const chr_handle *h, chr_stats_t *out)
{
    if (!h || !out) return fail(CHR_ERR_INVALID, "chr_stats: NULL argument");
    memset(out, 0, sizeof(*out));
    out->dims = h->dims;
    out->nlevels = h->nlevels;
    out->n_iso = h->n_iso;
    out->topo_mode = h->topo_mode;
    out->nbricks = (uint64_t)h->g.nbricks;
    for (uint32_t l = 0; l < h->nlevels; l++) {
        out->eb[l] = h->eb[l];
        out->payload_words[l] = h->nwords[l];
        out->exceptions[l] = h->nexc[l];
        out->level_bytes[l] = level_bytes(h, l);
    }
    out->eb_translated = h->eb_translated;
    out->topo_accuracy = h->topo_accuracy;
    out->translate_D_count = h->D_count;
    return CHR_OK;
}

chr_status chr_serialize(const chr_handle *h, void *host_buf, size_t cap, size_t *need, void *stream)
{
    NvtxRange nvtx_("chr_serialize");
    if (!h || !need) return fail(CHR_ERR_INVALID, "chr_serialize: NULL handle or size");
    size_t total = header_bytes(h->nlevels, h->n_iso);
    for (uint32_t l = 0; l < h->nlevels; l++) total += level_bytes(h, l);
    if (h->has_index) total += (size_t)h->nlevels * h->g.nbricks * 8;
    *need = total;
    if (!host_buf || cap < total) return CHR_OK;
    std::vector<char> hdr;
    Writer w{&hdr};
    hdr.insert(hdr.end(), {'C', 'H', 'R', '1'});
    w.put<uint32_t>(h->has_index ? 2 : 1);
    w.put<int64_t>(h->dims.nx);
    w.put<int64_t>(h->dims.ny);
    w.put<int64_t>(h->dims.nz);
    w.put<uint32_t>(h->nlevels);
    w.put<uint32_t>(h->n_iso);
    w.put<uint32_t>(h->topo_mode);
    w.put<uint32_t>(h->flags);
    w.put<float>(h->topo_accuracy);
    w.put<float>(h->eb_translated);
    w.put<uint64_t>(h->D_count);
    for (uint32_t l = 0; l < h->nlevels; l++) w.put<float>(h->eb[l]);
    for (uint32_t j = 0; j < h->n_iso; j++) w.put<float>(h->iso[j]);
    for (uint32_t l = 0; l < h->nlevels; l++) {
        w.put<uint64_t>(h->nwords[l]);
        w.put<uint64_t>(h->nexc[l]);
    }
    char *dst = (char *)host_buf;
    memcpy(dst, hdr.data(), hdr.size());
    size_t off = hdr.size();
    cudaStream_t s = (cudaStream_t)stream;
    for (uint32_t l = 0; l < h->nlevels; l++) {
        const size_t nr = (size_t)h->g.nbricks * 16, nw = (size_t)h->nwords[l] * 4, ne = (size_t)h->nexc[l];
        CHR_CUDA(cudaMemcpyAsync(dst + off, h->d_recs[l], nr, cudaMemcpyDeviceToHost, s), "chr_serialize");
        off += nr;
        if (nw) CHR_CUDA(cudaMemcpyAsync(dst + off, h->d_words[l], nw, cudaMemcpyDeviceToHost, s), "chr_serialize");
        off += nw;
        if (ne) CHR_CUDA(cudaMemcpyAsync(dst + off, h->d_exc_idx[l], ne * 2, cudaMemcpyDeviceToHost, s), "chr_serialize");
        const size_t idx = (ne * 2 + 3) & ~size_t(3);
        if (idx > ne * 2) memset(dst + off + ne * 2, 0, idx - ne * 2);
        off += idx;
        if (ne) CHR_CUDA(cudaMemcpyAsync(dst + off, h->d_exc_val[l], ne * 4, cudaMemcpyDeviceToHost, s), "chr_serialize");
        off += ne * 4;
    }
    if (h->has_index)
        for (uint32_t l = 0; l < h->nlevels; l++) {
            CHR_CUDA(cudaMemcpyAsync(dst + off, h->d_index[l], (size_t)h->g.nbricks * 8, cudaMemcpyDeviceToHost, s),
                     "chr_serialize");
            off += (size_t)h->g.nbricks * 8;
        }
    CHR_CUDA(cudaStreamSynchronize(s), "chr_serialize");
    return CHR_OK;
}

chr_status chr_deserialize(const void *host_buf, size_t n, const chr_allocator *alloc, void *stream, chr_handle **out)
{
    NvtxRange nvtx_("chr_deserialize");
    if (!out) return fail(CHR_ERR_INVALID, "chr_deserialize: out is NULL");
    *out = nullptr;
    if (!host_buf) return fail(CHR_ERR_INVALID, "chr_deserialize: NULL buffer");
    const char *src = (const char *)host_buf;
    size_t off = 0;
    auto take = [&](void *dst, size_t k) -> bool {
        if (off + k > n) return false;
        memcpy(dst, src + off, k);
        off += k;
        return true;
    };
    char magic[4];
    uint32_t version = 0, nlevels = 0, n_iso = 0, topo = 0, flags = 0;
    chr_dims dims;
    float acc = 1.0f, ebt = INFINITY;
    uint64_t dcount = 0;
    if (!take(magic, 4) || memcmp(magic, "CHR1", 4) != 0) return fail(CHR_ERR_CORRUPT, "chr_deserialize: bad magic");
    if (!take(&version, 4) || (version != 1 && version != 2))
        return fail(CHR_ERR_CORRUPT, "chr_deserialize: unsupported version");
    if (!take(&dims.nx, 8) || !take(&dims.ny, 8) || !take(&dims.nz, 8) || !take(&nlevels, 4) || !take(&n_iso, 4) ||
        !take(&topo, 4) || !take(&flags, 4) || !take(&acc, 4) || !take(&ebt, 4) || !take(&dcount, 8))
        return fail(CHR_ERR_CORRUPT, "chr_deserialize: truncated header");
    std::string why;
    if (!dims_ok(dims, why)) return fail(CHR_ERR_CORRUPT, "chr_deserialize: " + why);
    if (nlevels < 1 || nlevels > CHR_MAX_LEVELS || n_iso > CHR_MAX_ISO || topo > CHR_TOPO_TRANSLATE || flags != 0)
        return fail(CHR_ERR_CORRUPT, "chr_deserialize: bad level/isovalue/mode fields");
    cudaStream_t s = (cudaStream_t)stream;
    chr_handle *h = new_handle(dims, alloc, s);
    h->nlevels = nlevels;
    h->n_iso = n_iso;
    h->topo_mode = topo;
    h->topo_accuracy = acc;
    h->eb_translated = ebt;
    h->D_count = dcount;
    bool ok = true;
    for (uint32_t l = 0; l < nlevels && ok; l++) ok = take(&h->eb[l], 4) && h->eb[l] >= 0.0f && h->eb[l] < 1e37f;
    for (uint32_t j = 0; j < n_iso && ok; j++) ok = take(&h->iso[j], 4);
    for (uint32_t l = 0; l < nlevels && ok; l++) ok = take(&h->nwords[l], 8) && take(&h->nexc[l], 8);
    if (!ok) {
        delete h;
        return fail(CHR_ERR_CORRUPT, "chr_deserialize: truncated or invalid header arrays");
    }
    set_constants(h);
    const Grid &g = h->g;
    // every level's place in the buffer (cheap size checks first)
    std::vector<size_t> level_off(nlevels);
    for (uint32_t l = 0; l < nlevels; l++) {
        level_off[l] = off;
        if (h->nexc[l] > (uint64_t)g.N || h->nwords[l] > (uint64_t)g.nbricks * 512 || off + level_bytes(h, l) > n) {
            delete h;
            return fail(CHR_ERR_CORRUPT, "chr_deserialize: level sizes inconsistent with the buffer");
        }
        off += level_bytes(h, l);
    }
    // version 2: every level's value index follows the levels (any values
    // are safe to upload: the index only decides which bricks are classified)
    const bool with_index = (version == 2);
    const size_t index_off = off, index_bytes = (size_t)g.nbricks * 8;
    if (with_index && off + index_bytes * nlevels > n) {
        delete h;
        return fail(CHR_ERR_CORRUPT, "chr_deserialize: truncated value index");
    }
    // The copies are issued first and the host checks every level while
    // they are in flight: the device only holds the bytes, no kernel reads
    // them before this call has returned the handle, and a failed check
    // waits for the copies and frees the buffers.  A failed check is
    // reported ahead of a failed allocation or copy.
    Alloc al(alloc, s);
    bool oom = !alloc_records(h, al, with_index) || !alloc_payload(h, al);
    cudaError_t ce = cudaSuccess;
    for (uint32_t l = 0; l < nlevels && !oom && ce == cudaSuccess && with_index; l++)
        ce = cudaMemcpyAsync(h->d_index[l], src + index_off + index_bytes * l, index_bytes, cudaMemcpyHostToDevice, s);
    for (uint32_t l = 0; l < nlevels && !oom && ce == cudaSuccess; l++) {
        size_t o = level_off[l];
        const size_t nr = (size_t)g.nbricks * 16, nw = (size_t)h->nwords[l] * 4, ne = (size_t)h->nexc[l];
        ce = cudaMemcpyAsync(h->d_recs[l], src + o, nr, cudaMemcpyHostToDevice, s);
        o += nr;
        if (ce == cudaSuccess && nw) ce = cudaMemcpyAsync(h->d_words[l], src + o, nw, cudaMemcpyHostToDevice, s);
        o += nw;
        if (ce == cudaSuccess && ne) ce = cudaMemcpyAsync(h->d_exc_idx[l], src + o, ne * 2, cudaMemcpyHostToDevice, s);
        o += (ne * 2 + 3) & ~size_t(3);
        if (ce == cudaSuccess && ne) ce = cudaMemcpyAsync(h->d_exc_val[l], src + o, ne * 4, cudaMemcpyHostToDevice, s);
    }
    bool corrupt = false;
    for (uint32_t l = 0; l < nlevels && !corrupt; l++) {
        const size_t nr = (size_t)g.nbricks * 16;
        const uint32_t *rec = reinterpret_cast<const uint32_t *>(src + level_off[l]);
        const uint16_t *eidx = reinterpret_cast<const uint16_t *>(src + level_off[l] + nr + h->nwords[l] * 4);
        uint64_t wsum = 0, esum = 0;
        corrupt = !validate_level(rec, eidx, g, h->nexc[l], wsum, esum) || 16 * wsum != h->nwords[l] ||
                  esum != h->nexc[l];
    }
    // (always: the buffers are freed only after their copies are done)
    const cudaError_t se = oom ? cudaSuccess : cudaStreamSynchronize(s);
    if (corrupt || oom || ce != cudaSuccess || se != cudaSuccess) {
        free_handle_buffers(h);
        delete h;
        if (corrupt)
            return fail(CHR_ERR_CORRUPT, "chr_deserialize: records inconsistent (widths, prefix sums or exception slots)");
        if (oom) return fail(CHR_ERR_OOM, "chr_deserialize: allocator returned NULL");
        return cuda_fail(ce != cudaSuccess ? ce : se, "chr_deserialize");
    }
    *out = h;
    return CHR_OK;
}

void chr_free(chr_handle *h)
{
    if (!h) return;
    free_handle_buffers(h);
    delete h;
}

}  // extern "C"

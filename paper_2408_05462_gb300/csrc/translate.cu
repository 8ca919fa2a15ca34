// Error-bound translation (paper Sec. 2.2): the multiset D of d0 = k - s0 and
// d1 = s1 - k over every grid edge with s0 < k < s1, and its smallest or n-th
// smallest element.  D is never materialised whole (non-negative floats order
// like their bit patterns): one walk over the edges takes the minimum
// (accuracy 1).  For the n-th smallest, a walk over a sample of the field
// (every 16th item) builds a 4096-bin histogram of the elements' top 12
// bits, from which a range of buckets that should hold rank n is chosen; one
// walk over the whole field then counts the elements below the range and
// appends those inside it to a compact array, and small histogram passes
// over that array select the element exactly.  When the range misses rank n
// (an unrepresentative sample), the exact two-walk selection runs instead: a
// 4096-bin histogram of the whole field names the bucket that holds rank n,
// a second walk appends that bucket's elements, and two histogram passes
// over them (bits 10..19, then 0..9) select the element.
//
// Each vertex v is summarised against the sorted isovalues by a = #{k < v}
// and b = #{k > v}.  An edge (s, t) then holds c1 = a_t + b_s - nK isovalues
// strictly between with s the lower end, and c2 = a_s + b_t - nK with t the
// lower end (at most one is positive; a NaN end has a = b = 0, so neither
// is); they are the sorted isovalues of index nK - b_s .. a_t - 1 (resp.
// nK - b_t .. a_s - 1).  The smallest d0 of such an edge belongs to the
// smallest isovalue above s and the smallest d1 to the largest below t:
// up(s) = K[nK - b_s] - s and dn(t) = t - K[a_t - 1] per vertex (both rounded
// down, like every element of D).  The minimum pass needs nothing else; the
// histogram and collecting walks take these two elements of every crossing
// edge the same way and compute the others (edges across two isovalues or
// more) from the two end values.
//
// Tiling: a block of 16 warps walks a tile of 32 x-columns by 16 rows along z.
// Lane 31 and warp 15 are halo: they read the next tile's first column and
// row so that every owned vertex (31 x 15 per plane) finds its +x neighbour
// by a warp shuffle and its +y neighbour in shared memory; its +z neighbour
// is the next plane, already in registers.  The field is read once per pass
// (plus the one-column, one-row and one-plane halos).
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace chr {

namespace {

constexpr int kTrWarps = 16;           // rows per tile, one warp each
constexpr int kTrOwnX = 31;            // owned columns per tile (lane 31 is halo)
constexpr int kTrOwnY = kTrWarps - 1;  // owned rows per tile (warp 15 is halo)
constexpr int kTrG = 4;                // planes per shared-memory exchange
constexpr int kTrBlocksPerSm = 2;

struct TrParams {
    const float *f;
    int64_t nx, ny, nz;
    int32_t nK;
    float Klt[CHR_MAX_ISO];  // sorted isovalues, +inf past nK (never below a vertex)
    float Kgt[CHR_MAX_ISO];  // sorted isovalues, -inf past nK (never above a vertex)
    uint32_t prefix;         // collect: the top 12 bits of the elements kept
    uint32_t lo_bits, hi_bits;  // range: elements below lo_bits are counted, those in [lo_bits, hi_bits) kept
    int64_t tiles_x, tiles_y, zc, items;
    int64_t item_step;       // every item_step-th item (1: all; more: a sample)
    TranslateScratch sc;
};

// a = #{k < v} in bits 0-7, b = #{k > v} in bits 8-15 (NK >= nK, padded)
template <int NK>
__device__ __forceinline__ uint32_t below_above(float v, const TrParams &p)
{
    uint32_t a = 0, b = 0;
#pragma unroll
    for (int j = 0; j < NK; j++) {
        a += (p.Klt[j] < v) ? 1u : 0u;
        b += (v < p.Kgt[j]) ? 1u : 0u;
    }
    return a | (b << 8);
}

__device__ __forceinline__ uint32_t tr_lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

constexpr int kTrHistBins = 4096;  // the first walk's key: the top 12 bits
constexpr int kTrAppBuf = 4096;    // a block's appended elements staged in shared memory

// MODE: kTrMin (the minimum), kTrHist (the 12-bit histogram), kTrCollect
// (the elements whose top 12 bits are p.prefix, appended to p.sc.coll),
// kTrRange (the elements below p.lo_bits counted, those in [p.lo_bits,
// p.hi_bits) appended less p.lo_bits).
enum { kTrMin = 0, kTrHist = 1, kTrCollect = 2, kTrRange = 3 };

template <int NK, int MODE>
__global__ void __launch_bounds__(kTrWarps * 32, kTrBlocksPerSm) k_translate(const __grid_constant__ TrParams p)
{
    constexpr bool MIN = MODE == kTrMin;
    constexpr bool APP = MODE == kTrCollect || MODE == kTrRange;
    __shared__ uint32_t s_x[3][kTrG][kTrWarps][32];  // exchanged words per vertex: ab, up, dn
    __shared__ unsigned int s_hist[MODE == kTrHist ? kTrHistBins : 1];
    __shared__ float s_kup[CHR_MAX_ISO + 1];  // sorted isovalues, +inf at nK
    __shared__ float s_kdn[CHR_MAX_ISO + 1];  // -inf, then the sorted isovalues
    __shared__ unsigned long long s_cnt, s_lo;
    __shared__ unsigned int s_min;
    // appended elements: staged in s_app (s_napp reserved, the first s_valid
    // of them written) and copied out when half full and at the end, so that
    // the global counter takes one atomic per copy instead of one per group
    // of lanes; a group that does not fit goes straight to global memory
    __shared__ uint32_t s_app[APP ? kTrAppBuf : 1];
    __shared__ unsigned int s_napp, s_valid;
    __shared__ unsigned long long s_flush;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (MODE == kTrHist)
        for (int i = threadIdx.x; i < kTrHistBins; i += blockDim.x) s_hist[i] = 0u;
    if (threadIdx.x <= CHR_MAX_ISO) {
        const int i = threadIdx.x;
        s_kup[i] = (i < p.nK) ? p.Klt[i] : __int_as_float(0x7f800000);
        s_kdn[i] = (i == 0) ? __int_as_float(0xff800000) : p.Klt[i - 1];
    }
    if (threadIdx.x == 0) {
        s_cnt = 0ull;
        s_lo = 0ull;
        s_min = 0xffffffffu;
        s_napp = 0u;
        s_valid = kTrAppBuf;
    }
    __syncthreads();

    unsigned long long cnt = 0, cnt_lo = 0;
    uint32_t lo32 = 0;  // range: elements below lo_bits in the current item
    unsigned int mn = 0xffffffffu;
    const int nK = p.nK;
    const int64_t plane = p.nx * p.ny;

    // v appended where `want`, one shared atomic per group of lanes that
    // append together.  CONV: all 32 lanes call it together
    auto append = [&](bool want, uint32_t v, auto conv) {
        const uint32_t m = decltype(conv)::value ? __ballot_sync(CHR_FULL_MASK, want) : __ballot_sync(__activemask(), want);
        if (want) {
            const int leader = __ffs(m) - 1;
            const uint32_t n = __popc(m), rank = __popc(m & tr_lanemask_lt());
            uint32_t b = 0;
            if (lane == leader) {
                b = atomicAdd(&s_napp, n);
                if (b < kTrAppBuf && b + n > kTrAppBuf) s_valid = b;  // (the one group that straddles the end)
            }
            b = __shfl_sync(m, b, leader);
            if (b + n <= kTrAppBuf) {
                s_app[b + rank] = v;
            } else {
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(p.sc.ncoll, (unsigned long long)n);
                base = __shfl_sync(m, base, leader);
                if (base + rank < p.sc.cap) p.sc.coll[base + rank] = v;
            }
        }
    };
    // the staged elements out (every thread of the block, after a barrier)
    auto flush = [&]() {
        const uint32_t n = min(s_napp, s_valid);
        if (threadIdx.x == 0) s_flush = n ? atomicAdd(p.sc.ncoll, (unsigned long long)n) : 0ull;
        __syncthreads();
        const unsigned long long base = s_flush;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
            if (base + i < p.sc.cap) p.sc.coll[base + i] = s_app[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            s_napp = 0u;
            s_valid = kTrAppBuf;
        }
        __syncthreads();
    };
    // one element of D (where `valid`): into the histogram, or appended when
    // its top 12 bits match (collect) or when it lies in the range (range)
    auto put = [&](bool valid, uint32_t bits, auto conv) {
        if (MODE == kTrHist) {
            if (valid) atomicAdd(&s_hist[bits >> 20], 1u);
        } else if (MODE == kTrCollect) {
            append(valid && (bits >> 20) == p.prefix, bits & 0xfffffu, conv);
        } else if (MODE == kTrRange) {
            const bool below = valid && bits < p.lo_bits;
            lo32 += below ? 1u : 0u;
            append(valid && !below && bits < p.hi_bits, bits - p.lo_bits, conv);
        }
    };
    // one edge (where `on`): s the vertex, t its neighbour, each given by its
    // exchanged words; `ends` gives their values (read only for an edge
    // across two isovalues or more)
    auto edge = [&](bool on, uint32_t ab_s, uint32_t up_s, uint32_t dn_s, uint32_t ab_t, uint32_t up_t,
                    uint32_t dn_t, auto &&ends, uint32_t &c32) {
        const int as = (int)(ab_s & 0xffu), bs = (int)(ab_s >> 8), at = (int)(ab_t & 0xffu), bt = (int)(ab_t >> 8);
        const int c1 = on ? at + bs - nK : 0, c2 = on ? as + bt - nK : 0;
        if (MIN) {
            c32 += (uint32_t)(max(c1, 0) + max(c2, 0));
            if (c1 > 0) mn = min(mn, min(up_s, dn_t));
            if (c2 > 0) mn = min(mn, min(up_t, dn_s));
        } else {
            if (MODE == kTrHist || MODE == kTrRange) c32 += (uint32_t)(max(c1, 0) + max(c2, 0));
            const bool s_low = c1 > 0;
            const int c = s_low ? c1 : c2;
            // d0 of the lowest crossing isovalue and d1 of the highest
            put(c > 0, s_low ? up_s : up_t, std::true_type{});
            put(c > 0, s_low ? dn_t : dn_s, std::true_type{});
            if (c > 1) {  // the other crossing isovalues K[i0 + 1 ..] (d0) and K[.. i0 + c - 2] (d1)
                float vs, vt;
                ends(vs, vt);
                const float lo = s_low ? vs : vt, hi = s_low ? vt : vs;
                const int i0 = nK - (s_low ? bs : bt);
                for (int i = 1; i < c; i++) {
                    put(true, __float_as_uint(__fsub_rd(s_kup[i0 + i], lo)), std::false_type{});
                    put(true, __float_as_uint(__fsub_rd(hi, s_kup[i0 + i - 1])), std::false_type{});
                }
            }
        }
    };

    for (int64_t it = (int64_t)blockIdx.x * p.item_step; it < p.items; it += (int64_t)gridDim.x * p.item_step) {
        const int64_t tx = it % p.tiles_x, r = it / p.tiles_x;
        const int64_t ty = r % p.tiles_y, tz = r / p.tiles_y;
        const int64_t x = tx * kTrOwnX + lane, y = ty * kTrOwnY + w;
        const int64_t z0 = tz * p.zc, z1 = min(z0 + p.zc, p.nz);  // owned planes [z0, z1)
        const int64_t zl = min(z1, p.nz - 1);                      // last plane read
        const bool valid = x < p.nx && y < p.ny;
        const bool own = valid && lane < kTrOwnX && w < kTrOwnY;
        const bool hx = own && x + 1 < p.nx, hy = own && y + 1 < p.ny;
        const float *src = p.f + (valid ? y * p.nx + x : 0);
        auto ld = [&](int64_t z) -> float {
            return (valid && z <= zl) ? __ldg(src + z * plane) : __int_as_float(0x7fffffff);
        };
        // per-vertex words: ab, up, dn
        auto attr = [&](float v, uint32_t &ab, uint32_t &e1, uint32_t &e2) {
            ab = below_above<NK>(v, p);
            e1 = __float_as_uint(__fsub_rd(s_kup[nK - (int)(ab >> 8)], v));
            e2 = __float_as_uint(__fsub_rd(v, s_kdn[ab & 0xffu]));
        };

        uint32_t ab[kTrG + 1], e1[kTrG + 1], e2[kTrG + 1];
        attr(ld(z0), ab[0], e1[0], e2[0]);
        float vn[kTrG];
#pragma unroll
        for (int i = 0; i < kTrG; i++) vn[i] = ld(z0 + 1 + i);
        uint32_t c32 = 0;
        for (int64_t zb = z0; zb < z1; zb += kTrG) {
#pragma unroll
            for (int i = 0; i < kTrG; i++) attr(vn[i], ab[i + 1], e1[i + 1], e2[i + 1]);
#pragma unroll
            for (int i = 0; i < kTrG; i++) vn[i] = ld(zb + kTrG + 1 + i);  // in flight during the edges
#pragma unroll
            for (int i = 0; i < kTrG; i++) {
                s_x[0][i][w][lane] = ab[i];
                s_x[1][i][w][lane] = e1[i];
                s_x[2][i][w][lane] = e2[i];
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kTrG; i++) {
                const uint32_t xab = __shfl_down_sync(CHR_FULL_MASK, ab[i], 1);
                const uint32_t xe1 = __shfl_down_sync(CHR_FULL_MASK, e1[i], 1);
                const uint32_t xe2 = __shfl_down_sync(CHR_FULL_MASK, e2[i], 1);
                const int wy = (w + 1 < kTrWarps) ? w + 1 : w;  // (the halo warp's reads go unused)
                const uint32_t yab = s_x[0][i][wy][lane], ye1 = s_x[1][i][wy][lane], ye2 = s_x[2][i][wy][lane];
                const int64_t z = zb + i;
                const bool oz = own && z < z1;
                // the end values of the +x, +y and +z edges from vertex (x, y, z)
                auto ends_at = [&](int64_t step) {
                    return [&, step](float &vs, float &vt) {
                        vs = __ldg(src + z * plane);
                        vt = __ldg(src + z * plane + step);
                    };
                };
                if (MIN) {
                    if (oz) {
                        if (hx) edge(true, ab[i], e1[i], e2[i], xab, xe1, xe2, ends_at(1), c32);
                        if (hy) edge(true, ab[i], e1[i], e2[i], yab, ye1, ye2, ends_at(p.nx), c32);
                        if (z + 1 < p.nz) edge(true, ab[i], e1[i], e2[i], ab[i + 1], e1[i + 1], e2[i + 1], ends_at(plane), c32);
                    }
                } else {  // every lane takes every edge (the collecting walk's ballots take the whole warp)
                    edge(oz && hx, ab[i], e1[i], e2[i], xab, xe1, xe2, ends_at(1), c32);
                    edge(oz && hy, ab[i], e1[i], e2[i], yab, ye1, ye2, ends_at(p.nx), c32);
                    edge(oz && z + 1 < p.nz, ab[i], e1[i], e2[i], ab[i + 1], e1[i + 1], e2[i + 1], ends_at(plane),
                         c32);
                }
            }
            __syncthreads();
            if (APP && s_napp >= kTrAppBuf / 2) flush();  // (uniform: read after the barrier)
            ab[0] = ab[kTrG];
            e1[0] = e1[kTrG];
            e2[0] = e2[kTrG];
        }
        cnt += 2ull * c32;  // d0 and d1 per crossing; c32 <= 3 * 16 per plane, and an item spans <= 2^20 planes
        cnt_lo += lo32;
        lo32 = 0;
    }

    if (APP) {
        __syncthreads();
        if (s_napp) flush();
    }

    // block reduction, then one global update per block
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(CHR_FULL_MASK, cnt, o);
        if (MODE == kTrRange) cnt_lo += __shfl_xor_sync(CHR_FULL_MASK, cnt_lo, o);
        mn = min(mn, __shfl_xor_sync(CHR_FULL_MASK, mn, o));
    }
    if (lane == 0) {
        if (cnt) atomicAdd(&s_cnt, cnt);
        if (MODE == kTrRange && cnt_lo) atomicAdd(&s_lo, cnt_lo);
        if (MIN) atomicMin(&s_min, mn);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cnt && MODE != kTrCollect) atomicAdd(p.sc.count, s_cnt);
        if (MODE == kTrRange && s_lo) atomicAdd(p.sc.count_lo, s_lo);
        if (MIN) atomicMin(p.sc.minbits, s_min);
    }
    if (MODE == kTrHist)
        for (int i = threadIdx.x; i < kTrHistBins; i += blockDim.x)
            if (s_hist[i]) atomicAdd(p.sc.hist + i, (unsigned long long)s_hist[i]);
}

// Histogram of bits [shift, shift + 10) of the collected values, over those
// whose bits from shift + 10 up equal `above`.
__global__ void __launch_bounds__(256) k_select_hist(const uint32_t *coll, unsigned long long n, int shift,
                                                     uint32_t above, unsigned long long *hist)
{
    __shared__ unsigned int s_h[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s_h[i] = 0u;
    __syncthreads();
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t v = coll[i];
        if ((v >> (shift + 10)) == above) atomicAdd(&s_h[(v >> shift) & 1023u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += blockDim.x)
        if (s_h[i]) atomicAdd(hist + i, (unsigned long long)s_h[i]);
}

template <int NK>
void launch_nk(const TrParams &p, int mode, unsigned blocks, cudaStream_t s)
{
    if (mode == kTrMin)
        k_translate<NK, kTrMin><<<blocks, kTrWarps * 32, 0, s>>>(p);
    else if (mode == kTrHist)
        k_translate<NK, kTrHist><<<blocks, kTrWarps * 32, 0, s>>>(p);
    else if (mode == kTrCollect)
        k_translate<NK, kTrCollect><<<blocks, kTrWarps * 32, 0, s>>>(p);
    else
        k_translate<NK, kTrRange><<<blocks, kTrWarps * 32, 0, s>>>(p);
}

}  // namespace

size_t translate_scratch_bytes() { return kTrHistBins * sizeof(unsigned long long) + 64; }

cudaError_t launch_translate_select(const uint32_t *coll, unsigned long long n, int shift, uint32_t above,
                                    unsigned long long *hist, cudaStream_t s)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long want = (n + 255) / 256;
    const unsigned blocks = (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>(want, 4ull * sms));
    k_select_hist<<<blocks, 256, 0, s>>>(coll, n, shift, above, hist);
    return cudaGetLastError();
}

cudaError_t launch_translate_pass(const float *field, const Grid &g, const float *K, int nK, int mode,
                                  uint32_t prefix, TranslateScratch sc, cudaStream_t s, uint32_t lo_bits,
                                  uint32_t hi_bits, int64_t item_step, int64_t *n_items)
{
    if (nK < 1 || nK > CHR_MAX_ISO) return cudaErrorInvalidValue;
    TrParams p;
    p.f = field;
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.nK = nK;
    float ks[CHR_MAX_ISO];
    std::copy(K, K + nK, ks);
    std::sort(ks, ks + nK);
    for (int j = 0; j < CHR_MAX_ISO; j++) {
        p.Klt[j] = (j < nK) ? ks[j] : INFINITY;
        p.Kgt[j] = (j < nK) ? ks[j] : -INFINITY;
    }
    p.prefix = prefix;
    p.lo_bits = lo_bits;
    p.hi_bits = hi_bits;
    p.item_step = item_step < 1 ? 1 : item_step;
    p.sc = sc;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // items: tiles x chunks of z, about 8 per resident block; a chunk's
    // extent is capped so that a thread's per-item count fits 32 bits
    const int64_t grid = (int64_t)sms * kTrBlocksPerSm;
    p.tiles_x = (g.nx + kTrOwnX - 1) / kTrOwnX;
    p.tiles_y = (g.ny + kTrOwnY - 1) / kTrOwnY;
    const int64_t tiles = p.tiles_x * p.tiles_y;
    int64_t chunks = std::min<int64_t>(std::max<int64_t>((8 * grid + tiles - 1) / tiles, 1), g.nz);
    p.zc = std::min<int64_t>((g.nz + chunks - 1) / chunks, 1 << 20);
    chunks = (g.nz + p.zc - 1) / p.zc;
    p.items = tiles * chunks;
    if (n_items) *n_items = p.items;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((p.items + p.item_step - 1) / p.item_step, grid));
    if (nK <= 1)
        launch_nk<1>(p, mode, blocks, s);
    else if (nK <= 2)
        launch_nk<2>(p, mode, blocks, s);
    else if (nK <= 4)
        launch_nk<4>(p, mode, blocks, s);
    else if (nK <= 8)
        launch_nk<8>(p, mode, blocks, s);
    else
        launch_nk<16>(p, mode, blocks, s);
    return cudaGetLastError();
}

}  // namespace chr

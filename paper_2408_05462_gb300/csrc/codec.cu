// CHR codec kernels: encode (quantise + level chain + sign fix + Lorenzo +
// pack), the record scans, and decode (unpack + inverse Lorenzo + level chain
// + exact vertices).  Paper Sec. 2 (CHR, accuracy levels) and Sec. 2.2
// (topology preservation); the format is this library's (see chr.h).
//
// Work decomposition: one warp owns one 8^3 brick (512 vertices), each lane
// two x-rows of 8 vertices: row r0 = lane (y = lane&7, z = lane>>3) and
// row r1 = lane + 32 (z + 4).  A block of 8 warps takes 8 bricks that follow
// each other along x, so the rows a block touches are 256-byte runs.
#include "common.cuh"
#include "internal.h"

namespace chr {

namespace {

CHR_BOUNDS_WORD();

struct BrickCoord {
    int32_t bx, by, bz;
    int64_t b;  // linear brick index
};

// Minimum / maximum of a float over the warp (one redux instruction; the
// inputs here are never NaN).
__device__ __forceinline__ float warp_min_f32(float v)
{
    float r;
    asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float warp_max_f32(float v)
{
    float r;
    asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// max(a, b), NaN when either is NaN
__device__ __forceinline__ float fmax_nan(float a, float b)
{
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Number of candidate isovalues strictly above v (K sorted ascending).  Two
// values lie on the same side of every k exactly when these counts agree,
// because {j : v < K[j]} is always a suffix of the sorted K.
// K[j] for j >= nK is -inf (never above anything), so NK may be any bound
// >= nK.
template <int NK>
__device__ __forceinline__ int count_above(float v, const float *K)
{
    int c = 0;
#pragma unroll
    for (int j = 0; j < NK; j++) c += (v < K[j]) ? 1 : 0;
    return c;
}

// count_above of the row's 8 values, one byte each
template <int NK>
__device__ __forceinline__ void count_above_row(const float (&f)[8], const float *K, uint32_t (&cfp)[2])
{
#pragma unroll
    for (int x = 0; x < 8; x++) cfp[x >> 2] |= (uint32_t)count_above<NK>(f[x], K) << (8 * (x & 3));
}

// One level of the residual chain for one vertex (paper Sec. 2 accuracy
// levels; Sec. 2.2 sign preservation).  Every float operation is one IEEE
// binary32 operation rounded to nearest-even.  Returns true for a vertex
// stored exactly (bound or sign check failed, or not quantisable); its code
// is the rounded value (0 when not quantisable) and R takes f.
// The sign check compares the count of candidates above R with f's count cf.
// Both counts agree exactly when kdn <= R < kup, kup the smallest candidate
// above f (+inf if none) and kdn the largest at or below it (-inf if none):
// the same test without a second count.
__device__ __forceinline__ bool encode_step(float f, float Rprev, float e, float two_e, float inv2e, bool fix,
                                            float kdn, float kup, int32_t &q, float &R)
{
    // (level 0 starts from Rprev = +0: f - (+0) is f and (+0) + P is P
    // exactly, P never being -0, so it takes the same operations)
    const float r = __fsub_rn(f, Rprev);
    const float x = __fmul_rn(r, inv2e);
    q = 0;
    R = f;
    if (!(fabsf(x) <= CHR_QMAX)) return true;
    const int32_t qi = __float2int_rn(x);  // round half to even
    q = qi;  // kept by an exception too, so the neighbours' prediction stays smooth
    const float P = __fmul_rn(__int2float_rn(qi), two_e);
    const float Rn = __fadd_rn(Rprev, P);
    if (!(fabsf(__fsub_rn(f, Rn)) < e)) return true;
    if (fix && !(Rn >= kdn && Rn < kup)) return true;
    R = Rn;
    return false;
}

// One 8^3 brick per 64 threads (two warps), one x-row of 8 vertices per
// thread: row r = ly + 8*lz, so a warp holds z = 0..3 or z = 4..7 of its
// brick.  A block of 256 threads encodes 4 bricks that follow each other
// along x.  Every thread of the block runs the same level loop (threads of a
// brick past the grid only idle), because the bricks' two warps meet at
// block barriers to exchange the z = 3 row, their maxima and their
// exception counts.
constexpr int kEncBricks = 4;  // bricks per block

// The two warps of brick j meet at their own barrier (1 + j): bricks of a
// block share nothing inside the level loop, so none waits for another.
__device__ __forceinline__ void brick_sync(int j)
{
    asm volatile("bar.sync %0, 64;" ::"r"(1 + j) : "memory");
}

// Row r's 8 codes at width W <= 8 are bits [8Wr, 8Wr + 8W) of the brick's
// stream: the W bytes from byte Wr of its slot (words are little-endian),
// written straight from the row's bits.
template <int W>
__device__ __forceinline__ void store_row(uint32_t *slot, int r, const uint32_t (&zz)[8])
{
    // every code is below 2^W, so the row's two 32-bit halves are built
    // directly (a code that straddles bit 32 goes to both)
    uint32_t lo = 0u, hi = 0u;
#pragma unroll
    for (int x = 0; x < 8; x++) {
        const int sh = W * x;
        if (sh + W <= 32) {
            lo |= zz[x] << sh;
        } else if (sh >= 32) {
            hi |= zz[x] << (sh - 32);
        } else {
            lo |= zz[x] << sh;
            hi |= zz[x] >> (32 - sh);
        }
    }
    const uint64_t row = ((uint64_t)hi << 32) | lo;
    unsigned char *dst = reinterpret_cast<unsigned char *>(slot) + W * r;
    if (W == 1) {
        *dst = (unsigned char)row;
    } else if (W == 2 || W == 6) {
#pragma unroll
        for (int b = 0; b < W / 2; b++) reinterpret_cast<uint16_t *>(dst)[b] = (uint16_t)(row >> (16 * b));
    } else if (W == 4) {
        *reinterpret_cast<uint32_t *>(dst) = (uint32_t)row;
    } else if (W == 8) {
        *reinterpret_cast<uint64_t *>(dst) = row;
    } else {
#pragma unroll
        for (int b = 0; b < W; b++) dst[b] = (unsigned char)(row >> (8 * b));
    }
}

template <bool FULL>
__global__ void __launch_bounds__(256, 4) k_encode(const __grid_constant__ CodecParams p)
{
    __shared__ __align__(16) int32_t s_zrow[kEncBricks][8][8];  // z = 3 rows after the x and y differences
    __shared__ uint32_t s_red[kEncBricks][2][4];                // per warp: max L, max plain, exceptions, -
    __shared__ __align__(16) uint32_t s_pk[kEncBricks][512];    // packed words of each brick (zero between levels)
    __shared__ float s_kup[CHR_MAX_ISO + 1], s_kdn[CHR_MAX_ISO + 1];  // by count of candidates above f
    __shared__ float2 s_rng[kEncBricks][3][4];                  // per warp, then the z = 0 parts: ranges for the index

    const int tid = threadIdx.x, lane = tid & 31;
    const int j = tid >> 6, r = tid & 63, wb = r >> 5;
    const int ly = r & 7, lz = r >> 3;
    const int ngx = (p.nbx + kEncBricks - 1) / kEncBricks;
    const int64_t g = blockIdx.x;
    BrickCoord c;
    c.bx = (int32_t)(g % ngx) * kEncBricks + j;
    const int64_t rest = g / ngx;
    c.by = (int32_t)(rest % p.nby);
    c.bz = (int32_t)(rest / p.nby);
    c.b = c.bx + (int64_t)p.nbx * (c.by + (int64_t)p.nby * c.bz);
    bool mine = c.bx < p.nbx;
    if (mine) {
        const bool full = ((int64_t)c.bx * 8 + 8 <= p.nx) && ((int64_t)c.by * 8 + 8 <= p.ny) && ((int64_t)c.bz * 8 + 8 <= p.nz);
        mine = (full == FULL);
    }
    if (tid <= CHR_MAX_ISO) {  // sign-check intervals by count of candidates above (sorted on the host)
        s_kup[tid] = p.kup[tid];
        s_kdn[tid] = p.kdn[tid];
    }
    *reinterpret_cast<uint4 *>(&s_pk[j][8 * r]) = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(&s_pk[j][8 * r + 4]) = make_uint4(0u, 0u, 0u, 0u);
    if (!__syncthreads_or(mine)) return;  // uniform: no brick of this block is ours

    // load this thread's row
    const int64_t x0 = (int64_t)c.bx * 8, y = (int64_t)c.by * 8 + ly, z = (int64_t)c.bz * 8 + lz;
    float f[8];
    uint32_t valid = 0;
#pragma unroll
    for (int x = 0; x < 8; x++) f[x] = 0.0f;
    if (mine && y < p.ny && z < p.nz) {
        const float *row = p.f + x0 + p.nx * (y + p.ny * z);
        const int ex = (int)((p.nx - x0) < 8 ? (p.nx - x0) : 8);
        if (FULL && (p.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(p.f) & 15u) == 0) {
            const float4 a = ld_stream_f4(reinterpret_cast<const float4 *>(row));
            const float4 b = ld_stream_f4(reinterpret_cast<const float4 *>(row + 4));
            f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
            f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
            valid = 0xffu;
        } else {
#pragma unroll
            for (int x = 0; x < 8; x++)
                if (x < ex) {
                    f[x] = __ldg(row + x);
                    valid |= 1u << x;
                }
        }
    }
    // a full brick's rows are whole (the threads of a brick that is not
    // this kernel's compute on zeros and write nothing)
    if (FULL) valid = 0xffu;

    const bool fix = p.fix != 0;
    uint32_t cfp[2] = {0u, 0u};  // count_above(f), one byte per vertex
    if (fix) {
        if (p.nK <= 1) count_above_row<1>(f, p.K, cfp);
        else if (p.nK <= 2) count_above_row<2>(f, p.K, cfp);
        else if (p.nK <= 4) count_above_row<4>(f, p.K, cfp);
        else if (p.nK <= 8) count_above_row<8>(f, p.K, cfp);
        else count_above_row<CHR_MAX_ISO>(f, p.K, cfp);
    }
    float R[8];
#pragma unroll
    for (int x = 0; x < 8; x++) R[x] = 0.0f;

    for (int l = 0; l < p.nlevels; l++) {
        int32_t q[8];
        uint32_t excm = 0;
        const float e = p.e[l], two_e = p.two_e[l], inv2e = p.inv2e[l];
#pragma unroll
        for (int x = 0; x < 8; x++) {
            q[x] = 0;
            if ((valid >> x) & 1u) {
                float Rn;
                int32_t qq;
                const int cf = (int)((cfp[x >> 2] >> (8 * (x & 3))) & 0xffu);
                const bool ex = encode_step(f[x], R[x], e, two_e, inv2e, fix, fix ? s_kdn[cf] : 0.0f,
                                            fix ? s_kup[cf] : 0.0f, qq, Rn);
                q[x] = qq;
                R[x] = Rn;
                if (ex) excm |= 1u << x;
            }
        }

        // Lorenzo residual: first differences along x, y (lanes 1 apart) and z
        // (lanes 8 apart; the z = 4 rows take the z = 3 rows from shared memory)
        int32_t d[8];
#pragma unroll
        for (int x = 7; x > 0; x--) d[x] = (int32_t)((uint32_t)q[x] - (uint32_t)q[x - 1]);
        d[0] = q[0];
#pragma unroll
        for (int x = 0; x < 8; x++) {
            const int32_t up = __shfl_up_sync(CHR_FULL_MASK, d[x], 1, 8);
            if (ly > 0) d[x] = (int32_t)((uint32_t)d[x] - (uint32_t)up);
        }
        if (lz == 3)
#pragma unroll
            for (int x = 0; x < 8; x++) s_zrow[j][ly][x] = d[x];
        int32_t below[8];
#pragma unroll
        for (int x = 0; x < 8; x++) below[x] = __shfl_up_sync(CHR_FULL_MASK, d[x], 8);
        brick_sync(j);
        if (lz == 4)
#pragma unroll
            for (int x = 0; x < 8; x++) below[x] = s_zrow[j][ly][x];
        if (lz > 0)
#pragma unroll
            for (int x = 0; x < 8; x++) d[x] = (int32_t)((uint32_t)d[x] - (uint32_t)below[x]);

        // the widths: bitlen of the largest zig-zag code = bitlen of their OR
        uint32_t maxl = 0, maxn = 0;
#pragma unroll
        for (int x = 0; x < 8; x++) {
            const bool live = ((valid >> x) & 1u) && !(r == 0 && x == 0);
            if (!live) d[x] = 0;  // d is only read for packing from here on
            maxl |= zigzag(d[x]);
            maxn |= live ? zigzag(q[x]) : 0u;
        }
        const uint32_t cnt = __popc(excm);
        const uint32_t inc = warp_incl_scan_u32(cnt, lane);
        maxl = __reduce_or_sync(CHR_FULL_MASK, maxl);
        maxn = __reduce_or_sync(CHR_FULL_MASK, maxn);
        if (lane == 31) {
            s_red[j][wb][0] = maxl;
            s_red[j][wb][1] = maxn;
            s_red[j][wb][2] = inc;
        }
        brick_sync(j);
        maxl = s_red[j][0][0] | s_red[j][1][0];
        maxn = s_red[j][0][1] | s_red[j][1][1];
        const uint32_t tot0 = s_red[j][0][2];
        const uint32_t nexc = tot0 + s_red[j][1][2];
        const uint32_t exc_rank = inc - cnt + (wb ? tot0 : 0u);
        const int wl = bitlen(maxl), wn = bitlen(maxn);
        const int mode = (wl < wn) ? 1 : 0;
        const int w = mode ? wl : wn;
        if (mine && r == 0)
            p.recs[l][c.b] = make_uint4(0u, 0u, (uint32_t)q[0], (uint32_t)w | ((uint32_t)mode << 8) | (nexc << 16));
        // pack: row r's 8 codes are bits [8*r*w, 8*r*w + 8*w) of the brick's
        // stream.  Widths up to 8 go straight to the brick's slot, a row per
        // thread; wider rows are ORed into the zeroed shared words, then the
        // brick's 16*w words are copied out (and zeroed for the next level)
        uint32_t zz[8];
#pragma unroll
        for (int x = 0; x < 8; x++) {
            const bool live = ((valid >> x) & 1u) && !(r == 0 && x == 0);
            zz[x] = mode ? zigzag(d[x]) : (live ? zigzag(q[x]) : 0u);
        }
        uint32_t *slot = p.slot_words[l] + 512ull * c.b;
        if (w <= 8) {
            if (mine) switch (w) {  // (uniform across the brick)
                    case 1: store_row<1>(slot, r, zz); break;
                    case 2: store_row<2>(slot, r, zz); break;
                    case 3: store_row<3>(slot, r, zz); break;
                    case 4: store_row<4>(slot, r, zz); break;
                    case 5: store_row<5>(slot, r, zz); break;
                    case 6: store_row<6>(slot, r, zz); break;
                    case 7: store_row<7>(slot, r, zz); break;
                    case 8: store_row<8>(slot, r, zz); break;
                    default: break;  // w = 0: no words
                }
        } else {
            const uint32_t bit0 = 8u * (uint32_t)r * (uint32_t)w;
            uint32_t wi = bit0 >> 5;
            int pos = (int)(bit0 & 31u);
            uint64_t acc = 0;
#pragma unroll
            for (int x = 0; x < 8; x++) {
                acc |= (uint64_t)zz[x] << pos;
                pos += w;
                if (pos >= 32) {
                    if ((uint32_t)acc && CHR_IN_BOUNDS(wi < 512u)) atomicOr(&s_pk[j][wi], (uint32_t)acc);
                    acc >>= 32;
                    pos -= 32;
                    wi++;
                }
            }
            if (pos > 0 && (uint32_t)acc && CHR_IN_BOUNDS(wi < 512u)) atomicOr(&s_pk[j][wi], (uint32_t)acc);
            brick_sync(j);
            const int nw = 16 * w;
            for (int jw = r; jw < nw; jw += 64) {
                if (mine) slot[jw] = s_pk[j][jw];
                s_pk[j][jw] = 0u;
            }
        }
        if (mine && cnt) {
            uint32_t pos = exc_rank;
#pragma unroll
            for (int x = 0; x < 8; x++) {
                if (((excm >> x) & 1u) && CHR_IN_BOUNDS(pos < 512u)) {
                    p.slot_idx[l][512ull * c.b + pos] = (uint16_t)(8 * r + x);
                    p.slot_val[l][512ull * c.b + pos] = __float_as_uint(f[x]);
                    pos++;
                }
            }
        }
        // The value index (Sec. 2.1: which bricks an isovalue can cross).
        // Ranges of R over 8 vertex subsets of the brick, NaN as +inf and -0
        // as +0: all of it, the planes x = 0, y = 0, z = 0, the lines
        // x = y = 0, x = z = 0, y = z = 0 and the corner; k_brick_index
        // assembles each brick's cell-vertex range from its own range and
        // its neighbours' planes, lines and corner.  One warp-wide float
        // reduction per range and end (non-members contribute the empty
        // range): the whole warp, its y = 0 lanes, its z = 0 lanes (warp 0);
        // thread 0 holds the y = z = 0 line and the corner itself.
        if (p.idx_part) {
            const float inf = __int_as_float(0x7f800000);
            float mn = inf, mx = -inf, a0 = inf, b0 = -inf;
#pragma unroll
            for (int x = 0; x < 8; x++)
                if ((valid >> x) & 1u) {
                    mn = fminf(mn, R[x]);      // a NaN never lowers it (as +inf would not)
                    mx = fmax_nan(mx, R[x]);   // NaN once any value is
                }
            // NaN as +inf; +0 added to the extremes, which are zeros exactly
            // when some value is a zero (either sign) and none is beyond it
            mn = __fadd_rn(mn, 0.0f);
            mx = __fadd_rn(isnan(mx) ? inf : mx, 0.0f);
            if (valid & 1u) a0 = b0 = isnan(R[0]) ? inf : __fadd_rn(R[0], 0.0f);
            if (r == 0) {  // the y = z = 0 line and the corner
                s_rng[j][2][0] = make_float2(mn, mx);
                s_rng[j][2][1] = make_float2(a0, b0);
            }
            const bool y0 = ly == 0, z0 = lz == 0;
            float2 t;
            t = make_float2(warp_min_f32(mn), warp_max_f32(mx));
            if (lane == 0) s_rng[j][wb][0] = t;  // this warp's whole part
            t = make_float2(warp_min_f32(a0), warp_max_f32(b0));
            if (lane == 0) s_rng[j][wb][1] = t;  // x = 0 plane
            t = make_float2(warp_min_f32(y0 ? mn : inf), warp_max_f32(y0 ? mx : -inf));
            if (lane == 0) s_rng[j][wb][2] = t;  // y = 0 plane
            t = make_float2(warp_min_f32(y0 ? a0 : inf), warp_max_f32(y0 ? b0 : -inf));
            if (lane == 0) s_rng[j][wb][3] = t;  // x = y = 0 line
            if (wb == 0) {                       // (the z = 0 rows are warp 0's lanes 0..7)
                t = make_float2(warp_min_f32(z0 ? mn : inf), warp_max_f32(z0 ? mx : -inf));
                if (lane == 0) s_rng[j][2][2] = t;  // z = 0 plane
                t = make_float2(warp_min_f32(z0 ? a0 : inf), warp_max_f32(z0 ? b0 : -inf));
                if (lane == 0) s_rng[j][2][3] = t;  // x = z = 0 line
            }
        }
        brick_sync(j);  // s_pk, s_zrow, s_red and s_rng are reused by the next level
        if (p.idx_part && mine && r == 0) {  // (thread 0 holds the z = 0 rows' and its own parts)
            auto un = [](float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fmaxf(a.y, b.y)); };
            float4 *dst = reinterpret_cast<float4 *>(p.idx_part + ((size_t)l * p.nbx * p.nby * p.nbz + c.b) * kIdxParts);
            const float2 all = un(s_rng[j][0][0], s_rng[j][1][0]), x0 = un(s_rng[j][0][1], s_rng[j][1][1]);
            const float2 y0 = un(s_rng[j][0][2], s_rng[j][1][2]), x0y0 = un(s_rng[j][0][3], s_rng[j][1][3]);
            const float2 z0 = s_rng[j][2][2], x0z0 = s_rng[j][2][3], y0z0 = s_rng[j][2][0], c0 = s_rng[j][2][1];
            dst[0] = make_float4(all.x, all.y, x0.x, x0.y);
            dst[1] = make_float4(y0.x, y0.y, z0.x, z0.y);
            dst[2] = make_float4(x0y0.x, x0y0.y, x0z0.x, x0z0.y);
            dst[3] = make_float4(y0z0.x, y0z0.y, c0.x, c0.y);
        }
    }
}

// Moves every brick's slot contents to its place in the dense stream: 16*w
// words to words + 16*wsum, and the exceptions to exc_off.  A warp takes
// kCompactBricks bricks in linear order at one level (blockIdx.y) and issues
// the loads of all of them (records, then payloads and first exceptions)
// before any store, so each warp keeps several bricks' bytes in flight.
constexpr int kCompactBricks = 4;

__global__ void __launch_bounds__(256) k_compact(const __grid_constant__ CodecParams p)
{
    const int lane = threadIdx.x & 31;
    const int l = blockIdx.y;
    const int64_t nbricks = (int64_t)p.nbx * p.nby * p.nbz;
    const int64_t b0 = ((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kCompactBricks;
    if (b0 >= nbricks) return;
    const int nb = (int)((nbricks - b0) < kCompactBricks ? (nbricks - b0) : kCompactBricks);
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (lane < nb) r = p.recs[l][b0 + lane];
    uint4 rec[kCompactBricks], v[kCompactBricks];
    uint16_t ei[kCompactBricks];
    uint32_t ev[kCompactBricks];
#pragma unroll
    for (int k = 0; k < kCompactBricks; k++) {
        v[k] = make_uint4(0u, 0u, 0u, 0u);
        ei[k] = 0;
        ev[k] = 0u;
        rec[k].z = 0u;
        rec[k].x = __shfl_sync(CHR_FULL_MASK, r.x, k);
        rec[k].y = __shfl_sync(CHR_FULL_MASK, r.y, k);
        rec[k].w = __shfl_sync(CHR_FULL_MASK, r.w, k);
        const int w = min((int)(rec[k].w & 0xffu), 32), nexc = (int)(rec[k].w >> 16);
        const size_t slot = 512ull * (uint64_t)(b0 + k);
        if (k < nb && lane < 4 * w) v[k] = ld_stream_u4(reinterpret_cast<const uint4 *>(p.slot_words[l] + slot) + lane);
        if (k < nb && lane < nexc) {
            ei[k] = p.slot_idx[l][slot + lane];
            ev[k] = p.slot_val[l][slot + lane];
        }
    }
#pragma unroll
    for (int k = 0; k < kCompactBricks; k++) {
        if (k >= nb) break;
        const int w = min((int)(rec[k].w & 0xffu), 32), nexc = (int)(rec[k].w >> 16);
        const size_t slot = 512ull * (uint64_t)(b0 + k);
        const uint4 *src = reinterpret_cast<const uint4 *>(p.slot_words[l] + slot);
        uint4 *dst = reinterpret_cast<uint4 *>(p.words[l] + 16ull * rec[k].x);
        if (lane < 4 * w) __stcs(dst + lane, v[k]);
        for (int j = lane + 32; j < 4 * w; j += 32) __stcs(dst + j, ld_stream_u4(src + j));  // w > 8
        if (lane < nexc) {
            p.exc_idx[l][rec[k].y + lane] = ei[k];
            p.exc_val[l][rec[k].y + lane] = ev[k];
        }
        for (int j = lane + 32; j < nexc; j += 32) {
            p.exc_idx[l][rec[k].y + j] = p.slot_idx[l][slot + j];
            p.exc_val[l][rec[k].y + j] = p.slot_val[l][slot + j];
        }
    }
}

constexpr int kDecGroup = 3;       // levels whose loads are in flight together
constexpr int kLevelWords = 516;   // shared words per level and warp: 512 payload + read-ahead slack
constexpr int kExcPrefetch = 1;    // exception entries per lane and level loaded ahead (32 per brick)
// k_decode stages only codes of width up to 8 (128 words a level, plus
// read-ahead, a 16-byte multiple) and reads wider levels from global memory;
// a separate 512-float buffer per warp takes the exception patch and the
// rows on their way out.  The smaller footprint leaves more of the SM's
// memory to the L1 cache.
constexpr int kNarrowLevelWords = 132;
constexpr int kDecodeSmem = kWarpsPerBlock * (kDecGroup * kNarrowLevelWords + 512) * 4;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The 8 codes of packed row L (slots 8L..8L+7: bits [8WL, 8WL + 8W) of the
// brick's stream) for a width W <= 8 known at compile time.  A row starts
// on a byte boundary, so one 64-bit window cut from three words holds it
// and every code sits at a fixed offset in the window.
template <int W>
__device__ __forceinline__ void unpack_row(const uint32_t *buf, int L, uint32_t (&q)[8])
{
    const uint32_t bit0 = 8u * W * (uint32_t)L;
    const uint32_t wd = bit0 >> 5, off = bit0 & 31u;
    const uint32_t a = buf[wd], b = buf[wd + 1];
    const uint32_t lo = __funnelshift_r(a, b, off);
    uint64_t win = lo;
    if (W > 4) win |= (uint64_t)__funnelshift_r(b, buf[wd + 2], off) << 32;  // 8W > 32 bits
#pragma unroll
    for (int x = 0; x < 8; x++) q[x] = (uint32_t)unzigzag((uint32_t)(win >> (W * x)) & ((1u << W) - 1u));
}

template <int W>
__device__ __forceinline__ void unpack_rows(const uint32_t *buf, int lane, uint32_t (&q)[2][8])
{
    unpack_row<W>(buf, lane, q[0]);
    unpack_row<W>(buf, lane + 32, q[1]);
}

// Decode one brick per warp.  For each group of up to three levels every
// load is issued before any is consumed: the records (one lane per level),
// the packed words (cp.async straight into shared memory) and the first 32
// exception entries of each level (registers), so a brick costs about two
// memory round trips instead of three per level.
// LW: shared words a level for its packed codes; kLevelWords holds any
// width, a smaller LW widths up to 8 (see kNarrowLevelWords).
template <int LW>
__device__ __forceinline__ void decode_brick(const CodecParams &p, const BrickCoord &c, uint32_t *s_dyn);

__global__ void __launch_bounds__(256, 4) k_decode(const __grid_constant__ CodecParams p)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    BrickCoord c;
    // bricks of the output box: groups of 8 along x inside the box's brick range
    const int warp = threadIdx.x >> 5;
    const int ngx = (p.box_bricks[0] + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int64_t g = blockIdx.x;
    const int32_t gx = (int32_t)(g % ngx);
    const int64_t rest = g / ngx;
    const int32_t lbx = gx * kWarpsPerBlock + warp;
    if (lbx >= p.box_bricks[0]) return;
    c.bx = p.box_brick0[0] + lbx;
    c.by = p.box_brick0[1] + (int32_t)(rest % p.box_bricks[1]);
    c.bz = p.box_brick0[2] + (int32_t)(rest / p.box_bricks[1]);
    c.b = c.bx + (int64_t)p.nbx * (c.by + (int64_t)p.nby * c.bz);
    decode_brick<kNarrowLevelWords>(p, c, s_dyn);
}

// Many CHRs in one launch: warp w of the grid decodes brick w of the
// concatenated brick list (box i owns bricks brick_start[i] ..
// brick_start[i+1]-1, x fastest), so small boxes leave no warp idle.
template <int WPB>
__global__ void __launch_bounds__(WPB * 32, 32 / WPB) k_decode_batched(const CodecParams *__restrict__ descs,
                                                                      const int64_t *__restrict__ brick_start,
                                                                      int32_t nboxes)
{
    extern __shared__ __align__(16) uint32_t s_dyn[];
    const int64_t w = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
    if (w >= brick_start[nboxes]) return;
    int lo = 0, hi = nboxes - 1;  // the last box whose start is <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (brick_start[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const CodecParams &p = descs[lo];
    const int64_t lb = w - brick_start[lo];
    BrickCoord c;
    c.bx = (int32_t)(lb % p.nbx);
    c.by = (int32_t)((lb / p.nbx) % p.nby);
    c.bz = (int32_t)(lb / ((int64_t)p.nbx * p.nby));
    c.b = lb;
    decode_brick<kNarrowLevelWords>(p, c, s_dyn);
}

// Decode brick c of p into p.out (and its value range into p.range), by one warp.
template <int LW>
__device__ __forceinline__ void decode_brick(const CodecParams &p, const BrickCoord &c, uint32_t *s_dyn)
{
    constexpr bool WIDE = LW >= kLevelWords;  // every width staged; the level buffers double as the float buffer
    constexpr int kWarpW = WIDE ? kDecGroup * LW : kDecGroup * LW + 512;
    float *fbw = reinterpret_cast<float *>(s_dyn + (threadIdx.x >> 5) * kWarpW + (WIDE ? 0 : kDecGroup * LW));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ly = lane & 7;

    float R[2][8];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int x = 0; x < 8; x++) R[s][x] = 0.0f;

    for (int g0 = 0; g0 < p.nlevels; g0 += kDecGroup) {
        const int ng = min(kDecGroup, p.nlevels - g0);
        // records: lane l holds level g0 + l
        uint4 myrec = make_uint4(0, 0, 0, 0);
        if (lane < ng) myrec = __ldg(p.recs[g0 + lane] + c.b);
        uint4 rec[kDecGroup];
        uint16_t eidx[kDecGroup][kExcPrefetch];
        uint32_t eval[kDecGroup][kExcPrefetch];
#pragma unroll
        for (int u = 0; u < kDecGroup; u++) {
            rec[u].x = __shfl_sync(CHR_FULL_MASK, myrec.x, u);
            rec[u].y = __shfl_sync(CHR_FULL_MASK, myrec.y, u);
            rec[u].z = __shfl_sync(CHR_FULL_MASK, myrec.z, u);
            rec[u].w = __shfl_sync(CHR_FULL_MASK, myrec.w, u);
        }
        // issue payload copies and exception loads of the whole group
#pragma unroll
        for (int u = 0; u < kDecGroup; u++) {
            if (u >= ng) break;
            const int l = g0 + u;
            const int w = min((int)(rec[u].w & 0xffu), 32);
            const int nexc = (int)(rec[u].w >> 16);
            const uint4 *src = reinterpret_cast<const uint4 *>(p.words[l] + 16ull * rec[u].x);
            uint32_t *dst = (s_dyn + warp * kWarpW) + u * LW;
            if (WIDE || w <= 8)
                for (int j = lane; j < 4 * w; j += 32) cp_async16(dst + 4 * j, src + j);
#pragma unroll
            for (int e = 0; e < kExcPrefetch; e++) {
                const int jj = lane + 32 * e;
                eidx[u][e] = 0xffffu;
                eval[u][e] = 0u;
                if (jj < nexc) {
                    eidx[u][e] = __ldg(p.exc_idx[l] + rec[u].y + jj);
                    eval[u][e] = __ldg(p.exc_val[l] + rec[u].y + jj);
                }
            }
        }
        cp_async_wait_all();
        __syncwarp();

#pragma unroll
        for (int u = 0; u < kDecGroup; u++) {
            if (u >= ng) break;
            const int l = g0 + u;
            const int w = min((int)(rec[u].w & 0xffu), 32), mode = (int)((rec[u].w >> 8) & 0xffu);
            const int nexc = (int)(rec[u].w >> 16);
            const uint32_t *buf = (WIDE || w <= 8) ? (s_dyn + warp * kWarpW) + u * LW : p.words[l] + 16ull * rec[u].x;
            uint32_t q[2][8];  // unsigned: prefix sums wrap like the encoder's int32
            switch (w) {  // (uniform across the warp) the common narrow widths with fixed offsets
                case 1: unpack_rows<1>(buf, lane, q); break;
                case 2: unpack_rows<2>(buf, lane, q); break;
                case 3: unpack_rows<3>(buf, lane, q); break;
                case 4: unpack_rows<4>(buf, lane, q); break;
                case 5: unpack_rows<5>(buf, lane, q); break;
                case 6: unpack_rows<6>(buf, lane, q); break;
                case 7: unpack_rows<7>(buf, lane, q); break;
                case 8: unpack_rows<8>(buf, lane, q); break;
                case 0:
#pragma unroll
                    for (int s = 0; s < 2; s++)
#pragma unroll
                        for (int x = 0; x < 8; x++) q[s][x] = 0u;
                    break;
                default: {
                    const uint32_t mask = width_mask(w);
#pragma unroll
                    for (int s = 0; s < 2; s++)
#pragma unroll
                        for (int x = 0; x < 8; x++) {
                            const int slot = 8 * (lane + 32 * s) + x;
                            const int pos = slot * w;
                            const int wd = pos >> 5;
                            // (from global memory, the word after a code's first is read only when
                            // the code reaches into it: the payload ends with its last code)
                            const uint32_t hi1 = (WIDE || (pos & 31) + w > 32) ? buf[wd + 1] : 0u;
                            const uint32_t z = __funnelshift_r(buf[wd], hi1, pos & 31) & mask;
                            q[s][x] = (uint32_t)unzigzag(z);
                        }
                }
            }
            if (lane == 0) q[0][0] = rec[u].z;  // anchor

            if (mode == 1) {  // inverse Lorenzo: inclusive prefix sums along x, y, z
#pragma unroll
                for (int s = 0; s < 2; s++)
#pragma unroll
                    for (int x = 1; x < 8; x++) q[s][x] += q[s][x - 1];
#pragma unroll
                for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                    for (int s = 0; s < 2; s++)
#pragma unroll
                        for (int x = 0; x < 8; x++) {
                            uint32_t t = __shfl_up_sync(CHR_FULL_MASK, q[s][x], o, 8);
                            if (ly >= o) q[s][x] += t;
                        }
#pragma unroll
                for (int o = 8; o < 32; o <<= 1)
#pragma unroll
                    for (int s = 0; s < 2; s++)
#pragma unroll
                        for (int x = 0; x < 8; x++) {
                            uint32_t t = __shfl_up_sync(CHR_FULL_MASK, q[s][x], o);
                            if (lane >= o) q[s][x] += t;
                        }
#pragma unroll
                for (int x = 0; x < 8; x++) q[1][x] += __shfl_sync(CHR_FULL_MASK, q[0][x], 24 + ly);
            }

            const float two_e = p.two_e[l];
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int x = 0; x < 8; x++) {
                    const float P = __fmul_rn(__int2float_rn((int32_t)q[s][x]), two_e);
                    R[s][x] = (l == 0) ? P : __fadd_rn(R[s][x], P);
                }

            if (nexc > 0) {  // vertices stored exactly at this level
                __syncwarp();
                float *fb = WIDE ? reinterpret_cast<float *>((s_dyn + warp * kWarpW) + u * LW) : fbw;  // (payload no longer needed)
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    const int slot = 8 * (lane + 32 * s);
                    *reinterpret_cast<float4 *>(fb + slot) = make_float4(R[s][0], R[s][1], R[s][2], R[s][3]);
                    *reinterpret_cast<float4 *>(fb + slot + 4) = make_float4(R[s][4], R[s][5], R[s][6], R[s][7]);
                }
                __syncwarp();
#pragma unroll
                for (int e = 0; e < kExcPrefetch; e++)
                    if (lane + 32 * e < nexc) fb[eidx[u][e] & 511] = __uint_as_float(eval[u][e]);
                for (int j = lane + 32 * kExcPrefetch; j < nexc; j += 32)
                    fb[__ldg(p.exc_idx[l] + rec[u].y + j) & 511] = __uint_as_float(__ldg(p.exc_val[l] + rec[u].y + j));
                __syncwarp();
#pragma unroll
                for (int s = 0; s < 2; s++) {
                    const int slot = 8 * (lane + 32 * s);
                    const float4 a = *reinterpret_cast<const float4 *>(fb + slot);
                    const float4 b = *reinterpret_cast<const float4 *>(fb + slot + 4);
                    R[s][0] = a.x; R[s][1] = a.y; R[s][2] = a.z; R[s][3] = a.w;
                    R[s][4] = b.x; R[s][5] = b.y; R[s][6] = b.z; R[s][7] = b.w;
                }
            }
        }
        __syncwarp();  // shared buffers are refilled by the next group
    }

    const int64_t x0 = (int64_t)c.bx * 8;
    if (p.range) {
        // the brick's value range over its grid vertices; NaN is never below
        // an isovalue, so it counts as +inf
        const int exg = (int)((p.nx - x0) < 8 ? (p.nx - x0) : 8);
        float mn = __int_as_float(0x7f800000), mx = -mn;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int64_t y = (int64_t)c.by * 8 + ly, z = (int64_t)c.bz * 8 + (lane >> 3) + 4 * s;
            if (y >= p.ny || z >= p.nz) continue;
#pragma unroll
            for (int x = 0; x < 8; x++) {
                const float v = isnan(R[s][x]) ? __int_as_float(0x7f800000) : R[s][x];
                if (x < exg) {
                    mn = fminf(mn, v);
                    mx = fmaxf(mx, v);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(CHR_FULL_MASK, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(CHR_FULL_MASK, mx, o));
        }
        if (lane == 0) p.range[c.b] = make_float2(mn, mx);
    }
    if (!p.out) return;
    // store the lane's two rows (the part inside the output box)
    const int64_t bx0 = x0 - p.box_org[0];
    int xlo = (int)(bx0 < 0 ? -bx0 : 0);
    int xhi = (int)((p.nx - x0) < 8 ? (p.nx - x0) : 8);
    if (bx0 + xhi > p.box_dim[0]) xhi = (int)(p.box_dim[0] - bx0);
    const bool vec = (xlo == 0) && (xhi == 8) && ((p.out_sx & 3) == 0) && ((p.out_sy & 3) == 0) &&
                     ((bx0 & 3) == 0) && ((reinterpret_cast<uintptr_t>(p.out) & 15u) == 0);
    if (vec) {  // (uniform across the warp)
        // through the warp's float buffer, so that two neighbouring
        // lanes write one row's 32 bytes (whole sectors) per store
        float *fb = WIDE ? reinterpret_cast<float *>(s_dyn + warp * kWarpW) : fbw;
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int slot = 8 * (lane + 32 * s);
            *reinterpret_cast<float4 *>(fb + slot) = make_float4(R[s][0], R[s][1], R[s][2], R[s][3]);
            *reinterpret_cast<float4 *>(fb + slot + 4) = make_float4(R[s][4], R[s][5], R[s][6], R[s][7]);
        }
        __syncwarp();
        const int half = lane & 1;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int r = (lane >> 1) + 16 * k;  // row r: y = r & 7, z = r >> 3
            const int64_t y = (int64_t)c.by * 8 + (r & 7) - p.box_org[1];
            const int64_t z = (int64_t)c.bz * 8 + (r >> 3) - p.box_org[2];
            if (y < 0 || z < 0 || y >= p.box_dim[1] || z >= p.box_dim[2]) continue;
            if (y + p.box_org[1] >= p.ny || z + p.box_org[2] >= p.nz) continue;
            __stcs(reinterpret_cast<float4 *>(p.out + bx0 + p.out_sx * y + p.out_sy * z) + half,
                   *reinterpret_cast<const float4 *>(fb + 8 * r + 4 * half));
        }
        return;
    }
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const int64_t y = (int64_t)c.by * 8 + ly - p.box_org[1];
        const int64_t z = (int64_t)c.bz * 8 + (lane >> 3) + 4 * s - p.box_org[2];
        if (y < 0 || z < 0 || y >= p.box_dim[1] || z >= p.box_dim[2]) continue;
        if (y + p.box_org[1] >= p.ny || z + p.box_org[2] >= p.nz) continue;
        float *row = p.out + bx0 + p.out_sx * y + p.out_sy * z;
        if (vec) {
            __stcs(reinterpret_cast<float4 *>(row), make_float4(R[s][0], R[s][1], R[s][2], R[s][3]));
            __stcs(reinterpret_cast<float4 *>(row + 4), make_float4(R[s][4], R[s][5], R[s][6], R[s][7]));
        } else {
#pragma unroll
            for (int x = 0; x < 8; x++)
                if (x >= xlo && x < xhi) row[x] = R[s][x];
        }
    }
}

// ---- record scans: wsum / exc_off = exclusive prefix over bricks ----------

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanChunk = kScanThreads * kScanPerThread;  // bricks per block

struct ScanArgs {
    uint4 *recs[CHR_MAX_LEVELS];
    int64_t nbricks;
    int64_t nchunks;
    uint2 *chunk;  // [nlevels][nchunks] (sum w, sum nexc) -> exclusive offsets
    uint64_t *totals;
};

__device__ __forceinline__ uint2 rec_counts(const uint4 &r) { return make_uint2(r.w & 0xffu, r.w >> 16); }

// block-wide exclusive scan of (w, nexc) pairs packed in 64 bits
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *s_warp, uint64_t &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t inc = warp_incl_scan_u64(v, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint64_t t = (lane < kScanThreads / 32) ? s_warp[lane] : 0;
        uint64_t ti = warp_incl_scan_u64(t, lane);
        if (lane < kScanThreads / 32) s_warp[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) s_warp[kScanThreads / 32] = ti;
    }
    __syncthreads();
    total = s_warp[kScanThreads / 32];
    uint64_t r = s_warp[warp] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const __grid_constant__ ScanArgs a)
{
    __shared__ uint64_t s_warp[kScanThreads / 32 + 1];
    const int l = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPerThread;
    uint64_t v = 0;
    for (int i = 0; i < kScanPerThread; i++) {
        int64_t b = base + i;
        if (b < a.nbricks) {
            uint2 c = rec_counts(a.recs[l][b]);
            v += (uint64_t)c.x | ((uint64_t)c.y << 32);
        }
    }
    uint64_t total;
    block_excl_scan(v, s_warp, total);
    if (threadIdx.x == 0) a.chunk[(int64_t)l * a.nchunks + blockIdx.x] = make_uint2((uint32_t)total, (uint32_t)(total >> 32));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const __grid_constant__ ScanArgs a)
{
    __shared__ uint64_t s_warp[kScanThreads / 32 + 1];
    const int l = blockIdx.x;
    uint2 *ch = a.chunk + (int64_t)l * a.nchunks;
    uint64_t carry_w = 0, carry_e = 0;
    for (int64_t c0 = 0; c0 < a.nchunks; c0 += kScanThreads) {
        int64_t c = c0 + threadIdx.x;
        uint2 v = (c < a.nchunks) ? ch[c] : make_uint2(0, 0);
        uint64_t packed = (uint64_t)v.x | ((uint64_t)v.y << 32);
        uint64_t total;
        uint64_t ex = block_excl_scan(packed, s_warp, total);
        if (c < a.nchunks) ch[c] = make_uint2((uint32_t)(carry_w + (ex & 0xffffffffull)), (uint32_t)(carry_e + (ex >> 32)));
        carry_w += total & 0xffffffffull;
        carry_e += total >> 32;
    }
    if (threadIdx.x == 0) {
        a.totals[2 * l] = carry_w;
        a.totals[2 * l + 1] = carry_e;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const __grid_constant__ ScanArgs a)
{
    __shared__ uint64_t s_warp[kScanThreads / 32 + 1];
    const int l = blockIdx.y;
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPerThread;
    uint4 r[kScanPerThread];
    uint64_t v = 0;
    for (int i = 0; i < kScanPerThread; i++) {
        int64_t b = base + i;
        r[i] = (b < a.nbricks) ? a.recs[l][b] : make_uint4(0, 0, 0, 0);
        uint2 c = rec_counts(r[i]);
        v += (uint64_t)c.x | ((uint64_t)c.y << 32);
    }
    uint64_t total;
    uint64_t ex = block_excl_scan(v, s_warp, total);
    const uint2 off = a.chunk[(int64_t)l * a.nchunks + blockIdx.x];
    uint32_t ws = off.x + (uint32_t)(ex & 0xffffffffull), es = off.y + (uint32_t)(ex >> 32);
    for (int i = 0; i < kScanPerThread; i++) {
        int64_t b = base + i;
        if (b < a.nbricks) {
            r[i].x = ws;
            r[i].y = es;
            a.recs[l][b] = r[i];
            uint2 c = rec_counts(r[i]);
            ws += c.x;
            es += c.y;
        }
    }
}

}  // namespace


// One thread per brick and level: the range over the vertices of the
// brick's cells (the brick, plus the first vertex plane of its +x, +y, +z
// neighbours), from the parts k_encode wrote: the brick's own range, the
// x = 0 plane of brick +x, the y = 0 plane of +y, the z = 0 plane of +z,
// the x = y = 0 line of +x+y, the x = z = 0 line of +x+z, the y = z = 0
// line of +y+z and the corner of +x+y+z.  A brick without cells (its first
// vertex on the grid's last plane) gets (+inf, -inf).
__global__ void __launch_bounds__(256) k_brick_index(const __grid_constant__ CodecParams p)
{
    const int64_t nb = (int64_t)p.nbx * p.nby * p.nbz;
    const int64_t b = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int l = blockIdx.y;
    if (b >= nb) return;
    const int32_t bx = (int32_t)(b % p.nbx), by = (int32_t)((b / p.nbx) % p.nby), bz = (int32_t)(b / ((int64_t)p.nbx * p.nby));
    float2 r = make_float2(__int_as_float(0x7f800000), __int_as_float(0xff800000));
    if ((int64_t)bx * 8 < p.nx - 1 && (int64_t)by * 8 < p.ny - 1 && (int64_t)bz * 8 < p.nz - 1) {
        const float2 *P = p.idx_part + (size_t)l * nb * kIdxParts;
        const bool ex = bx + 1 < p.nbx, ey = by + 1 < p.nby, ez = bz + 1 < p.nbz;
        const int64_t sx = 1, sy = p.nbx, sz = (int64_t)p.nbx * p.nby;
        auto add = [&](int64_t bb, int part) {
            const float2 v = P[bb * kIdxParts + part];
            r.x = fminf(r.x, v.x);
            r.y = fmaxf(r.y, v.y);
        };
        add(b, 0);
        if (ex) add(b + sx, 1);
        if (ey) add(b + sy, 2);
        if (ez) add(b + sz, 3);
        if (ex && ey) add(b + sx + sy, 4);
        if (ex && ez) add(b + sx + sz, 5);
        if (ey && ez) add(b + sy + sz, 6);
        if (ex && ey && ez) add(b + sx + sy + sz, 7);
    }
    p.index[l][b] = r;
}

cudaError_t launch_brick_index(const CodecParams &p, cudaStream_t s)
{
    const int64_t nb = (int64_t)p.nbx * p.nby * p.nbz;
    k_brick_index<<<dim3((unsigned)((nb + 255) / 256), (unsigned)p.nlevels), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_encode(const CodecParams &p, cudaStream_t s)
{
    const dim3 g((unsigned)((int64_t)((p.nbx + kEncBricks - 1) / kEncBricks) * p.nby * p.nbz));
    k_encode<true><<<g, 256, 0, s>>>(p);
    if ((p.nx & 7) || (p.ny & 7) || (p.nz & 7)) k_encode<false><<<g, 256, 0, s>>>(p);
    return cudaGetLastError();
}

uint32_t codec_bounds_word(bool reset)
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

cudaError_t launch_compact(const CodecParams &p, cudaStream_t s)
{
    const int64_t nbricks = (int64_t)p.nbx * p.nby * p.nbz;
    const int64_t per_block = (int64_t)kWarpsPerBlock * kCompactBricks;
    k_compact<<<dim3((unsigned)((nbricks + per_block - 1) / per_block), (unsigned)p.nlevels), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_decode(const CodecParams &p, cudaStream_t s)
{
    const dim3 grid((unsigned)((int64_t)((p.box_bricks[0] + kWarpsPerBlock - 1) / kWarpsPerBlock) * p.box_bricks[1] *
                               p.box_bricks[2]));
    static bool attr[kMaxDevices] = {};
    const int dev = current_device();
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, kDecodeSmem);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    k_decode<<<grid, 256, kDecodeSmem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_decode_batched(const CodecParams *d_descs, const int64_t *d_brick_start, int32_t nboxes,
                                  int64_t total_bricks, int warps_per_block, cudaStream_t s)
{
    static bool attr[kMaxDevices] = {};
    const int dev = current_device();
    if (!attr[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_decode_batched<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             8 * (kDecGroup * kNarrowLevelWords + 512) * 4);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_decode_batched<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * (kDecGroup * kNarrowLevelWords + 512) * 4);
        if (e != cudaSuccess) return e;
        attr[dev] = true;
    }
    if (total_bricks == 0) return cudaSuccess;
    if (warps_per_block == 4) {
        const unsigned grid = (unsigned)((total_bricks + 3) / 4);
        k_decode_batched<4><<<grid, 128, 4 * (kDecGroup * kNarrowLevelWords + 512) * 4, s>>>(d_descs, d_brick_start, nboxes);
    } else {
        const unsigned grid = (unsigned)((total_bricks + 7) / 8);
        k_decode_batched<8><<<grid, 256, 8 * (kDecGroup * kNarrowLevelWords + 512) * 4, s>>>(d_descs, d_brick_start, nboxes);
    }
    return cudaGetLastError();
}

size_t scan_scratch_bytes(int64_t nbricks, int nlevels)
{
    int64_t nchunks = (nbricks + kScanChunk - 1) / kScanChunk;
    return (size_t)nchunks * nlevels * sizeof(uint2) + 256;
}

cudaError_t launch_scan_records(uint4 *const *recs, int nlevels, int64_t nbricks, void *scratch, uint64_t *totals,
                                cudaStream_t s)
{
    ScanArgs a;
    for (int l = 0; l < CHR_MAX_LEVELS; l++) a.recs[l] = (l < nlevels) ? recs[l] : nullptr;
    a.nbricks = nbricks;
    a.nchunks = (nbricks + kScanChunk - 1) / kScanChunk;
    a.chunk = reinterpret_cast<uint2 *>(scratch);
    a.totals = totals;
    dim3 g((unsigned)a.nchunks, (unsigned)nlevels);
    k_scan_reduce<<<g, kScanThreads, 0, s>>>(a);
    k_scan_chunks<<<nlevels, kScanThreads, 0, s>>>(a);
    k_scan_apply<<<g, kScanThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace chr

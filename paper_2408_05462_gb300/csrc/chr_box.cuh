// Decoding a marching-cubes tile's vertex box straight from a CHR level
// (paper Sec. 2: the visualization side reconstructs the requested level
// and generates the isosurface from it).  Used by the one-pass
// decode + marching-cubes kernel in mc.cu: the reconstructed field never
// goes to memory.
//
// A tile is 4 cell bricks along x (32x8x8 cells); its cells touch the
// vertices [x0, x0+32] x [y0, y0+8] x [z0, z0+8]: its 4 own vertex bricks
// in full, plus the first vertex plane of the bricks after them along x, y
// and z (and the lines and the corner where those meet).  A code is the
// 3-D inclusive prefix sum (within its brick) of the brick's Lorenzo
// residuals, or the residual itself in plain mode, so on a brick's first
// plane along one axis it is a 2-D prefix sum of that plane's residuals,
// and on a first line a 1-D one: the halo costs a prefix over 2 of the 3
// axes (or 1) of the slots it needs, each read at its own bit offset.
// Every value is computed with exactly the decoder's integer and float
// operations (codec.cu: k_decode), so the box holds the bits
// chr_reconstruct would write.
//
// The 20 bricks a tile reads are numbered id = dx + 5*(dy + 2*dz) for the
// brick at (bx0 + dx, by + dy, bz + dz), dx in 0..4, dy, dz in 0..1; their
// records of every level are read into shared memory (s_rec[l][id]) before
// the tile is decoded, so the decoding warps start with the payloads.
//
// The box: float [9][9][VX] (z, y, x), the tile's vertex (x0 + x, y0 + y,
// z0 + z) at x + VX*y + PLANE*z; vertices outside the grid are 0.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace chr {

namespace {

// Where the decoder reads level l of a CHR (device pointers), for levels
// 0..nlevels-1.
struct ChrLevels {
    const uint4 *recs[CHR_MAX_LEVELS];
    const uint32_t *words[CHR_MAX_LEVELS];
    const uint16_t *exc_idx[CHR_MAX_LEVELS];
    const uint32_t *exc_val[CHR_MAX_LEVELS];
    float two_e[CHR_MAX_LEVELS];
    int32_t nlevels;
    int32_t nbx, nby, nbz;
};

constexpr int kTileBricks = 20;  // bricks whose records a tile reads

// A magnitude from which a tile takes the IEEE quotient path (2^124: two
// such values differ by at most 2^125 < 2^126, where the fast quotient
// is exact to 2 ulp).
constexpr float kHugeValue = 2.1267647932558654e37f;

// The records of every level of the tile's 20 bricks into s_rec, by one
// warp (zero records for bricks outside the grid).
__device__ __forceinline__ void load_tile_records(uint4 (*s_rec)[kTileBricks], const ChrLevels &L, int32_t bx0,
                                                  int32_t by, int32_t bz, int lane)
{
    for (int e = lane; e < kTileBricks * L.nlevels; e += 32) {
        const int l = e / kTileBricks, id = e - l * kTileBricks;
        const int dx = id % 5, dy = (id / 5) & 1, dz = id / 10;
        const int32_t x = bx0 + dx, y = by + dy, z = bz + dz;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        if (x < L.nbx && y < L.nby && z < L.nbz) r = __ldg(L.recs[l] + x + (int64_t)L.nbx * (y + (int64_t)L.nby * z));
        s_rec[l][id] = r;
    }
}

__device__ __forceinline__ void cp_async16_box(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all_box() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The 8 codes of packed row L of a brick (slots 8L..8L+7) at width W from
// its words (shared staging or global memory: reads run up to 2 words past
// the row, inside the staging slack or the payload array's 64-byte tail).
template <int W>
__device__ __forceinline__ void unpack_row_any(const uint32_t *wp, int L, uint32_t (&q)[8])
{
    const uint32_t bit0 = 8u * W * (uint32_t)L;
    const uint32_t wd = bit0 >> 5, off = bit0 & 31u;
    const uint32_t a = wp[wd], b = wp[wd + 1];
    uint64_t win = __funnelshift_r(a, b, off);
    if (W > 4) win |= (uint64_t)__funnelshift_r(b, wp[wd + 2], off) << 32;
#pragma unroll
    for (int x = 0; x < 8; x++) q[x] = (uint32_t)unzigzag((uint32_t)(win >> (W * x)) & ((1u << W) - 1u));
}

template <int W>
__device__ __forceinline__ void unpack_rows_any(const uint32_t *wp, int lane, uint32_t (&q)[2][8])
{
    unpack_row_any<W>(wp, lane, q[0]);
    unpack_row_any<W>(wp, lane + 32, q[1]);
}

constexpr int kOwnGroup = 3;      // levels of an own brick whose loads are issued together
constexpr int kStageSlack = 4;    // staging words after each level's payload (read-ahead of the unpack)

// One whole brick (slot id of s_rec) by one warp into the box columns
// col0..col0+7 (rows y, z = 0..7): lane holds rows (y, z) = (lane&7,
// lane>>3) and z + 4.  For each group of kOwnGroup levels, every load is
// issued before any is consumed: the payload words into the warp's staging
// area (cp.async; a level that does not fit is read from global memory)
// and the first 32 exception entries into registers.  Returns whether some
// value has magnitude >= kHugeValue.
template <int VX, int PLANE>
__device__ __forceinline__ bool box_own_brick(float *box, const ChrLevels &L, const uint4 (*s_rec)[kTileBricks], int id,
                                              int col0, int lane, uint32_t *stage, int stage_words)
{
    const int ly = lane & 7, lz = lane >> 3;
    float R[2][8];
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int x = 0; x < 8; x++) R[s][x] = 0.0f;
    float *row0 = box + col0 + VX * ly + PLANE * lz;
    float *row1 = row0 + 4 * PLANE;
    bool inbox = false;  // R is in the box (the last level had exceptions)
    for (int g0 = 0; g0 < L.nlevels; g0 += kOwnGroup) {
        const int ng = min(kOwnGroup, L.nlevels - g0);
        int soff[kOwnGroup];
        uint32_t eidx[kOwnGroup], eval[kOwnGroup];
        int off = 0;
#pragma unroll
        for (int u = 0; u < kOwnGroup; u++) {
            soff[u] = -1;
            eidx[u] = 0xffffffffu;
            eval[u] = 0u;
            if (u >= ng) continue;
            const int l = g0 + u;
            const uint4 rec = s_rec[l][id];
            const int w = min((int)(rec.w & 0xffu), 32), nexc = (int)(rec.w >> 16);
            if (off + 16 * w + kStageSlack <= stage_words) {
                const uint4 *src = reinterpret_cast<const uint4 *>(L.words[l] + 16ull * rec.x);
                for (int j = lane; j < 4 * w; j += 32) cp_async16_box(stage + off + 4 * j, src + j);
                soff[u] = off;
                off += 16 * w + kStageSlack;
            }
            if (lane < nexc) {
                eidx[u] = __ldg(L.exc_idx[l] + rec.y + lane);
                eval[u] = __ldg(L.exc_val[l] + rec.y + lane);
            }
        }
        cp_async_wait_all_box();
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kOwnGroup; u++) {
            if (u >= ng) break;
            const int l = g0 + u;
            const uint4 rec = s_rec[l][id];
            const int w = min((int)(rec.w & 0xffu), 32), mode = (int)((rec.w >> 8) & 0xffu);
            const int nexc = (int)(rec.w >> 16);
            const uint32_t *wp = (soff[u] >= 0) ? stage + soff[u] : L.words[l] + 16ull * rec.x;
            uint32_t q[2][8];
            switch (w) {
                case 1: unpack_rows_any<1>(wp, lane, q); break;
                case 2: unpack_rows_any<2>(wp, lane, q); break;
                case 3: unpack_rows_any<3>(wp, lane, q); break;
                case 4: unpack_rows_any<4>(wp, lane, q); break;
                case 5: unpack_rows_any<5>(wp, lane, q); break;
                case 6: unpack_rows_any<6>(wp, lane, q); break;
                case 7: unpack_rows_any<7>(wp, lane, q); break;
                case 8: unpack_rows_any<8>(wp, lane, q); break;
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
                            const uint32_t pos = (uint32_t)(8 * (lane + 32 * s) + x) * (uint32_t)w;
                            const uint32_t wd = pos >> 5;
                            q[s][x] = (uint32_t)unzigzag(__funnelshift_r(wp[wd], wp[wd + 1], pos & 31u) & mask);
                        }
                }
            }
            if (lane == 0) q[0][0] = rec.z;  // anchor
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
                            const uint32_t t = __shfl_up_sync(CHR_FULL_MASK, q[s][x], o, 8);
                            if (ly >= o) q[s][x] += t;
                        }
#pragma unroll
                for (int o = 8; o < 32; o <<= 1)
#pragma unroll
                    for (int s = 0; s < 2; s++)
#pragma unroll
                        for (int x = 0; x < 8; x++) {
                            const uint32_t t = __shfl_up_sync(CHR_FULL_MASK, q[s][x], o);
                            if (lane >= o) q[s][x] += t;
                        }
#pragma unroll
                for (int x = 0; x < 8; x++) q[1][x] += __shfl_sync(CHR_FULL_MASK, q[0][x], 24 + ly);
            }
            const float two_e = L.two_e[l];
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int x = 0; x < 8; x++) {
                    const float P = __fmul_rn(__int2float_rn((int32_t)q[s][x]), two_e);
                    R[s][x] = (l == 0) ? P : __fadd_rn(R[s][x], P);
                }
            inbox = nexc > 0;
            if (inbox) {  // vertices stored exactly at this level: through the box
                *reinterpret_cast<float4 *>(row0) = make_float4(R[0][0], R[0][1], R[0][2], R[0][3]);
                *reinterpret_cast<float4 *>(row0 + 4) = make_float4(R[0][4], R[0][5], R[0][6], R[0][7]);
                *reinterpret_cast<float4 *>(row1) = make_float4(R[1][0], R[1][1], R[1][2], R[1][3]);
                *reinterpret_cast<float4 *>(row1 + 4) = make_float4(R[1][4], R[1][5], R[1][6], R[1][7]);
                __syncwarp();
                if (eidx[u] != 0xffffffffu) {
                    const uint32_t s = eidx[u] & 511u;
                    box[col0 + (s & 7u) + VX * ((s >> 3) & 7u) + PLANE * (s >> 6)] = __uint_as_float(eval[u]);
                }
                for (int e = lane + 32; e < nexc; e += 32) {
                    const uint32_t s = __ldg(L.exc_idx[l] + rec.y + e) & 511u;
                    box[col0 + (s & 7u) + VX * ((s >> 3) & 7u) + PLANE * (s >> 6)] =
                        __uint_as_float(__ldg(L.exc_val[l] + rec.y + e));
                }
                __syncwarp();
                const float4 a0 = *reinterpret_cast<const float4 *>(row0), b0 = *reinterpret_cast<const float4 *>(row0 + 4);
                const float4 a1 = *reinterpret_cast<const float4 *>(row1), b1 = *reinterpret_cast<const float4 *>(row1 + 4);
                R[0][0] = a0.x; R[0][1] = a0.y; R[0][2] = a0.z; R[0][3] = a0.w;
                R[0][4] = b0.x; R[0][5] = b0.y; R[0][6] = b0.z; R[0][7] = b0.w;
                R[1][0] = a1.x; R[1][1] = a1.y; R[1][2] = a1.z; R[1][3] = a1.w;
                R[1][4] = b1.x; R[1][5] = b1.y; R[1][6] = b1.z; R[1][7] = b1.w;
            }
        }
        __syncwarp();  // the staging area is refilled by the next group
    }
    if (!inbox) {
        *reinterpret_cast<float4 *>(row0) = make_float4(R[0][0], R[0][1], R[0][2], R[0][3]);
        *reinterpret_cast<float4 *>(row0 + 4) = make_float4(R[0][4], R[0][5], R[0][6], R[0][7]);
        *reinterpret_cast<float4 *>(row1) = make_float4(R[1][0], R[1][1], R[1][2], R[1][3]);
        *reinterpret_cast<float4 *>(row1 + 4) = make_float4(R[1][4], R[1][5], R[1][6], R[1][7]);
    }
    bool huge = false;
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int x = 0; x < 8; x++) huge |= fabsf(R[s][x]) >= kHugeValue;
    return huge;
}

// One halo piece per group of lanes: a brick's first plane along one axis
// (PLANE: all 32 lanes, lane (a, c) = (lane & 7, lane >> 3) holding the
// plane's rows c and c + 4), or up to four first lines (lanes 8g..8g+7 =
// positions 0..7 of line g).  id: the brick's slot in s_rec (-1: outside
// the grid, the positions get 0).  axa / axb: the brick axes (0 x, 1 y,
// 2 z) that a and the row index run along; the others are 0.  base, da,
// db: box index of position (0, 0) and its steps along a and along the
// rows.  len: the group's positions along a (1 for the corner).
struct HaloPiece {
    int id;
    int axa, axb;
    int base, da, db, len;
};

constexpr int kHaloGroup = 4;  // levels of a halo piece whose loads are issued together

template <bool PLANE, int VX, int PLANE_STRIDE>
__device__ __forceinline__ bool box_halo(float *box, const ChrLevels &L, const uint4 (*s_rec)[kTileBricks],
                                         const HaloPiece &hp, int lane)
{
    constexpr int GS = PLANE ? 32 : 8;  // lanes per group (one brick)
    const int a = lane & 7, c = PLANE ? (lane >> 3) : 0, gi = PLANE ? lane : a;
    const bool live = hp.id >= 0 && a < hp.len;
    const int sa = 1 << (3 * hp.axa), sb = PLANE ? (1 << (3 * hp.axb)) : 0;
    const int slot0 = a * sa + c * sb, slot1 = slot0 + 4 * sb;
    const int pos0 = hp.base + a * hp.da + c * hp.db, pos1 = pos0 + 4 * hp.db;
    // an exception entry of this group's brick lies on the piece when the
    // fixed axes are 0; its box index
    auto on_piece = [&](uint32_t s, int &pos) -> bool {
        const int cx = (int)(s & 7u), cy = (int)((s >> 3) & 7u), cz = (int)(s >> 6);
        const int ea = (hp.axa == 0) ? cx : (hp.axa == 1) ? cy : cz;
        const int eb = PLANE ? ((hp.axb == 0) ? cx : (hp.axb == 1) ? cy : cz) : 0;
        pos = hp.base + ea * hp.da + eb * hp.db;
        return (cx + cy + cz - ea - eb) == 0 && ea < hp.len;
    };
    float R0 = 0.0f, R1 = 0.0f;
    for (int g0 = 0; g0 < L.nlevels; g0 += kHaloGroup) {
        // every load of the group first: code words and the first GS exception entries
        uint32_t w00[kHaloGroup], w01[kHaloGroup], w10[kHaloGroup], w11[kHaloGroup];
        uint32_t eidx[kHaloGroup], eval[kHaloGroup];
#pragma unroll
        for (int u = 0; u < kHaloGroup; u++) {
            w00[u] = w01[u] = w10[u] = w11[u] = 0u;
            eidx[u] = 0xffffffffu;
            eval[u] = 0u;
            const int l = g0 + u;
            if (l >= L.nlevels || hp.id < 0) continue;
            const uint4 rec = s_rec[l][hp.id];
            const uint32_t w = min(rec.w & 0xffu, 32u), nexc = rec.w >> 16;
            const uint32_t *wp = L.words[l] + 16ull * rec.x;
            if (live && w > 0) {
                const uint32_t p0 = (uint32_t)slot0 * w >> 5;
                w00[u] = __ldg(wp + p0);
                w01[u] = __ldg(wp + p0 + 1);
                if (PLANE) {
                    const uint32_t p1 = (uint32_t)slot1 * w >> 5;
                    w10[u] = __ldg(wp + p1);
                    w11[u] = __ldg(wp + p1 + 1);
                }
            }
            if ((uint32_t)gi < nexc) {
                eidx[u] = __ldg(L.exc_idx[l] + rec.y + gi);
                eval[u] = __ldg(L.exc_val[l] + rec.y + gi);
            }
        }
#pragma unroll
        for (int u = 0; u < kHaloGroup; u++) {
            const int l = g0 + u;
            if (l >= L.nlevels) break;
            uint4 rec = make_uint4(0u, 0u, 0u, 0u);
            if (hp.id >= 0) rec = s_rec[l][hp.id];
            const uint32_t w = min(rec.w & 0xffu, 32u), mode = (rec.w >> 8) & 0xffu;
            const uint32_t mask = width_mask((int)w);
            uint32_t q0 = 0u, q1 = 0u;
            if (live && w > 0) {
                q0 = (uint32_t)unzigzag(__funnelshift_r(w00[u], w01[u], ((uint32_t)slot0 * w) & 31u) & mask);
                if (PLANE) q1 = (uint32_t)unzigzag(__funnelshift_r(w10[u], w11[u], ((uint32_t)slot1 * w) & 31u) & mask);
            }
            if (slot0 == 0) q0 = rec.z;  // anchor
            {  // Lorenzo: prefix along a, then (planes) along the rows; every
               // lane shuffles (the groups of a line task may differ in mode)
                uint32_t p0 = q0, p1 = q1;
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    const uint32_t t0 = __shfl_up_sync(CHR_FULL_MASK, p0, o, 8);
                    const uint32_t t1 = PLANE ? __shfl_up_sync(CHR_FULL_MASK, p1, o, 8) : 0u;
                    if (a >= o) {
                        p0 += t0;
                        p1 += t1;
                    }
                }
                if (PLANE) {
#pragma unroll
                    for (int o = 8; o < 32; o <<= 1) {
                        const uint32_t t0 = __shfl_up_sync(CHR_FULL_MASK, p0, o);
                        const uint32_t t1 = __shfl_up_sync(CHR_FULL_MASK, p1, o);
                        if (lane >= o) {
                            p0 += t0;
                            p1 += t1;
                        }
                    }
                    p1 += __shfl_sync(CHR_FULL_MASK, p0, 24 + a);
                }
                if (mode == 1) {
                    q0 = p0;
                    q1 = p1;
                }
            }
            const float two_e = L.two_e[l];
            const float P0 = __fmul_rn(__int2float_rn((int32_t)q0), two_e);
            const float P1 = __fmul_rn(__int2float_rn((int32_t)q1), two_e);
            if (live) {
                R0 = (l == 0) ? P0 : __fadd_rn(box[pos0], P0);
                box[pos0] = R0;
                if (PLANE) {
                    R1 = (l == 0) ? P1 : __fadd_rn(box[pos1], P1);
                    box[pos1] = R1;
                }
            }
            // vertices of the piece stored exactly at this level
            const uint32_t nexc = (hp.id >= 0) ? (rec.w >> 16) : 0u;
            if (__any_sync(CHR_FULL_MASK, nexc > 0)) {
                __syncwarp();
                int pos;
                if (eidx[u] != 0xffffffffu && on_piece(eidx[u] & 511u, pos)) box[pos] = __uint_as_float(eval[u]);
                for (uint32_t e = (uint32_t)gi + GS; e < nexc; e += GS) {  // past the first GS entries
                    const uint32_t s = __ldg(L.exc_idx[l] + rec.y + e) & 511u;
                    if (on_piece(s, pos)) box[pos] = __uint_as_float(__ldg(L.exc_val[l] + rec.y + e));
                }
                __syncwarp();
                if (live) {
                    R0 = box[pos0];
                    if (PLANE) R1 = box[pos1];
                }
            }
        }
    }
    if (hp.id < 0 && a < hp.len) {  // outside the grid
        box[pos0] = 0.0f;
        if (PLANE) box[pos1] = 0.0f;
    }
    return live && (fabsf(R0) >= kHugeValue || (PLANE && fabsf(R1) >= kHugeValue));
}

}  // namespace

}  // namespace chr

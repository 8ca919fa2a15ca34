/*
 * CPU oracle for topology-preserving compression and marching cubes
 * (Li & Chen, "Accelerating In-transit Isosurface Generation With Topology
 * Preserving Compression", arXiv 2408.05462).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU baseline leg
 * of the benchmark do.  It shares no code, header or table with the CUDA
 * path.  Every loop is written in the order the method is described, with no
 * blocking or fusion, so that a reader can check it against the text.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -frounding-math -fPIC -shared.
 * fp32 arithmetic is plain C float arithmetic with FLT_EVAL_METHOD == 0 and
 * no contraction into FMA, so every float operation below is one IEEE-754
 * binary32 operation rounded to nearest-even (except sub_down, which rounds
 * toward -inf on purpose).
 *
 * What each function follows:
 *   orc_encode        paper Sec. 2 (CHR: error-bounded levels, "desired ...
 *                     accuracy") and Sec. 2.2 (topology preservation: the
 *                     same marching-cubes case in every cell).  The codec
 *                     itself (residual level chain, 8^3 bricks, Lorenzo
 *                     prediction, zig-zag bit packing) is this library's
 *                     reading: the paper names prediction-based compressors
 *                     of the SZ family (Sec. 1) but defines no format.
 *   orc_decode        inverse of orc_encode (Sec. 2, reconstruction on the
 *                     visualization side).
 *   orc_cell_triangles / orc_mc
 *                     marching cubes (Sec. 2.2, Lorensen & Cline), written
 *                     without a case table: every cell is triangulated on the
 *                     fly by walking its six faces.
 *   orc_translate_D / orc_translate_eb
 *                     Sec. 2.2, error-bound translation: the array D of the
 *                     distances d0, d1 from the isovalue to both ends of every
 *                     edge with s0 < k < s1, and its smallest (or n-th
 *                     smallest) element.
 *   orc_cases         the marching-cubes case byte of every cell (Sec. 2.2:
 *                     topology preservation keeps these bytes).
 *   orc_brick_index   Sec. 2.1, the CHR's index over its blocks for the
 *                     candidate isovalues ("isovalue based data pruning"):
 *                     per 8^3 brick the value range over the vertices of
 *                     its cells.
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BRICK 8
#define ORC_SLOTS 512
#define ORC_QMAX 8388607.0f /* 2^23 - 1: |q| stays exact in a float */

/* ------------------------------------------------------------------ */
/* Grid helpers                                                        */
/* ------------------------------------------------------------------ */

static int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

int64_t orc_nbricks(int64_t nx, int64_t ny, int64_t nz)
{
    return cdiv64(nx, ORC_BRICK) * cdiv64(ny, ORC_BRICK) * cdiv64(nz, ORC_BRICK);
}

/* ------------------------------------------------------------------ */
/* Codec: one level of the error-bounded residual chain (Sec. 2)       */
/* ------------------------------------------------------------------ */

/*
 * Level `lvl` of one vertex.  r is the residual left by the previous level
 * (the value itself at level 0); it is quantised with step 2e, the
 * reconstruction R is checked strictly against the bound (|f - R| < e), and
 * with the topology fix on, against every candidate isovalue k: the inside
 * bit (v < k) of R must equal that of f (Sec. 2.2).  A vertex that fails any
 * check becomes an exception: R takes f exactly, and the code keeps the
 * rounded value when there is one (0 when r cannot be quantised), so the
 * prediction of its neighbours is not disturbed.
 * Returns 1 for an exception.
 */
static int level_step(float f, float Rprev, int lvl, float e, float two_e, float inv2e,
                      const float *K, int nK, int fix, int32_t *q_out, float *R_out)
{
    int exc = 0;
    int32_t q = 0;
    float R = 0.0f;
    float r = (lvl == 0) ? f : (f - Rprev);
    float x = r * inv2e;
    if (!(fabsf(x) <= ORC_QMAX)) {
        exc = 1; /* also NaN and Inf */
    } else {
        q = (int32_t)rintf(x); /* round half to even */
        float P = (float)q * two_e;
        R = (lvl == 0) ? P : (Rprev + P);
        float err = f - R;
        if (!(fabsf(err) < e)) {
            exc = 1;
        } else if (fix) {
            for (int j = 0; j < nK; j++) {
                if ((R < K[j]) != (f < K[j])) {
                    exc = 1;
                    break;
                }
            }
        }
    }
    if (exc) R = f; /* q stays the rounded code, or 0 if r was not quantisable */
    *q_out = q;
    *R_out = R;
    return exc;
}

/* zig-zag map of a signed code to an unsigned one: 0,-1,1,-2,... -> 0,1,2,3 */
static uint32_t zigzag(int64_t d) { return (uint32_t)(d >= 0 ? 2 * d : -2 * d - 1); }

static int32_t unzigzag(uint32_t z) { return (z & 1u) ? -(int32_t)(z >> 1) - 1 : (int32_t)(z >> 1); }

static int bit_length(uint32_t v)
{
    int n = 0;
    while (v) {
        n++;
        v >>= 1;
    }
    return n;
}

/*
 * Brick geometry.  Brick (bx,by,bz) holds vertices 8b..8b+7 along each axis;
 * slot s = lx + 8*ly + 64*lz.  Slots past the grid edge are padding.
 */
typedef struct {
    int64_t nx, ny, nz;
    int64_t nbx, nby, nbz;
} grid_t;

static grid_t make_grid(int64_t nx, int64_t ny, int64_t nz)
{
    grid_t g = {nx, ny, nz, cdiv64(nx, ORC_BRICK), cdiv64(ny, ORC_BRICK), cdiv64(nz, ORC_BRICK)};
    return g;
}

/* global vertex index of slot s of brick b, or -1 for padding */
static int64_t slot_vertex(const grid_t *g, int64_t b, int s)
{
    int64_t bx = b % g->nbx, by = (b / g->nbx) % g->nby, bz = b / (g->nbx * g->nby);
    int64_t x = bx * ORC_BRICK + (s & 7), y = by * ORC_BRICK + ((s >> 3) & 7), z = bz * ORC_BRICK + (s >> 6);
    if (x >= g->nx || y >= g->ny || z >= g->nz) return -1;
    return x + g->nx * (y + g->ny * z);
}

/*
 * 3-D Lorenzo prediction residual of slot (lx,ly,lz) of one brick, with the
 * codes outside the brick taken as zero:
 *   d = q(x,y,z) - q(x-1,y,z) - q(x,y-1,z) - q(x,y,z-1)
 *       + q(x-1,y-1,z) + q(x-1,y,z-1) + q(x,y-1,z-1) - q(x-1,y-1,z-1).
 */
static int64_t lorenzo_residual(const int32_t *qb, int lx, int ly, int lz)
{
    int64_t acc = 0;
    for (int dz = 0; dz <= 1; dz++)
        for (int dy = 0; dy <= 1; dy++)
            for (int dx = 0; dx <= 1; dx++) {
                int x = lx - dx, y = ly - dy, z = lz - dz;
                if (x < 0 || y < 0 || z < 0) continue;
                int sign = ((dx + dy + dz) & 1) ? -1 : 1;
                acc += sign * (int64_t)qb[x + 8 * y + 64 * z];
            }
    return acc;
}

/*
 * Encode an nx*ny*nz float field (x fastest) into `nlevels` levels.
 *
 * Inputs: eb[l] the absolute bound of level l (finite, > 0, non-increasing),
 * K[0..nK) the candidate isovalues, fix = 1 for the per-vertex topology fix.
 * Per level l, per brick b (bricks in x-fastest order) the outputs are
 *   recs[(l*nb + b)*4 + 0] = sum of the widths w of bricks before b
 *                            (the brick's payload starts at word 16*that)
 *   recs[...+1] = exceptions of this level in bricks before b
 *   recs[...+2] = anchor: the code at local (0,0,0), as int32 bits
 *   recs[...+3] = w | mode << 8 | nexc << 16
 *   words  + l*nb*512 : the level's packed stream, 16*w words per brick
 *   exc_idx/exc_val + l*N : the exceptions (slot, exact value bits) in
 *                            brick order then slot order
 *   Rout + l*N : the level's reconstruction as the decoder will produce it
 *   nwords[l], nexc[l] : totals.
 * Mode 1 (Lorenzo) stores d = q - prediction; mode 0 stores q itself; the
 * brick takes the mode with the smaller w, mode 0 on a tie.  Slot 0 always
 * packs 0 (its code is the anchor); padding slots pack 0.  Slot s packs its
 * zig-zag code in bits [s*w, s*w + w) of the little-endian word stream.
 * Returns 0, or -1 for bad arguments.
 */
int orc_encode(const float *f, int64_t nx, int64_t ny, int64_t nz, int nlevels, const float *eb, const float *K,
               int nK, int fix, uint32_t *recs, uint32_t *words, uint16_t *exc_idx, uint32_t *exc_val, float *Rout,
               int64_t *nwords, int64_t *nexc)
{
    if (nx < 1 || ny < 1 || nz < 1 || nlevels < 1) return -1;
    grid_t g = make_grid(nx, ny, nz);
    int64_t N = nx * ny * nz, nb = g.nbx * g.nby * g.nbz;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *isexc = (uint8_t *)malloc((size_t)N);
    if (!q || !isexc) {
        free(q);
        free(isexc);
        return -1;
    }
    for (int l = 0; l < nlevels; l++) {
        float e = eb[l];
        float two_e = 2.0f * e;
        float inv2e = 1.0f / two_e;
        float *R = Rout + (int64_t)l * N;
        const float *Rprev = (l == 0) ? NULL : Rout + (int64_t)(l - 1) * N;

        /* quantise every vertex, check it, fix its sign (Sec. 2, Sec. 2.2) */
        for (int64_t i = 0; i < N; i++)
            isexc[i] = (uint8_t)level_step(f[i], Rprev ? Rprev[i] : 0.0f, l, e, two_e, inv2e, K, nK, fix, &q[i], &R[i]);

        /* predict, zig-zag, size and pack every brick */
        uint32_t *W = words + (int64_t)l * nb * ORC_SLOTS;
        uint16_t *EI = exc_idx + (int64_t)l * N;
        uint32_t *EV = exc_val + (int64_t)l * N;
        int64_t wsum = 0, esum = 0;
        for (int64_t b = 0; b < nb; b++) {
            int32_t qb[ORC_SLOTS];
            int inside[ORC_SLOTS];
            for (int s = 0; s < ORC_SLOTS; s++) {
                int64_t v = slot_vertex(&g, b, s);
                inside[s] = (v >= 0);
                qb[s] = (v >= 0) ? q[v] : 0;
            }
            uint32_t zl[ORC_SLOTS], zn[ORC_SLOTS];
            uint32_t maxl = 0, maxn = 0;
            for (int s = 0; s < ORC_SLOTS; s++) {
                int64_t dl = 0, dn = 0;
                if (inside[s] && s != 0) {
                    dl = lorenzo_residual(qb, s & 7, (s >> 3) & 7, s >> 6);
                    dn = qb[s];
                }
                zl[s] = zigzag(dl);
                zn[s] = zigzag(dn);
                if (zl[s] > maxl) maxl = zl[s];
                if (zn[s] > maxn) maxn = zn[s];
            }
            int wl = bit_length(maxl), wn = bit_length(maxn);
            int mode = (wl < wn) ? 1 : 0;
            int w = mode ? wl : wn;
            const uint32_t *z = mode ? zl : zn;
            /* pack */
            uint32_t *P = W + 16 * wsum;
            for (int j = 0; j < 16 * w; j++) P[j] = 0;
            for (int s = 0; s < ORC_SLOTS; s++) {
                for (int bit = 0; bit < w; bit++) {
                    if ((z[s] >> bit) & 1u) {
                        int64_t pos = (int64_t)s * w + bit;
                        P[pos >> 5] |= 1u << (pos & 31);
                    }
                }
            }
            /* exceptions of this brick, slot order */
            int ne = 0;
            for (int s = 0; s < ORC_SLOTS; s++) {
                int64_t v = slot_vertex(&g, b, s);
                if (v >= 0 && isexc[v]) {
                    uint32_t bits;
                    memcpy(&bits, &f[v], 4);
                    EI[esum + ne] = (uint16_t)s;
                    EV[esum + ne] = bits;
                    ne++;
                }
            }
            uint32_t *rec = recs + ((int64_t)l * nb + b) * 4;
            rec[0] = (uint32_t)wsum;
            rec[1] = (uint32_t)esum;
            rec[2] = (uint32_t)qb[0];
            rec[3] = (uint32_t)w | ((uint32_t)mode << 8) | ((uint32_t)ne << 16);
            wsum += w;
            esum += ne;
        }
        nwords[l] = 16 * wsum;
        nexc[l] = esum;
    }
    free(q);
    free(isexc);
    return 0;
}

/*
 * Decode level `level` (0-based) of an encoded field into out[N]: for levels
 * 0..level in turn, unpack each brick, undo the prediction with inclusive
 * prefix sums along x, then y, then z (the exact inverse of the Lorenzo
 * residual above), add code*2e to the running reconstruction and overwrite
 * the level's exceptions with their exact values.
 * recs as from orc_encode; words_cat/exc_*_cat hold the levels back to back,
 * starting at word_base[l] / exc_base[l].
 */
int orc_decode(const uint32_t *recs, const uint32_t *words_cat, const int64_t *word_base, const uint16_t *exc_idx_cat,
               const uint32_t *exc_val_cat, const int64_t *exc_base, int64_t nx, int64_t ny, int64_t nz,
               const float *eb, int level, float *out)
{
    grid_t g = make_grid(nx, ny, nz);
    int64_t nb = g.nbx * g.nby * g.nbz;
    for (int l = 0; l <= level; l++) {
        float two_e = 2.0f * eb[l];
        const uint32_t *W = words_cat + word_base[l];
        const uint16_t *EI = exc_idx_cat + exc_base[l];
        const uint32_t *EV = exc_val_cat + exc_base[l];
        for (int64_t b = 0; b < nb; b++) {
            const uint32_t *rec = recs + ((int64_t)l * nb + b) * 4;
            int w = (int)(rec[3] & 0xff), mode = (int)((rec[3] >> 8) & 0xff), ne = (int)(rec[3] >> 16);
            const uint32_t *P = W + 16 * (int64_t)rec[0];
            uint32_t qb[ORC_SLOTS]; /* unsigned: prefix sums wrap like int32 */
            for (int s = 0; s < ORC_SLOTS; s++) {
                uint32_t z = 0;
                for (int bit = 0; bit < w; bit++) {
                    int64_t pos = (int64_t)s * w + bit;
                    z |= ((P[pos >> 5] >> (pos & 31)) & 1u) << bit;
                }
                qb[s] = (uint32_t)unzigzag(z);
            }
            qb[0] = rec[2];
            if (mode == 1) {
                for (int s = 0; s < ORC_SLOTS; s++) /* along x */
                    if ((s & 7) > 0) qb[s] += qb[s - 1];
                for (int s = 0; s < ORC_SLOTS; s++) /* along y */
                    if (((s >> 3) & 7) > 0) qb[s] += qb[s - 8];
                for (int s = 0; s < ORC_SLOTS; s++) /* along z */
                    if ((s >> 6) > 0) qb[s] += qb[s - 64];
            }
            for (int s = 0; s < ORC_SLOTS; s++) {
                int64_t v = slot_vertex(&g, b, s);
                if (v < 0) continue;
                float P2 = (float)(int32_t)qb[s] * two_e;
                out[v] = (l == 0) ? P2 : (out[v] + P2);
            }
            for (int j = 0; j < ne; j++) {
                int64_t v = slot_vertex(&g, b, EI[rec[1] + j]);
                uint32_t bits = EV[rec[1] + j];
                memcpy(&out[v], &bits, 4);
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Marching cubes without a table (Sec. 2.2; Lorensen & Cline)         */
/* ------------------------------------------------------------------ */

/*
 * Corner j of a cell sits at offset (j&1, j>>1&1, j>>2&1).  Edge numbers:
 * axis*4 + m, where m holds the offsets along the two other axes, the lower
 * axis in bit 0.  An edge runs from its corner with offset 0 along its axis
 * to the corner with offset 1.
 */
static int corner_off(int j, int axis) { return (j >> axis) & 1; }

static int edge_between(int ca, int cb)
{
    int diff = ca ^ cb;
    int axis = (diff == 1) ? 0 : (diff == 2) ? 1 : 2;
    int others[2], n = 0;
    for (int a = 0; a < 3; a++)
        if (a != axis) others[n++] = a;
    return axis * 4 + corner_off(ca, others[0]) + 2 * corner_off(ca, others[1]);
}

/*
 * Triangles of one cell with inside-bit pattern `caseb` (bit j = corner j is
 * inside, i.e. its value is below the isovalue).  Face rule: walking each
 * face's four corners counter-clockwise as seen from outside the cell, every
 * maximal run of inside corners gives one segment, from the crossing point on
 * the edge where the walk enters the run to the one where it leaves it.  The
 * inside corners then lie to the right of the segment, and a face with two
 * diagonal inside corners keeps them apart.  Each crossing point leaves one
 * segment and ends one; following them gives closed cycles.  Cycles are taken
 * in order of their smallest edge number and listed from it.  Each cycle is
 * fanned from its apex: the first vertex in that listing none of whose
 * diagonals joins two points on a common face of the cell (a diagonal on a
 * face could be drawn by the neighbouring cell too, and four triangles would
 * then meet at one edge).  Triangles (apex, v_i, v_i+1) follow the cycle.
 * edges[3*t .. 3*t+2] receives triangle t.  Returns the number of triangles,
 * or -1 if some cycle has no such apex (no case has one).
 */
static int edges_share_face(int ea, int eb)
{
    int fa[2][2], fb[2][2];
    int *src[2] = {&ea, &eb};
    for (int k = 0; k < 2; k++) {
        int e = *src[k], axis = e >> 2, m = e & 3, n = 0;
        int(*fs)[2] = k ? fb : fa;
        for (int a = 0; a < 3; a++) {
            if (a == axis) continue;
            fs[n][0] = a;
            fs[n][1] = (n == 0) ? (m & 1) : ((m >> 1) & 1);
            n++;
        }
    }
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++)
            if (fa[i][0] == fb[j][0] && fa[i][1] == fb[j][1]) return 1;
    return 0;
}

int orc_cell_triangles(int caseb, int8_t *edges)
{
    int next[12];
    for (int e = 0; e < 12; e++) next[e] = -1;
    for (int axis = 0; axis < 3; axis++) {
        int u = (axis + 1) % 3, v = (axis + 2) % 3;
        for (int side = 0; side < 2; side++) {
            /* counter-clockwise seen from outside: (u,v) = 00,10,11,01 on the
               +axis face; the reverse turn on the -axis face */
            static const int ccw_pos[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
            static const int ccw_neg[4][2] = {{0, 0}, {0, 1}, {1, 1}, {1, 0}};
            int c[4], in[4];
            for (int i = 0; i < 4; i++) {
                const int *p = side ? ccw_pos[i] : ccw_neg[i];
                c[i] = (side << axis) | (p[0] << u) | (p[1] << v);
                in[i] = (caseb >> c[i]) & 1;
            }
            for (int i = 0; i < 4; i++) {
                if (!in[i] || in[(i + 3) % 4]) continue; /* not the first corner of a run */
                int j = i;
                while (in[(j + 1) % 4]) j = (j + 1) % 4;
                int enter = edge_between(c[(i + 3) % 4], c[i]);
                int leave = edge_between(c[j], c[(j + 1) % 4]);
                next[enter] = leave;
            }
        }
    }
    int visited[12] = {0};
    int ntri = 0;
    for (int start = 0; start < 12; start++) {
        if (next[start] < 0 || visited[start]) continue;
        int cyc[12], len = 0;
        int e = start;
        do {
            visited[e] = 1;
            cyc[len++] = e;
            e = next[e];
        } while (e != start && len < 12);
        int apex = -1;
        for (int i = 0; i < len && apex < 0; i++) {
            int ok = 1;
            for (int j = 0; j < len; j++) {
                if (j == i || j == (i + 1) % len || j == (i + len - 1) % len) continue;
                if (edges_share_face(cyc[i], cyc[j])) ok = 0;
            }
            if (ok) apex = i;
        }
        if (apex < 0) return -1;
        for (int i = 1; i + 1 < len; i++) {
            edges[3 * ntri + 0] = (int8_t)cyc[apex];
            edges[3 * ntri + 1] = (int8_t)cyc[(apex + i) % len];
            edges[3 * ntri + 2] = (int8_t)cyc[(apex + i + 1) % len];
            ntri++;
        }
    }
    return ntri;
}

/*
 * Marching cubes over the whole grid for isovalue k.  Inside bit of a vertex:
 * v < k (NaN is outside).  Cells in ascending index x + (nx-1)*(y + (ny-1)*z);
 * triangles of a cell in orc_cell_triangles order.  A vertex on edge (v0,v1)
 * sits at v0 + t*(v1 - v0), t = (k - f0)/(f1 - f0), computed in double from
 * the float values (the exact point, up to double rounding).
 * Outputs (each may be NULL): pos[T*9] (x,y,z of the three corners in grid
 * units), cell[T], edge_id[T*3] = 3*index(v0) + axis.  At most cap triangles
 * are written; the return value is the full count.
 */
int64_t orc_mc(const float *f, int64_t nx, int64_t ny, int64_t nz, float k, double *pos, int64_t *cell,
               int64_t *edge_id, int64_t cap)
{
    int64_t T = 0;
    if (nx < 2 || ny < 2 || nz < 2) return 0;
    for (int64_t z = 0; z + 1 < nz; z++)
        for (int64_t y = 0; y + 1 < ny; y++)
            for (int64_t x = 0; x + 1 < nx; x++) {
                int caseb = 0;
                for (int j = 0; j < 8; j++) {
                    int64_t v = (x + corner_off(j, 0)) + nx * ((y + corner_off(j, 1)) + ny * (z + corner_off(j, 2)));
                    if (f[v] < k) caseb |= 1 << j;
                }
                if (caseb == 0 || caseb == 255) continue;
                int8_t edges[36];
                int nt = orc_cell_triangles(caseb, edges);
                if (nt < 0) return -1;
                for (int t = 0; t < nt; t++, T++) {
                    if (T >= cap) continue;
                    if (cell) cell[T] = x + (nx - 1) * (y + (ny - 1) * z);
                    for (int c = 0; c < 3; c++) {
                        int e = edges[3 * t + c];
                        int axis = e >> 2, m = e & 3;
                        int o[3] = {0, 0, 0};
                        int others[2], n = 0;
                        for (int a = 0; a < 3; a++)
                            if (a != axis) others[n++] = a;
                        o[others[0]] = m & 1;
                        o[others[1]] = (m >> 1) & 1;
                        int64_t p0[3] = {x + o[0], y + o[1], z + o[2]};
                        int64_t i0 = p0[0] + nx * (p0[1] + ny * p0[2]);
                        int64_t step = (axis == 0) ? 1 : (axis == 1) ? nx : nx * ny;
                        double f0 = f[i0], f1 = f[i0 + step];
                        double tt = ((double)k - f0) / (f1 - f0);
                        if (pos) {
                            for (int a = 0; a < 3; a++) pos[T * 9 + c * 3 + a] = (double)p0[a];
                            pos[T * 9 + c * 3 + axis] += tt;
                        }
                        if (edge_id) edge_id[T * 3 + c] = 3 * i0 + axis;
                    }
                }
            }
    return T;
}

/* ------------------------------------------------------------------ */
/* Error-bound translation (Sec. 2.2)                                  */
/* ------------------------------------------------------------------ */

/* a - b rounded toward -inf, so that the float never exceeds the true gap */
static float sub_down(float a, float b)
{
    int old = fegetround();
    fesetround(FE_DOWNWARD);
    volatile float va = a, vb = b;
    volatile float d = va - vb;
    fesetround(old);
    return d;
}

/*
 * The array D of Sec. 2.2: for every grid edge (x-, y- and z-neighbours) and
 * every candidate isovalue k with s0 < k < s1 (s0 the smaller end), both
 * d0 = k - s0 and d1 = s1 - k.  Order: vertex index, then axis, then k,
 * d0 before d1.  At most cap values are written; returns |D|.
 */
int64_t orc_translate_D(const float *f, int64_t nx, int64_t ny, int64_t nz, const float *K, int nK, float *D,
                        int64_t cap)
{
    int64_t n = 0;
    for (int64_t z = 0; z < nz; z++)
        for (int64_t y = 0; y < ny; y++)
            for (int64_t x = 0; x < nx; x++) {
                int64_t i = x + nx * (y + ny * z);
                int64_t nbr[3] = {x + 1 < nx ? i + 1 : -1, y + 1 < ny ? i + nx : -1, z + 1 < nz ? i + nx * ny : -1};
                for (int a = 0; a < 3; a++) {
                    if (nbr[a] < 0) continue;
                    float s0 = f[i], s1 = f[nbr[a]];
                    if (s1 < s0) {
                        float t = s0;
                        s0 = s1;
                        s1 = t;
                    }
                    for (int j = 0; j < nK; j++) {
                        float k = K[j];
                        if (s0 < k && k < s1) {
                            if (n < cap) D[n] = sub_down(k, s0);
                            n++;
                            if (n < cap) D[n] = sub_down(s1, k);
                            n++;
                        }
                    }
                }
            }
    return n;
}

static int cmp_float(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/*
 * The translated bound: the element of rank n = floor((1 - accuracy) * |D|)
 * (0-based, ascending) of D, clamped to the last element; accuracy 1 gives
 * min D.  An empty D gives +inf (no edge crosses any isovalue).
 * count_out receives |D|.
 */
float orc_translate_eb(const float *f, int64_t nx, int64_t ny, int64_t nz, const float *K, int nK, float accuracy,
                       int64_t *count_out)
{
    int64_t n = orc_translate_D(f, nx, ny, nz, K, nK, NULL, 0);
    if (count_out) *count_out = n;
    if (n == 0) return INFINITY;
    float *D = (float *)malloc(sizeof(float) * (size_t)n);
    if (!D) return NAN;
    orc_translate_D(f, nx, ny, nz, K, nK, D, n);
    qsort(D, (size_t)n, sizeof(float), cmp_float);
    double r = floor((1.0 - (double)accuracy) * (double)n);
    int64_t rank = (r < 0) ? 0 : (int64_t)r;
    if (rank > n - 1) rank = n - 1;
    float eb = D[rank];
    free(D);
    return eb;
}

/* ------------------------------------------------------------------ */
/* Adjoints (reading of the paper: attributing isosurface error to the */
/* grid points, Sec. 2.2 error translation run backwards)              */
/* ------------------------------------------------------------------ */

/*
 * Adjoint of orc_mc's vertex positions with respect to the field.  A vertex
 * on edge (i0, i1) along `axis` sits at p_axis = x0 + t, t = (k-f0)/(f1-f0),
 * so dp_axis/df0 = (t-1)/(f1-f0) and dp_axis/df1 = -t/(f1-f0); the other two
 * coordinates do not depend on the field.  grad_pos[T*9] holds dL/dp in the
 * order orc_mc emits; grad_field[N] receives dL/df (overwritten).
 * Returns the number of triangles, or -1.
 */
int64_t orc_mc_backward(const float *f, int64_t nx, int64_t ny, int64_t nz, float k, const double *grad_pos,
                        double *grad_field)
{
    int64_t N = nx * ny * nz, T = 0;
    for (int64_t i = 0; i < N; i++) grad_field[i] = 0.0;
    if (nx < 2 || ny < 2 || nz < 2) return 0;
    for (int64_t z = 0; z + 1 < nz; z++)
        for (int64_t y = 0; y + 1 < ny; y++)
            for (int64_t x = 0; x + 1 < nx; x++) {
                int caseb = 0;
                for (int j = 0; j < 8; j++) {
                    int64_t v = (x + corner_off(j, 0)) + nx * ((y + corner_off(j, 1)) + ny * (z + corner_off(j, 2)));
                    if (f[v] < k) caseb |= 1 << j;
                }
                if (caseb == 0 || caseb == 255) continue;
                int8_t edges[36];
                int nt = orc_cell_triangles(caseb, edges);
                if (nt < 0) return -1;
                for (int t = 0; t < nt; t++, T++) {
                    for (int c = 0; c < 3; c++) {
                        int e = edges[3 * t + c];
                        int axis = e >> 2, m = e & 3;
                        int o[3] = {0, 0, 0};
                        int others[2], n = 0;
                        for (int a = 0; a < 3; a++)
                            if (a != axis) others[n++] = a;
                        o[others[0]] = m & 1;
                        o[others[1]] = (m >> 1) & 1;
                        int64_t i0 = (x + o[0]) + nx * ((y + o[1]) + ny * (z + o[2]));
                        int64_t step = (axis == 0) ? 1 : (axis == 1) ? nx : nx * ny;
                        double f0 = f[i0], f1 = f[i0 + step];
                        double tt = ((double)k - f0) / (f1 - f0);
                        double g = grad_pos[T * 9 + c * 3 + axis];
                        grad_field[i0] += g * (tt - 1.0) / (f1 - f0);
                        grad_field[i0 + step] += g * (-tt) / (f1 - f0);
                    }
                }
            }
    return T;
}

/*
 * Mean first-order distance of points to the isosurface of an original
 * field: for each point p, |F(p) - k| / |grad F(p)|, F the trilinear
 * interpolant of f in the cell with lower corner clamp(floor(p), 0, n-2)
 * (grid units); points where grad F vanishes count as distance 0.  Returns
 * the mean over the npts points; grad_pts (may be NULL) receives
 * d(mean)/dp = (1/npts) [ s G/|G| - |F-k| H G / |G|^3 ], s = sign(F-k),
 * G = grad F, H = the Hessian of F (trilinear: only mixed second
 * derivatives are non-zero).
 */
double orc_dist_loss(const float *f, int64_t nx, int64_t ny, int64_t nz, float k, const double *pts, int64_t npts,
                     double *grad_pts)
{
    double sum = 0.0;
    const int64_t n[3] = {nx, ny, nz};
    for (int64_t v = 0; v < npts; v++) {
        const double *p = pts + 3 * v;
        int64_t c[3];
        double u[3];
        for (int a = 0; a < 3; a++) {
            double fl = floor(p[a]);
            if (fl < 0) fl = 0;
            if (fl > (double)(n[a] - 2)) fl = (double)(n[a] - 2);
            c[a] = (int64_t)fl;
            u[a] = p[a] - fl;
        }
        double val[2][2][2]; /* [dz][dy][dx] */
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < 2; dy++)
                for (int dx = 0; dx < 2; dx++)
                    val[dz][dy][dx] = f[(c[0] + dx) + nx * ((c[1] + dy) + ny * (c[2] + dz))];
        double w[3][2];
        for (int a = 0; a < 3; a++) {
            w[a][0] = 1.0 - u[a];
            w[a][1] = u[a];
        }
        double F = 0, G[3] = {0, 0, 0}, H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < 2; dy++)
                for (int dx = 0; dx < 2; dx++) {
                    double fv = val[dz][dy][dx];
                    double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
                    F += w[0][dx] * w[1][dy] * w[2][dz] * fv;
                    G[0] += sx * w[1][dy] * w[2][dz] * fv;
                    G[1] += w[0][dx] * sy * w[2][dz] * fv;
                    G[2] += w[0][dx] * w[1][dy] * sz * fv;
                    H[0][1] += sx * sy * w[2][dz] * fv;
                    H[0][2] += sx * w[1][dy] * sz * fv;
                    H[1][2] += w[0][dx] * sy * sz * fv;
                }
        H[1][0] = H[0][1];
        H[2][0] = H[0][2];
        H[2][1] = H[1][2];
        double gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
        double r = F - (double)k;
        if (gn == 0.0) {
            if (grad_pts)
                for (int a = 0; a < 3; a++) grad_pts[3 * v + a] = 0.0;
            continue;
        }
        sum += fabs(r) / gn;
        if (grad_pts) {
            double s = (r > 0) ? 1.0 : (r < 0) ? -1.0 : 0.0;
            for (int a = 0; a < 3; a++) {
                double hg = H[a][0] * G[0] + H[a][1] * G[1] + H[a][2] * G[2];
                grad_pts[3 * v + a] = (s * G[a] / gn - fabs(r) * hg / (gn * gn * gn)) / (double)npts;
            }
        }
    }
    return npts ? sum / (double)npts : 0.0;
}

/* ------------------------------------------------------------------ */
/* Case bytes and the per-brick index (Sec. 2.1, Sec. 2.2)             */
/* ------------------------------------------------------------------ */

/*
 * Case byte of every cell for isovalue k: bit j set when corner j (offset
 * (j&1, j>>1&1, j>>2&1)) is inside, v < k (NaN is outside).  cases[c] for
 * cell c = x + (nx-1)*(y + (ny-1)*z).  A cell is active (carries triangles)
 * when its byte is neither 0 nor 255.
 */
void orc_cases(const float *f, int64_t nx, int64_t ny, int64_t nz, float k, uint8_t *cases)
{
    if (nx < 2 || ny < 2 || nz < 2) return;
    for (int64_t z = 0; z + 1 < nz; z++)
        for (int64_t y = 0; y + 1 < ny; y++)
            for (int64_t x = 0; x + 1 < nx; x++) {
                int caseb = 0;
                for (int j = 0; j < 8; j++) {
                    int64_t v = (x + corner_off(j, 0)) + nx * ((y + corner_off(j, 1)) + ny * (z + corner_off(j, 2)));
                    if (f[v] < k) caseb |= 1 << j;
                }
                cases[x + (nx - 1) * (y + (ny - 1) * z)] = (uint8_t)caseb;
            }
}

/*
 * Per-brick value index of a field.  Brick b = bx + nbx*(by + nby*bz)
 * (nbx = ceil(nx/8), ...) owns the cells whose lower corner lies in it,
 * x in [8bx, min(8bx+8, nx-1)) and likewise along y and z; those cells
 * touch the vertices x in [8bx, min(8bx+8, nx-1)] (the brick and the first
 * vertex plane of its +x, +y and +z neighbours).  lo[b], hi[b]: the
 * smallest and largest value over those vertices, NaN counted as +inf, a
 * zero stored as +0 (-0 and +0 are the same value).  A
 * brick without cells gets lo = +inf, hi = -inf.  A cell of brick b is
 * active for k only if one corner has v < k and another v >= k (or NaN),
 * hence only if lo[b] < k <= hi[b].
 */
void orc_brick_index(const float *f, int64_t nx, int64_t ny, int64_t nz, float *lo, float *hi)
{
    const int64_t nbx = cdiv64(nx, ORC_BRICK), nby = cdiv64(ny, ORC_BRICK), nbz = cdiv64(nz, ORC_BRICK);
    for (int64_t bz = 0; bz < nbz; bz++)
        for (int64_t by = 0; by < nby; by++)
            for (int64_t bx = 0; bx < nbx; bx++) {
                const int64_t b = bx + nbx * (by + nby * bz);
                float mn = INFINITY, mx = -INFINITY;
                const int64_t x0 = 8 * bx, y0 = 8 * by, z0 = 8 * bz;
                if (x0 < nx - 1 && y0 < ny - 1 && z0 < nz - 1) {
                    const int64_t x1 = (x0 + 8 < nx - 1) ? x0 + 8 : nx - 1;
                    const int64_t y1 = (y0 + 8 < ny - 1) ? y0 + 8 : ny - 1;
                    const int64_t z1 = (z0 + 8 < nz - 1) ? z0 + 8 : nz - 1;
                    for (int64_t z = z0; z <= z1; z++)
                        for (int64_t y = y0; y <= y1; y++)
                            for (int64_t x = x0; x <= x1; x++) {
                                float v = f[x + nx * (y + ny * z)];
                                if (isnan(v)) v = INFINITY;
                                v = v + 0.0f; /* -0 and +0 are one value: +0 stands for both */
                                if (v < mn) mn = v;
                                if (v > mx) mx = v;
                            }
                }
                lo[b] = mn;
                hi[b] = mx;
            }
}

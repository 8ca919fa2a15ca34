"""Pins for the oracle's case bytes and per-brick value index (paper Sec. 2.1,
the CHR's index for isovalue-based pruning; Sec. 2.2, the cases that
topology preservation keeps).

Checks from outside the oracle: single cells with hand-set corners, the
triangle count of mc() as the sum over cells of the cases' triangle counts,
the complement symmetry of the inside test, bricks worked by hand at the
grid's edges, and on tiny random grids (with NaN, infinities and vertices
equal to k) a brute force over cells: every active cell lies in a brick
whose range straddles k, and each bound equals the extreme over the corners
of the brick's cells."""
import numpy as np
import pytest

import oracle


def _corner_grid(inside_corners, k=0.0, nan_corners=(), equal_corners=()):
    """2x2x2 grid, [z, y, x]; corner j at (j&1, j>>1&1, j>>2&1)."""
    f = np.full((2, 2, 2), 1.0, np.float32)
    for j in inside_corners:
        f[j >> 2 & 1, j >> 1 & 1, j & 1] = -1.0
    for j in nan_corners:
        f[j >> 2 & 1, j >> 1 & 1, j & 1] = np.nan
    for j in equal_corners:
        f[j >> 2 & 1, j >> 1 & 1, j & 1] = k
    return f


@pytest.mark.parametrize("corners,byte", [((), 0), ((0,), 1), ((1,), 2), ((2,), 4), ((4,), 16), ((6,), 64),
                                          ((7,), 128), ((1, 2, 4), 2 + 4 + 16), (tuple(range(8)), 255)])
def test_cases_single_cell_by_hand(corners, byte):
    assert int(oracle.cases(_corner_grid(corners), 0.0)[0, 0, 0]) == byte


def test_cases_nan_and_equal_are_outside():
    # corner 3 NaN, corner 5 equal to k: both outside; corner 0 inside
    f = _corner_grid((0,), nan_corners=(3,), equal_corners=(5,))
    assert int(oracle.cases(f, 0.0)[0, 0, 0]) == 1


def test_cases_layout_and_triangle_count():
    rng = np.random.default_rng(7)
    f = rng.standard_normal((6, 7, 9)).astype(np.float32)
    c = oracle.cases(f, 0.25)
    assert c.shape == (5, 6, 8)
    # cell (x, y, z) = (3, 2, 1): its byte from the corners read off the grid by hand
    x, y, z = 3, 2, 1
    want = 0
    for j in range(8):
        if f[z + (j >> 2 & 1), y + (j >> 1 & 1), x + (j & 1)] < 0.25:
            want |= 1 << j
    assert int(c[z, y, x]) == want
    ntri = np.array([len(oracle.cell_triangles(b)) for b in range(256)])
    assert int(ntri[c].sum()) == oracle.mc_count(f, 0.25)


def test_cases_complement():
    rng = np.random.default_rng(8)
    f = rng.standard_normal((5, 6, 7)).astype(np.float32)
    k = np.float32(0.1)
    # no vertex equals k, so every corner is inside exactly once
    assert not (f == k).any()
    assert np.array_equal(oracle.cases(f, k) ^ oracle.cases(-f, -k), np.full((4, 5, 6), 255, np.uint8))


def test_index_hand_worked_spikes():
    # 10^3 grid: bricks 0 and 1 along each axis; brick 0 has cells 0..7 and
    # touches vertices 0..8, brick 1 has cell 8 and touches vertices 8..9
    f = np.zeros((10, 10, 10), np.float32)
    f[7, 7, 7] = 5.0    # only brick (0,0,0) touches it
    f[8, 8, 8] = 6.0    # every brick touches it
    f[9, 9, 9] = -4.0   # only brick (1,1,1)
    f[0, 0, 9] = -2.0   # x = 9: bricks with bx = 1, by = bz = 0
    lo, hi = oracle.brick_index(f)
    assert lo.shape == (2, 2, 2)
    want_hi = np.full((2, 2, 2), 6.0, np.float32)
    want_hi[0, 0, 0] = 6.0
    want_lo = np.zeros((2, 2, 2), np.float32)
    want_lo[1, 1, 1] = -4.0
    want_lo[0, 0, 1] = -2.0
    assert np.array_equal(hi, want_hi)
    assert np.array_equal(lo, want_lo)
    f[8, 8, 8] = 0.0
    lo, hi = oracle.brick_index(f)
    assert hi[0, 0, 0] == 5.0 and hi[1, 1, 1] == 0.0 and hi[0, 1, 0] == 0.0


def test_index_nan_and_cellless_brick():
    # nx = 9: brick 1 along x holds the vertex column x = 8 only, no cell
    f = np.zeros((9, 9, 9), np.float32)
    f[3, 4, 8] = np.nan
    lo, hi = oracle.brick_index(f)
    assert lo.shape == (2, 2, 2)
    assert lo[0, 0, 0] == 0.0 and hi[0, 0, 0] == np.inf  # NaN counts as +inf
    for b in [(0, 0, 1), (0, 1, 0), (1, 0, 0), (1, 1, 1)]:
        assert lo[b] == np.inf and hi[b] == -np.inf


def _brute_index(f):
    """Extremes over the 8 corners of every cell, grouped by the cell's brick."""
    nz, ny, nx = f.shape
    nbx, nby, nbz = -(-nx // 8), -(-ny // 8), -(-nz // 8)
    lo = np.full((nbz, nby, nbx), np.inf, np.float32)
    hi = np.full((nbz, nby, nbx), -np.inf, np.float32)
    g = np.where(np.isnan(f), np.float32(np.inf), f)
    for z in range(nz - 1):
        for y in range(ny - 1):
            for x in range(nx - 1):
                c = g[z:z + 2, y:y + 2, x:x + 2]
                b = (z // 8, y // 8, x // 8)
                lo[b] = min(lo[b], c.min())
                hi[b] = max(hi[b], c.max())
    return lo, hi


@pytest.mark.parametrize("shape,seed", [((9, 10, 17), 1), ((17, 9, 12), 2), ((8, 18, 9), 3)])
def test_index_brute_force(shape, seed):
    rng = np.random.default_rng(seed)
    f = rng.integers(-3, 4, size=shape).astype(np.float32)
    flat = f.reshape(-1)
    flat[rng.choice(flat.size, 5, replace=False)] = np.nan
    flat[rng.choice(flat.size, 2, replace=False)] = np.inf
    flat[rng.choice(flat.size, 2, replace=False)] = -np.inf
    lo, hi = oracle.brick_index(f)
    blo, bhi = _brute_index(f)
    assert np.array_equal(lo, blo) and np.array_equal(hi, bhi)
    # no active cell outside the bricks whose range straddles k (k equal to vertex values too)
    for k in (-2.0, -0.5, 0.0, 1.0, 3.0):
        c = oracle.cases(f, k)
        active = (c != 0) & (c != 255)
        z, y, x = np.nonzero(active)
        straddle = (lo < k) & (k <= hi)
        assert straddle[z // 8, y // 8, x // 8].all()


def test_index_zero_is_positive_zero():
    # bricks whose extreme is a zero store +0 whichever zero the grid holds
    f = np.ones((9, 9, 9), np.float32)
    f[2, 2, 2] = -0.0
    lo, hi = oracle.brick_index(-f * 0.0)  # every vertex -0
    assert np.all(lo[0, 0, 0].view(np.uint32) == 0) and np.all(hi[0, 0, 0].view(np.uint32) == 0)
    lo, hi = oracle.brick_index(f)
    assert lo[0, 0, 0].view(np.uint32) == 0 and hi[0, 0, 0] == 1.0

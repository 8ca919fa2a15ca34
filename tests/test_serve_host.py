"""Host-side logic of the request loop: the brick-index dilation, the
triangle bound of a box against brute force over a field, and the request
generator.  No GPU."""
import numpy as np
import pytest

from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, serve, synth


@pytest.fixture(scope="module", autouse=True)
def _lib():
    chr_build.build()  # the native bound lives in libchr; nvcc builds it without a GPU


def _range_index(f):
    """Per-brick (min, max) of f[z, y, x] with NaN as +inf: what
    chr_brick_range computes, written out with numpy."""
    nz, ny, nx = f.shape
    nb = [(s + 7) // 8 for s in (nz, ny, nx)]
    g = np.where(np.isnan(f), np.inf, f).astype(np.float32)
    out = np.zeros(nb + [2], np.float32)
    for bz in range(nb[0]):
        for by in range(nb[1]):
            for bx in range(nb[2]):
                blk = g[8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
                out[bz, by, bx] = (blk.min(), blk.max())
    return out


def _active_cells(f, k):
    """Cells (lower corner z, y, x) with a corner below k and one not below."""
    below = f < k
    c = [below[dz:dz + f.shape[0] - 1, dy:dy + f.shape[1] - 1, dx:dx + f.shape[2] - 1]
         for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)]
    anyb = np.logical_or.reduce(c)
    allb = np.logical_and.reduce(c)
    return anyb & ~allb


def _timestep(f):
    return serve.Timestep(0, None, f.shape, [serve.dilate_range(_range_index(f))], 0)


def _bound_reference(mn, mx, origin, size, k):
    """The bound written out with numpy: 5 x the box's cells in bricks whose
    widened range straddles k."""
    total = 0
    per_axis = []
    for a, nb in zip(range(3), (mn.shape[2], mn.shape[1], mn.shape[0])):
        o, n = origin[a], size[a]
        cells = np.zeros(nb, np.int64)
        for c in range(o, o + n - 1):
            cells[c // 8] += 1
        per_axis.append(cells)
    act = (mn < np.float32(k)) & (mx >= np.float32(k))
    total = np.einsum("zyx,z,y,x->", act.astype(np.int64), per_axis[2], per_axis[1], per_axis[0])
    return 5 * int(total)


def test_native_bound_equals_the_reference():
    g = np.random.Generator(np.random.PCG64(4))
    for shape in [(5, 7, 9), (1, 1, 1), (3, 1, 4)]:
        mid = g.normal(size=shape).astype(np.float32)
        mn, mx = (mid - 0.4).astype(np.float32), (mid + 0.4).astype(np.float32)
        nbz, nby, nbx = shape
        for _ in range(50):
            size = tuple(int(g.integers(2, 8 * s + 1)) for s in (nbx, nby, nbz))
            org = tuple(int(g.integers(0, 8 * s - b + 1)) for s, b in zip((nbx, nby, nbz), size))
            k = float(g.uniform(-1.5, 1.5))
            assert chr.chr_box_tri_bound(mn, mx, org, size, k) == _bound_reference(mn, mx, org, size, k)
    assert chr.chr_box_tri_bound(mn, mx, (0, 0, 0), (1, 4, 4), 0.0) == 0


def test_tri_bound_covers_every_active_cell():
    f = synth.turbulence((45, 38, 29), seed=21)
    nz, ny, nx = f.shape
    ts = _timestep(f)
    g = np.random.Generator(np.random.PCG64(3))
    for _ in range(40):
        k = float(g.uniform(-1.5, 1.5))
        size = tuple(int(g.integers(2, s + 1)) for s in (nx, ny, nz))
        org = tuple(int(g.integers(0, s - b + 1)) for s, b in zip((nx, ny, nz), size))
        box = f[org[2]:org[2] + size[2], org[1]:org[1] + size[1], org[0]:org[0] + size[0]]
        active = int(_active_cells(box, np.float32(k)).sum())
        bound = ts.tri_bound(0, k, org, size)
        assert bound >= 5 * active
        assert bound <= 5 * (size[0] - 1) * (size[1] - 1) * (size[2] - 1)


def test_tri_bound_is_zero_away_from_the_range():
    f = synth.gaussian_blobs(40, seed=8)
    ts = _timestep(f)
    assert ts.tri_bound(0, float(f.max()) + 1.0, (0, 0, 0), (40, 40, 40)) == 0
    assert ts.tri_bound(0, float(f.min()) - 1.0, (3, 4, 5), (30, 20, 10)) == 0
    # the plane z = 12.5 lies in brick layer 1 (vertices 8..15); layer 0's
    # range is widened by all of layer 1, so the cells of layers 0 and 1 count
    # and those of layers 2 and 3 do not
    p = synth.plane_field((32, 32, 32), (0, 0, 1), 12.5)
    tp = _timestep(p)
    assert tp.tri_bound(0, 0.0, (0, 0, 0), (32, 32, 32)) == 5 * 31 * 31 * 16
    assert tp.tri_bound(0, 0.0, (0, 0, 16), (32, 32, 16)) == 0


def test_nan_counts_as_not_below():
    f = np.zeros((16, 16, 16), np.float32)
    f[4, 4, 4] = np.nan
    ts = _timestep(f)
    # every vertex is >= -1 or NaN: nothing is below, nothing is active
    assert ts.tri_bound(0, -1.0, (0, 0, 0), (16, 16, 16)) == 0
    # below 0.5 everywhere but at the NaN: the cells around it may be active
    assert ts.tri_bound(0, 0.5, (0, 0, 0), (16, 16, 16)) > 0


def test_make_requests_is_seeded_and_in_bounds():
    a = serve.make_requests(50, 100.0, (300, 200, 100), [0, 1], seed=5)
    b = serve.make_requests(50, 100.0, (300, 200, 100), [0, 1], seed=5)
    assert a == b
    t = [r.arrival for r in a]
    assert all(x < y for x, y in zip(t, t[1:]))
    for r in a:
        assert -1.0 <= r.k <= 1.0 and 0 <= r.level < 4 and r.step in (0, 1)
        for o, s, n in zip(r.origin, r.size, (300, 200, 100)):
            assert 64 <= s <= 512 or s == n
            assert 0 <= o and o + s <= n
    burst = serve.make_requests(10, 0.0, (100, 100, 100), [0])
    assert all(r.arrival == 0.0 for r in burst)


def test_free_list_first_fit_and_merge():
    fl = serve.FreeList(4096)
    a = fl.alloc(100)
    b = fl.alloc(1000)
    c = fl.alloc(256)
    assert a == (0, 256) and b == (256, 1024) and c == (1280, 256)
    assert fl.alloc(4096) is None
    fl.release(*b)
    assert fl.alloc(2000) == (1536, 2048)       # the freed hole is too small; first fit goes past it
    assert fl.alloc(512) == (256, 512)          # the hole is used from its start
    fl.release(*a)
    assert fl.free == [(0, 256), (768, 512), (3584, 512)]
    fl.release(256, 512)                        # merges with both neighbours
    assert fl.free == [(0, 1280), (3584, 512)]
    fl.release(1280, 256)
    assert fl.free == [(0, 1536), (3584, 512)]
    fl.release(1536, 2048)
    assert fl.free == [(0, 4096)]
    g = np.random.Generator(np.random.PCG64(1))
    fl = serve.FreeList(1 << 20)
    live = []
    for _ in range(2000):
        if live and g.uniform() < 0.5:
            fl.release(*live.pop(int(g.integers(0, len(live)))))
        else:
            blk = fl.alloc(int(g.integers(1, 40000)))
            if blk is not None:
                live.append(blk)
        spans = sorted(live + fl.free)
        assert sum(n for _, n in spans) == fl.size
        assert all(o1 + n1 == o2 for (o1, n1), (o2, _) in zip(spans, spans[1:]))  # no overlap, no gap
    for blk in live:
        fl.release(*blk)
    assert fl.free == [(0, fl.size)]

"""Pins for the oracle's error-bound translation (paper Sec. 2.2: D holds
d0 = k - s0 and d1 = s1 - k for every edge with s0 < k < s1; its smallest
element, or its n-th smallest to tolerate some wrong cells, is the bound).

Checks: closed-form ramps whose D has known values and multiplicities,
downward rounding of a gap that float32 cannot hold, the sign property the
paper argues for, the counter-example where min D does not protect a
vertex that is on no crossing edge, hand-worked NaN and infinite ends and a
repeated isovalue, and D enumerated by brute force from exact rational gaps
on tiny grids (rounding to nearest instead of down would change about a
quarter of its elements)."""
import numpy as np
import pytest

import oracle
from paper_2408_05462_gb300 import synth


def _ramp(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float32)


def test_ramp_closed_form():
    nx, ny, nz = 7, 5, 3
    f = _ramp(nx, ny, nz)  # f = x; only x-edges between x=2 and x=3 straddle 2.25
    D = oracle.translate_D(f, [2.25])
    m = ny * nz
    assert D.size == 2 * m
    assert sorted(D.tolist()) == [0.25] * m + [0.75] * m
    assert oracle.translate_eb(f, [2.25], 1.0) == (0.25, 2 * m)
    # rank floor(0.5 * 2m) = m is the first 0.75
    assert oracle.translate_eb(f, [2.25], 0.5)[0] == 0.75
    # rank floor(0.25 * 2m) < m is still 0.25
    assert oracle.translate_eb(f, [2.25], 0.75)[0] == 0.25


def test_ramp_two_isovalues_and_vertex_on_k():
    nx, ny, nz = 9, 4, 2
    f = _ramp(nx, ny, nz)
    m = ny * nz
    D = oracle.translate_D(f, [2.25, 4.5, 6.0])
    # 6.0 sits on the vertices x = 6: no edge has s0 < 6 < s1, it adds nothing
    assert sorted(D.tolist()) == sorted([0.25] * m + [0.75] * m + [0.5] * (2 * m))
    assert oracle.translate_eb(f, [2.25, 4.5, 6.0], 1.0)[0] == 0.25


def test_empty_D_is_infinite():
    f = np.full((4, 4, 4), 3.0, np.float32)
    eb, n = oracle.translate_eb(f, [1.0])
    assert n == 0 and np.isinf(eb)


def test_gap_rounds_down():
    # k - s0 = 2^25 + 3 is not a float32; nearest is 2^25 + 4, downward 2^25.
    k = np.float32(2.0 ** 25 + 4.0)
    f = np.array([1.0, 2.0 ** 26], np.float32).reshape(1, 1, 2)
    D = oracle.translate_D(f, [k])
    assert D.size == 2
    assert D[0] == np.float32(2.0 ** 25)
    assert float(D[0]) <= float(k) - 1.0
    assert float(D[1]) <= 2.0 ** 26 - float(k)


def test_min_D_preserves_crossing_edges():
    # the paper's argument: an error below both d0 and d1 keeps every
    # crossing edge crossing with the same orientation.
    f = synth.turbulence(24, seed=21)
    K = [-0.5, 0.5]
    eb, _ = oracle.translate_eb(f, K, 1.0)
    enc = oracle.encode(f, [np.float32(min(0.5, eb))], [], fix=False)
    R = enc.R[0]
    nz, ny, nx = f.shape
    for k in K:
        k = np.float32(k)
        for axis in range(3):
            sl0 = [slice(None)] * 3
            sl1 = [slice(None)] * 3
            sl0[2 - axis] = slice(0, -1)
            sl1[2 - axis] = slice(1, None)
            a, b = f[tuple(sl0)], f[tuple(sl1)]
            cross = (np.minimum(a, b) < k) & (k < np.maximum(a, b))
            ra, rb = R[tuple(sl0)], R[tuple(sl1)]
            assert np.array_equal((ra < k)[cross], (a < k)[cross])
            assert np.array_equal((rb < k)[cross], (b < k)[cross])


def test_min_D_is_not_enough_for_lone_vertices():
    # a vertex just above k whose neighbours are all above k is on no crossing
    # edge, so D does not see it; with 2e = 1 it quantises to 0 < k and a new
    # surface appears.  The per-vertex sign fix keeps it.
    k = np.float32(0.25)
    f = np.full((6, 6, 6), 10.0, np.float32)
    f[1, 1, 1:3] = [-0.25, 0.75]       # crossing edge: d0 = d1 = 0.5
    f[4, 4, 4] = 0.375                 # lone vertex above k
    eb, _ = oracle.translate_eb(f, [k], 1.0)
    assert eb == 0.5
    enc_t = oracle.encode(f, [np.float32(min(1.0, eb))], [], fix=False)
    assert enc_t.R[0][4, 4, 4] < k      # flipped
    assert oracle.mc_count(enc_t.R[0], k) > oracle.mc_count(f, k)
    enc_f = oracle.encode(f, [np.float32(1.0)], [k], fix=True)
    assert np.array_equal(enc_f.R[0] < k, f < k)
    assert oracle.mc_count(enc_f.R[0], k) == oracle.mc_count(f, k)


@pytest.mark.parametrize("acc", [0.99, 0.95, 0.8])
def test_nth_smallest_rank(acc):
    f = synth.turbulence(16, seed=4)
    K = [0.0, 1.0]
    D = np.sort(oracle.translate_D(f, K))
    eb, n = oracle.translate_eb(f, K, acc)
    rank = int(np.floor((1.0 - np.float64(np.float32(acc))) * n))
    # eb is the value at that rank: at most `rank` elements lie below it and
    # more than `rank` lie at or below it
    assert np.count_nonzero(D < eb) <= rank < np.count_nonzero(D <= eb)


def test_nan_and_infinite_ends():
    # NaN compares false with every k: an edge with a NaN end never crosses.
    # An infinite end makes its own difference +inf and leaves the other one
    # finite.
    f = np.array([np.nan, 1.0, 3.0], np.float32).reshape(1, 1, 3)
    assert sorted(oracle.translate_D(f, [2.0]).tolist()) == [1.0, 1.0]
    f = np.array([-np.inf, 0.0], np.float32).reshape(1, 1, 2)
    assert sorted(oracle.translate_D(f, [-1.0]).tolist()) == [1.0, np.inf]
    f = np.array([0.0, np.inf], np.float32).reshape(1, 1, 2)
    assert sorted(oracle.translate_D(f, [1.0]).tolist()) == [1.0, np.inf]
    f = np.array([np.inf, -np.inf], np.float32).reshape(1, 1, 2)
    assert oracle.translate_D(f, [5.0]).tolist() == [np.inf, np.inf]
    f = np.array([np.nan, np.inf], np.float32).reshape(1, 1, 2)
    assert oracle.translate_eb(f, [5.0], 1.0) == (np.inf, 0)


def test_repeated_isovalue_counts_twice():
    f = _ramp(7, 5, 3)
    once = np.sort(oracle.translate_D(f, [2.25]))
    twice = np.sort(oracle.translate_D(f, [2.25, 2.25]))
    assert np.array_equal(twice, np.sort(np.concatenate([once, once])))
    assert oracle.translate_eb(f, [2.25, 2.25], 1.0) == (0.25, 2 * once.size)


def _f32_down(q):
    """The largest float32 <= the rational q (math.inf stays inf)."""
    from fractions import Fraction
    if q == float("inf"):
        return np.float32(np.inf)
    c = np.float32(float(q))
    while Fraction(float(c)) > q:
        c = np.nextafter(c, np.float32(-np.inf))
    while Fraction(float(np.nextafter(c, np.float32(np.inf)))) <= q:
        c = np.nextafter(c, np.float32(np.inf))
    return c


def _brute_D(f, K):
    """D from its definition: every edge, every listed k strictly between the
    ends, both rounded-down gaps computed from exact rationals."""
    from fractions import Fraction
    nz, ny, nx = f.shape
    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
                    if x + dx >= nx or y + dy >= ny or z + dz >= nz:
                        continue
                    a, b = float(f[z, y, x]), float(f[z + dz, y + dy, x + dx])
                    if np.isnan(a) or np.isnan(b):
                        continue
                    lo, hi = min(a, b), max(a, b)
                    for k in K:
                        k = float(np.float32(k))
                        if lo < k < hi:
                            d0 = float("inf") if lo == -np.inf else Fraction(k) - Fraction(lo)
                            d1 = float("inf") if hi == np.inf else Fraction(hi) - Fraction(k)
                            out += [_f32_down(d0), _f32_down(d1)]
    return np.sort(np.array(out, np.float32))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_D_on_tiny_grids(seed):
    # values on a coarse grid of thirds so that ends often equal an isovalue
    # or each other, plus NaN and infinite vertices; isovalues unsorted and
    # one repeated
    rng = np.random.default_rng(seed)
    f = (rng.integers(-9, 10, size=(4, 5, 6)) / 3.0).astype(np.float32)
    f.ravel()[rng.choice(f.size, 6, replace=False)] = [np.nan, np.nan, np.inf, -np.inf, np.inf, -np.inf]
    K = [1.0, -2.0 / 3.0, 0.1, 1.0, 2.5]
    ref = _brute_D(f, K)
    got = np.sort(oracle.translate_D(f, K))
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    eb, n = oracle.translate_eb(f, K, 1.0)
    assert n == ref.size and np.float32(eb) == ref[0]

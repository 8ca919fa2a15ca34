"""Pins for the oracle's codec (paper Sec. 2 levels, Sec. 2.2 sign fix).

Each check comes from outside the oracle: the error bound re-checked in
float64, the sign rule of Sec. 2.2, closed forms of the Lorenzo residual on
plane and constant fields, exact integer round trips, a hand-derived
worked example (tests/golden/codec_worked_example.txt), and every int8 value
in every slot of a 2^3 brick against the Lorenzo residual written out by
inclusion-exclusion (mode, width, anchor, packed bits, exact decode)."""
import os

import numpy as np
import pytest

import oracle
from paper_2408_05462_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _check_bound(f, enc):
    f64 = f.astype(np.float64)
    fin = np.isfinite(f64)
    for l in range(enc.nlevels):
        R = enc.R[l].astype(np.float64)
        with np.errstate(invalid="ignore"):  # inf - inf and NaN at the non-finite inputs, checked below
            err = np.abs(f64 - R)
        assert np.all(err[fin] < float(enc.eb[l])), f"level {l}: max err {err[fin].max()} >= {enc.eb[l]}"
        # non-finite inputs come back bit-exact
        assert np.array_equal(f[~fin].view(np.uint32), enc.R[l][~fin].view(np.uint32))


def _check_signs(f, enc, K):
    for l in range(enc.nlevels):
        for k in K:
            k = np.float32(k)
            assert np.array_equal(enc.R[l] < k, f < k), f"level {l}, k {k}: sign flipped"


def _zz(d):
    d = np.asarray(d, np.int64)
    return np.where(d >= 0, 2 * d, -2 * d - 1)


def _bitlen(v):
    v = int(v)
    return v.bit_length()


@pytest.mark.parametrize("shape,seed", [((16, 16, 16), 1), ((21, 33, 40), 2), ((9, 8, 17), 3)])
def test_strict_bound_and_roundtrip_random(shape, seed):
    f = synth.uniform_noise(shape, seed, -3.0, 5.0)
    r = synth.value_range(f)
    eb = np.array([1e-2 * r, 1e-3 * r, 1e-4 * r], np.float32)
    K = [-1.0, 0.5, 2.0]
    enc = oracle.encode(f, eb, K, fix=True)
    _check_bound(f, enc)
    _check_signs(f, enc, K)
    for l in range(enc.nlevels):
        dec = oracle.decode(enc, l)
        assert np.array_equal(dec.view(np.uint32), enc.R[l].view(np.uint32))


def test_turbulence_and_blobs_bound():
    for f in (synth.turbulence(32, seed=7), synth.gaussian_blobs(24, seed=64)):
        r = synth.value_range(f)
        eb = np.array([1e-2 * r, 1e-3 * r], np.float32)
        K = [float(np.median(f)), float(np.percentile(f, 90))]
        enc = oracle.encode(f, eb, K)
        _check_bound(f, enc)
        _check_signs(f, enc, K)
        # errors shrink level by level
        e0 = np.abs(enc.R[0].astype(np.float64) - f).max()
        e1 = np.abs(enc.R[1].astype(np.float64) - f).max()
        assert e1 < e0


def test_adversarial_values():
    e = np.float32(0.25)
    two_e = np.float32(0.5)
    vals = [0.0, -0.0, 0.25, -0.25, 0.75, 1.25,          # exact ties x = n + 0.5 -> |err| = e
            1.0, np.nextafter(np.float32(1.0), np.float32(2)), np.nextafter(np.float32(1.0), np.float32(0)),
            np.nan, np.inf, -np.inf, 1e30, -1e30,        # non-finite and |x| > QMAX
            float(two_e) * 8388607.0, float(two_e) * 8388608.0, 3.0, -7.5]
    f = np.array(vals + [0.5] * (64 - len(vals)), np.float32).reshape(4, 4, 4)
    enc = oracle.encode(f, [e, np.float32(0.01)], [1.0], fix=True)
    _check_bound(f, enc)
    _check_signs(f, enc, [1.0])
    flat = f.ravel()
    slots = {int(s) for s in enc.exc_idx[0]}
    # index -> slot inside the single 8^3 brick: x + 8y + 64z
    def slot(i):
        x, y, z = i % 4, (i // 4) % 4, i // 16
        return x + 8 * y + 64 * z
    for i, v in enumerate(flat):
        if not np.isfinite(v) or abs(float(v)) * 2.0 > 8388607.0:
            assert slot(i) in slots, f"value {v} must be an exception"
    # a tie |f - R| == e exactly is an exception (strict bound)
    for i in (2, 3, 4, 5):
        assert slot(i) in slots
    # non-finite values are exceptions at every level and return bit-exact
    for l in range(2):
        s_l = {int(s) for s in enc.exc_idx[l]}
        for i, v in enumerate(flat):
            if not np.isfinite(v):
                assert slot(i) in s_l
        dec = oracle.decode(enc, l)
        assert np.array_equal(dec.view(np.uint32)[~np.isfinite(f)], f.view(np.uint32)[~np.isfinite(f)])


def test_constant_bricks_need_no_bits():
    # one constant per 8^3 brick, each an exact multiple of 2e: every code in a
    # brick equals its anchor, so both residual forms are zero and w == 0.
    nb = 3
    f = np.zeros((8 * nb, 8 * nb, 8 * nb), np.float32)
    consts = {}
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                c = float(bx - 2 * by + 3 * bz) * 0.5
                consts[(bx, by, bz)] = c
                f[8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8] = c
    enc = oracle.encode(f, [0.25], [], fix=False)   # 2e = 0.5
    assert np.all(enc.width(0) == 0)
    assert enc.words[0].size == 0
    for b, (key, c) in enumerate(sorted(consts.items(), key=lambda kv: (kv[0][2], kv[0][1], kv[0][0]))):
        assert int(np.int32(enc.recs[0][b, 2].view(np.int32))) == int(round(c / 0.5))
    assert np.array_equal(enc.R[0], f)


@pytest.mark.parametrize("a,b,c", [(1, 2, 3), (-5, 0, 7), (0, 0, 1), (40, -33, 2)])
def test_plane_field_lorenzo_closed_form(a, b, c):
    # codes q = a*x + b*y + c*z exactly (2e = 1, integer field).  The Lorenzo
    # residual of a linear function vanishes except on the three axes through
    # the brick origin, where it is a, b and c; the plain residual is q itself.
    n = 20
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    f = (a * x + b * y + c * z).astype(np.float32)
    enc = oracle.encode(f, [0.5], [], fix=False)
    assert enc.exc_idx[0].size == 0
    nbx = 3
    wl = _bitlen(max(_zz([a, b, c])))
    for bidx in range(enc.recs[0].shape[0]):
        bx, by, bz = bidx % nbx, (bidx // nbx) % nbx, bidx // (nbx * nbx)
        ex, ey, ez = min(8, n - 8 * bx), min(8, n - 8 * by), min(8, n - 8 * bz)
        lz, ly, lx = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
        q = a * (8 * bx + lx) + b * (8 * by + ly) + c * (8 * bz + lz)
        zn = _zz(q).ravel()[1:]  # slot 0 is the anchor
        wn = _bitlen(zn.max()) if zn.size else 0
        # which of the three axis residuals exist inside this (possibly partial) brick
        present = [a] * (ex > 1) + [b] * (ey > 1) + [c] * (ez > 1)
        wlb = _bitlen(max(_zz(present))) if present else 0
        w = int(enc.width(0)[bidx])
        mode = int(enc.mode(0)[bidx])
        exp_mode = 1 if wlb < wn else 0
        assert mode == exp_mode, (bidx, wlb, wn)
        assert w == (wlb if exp_mode else wn)
        assert int(enc.recs[0][bidx, 2].view(np.int32)) == int(q.ravel()[0])
    assert wl >= 0
    assert np.array_equal(oracle.decode(enc, 0), f)


def test_integer_fields_roundtrip_exactly():
    # with 2e = 1 an integer field quantises to itself: no exception, exact
    # reconstruction, large residuals exercise wide packing (w up to 26).
    g = np.random.Generator(np.random.PCG64(11))
    for shape, hi in [((8, 8, 8), 3), ((13, 10, 9), 1 << 10), ((16, 9, 11), (1 << 22) - 1)]:
        f = g.integers(-hi, hi + 1, size=shape).astype(np.float32)
        enc = oracle.encode(f, [0.5], [], fix=False)
        assert enc.exc_idx[0].size == 0
        assert np.array_equal(oracle.decode(enc, 0), f)
        assert enc.width(0).max() <= 27


def test_packing_is_minimal_width():
    # every brick's w is the bit length of its widest zig-zag code: decoding
    # with w-1 bits would lose the top bit of at least one slot.
    f = synth.uniform_noise((16, 16, 16), 5, -2, 2)
    enc = oracle.encode(f, [0.01], [], fix=False)
    W = enc.words[0]
    for b in range(enc.recs[0].shape[0]):
        w = int(enc.width(0)[b])
        if w == 0:
            continue
        base = 16 * int(enc.recs[0][b, 0])
        bits = np.unpackbits(W[base:base + 16 * w].view(np.uint8), bitorder="little")
        top = bits.reshape(512, w)[:, w - 1]
        assert top.any()


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "level":
                rows[("level", int(parts[1]), parts[2])] = parts[3:]
            else:
                rows[parts[0]] = parts[1:]
    return rows


def test_golden_worked_example():
    g = _read_golden("codec_worked_example.txt")
    nx, ny, nz = map(int, g["dims"])
    f = np.array(list(map(float, g["f"])), np.float32).reshape(nz, ny, nx)
    eb = np.array(list(map(float, g["eb"])), np.float32)
    K = list(map(float, g["K"]))
    enc = oracle.encode(f, eb, K, fix=True)
    for l in range(2):
        assert list(enc.recs[l][0]) == [int(v) for v in g[("level", l, "record")]]
        assert enc.words[l].size == int(g[("level", l, "nwords")][0])
        assert int(enc.words[l][0]) == int(g[("level", l, "word0")][0])
        assert np.all(enc.words[l][1:] == 0)
        assert [int(v) for v in enc.exc_idx[l]] == [int(v) for v in g[("level", l, "exc_idx")]]
        assert [int(v) for v in enc.exc_val[l]] == [int(v, 16) for v in g[("level", l, "exc_val")]]
        assert np.array_equal(enc.R[l].ravel(), np.array(list(map(float, g[("level", l, "R")])), np.float32))
        assert np.array_equal(oracle.decode(enc, l).ravel(), enc.R[l].ravel())


def test_sign_fix_off_can_flip_and_on_cannot():
    # values just above k quantise below it when the fix is off
    k = np.float32(0.3)
    f = np.full((8, 8, 8), 0.31, np.float32)  # 2e = 0.5 -> q = 1 -> R = 0.5?  use e s.t. R < k
    f[::2] = 0.26                             # x = 0.52 -> q 1 -> R 0.5 (>k), true 0.26 < k -> flip
    enc_off = oracle.encode(f, [0.25], [k], fix=False)
    enc_on = oracle.encode(f, [0.25], [k], fix=True)
    assert not np.array_equal(enc_off.R[0] < k, f < k)
    assert np.array_equal(enc_on.R[0] < k, f < k)
    _check_bound(f, enc_off)
    _check_bound(f, enc_on)


def _lorenzo_2x2x2(q):
    """3-D Lorenzo residual with zero outside the brick, written out by
    inclusion-exclusion over the up-to-seven lower neighbours."""
    d = np.zeros_like(q)
    for z in range(2):
        for y in range(2):
            for x in range(2):
                pred = 0
                for dz in (0, 1):
                    for dy in (0, 1):
                        for dx in (0, 1):
                            if dx == dy == dz == 0:
                                continue
                            if x - dx < 0 or y - dy < 0 or z - dz < 0:
                                continue
                            sign = 1 if (dx + dy + dz) % 2 == 1 else -1
                            pred += sign * int(q[z - dz, y - dy, x - dx])
                d[z, y, x] = int(q[z, y, x]) - pred
    return d


def test_brute_force_int8_bricks():
    # a 2^3 grid is one partial brick; with 2e = 1 its integer values are its
    # codes.  Every slot takes every int8 value, the others from a plane (the
    # Lorenzo form wins near it: widths 3 to 7) or from a seeded draw (the
    # plain codes win): the mode is the residual form of smaller width (a tie
    # keeps the plain codes), the anchor is the code at the origin and its
    # slot packs 0, slot s = x + 8*(y + 8*z) sits at bit s*w, and decoding is
    # exact.
    z, y, x = np.meshgrid(np.arange(2), np.arange(2), np.arange(2), indexing="ij")
    g = np.random.Generator(np.random.PCG64(8))
    seen = set()
    for base in (20 + 3 * x - 2 * y + 5 * z, g.integers(-128, 128, size=(2, 2, 2))):
        seen |= _brute_force_brick(base)
    assert {m for m, _ in seen} == {0, 1} and len({w for _, w in seen}) >= 5


def _brute_force_brick(base):
    seen = set()
    for slot in range(8):
        z, y, x = (slot >> 2) & 1, (slot >> 1) & 1, slot & 1
        for v in range(-128, 128):
            q = base.copy()
            q[z, y, x] = v
            f = q.astype(np.float32)
            enc = oracle.encode(f, [0.5], [], fix=False)
            assert enc.exc_idx[0].size == 0
            plain = q.copy()
            lor = _lorenzo_2x2x2(q)
            wp = _bitlen(_zz(plain.ravel()[1:]).max())
            wl = _bitlen(_zz(lor.ravel()[1:]).max())
            mode, w = (1, wl) if wl < wp else (0, wp)
            seen.add((mode, w))
            assert int(enc.mode(0)[0]) == mode and int(enc.width(0)[0]) == w, (slot, v)
            assert int(enc.recs[0][0, 2].view(np.int32)) == int(q[0, 0, 0])
            resid = (lor if mode else plain).copy()
            resid[0, 0, 0] = 0
            if w:
                bits = np.unpackbits(enc.words[0].view(np.uint8), bitorder="little")
                for zz in range(2):
                    for yy in range(2):
                        for xx in range(2):
                            s = xx + 8 * (yy + 8 * zz)
                            code = int(np.dot(bits[s * w:(s + 1) * w], 1 << np.arange(w)))
                            assert code == int(_zz(resid[zz, yy, xx])), (slot, v, s)
            assert np.array_equal(oracle.decode(enc, 0), f)
    return seen

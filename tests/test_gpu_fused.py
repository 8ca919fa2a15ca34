"""chr_isosurface's forms (paper Sec. 2: the visualization side reconstructs
the requested level and generates the isosurface) -- decode then marching
cubes, with or without the value index, and the one-pass fused kernel --
and the CHR's value index itself (Sec. 2.1, isovalue-based pruning).

* The index of every level equals the oracle's brick index of the oracle's
  reconstruction, bit for bit (odd sizes, bricks without cells, NaN and
  infinite vertices).
* Each form's triangles equal the oracle's marching cubes of the
  oracle's reconstruction (counts and order exactly, vertices within the
  tolerance of tests/helpers.py), at every level, for 1 to 6 isovalues, on
  grids of several tiles with ragged edges.
* Every form (with and without the index, fused or not) gives the same
  bits (triangles, counts, error word); a handle read back from
  its byte string (with its index, or stripped to a version-1 string
  without one) gives the same bits again.
* Bricks the index skips hold no triangle of the oracle's mesh, and on
  turbulence the index does skip some.
"""
import numpy as np
import pytest
import torch

import oracle
from helpers import compare_mesh
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()
    chr.lib()


def _bits(t):
    return t.contiguous().view(torch.int32)


def _dev(f):
    return torch.from_numpy(np.ascontiguousarray(f)).cuda()


def _adversarial(shape, seed):
    f = synth.turbulence(shape, seed=seed)
    rng = np.random.default_rng(seed)
    flat = f.reshape(-1)
    n = flat.size
    flat[rng.choice(n, max(n // 500, 1), replace=False)] = np.nan
    flat[rng.choice(n, max(n // 700, 1), replace=False)] = np.inf
    flat[rng.choice(n, max(n // 900, 1), replace=False)] = -np.inf
    return f


CASES = [
    ("blobs64", lambda: synth.gaussian_blobs(64, seed=64), None),
    ("odd", lambda: synth.turbulence((37, 50, 65), seed=3), None),
    ("ragged_tiles", lambda: synth.turbulence((70, 45, 33), seed=12), None),
    ("nx9_cellless", lambda: synth.turbulence((9, 33, 17), seed=7), None),
    ("small", lambda: synth.turbulence((17, 9, 23), seed=2), None),
]


def _isos(name, f):
    if name == "blobs64":
        return [0.5 * float(f.max())]
    return [-1.0, -0.5, 0.5, 1.0]


@pytest.mark.parametrize("name,make,_", CASES)
def test_index_matches_oracle(name, make, _):
    f = make()
    r = synth.value_range(f)
    K = _isos(name, f)
    eb = [1e-2 * r, 1e-3 * r, 1e-4 * r]
    h = chr.chr_compress(_dev(f), eb, K)
    enc = oracle.encode(f, eb, K, fix=True)
    for l in range(3):
        got = chr.chr_brick_index(h, l).cpu().numpy()
        lo, hi = oracle.brick_index(enc.R[l])
        assert np.array_equal(got[..., 0].view(np.uint32), lo.view(np.uint32)), (name, l)
        assert np.array_equal(got[..., 1].view(np.uint32), hi.view(np.uint32)), (name, l)
    h.free()


def test_index_nonfinite_values():
    f = _adversarial((41, 26, 19), seed=9)
    eb = [1e-2, 1e-3]
    K = [-0.5, 0.5]
    h = chr.chr_compress(_dev(f), eb, K)
    enc = oracle.encode(f, eb, K, fix=True)
    for l in range(2):
        got = chr.chr_brick_index(h, l).cpu().numpy()
        lo, hi = oracle.brick_index(enc.R[l])
        assert np.array_equal(got[..., 0].view(np.uint32), lo.view(np.uint32))
        assert np.array_equal(got[..., 1].view(np.uint32), hi.view(np.uint32))
    h.free()


@pytest.mark.parametrize("name,make,_", CASES)
def test_fused_matches_oracle_every_level(name, make, _):
    f = make()
    r = synth.value_range(f)
    K = _isos(name, f)
    eb = [1e-2 * r, 1e-3 * r, 1e-4 * r]
    h = chr.chr_compress(_dev(f), eb, K)
    enc = oracle.encode(f, eb, K, fix=True)
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
    for level in range(3):
        for flags in (0, chr.ISO_INDEX, chr.ISO_FUSED | chr.ISO_INDEX):
            t, c, e = chr.chr_isosurface(h, level, K, cap, flags=flags)
            torch.cuda.synchronize()
            assert int(e.item()) == 0
            tt = t.cpu().numpy()
            for j, k in enumerate(K):
                mesh = oracle.mc(enc.R[level], k)
                assert int(c[j]) == mesh.ntri, (name, level, k, flags)
                compare_mesh(tt[j, :mesh.ntri], mesh, (nx, ny, nz), f"{name} level {level} k={k} flags {flags}")
    h.free()


@pytest.mark.parametrize("isos", [[0.3], [-1.0, 0.5], [-1.0, -0.5, 0.5], [-1.0, -0.5, 0.5, 1.0],
                                  [-1.2, -0.6, 0.0, 0.2, 0.7], [-1.2, -0.6, 0.0, 0.2, 0.7, 1.1]])
def test_fused_isovalue_counts_against_oracle(isos):
    f = synth.turbulence((70, 45, 33), seed=12)
    r = synth.value_range(f)
    eb = [1e-2 * r, 1e-3 * r]
    h = chr.chr_compress(_dev(f), eb, [-1.0, -0.5, 0.5, 1.0])
    enc = oracle.encode(f, eb, [-1.0, -0.5, 0.5, 1.0], fix=True)
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
    for flags in (0, chr.ISO_INDEX, chr.ISO_FUSED | chr.ISO_INDEX):
        t, c, e = chr.chr_isosurface(h, 1, isos, cap, flags=flags)
        torch.cuda.synchronize()
        assert int(e.item()) == 0
        tt = t.cpu().numpy()
        for j, k in enumerate(isos):
            mesh = oracle.mc(enc.R[1], k)
            assert int(c[j]) == mesh.ntri, (k, flags)
            compare_mesh(tt[j, :mesh.ntri], mesh, (nx, ny, nz), f"k={k} flags {flags}")
    h.free()


def _three_ways(h, level, K, cap):
    """(default, with the index, one-pass fused, fused with the index)"""
    out = []
    for flags in (0, chr.ISO_INDEX, chr.ISO_FUSED, chr.ISO_FUSED | chr.ISO_INDEX):
        t, c, e = chr.chr_isosurface(h, level, K, cap, flags=flags)
        out.append((t, c, e))
    torch.cuda.synchronize()
    return out


def _assert_same(a, b, K, label):
    (t0, c0, e0), (t1, c1, e1) = a, b
    assert int(e0.item()) == int(e1.item()), label
    assert torch.equal(c0, c1), label
    for j in range(len(K)):
        n = min(int(c0[j]), t0.shape[1])
        assert torch.equal(_bits(t0[j, :n]), _bits(t1[j, :n])), (label, j)


@pytest.mark.parametrize("shape,seed", [((70, 45, 33), 12), ((130, 66, 34), 4), ((33, 17, 9), 5), ((64, 64, 64), 8)])
def test_fused_skip_and_unfused_agree_bitwise(shape, seed):
    f = synth.turbulence(shape, seed=seed)
    r = synth.value_range(f)
    K = [-1.0, -0.5, 0.5, 1.0]
    h = chr.chr_compress(_dev(f), [1e-2 * r, 1e-3 * r, 1e-4 * r], K)
    nx, ny, nz = shape[2], shape[1], shape[0]
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
    for level in range(3):
        ways = _three_ways(h, level, K, cap)
        for w in ways[1:]:
            _assert_same(ways[0], w, K, f"level {level}")
    # more than 4 isovalues, not the compression's candidates
    K6 = [-1.3, -0.7, -0.1, 0.2, 0.6, 1.4]
    ways = _three_ways(h, 2, K6, cap)
    for w in ways[1:]:
        _assert_same(ways[0], w, K6, "6 isovalues")
    h.free()


def test_fused_nonfinite_and_huge_values_agree_bitwise():
    f = _adversarial((41, 26, 19), seed=9)
    f[5:9, 3:12, 10:30] *= np.float32(5e37)  # values past 2^124: the IEEE quotient in those tiles
    K = [-0.5, 0.5, 2e37]
    h = chr.chr_compress(_dev(f), [1e-2, 1e-3], K)
    cap = 5 * 40 * 25 * 18
    for level in range(2):
        ways = _three_ways(h, level, K, cap)
        for w in ways[1:]:
            _assert_same(ways[0], w, K, "nonfinite")
    h.free()


def test_overflow_matches_unfused():
    f = synth.turbulence((70, 45, 33), seed=12)
    r = synth.value_range(f)
    K = [-0.5, 0.5]
    h = chr.chr_compress(_dev(f), [1e-2 * r], K)
    _, c, _ = chr.chr_isosurface(h, 0, K, 0)
    torch.cuda.synchronize()
    cap = int(c.min()) // 3
    ways = _three_ways(h, 0, K, cap)
    assert int(ways[0][2].item()) & chr.ERR_OVERFLOW_BIT
    for w in ways[1:]:
        _assert_same(ways[0], w, K, "overflow")
    h.free()


def test_serialized_handles_with_and_without_index():
    f = synth.turbulence((70, 45, 33), seed=13)
    r = synth.value_range(f)
    K = [-1.0, 0.5]
    h = chr.chr_compress(_dev(f), [1e-2 * r, 1e-3 * r], K)
    blob = chr.chr_serialize(h)
    parsed = chr.parse_serialized(blob)
    assert parsed["version"] == 2
    for l in range(2):
        idx = chr.chr_brick_index(h, l).cpu().numpy().reshape(-1, 2)
        assert np.array_equal(parsed["levels"][l]["index"].view(np.uint32), idx.view(np.uint32))
    h2 = chr.chr_deserialize(blob)
    assert chr.chr_serialize(h2) == blob
    # the same string as version 1: no index (nothing skipped), same output
    nb = parsed["levels"][0]["recs"].shape[0]
    v1 = bytearray(blob[:len(blob) - 2 * 8 * nb])
    v1[4:8] = (1).to_bytes(4, "little")
    h1 = chr.chr_deserialize(bytes(v1))
    with pytest.raises(chr.ChrError):
        chr.chr_brick_index(h1, 0)
    cap = 5 * 69 * 44 * 32
    ref = chr.chr_isosurface(h, 1, K, cap)
    for hh in (h2, h1):
        for flags in (0, chr.ISO_INDEX, chr.ISO_FUSED | chr.ISO_INDEX):
            _assert_same(ref, chr.chr_isosurface(hh, 1, K, cap, flags=flags), K, "deserialized")
    for x in (h, h1, h2):
        x.free()


def test_skipped_bricks_hold_no_oracle_triangle():
    f = synth.turbulence((96, 80, 72), seed=21)
    r = synth.value_range(f)
    K = [-1.0, -0.5, 0.5, 1.0]
    eb = [1e-2 * r, 1e-3 * r]
    h = chr.chr_compress(_dev(f), eb, K)
    enc = oracle.encode(f, eb, K, fix=True)
    idx = chr.chr_brick_index(h, 1).cpu().numpy()
    nz, ny, nx = f.shape
    skipped_pairs = 0
    for k in K:
        skip = ~((idx[..., 0] < k) & (k <= idx[..., 1]))
        mesh = oracle.mc(enc.R[1], k)
        cx = mesh.cell % (nx - 1)
        cy = (mesh.cell // (nx - 1)) % (ny - 1)
        cz = mesh.cell // ((nx - 1) * (ny - 1))
        assert not skip[cz // 8, cy // 8, cx // 8].any(), k
        has_cells = (np.arange(idx.shape[2]) * 8 < nx - 1)[None, None, :] & \
            (np.arange(idx.shape[1]) * 8 < ny - 1)[None, :, None] & (np.arange(idx.shape[0]) * 8 < nz - 1)[:, None, None]
        skipped_pairs += int((skip & has_cells).sum())
    assert skipped_pairs > 0
    h.free()

"""GPU parity: libchr (through its C ABI) against the CPU oracle on the same
seeded inputs.  Integer results (records, packed words, exceptions, triangle
counts, case-determined triangle order) must match bit for bit; decoded
fields bit for bit; vertex positions within 1e-5 of a cell edge plus one
float32 ulp of the coordinate (tests/helpers.py)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import brick_major_order, compare_mesh, vertex_tol
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()
    chr.lib()


def _dev(f):
    return torch.from_numpy(np.ascontiguousarray(f)).cuda()


def _extract(f, isovalues, cap=None):
    fd = _dev(f)
    if cap is None:
        nz, ny, nx = f.shape
        cap = 5 * (nx - 1) * (ny - 1) * (nz - 1) + 64  # at most 5 triangles per cell
    tris, counts, err = chr.isosurface_extract(fd, isovalues, cap)
    torch.cuda.synchronize()
    return tris.cpu().numpy(), counts.cpu().numpy(), int(err.item())


def _fields_mc():
    blobs = synth.gaussian_blobs(64, seed=64)
    turb = synth.turbulence((37, 50, 65), seed=3)
    noise = synth.uniform_noise((17, 9, 23), 5)
    return [
        ("blobs64", blobs, [0.5 * float(blobs.max())]),
        ("turb_odd_4iso", turb, [-1.0, -0.5, 0.5, 1.0]),
        ("turb_odd_6iso", turb, [-1.5, -0.25, 0.0, 0.3, 0.9, 2.0]),
        ("noise", noise, [0.0, 0.5]),
    ]


@pytest.mark.parametrize("name,f,isos", _fields_mc(), ids=lambda v: v if isinstance(v, str) else "")
def test_mc_matches_oracle(name, f, isos):
    nz, ny, nx = f.shape
    tris, counts, err = _extract(f, isos)
    assert err == 0
    for j, k in enumerate(isos):
        mesh = oracle.mc(f, k)
        assert int(counts[j]) == mesh.ntri, (name, k)
        compare_mesh(tris[j, :mesh.ntri], mesh, (nx, ny, nz), f"{name} k={k}")


@pytest.mark.parametrize("case", ["constant", "all_equal_k", "checker", "plane", "tiny"])
def test_mc_degenerate_fields(case):
    if case == "constant":
        f = np.full((9, 10, 11), 3.0, np.float32)
        k = 1.0
    elif case == "all_equal_k":
        f = np.full((9, 10, 11), 0.5, np.float32)
        k = 0.5
    elif case == "checker":
        z, y, x = np.meshgrid(np.arange(12), np.arange(13), np.arange(14), indexing="ij")
        f = np.where((x + y + z) % 2 == 0, -1.0, 1.0).astype(np.float32)
        k = 0.0
    elif case == "plane":
        f = synth.plane_field((40, 33, 20), (0, 0, 1), 10.375)
        k = 0.0
    else:
        f = synth.uniform_noise((2, 2, 2), 1)
        k = 0.0
    nz, ny, nx = f.shape
    tris, counts, err = _extract(f, [k])
    mesh = oracle.mc(f, k)
    assert err == 0 and int(counts[0]) == mesh.ntri
    compare_mesh(tris[0, :mesh.ntri], mesh, (nx, ny, nz), case)


def test_mc_overflow_reports_true_count_and_stays_in_bounds():
    f = synth.turbulence(32, seed=8)
    mesh = oracle.mc(f, 0.0)
    cap = mesh.ntri // 3
    fd = _dev(f)
    guard = 1 << 12
    buf = torch.full((cap * 9 + guard,), 7.0, dtype=torch.float32, device="cuda")
    tris = buf[:cap * 9].view(1, cap, 3, 3)
    tris, counts, err = chr.isosurface_extract(fd, [0.0], cap, tris=tris)
    torch.cuda.synchronize()
    assert int(counts[0]) == mesh.ntri
    assert int(err.item()) & chr.ERR_OVERFLOW_BIT
    assert torch.all(buf[cap * 9:] == 7.0)
    # the triangles that fit are the first `cap` of the full output
    full, counts2, err2 = _extract(f, [0.0])
    assert np.array_equal(tris.cpu().numpy()[0], full[0, :cap])


@pytest.mark.parametrize("isos", [[0.3], [-1.0, 0.5], [-1.0, -0.5, 0.5], [-1.0, -0.5, 0.5, 1.0],
                                  [-1.2, -0.6, 0.0, 0.2, 0.7], [-1.2, -0.6, 0.0, 0.2, 0.7, 1.1]])
def test_mc_workspace_layouts_agree(isos):
    # A small grid takes the single pass with either workspace (the full one
    # also holds the count pass's classification; the minimum one, the tile
    # arrays, about 50 bytes per 32x8x8-cell tile).  Same bits, the oracle's
    # triangles, and a workspace full of stale bytes reused call after call.
    f = synth.turbulence((70, 45, 33), seed=12)
    fd = _dev(f)
    cap = 5 * 69 * 44 * 32
    full = chr.isosurface_workspace_size(f.shape, len(isos))
    small = chr.isosurface_workspace_min_size(f.shape, len(isos))
    ntiles = (69 + 31) // 32 * ((44 + 7) // 8) * ((32 + 7) // 8)
    assert small <= 64 * ntiles + 1024
    assert full > small
    out = []
    for nbytes in (full, small, small, full):
        ws = torch.full((nbytes,), 0xA5, dtype=torch.uint8, device="cuda")
        t, c, e = chr.isosurface_extract(fd, isos, cap, workspace=ws)
        torch.cuda.synchronize()
        assert int(e.item()) == 0
        out.append((t, c))
    t1, c1 = out[0]
    for t2, c2 in out[1:]:
        assert torch.equal(c1, c2)
        for j in range(len(isos)):
            n = int(c1[j])
            assert torch.equal(t1[j, :n].view(torch.int32), t2[j, :n].view(torch.int32)), j
    nz, ny, nx = f.shape
    for j, k in enumerate(isos):
        n = int(c1[j])
        mesh = oracle.mc(f, k)
        assert n == mesh.ntri, k
        compare_mesh(t1[j, :n].cpu().numpy(), mesh, (nx, ny, nz), f"layouts k={k}")


@pytest.mark.parametrize("shape,isos,with_oracle", [((257, 129, 129), [0.3], True),
                                                    ((513, 257, 257), [-0.5, 0.5], False)])
def test_mc_two_pass_and_single_pass_agree_on_large_grids(shape, isos, with_oracle):
    # From 2048*n^3 tiles a group of n isovalues with the full workspace takes
    # the count pass, tile scan and stored-classification emit (2048 tiles
    # here for one isovalue, 16384 for two); the minimum workspace keeps the
    # single pass.  The two give the same bits; one isovalue also against the
    # oracle.
    f = synth.turbulence(shape, seed=31)
    fd = _dev(f)
    nz, ny, nx = f.shape
    ntiles = (nx - 1 + 31) // 32 * ((ny - 1 + 7) // 8) * ((nz - 1 + 7) // 8)
    assert ntiles >= 2048 * len(isos) ** 3
    _, c0, _ = chr.isosurface_extract(fd, isos, 0)
    torch.cuda.synchronize()
    cap = int(c0.max().item()) + 16
    res = []
    for size in (chr.isosurface_workspace_size, chr.isosurface_workspace_min_size):
        ws = torch.full((size(f.shape, len(isos)),), 0x5A, dtype=torch.uint8, device="cuda")
        t, c, e = chr.isosurface_extract(fd, isos, cap, workspace=ws)
        torch.cuda.synchronize()
        assert int(e.item()) == 0
        res.append((t, c))
    (t1, c1), (t2, c2) = res
    assert torch.equal(c1, c2)
    for j in range(len(isos)):
        n = int(c1[j])
        assert torch.equal(t1[j, :n].view(torch.int32), t2[j, :n].view(torch.int32)), j
    if with_oracle:
        mesh = oracle.mc(f, isos[0])
        assert int(c1[0]) == mesh.ntri
        compare_mesh(t1[0, :mesh.ntri].cpu().numpy(), mesh, (nx, ny, nz), "two-pass large grid")


def test_mc_huge_values_take_the_ieee_quotient():
    # Tiles holding a value of magnitude 2^125 or more divide with the IEEE
    # quotient (|f1 - f0| may reach 2^126, past the fast reciprocal's
    # range); the rest keep the fast one.  Half of this field is scaled by
    # 5e37 (values up to about 2e38, neighbour differences far from
    # overflow), half is not, so one call takes both paths.
    f = synth.turbulence((80, 24, 20), seed=41)
    f = (f / np.abs(f).max()).astype(np.float32)
    f[:, :, 40:] *= np.float32(5e37)
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1) + 64
    for isos in ([-0.3, 0.3], [np.float32(-0.3) * np.float32(5e37), np.float32(0.3) * np.float32(5e37)]):
        isos = [float(k) for k in isos]
        for size in (chr.isosurface_workspace_size, chr.isosurface_workspace_min_size):
            ws = torch.empty(size(f.shape, len(isos)), dtype=torch.uint8, device="cuda")
            tris, counts, err = chr.isosurface_extract(_dev(f), isos, cap, workspace=ws)
            torch.cuda.synchronize()
            assert int(err.item()) == 0
            t = tris.cpu().numpy()
            for j, k in enumerate(isos):
                mesh = oracle.mc(f, k)
                assert int(counts[j]) == mesh.ntri, k
                compare_mesh(t[j, :mesh.ntri], mesh, (nx, ny, nz), f"huge k={k}")


def test_mc_nan_and_inf_vertices():
    # NaN and +inf are outside (v < k is false), -inf inside.  The edge
    # fraction t = (k - f0) / (f1 - f0) is 0 when only the far end f1 is
    # infinite and NaN when the near end f0 is infinite (inf / inf) or either
    # end is NaN; only the coordinate on the edge's axis carries t, so only
    # that one may be NaN, on both sides alike
    f = synth.turbulence((40, 30, 20), seed=43)
    f.ravel()[::97] = np.nan
    f.ravel()[5::89] = np.inf
    f.ravel()[9::83] = -np.inf
    nz, ny, nx = f.shape
    isos = [-0.5, 0.5]
    tris, counts, err = chr.isosurface_extract(_dev(f), isos, 5 * (nx - 1) * (ny - 1) * (nz - 1) + 64)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    t = tris.cpu().numpy()
    for j, k in enumerate(isos):
        mesh = oracle.mc(f, k)
        assert int(counts[j]) == mesh.ntri, k
        n = mesh.ntri
        got = t[j, :n].astype(np.float64)
        ref = mesh.pos[brick_major_order(mesh.cell, (nx, ny, nz))]
        assert np.array_equal(np.isnan(got), np.isnan(ref)), k
        ok = ~np.isnan(ref)
        assert np.all(np.abs(got[ok] - ref[ok]) <= vertex_tol(ref)[ok]), k


def test_mc_dense_tiles_take_their_isovalues_one_at_a_time():
    # The emit pass compacts the active cells of all of a tile's isovalues
    # into one shared pool when they fit (about 2048 cells in all) and takes
    # the isovalues one at a time when they do not.  White noise at four
    # isovalues fills every tile's lists several times over (the slot-by-slot
    # path); the smooth part of the field leaves its tiles on the pooled
    # path.  Against the oracle, with a workspace full of stale bytes.
    f = synth.turbulence((70, 19, 20), seed=21)
    f = (f / np.abs(f).max()).astype(np.float32)
    f[:, :, :34] = synth.uniform_noise((20, 19, 34), 22)
    isos = [-0.6, -0.2, 0.2, 0.6]
    fd = _dev(f)
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1) + 64
    meshes = [oracle.mc(f, k) for k in isos]
    assert min(m.ntri for m in meshes) > 4 * 2048  # the noise tiles alone overflow the pool
    for size in (chr.isosurface_workspace_size, chr.isosurface_workspace_min_size):
        ws = torch.full((size(f.shape, len(isos)),), 0xFF, dtype=torch.uint8, device="cuda")
        tris, counts, err = chr.isosurface_extract(fd, isos, cap, workspace=ws)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        t = tris.cpu().numpy()
        for j, (k, mesh) in enumerate(zip(isos, meshes)):
            assert int(counts[j]) == mesh.ntri, (size.__name__, k)
            compare_mesh(t[j, :mesh.ntri], mesh, (nx, ny, nz), f"dense {size.__name__} k={k}")


def test_library_pool_allocator_gives_the_same_chr():
    # a NULL chr_allocator takes the library's own stream-ordered pool; the
    # CHR is the same bytes as with torch's allocator, and trimming the pool
    # after the handles are freed succeeds
    f = synth.turbulence((40, 33, 27), seed=5)
    r = synth.value_range(f)
    fd = _dev(f)
    eb, isos = [1e-2 * r, 1e-3 * r], [-0.5, 0.5]
    ref = chr.chr_compress(fd, eb, isos)
    want = chr.chr_serialize(ref)
    for _ in range(3):
        h = chr.chr_compress(fd, eb, isos, library_pool=True)
        assert chr.chr_serialize(h) == want
        R = h.reconstruct(1)
        assert torch.equal(R.view(torch.int32), ref.reconstruct(1).view(torch.int32))
        h.free()
    torch.cuda.synchronize()
    chr.chr_pool_trim(0)
    ref.free()


def _compare_codec(h, enc, f, label):
    parsed = chr.parse_serialized(chr.chr_serialize(h))
    assert parsed["nlevels"] == enc.nlevels
    for l in range(enc.nlevels):
        lv = parsed["levels"][l]
        assert np.array_equal(lv["recs"], enc.recs[l]), f"{label}: records differ at level {l}"
        assert np.array_equal(lv["words"], enc.words[l]), f"{label}: packed words differ at level {l}"
        assert np.array_equal(lv["exc_idx"], enc.exc_idx[l]), f"{label}: exception slots differ at level {l}"
        assert np.array_equal(lv["exc_val"], enc.exc_val[l]), f"{label}: exception values differ at level {l}"
        dec = h.reconstruct(l).cpu().numpy()
        assert np.array_equal(dec.view(np.uint32), enc.R[l].view(np.uint32)), f"{label}: level {l} decode differs"


def _codec_cases():
    blobs = synth.gaussian_blobs(64, seed=64)
    rb = synth.value_range(blobs)
    turb = synth.turbulence((37, 50, 65), seed=3)
    rt = synth.value_range(turb)
    adv = synth.uniform_noise((20, 19, 18), 2, -4, 4)
    adv.ravel()[::97] = np.nan
    adv.ravel()[5::101] = np.inf
    adv.ravel()[7::103] = -1e30
    adv.ravel()[11::89] = 0.5           # exactly on an isovalue
    adv.ravel()[13::83] = -0.0
    ints = np.random.Generator(np.random.PCG64(9)).integers(-(1 << 20), 1 << 20, size=(16, 24, 40)).astype(np.float32)
    return [
        ("blobs64", blobs, [1e-2 * rb, 1e-3 * rb], [0.5 * float(blobs.max())], "fix"),
        ("turb_odd", turb, [1e-2 * rt, 1e-3 * rt, 1e-4 * rt], [-1.0, -0.5, 0.5, 1.0], "fix"),
        ("turb_nofix", turb, [1e-2 * rt, 1e-3 * rt], [], "none"),
        ("adversarial", adv, [0.25, 0.01, 1e-4], [0.5, -1.0], "fix"),
        ("integers", ints, [0.5], [], "none"),
    ]


@pytest.mark.parametrize("name,f,eb,isos,topo", _codec_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_codec_matches_oracle(name, f, eb, isos, topo):
    eb = np.array(eb, np.float32)
    enc = oracle.encode(f, eb, isos, fix=(topo == "fix"))
    h = chr.chr_compress(_dev(f), eb, isos, topo=topo)
    _compare_codec(h, enc, f, name)
    st = h.stats()
    assert st["exceptions"] == [int(e.size) for e in enc.exc_idx]


def test_serialize_roundtrip_and_decode():
    f = synth.turbulence(40, seed=12)
    r = synth.value_range(f)
    h = chr.chr_compress(_dev(f), [1e-2 * r, 1e-3 * r], [0.0, 1.0])
    blob = chr.chr_serialize(h)
    h2 = chr.chr_deserialize(blob)
    assert chr.chr_serialize(h2) == blob
    for l in range(2):
        a = h.reconstruct(l).cpu().numpy()
        b = h2.reconstruct(l).cpu().numpy()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("acc", [1.0, 0.99, 0.95, 0.8])
def test_translate_matches_oracle(acc):
    f = synth.turbulence((33, 40, 29), seed=int(round(acc * 100)))
    K = [-0.5, 0.25, 1.0]
    eb_o, n_o = oracle.translate_eb(f, K, acc)
    eb_g, n_g = chr.chr_topo_translate(_dev(f), K, acc)
    assert n_g == n_o
    assert np.float32(eb_g).view(np.uint32) == np.float32(eb_o).view(np.uint32)


_TRANSLATE_CASES = [
    # (shape (nz, ny, nx), isovalues): several 31 x 15 tiles with ragged
    # edges and z chunks; 1, 2, 3, 5, 9 and 16 isovalues (every padded
    # count), unsorted and repeated ones
    ((130, 61, 97), [0.3]),
    ((70, 47, 64), [0.5, -0.5]),
    ((33, 17, 93), [1.0, -0.5, 0.25]),
    ((21, 90, 33), [-1.2, -0.4, 0.1, 0.6, 1.3]),
    ((40, 31, 62), [-1.5, -1.0, -0.6, -0.2, 0.0, 0.2, 0.6, 1.0, 1.5]),
    ((17, 29, 45), list(np.linspace(-1.6, 1.6, 15)) + [0.25]),
    ((25, 16, 40), [0.25, -0.75, 0.25, 1.0, -0.75]),
]


@pytest.mark.parametrize("case", range(len(_TRANSLATE_CASES)))
@pytest.mark.parametrize("acc", [1.0, 0.99, 0.8])
def test_translate_tiles_and_isovalue_counts(case, acc):
    shape, K = _TRANSLATE_CASES[case]
    f = synth.turbulence(shape, seed=200 + case)
    f = (f / np.abs(f).max() * 1.7).astype(np.float32)
    eb_o, n_o = oracle.translate_eb(f, K, acc)
    eb_g, n_g = chr.chr_topo_translate(_dev(f), [float(k) for k in K], acc)
    assert n_g == n_o
    assert np.float32(eb_g).view(np.uint32) == np.float32(eb_o).view(np.uint32)


@pytest.mark.parametrize("acc", [1.0, 0.5, 0.2, 0.05])
def test_translate_values_on_isovalues_and_non_finite(acc):
    # an integer field with integer isovalues: many ends equal an isovalue
    # (no crossing there: both inequalities are strict), D holds the small
    # integers, each accuracy picks another; then NaN (never crosses) and
    # -inf / +inf ends (d = +inf or a finite difference; at 0.05 the rank
    # falls among the +inf elements)
    rng = np.random.default_rng(9)
    f = rng.integers(-3, 4, size=(23, 19, 37)).astype(np.float32)
    K = [-2.0, 0.0, 1.0, 3.0]
    for g in (f, f.copy()):
        if g is not f:
            g.ravel()[::53] = np.nan
            g.ravel()[7::61] = np.inf
            g.ravel()[11::67] = -np.inf
        eb_o, n_o = oracle.translate_eb(g, K, acc)
        eb_g, n_g = chr.chr_topo_translate(_dev(g), K, acc)
        assert n_g == n_o
        assert np.float32(eb_g).view(np.uint32) == np.float32(eb_o).view(np.uint32)


@pytest.mark.parametrize("acc", [0.99, 0.95, 0.5, 0.05])
def test_translate_sampled_range_matches_oracle(acc):
    # large enough that the sampled walk sees thousands of elements, so the
    # n-th smallest comes from the range walk (the exact two walks are the
    # fallback); 4 isovalues
    f = synth.turbulence((96, 80, 112), seed=31)
    K = [-1.0, -0.5, 0.5, 1.0]
    eb_o, n_o = oracle.translate_eb(f, K, acc)
    eb_g, n_g = chr.chr_topo_translate(_dev(f), K, acc)
    assert n_g == n_o
    assert np.float32(eb_g).view(np.uint32) == np.float32(eb_o).view(np.uint32)


def test_translate_unrepresentative_sample_falls_back():
    # 16 tiles of 31 columns along x and one-plane z chunks: the sampled walk
    # (every 16th item) sees only the band x < 31, whose crossings are far
    # from the isovalue, while the rest of the field crosses it closely; the
    # range chosen from the sample misses rank n and the exact walks decide
    rng = np.random.default_rng(5)
    nz, ny, nx = 64, 15, 496
    f = (0.5 + 1e-3 * rng.standard_normal((nz, ny, nx))).astype(np.float32)
    band = np.where((np.indices((nz, ny, 31)).sum(axis=0) % 2) == 0, 5.0, -5.0).astype(np.float32)
    f[:, :, :31] = band + rng.uniform(-0.5, 0.5, (nz, ny, 31)).astype(np.float32)
    K = [0.5]
    for acc in (0.95, 0.5):
        eb_o, n_o = oracle.translate_eb(f, K, acc)
        eb_g, n_g = chr.chr_topo_translate(_dev(f), K, acc)
        assert n_g == n_o
        assert np.float32(eb_g).view(np.uint32) == np.float32(eb_o).view(np.uint32)


def test_compress_translate_mode_matches_oracle():
    f = synth.turbulence(36, seed=77)
    K = [-0.5, 0.5]
    eb_user = np.array([0.05, 0.005], np.float32)
    h = chr.chr_compress(_dev(f), eb_user, K, topo="translate", accuracy=0.95)
    eb_t, _ = oracle.translate_eb(f, K, 0.95)
    eff = np.minimum(eb_user, np.float32(eb_t)).astype(np.float32)
    st = h.stats()
    assert np.array_equal(np.array(st["eb"], np.float32), eff)
    enc = oracle.encode(f, eff, [], fix=False)
    _compare_codec(h, enc, f, "translate")


def test_sign_preservation_on_gpu_output():
    # topology preservation (Sec. 2.2): every case byte of every candidate
    # isovalue is unchanged at every level, so meshes have identical counts
    f = synth.turbulence(48, seed=31)
    r = synth.value_range(f)
    K = [-1.0, -0.5, 0.5, 1.0]
    h = chr.chr_compress(_dev(f), [1e-2 * r, 1e-3 * r, 1e-4 * r], K)
    _, counts_f, _ = _extract(f, K)
    for l in range(3):
        R = h.reconstruct(l)
        for k in K:
            assert torch.equal(R < k, _dev(f) < k)
        err = (R.double() - _dev(f).double()).abs().max().item()
        assert err < float(np.float32([1e-2 * r, 1e-3 * r, 1e-4 * r][l]))
        _, counts_r, _ = _extract(R.cpu().numpy(), K)
        assert np.array_equal(counts_r, counts_f)


def test_unaligned_views_take_the_scalar_paths():
    # a field that starts 4 bytes into its allocation (not 16-byte aligned)
    f = synth.turbulence((24, 20, 36), seed=41)
    K = [-0.5, 0.5]
    big = torch.zeros(f.size + 1, dtype=torch.float32, device="cuda")
    big[1:] = torch.from_numpy(f.ravel()).cuda()
    fv = big[1:].view(f.shape)
    assert fv.data_ptr() % 16 != 0
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1) + 1  # odd: isovalue 1 starts at an unaligned address
    tris, counts, err = chr.isosurface_extract(fv, K, cap)
    torch.cuda.synchronize()
    for j, k in enumerate(K):
        mesh = oracle.mc(f, k)
        assert int(counts[j]) == mesh.ntri
        compare_mesh(tris[j, :mesh.ntri].cpu().numpy(), mesh, (nx, ny, nz), f"unaligned k={k}")
    r = synth.value_range(f)
    eb = np.array([1e-2 * r, 1e-3 * r], np.float32)
    h = chr.chr_compress(fv, eb, K)
    enc = oracle.encode(f, eb, K)
    out_big = torch.zeros(f.size + 1, dtype=torch.float32, device="cuda")
    out = out_big[1:].view(f.shape)
    h.reconstruct(1, out)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), enc.R[1].view(np.uint32))

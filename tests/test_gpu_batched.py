"""The batched launch sequence (chr_batch_*): every item's decoded field and
triangles equal, bit for bit, those of chr_reconstruct + isosurface_extract
of that item alone, which the oracle checks in turn; the graph and direct
launches agree; autotuning changes no result; overflow is reported; and the
full 256-box workload matches the per-box path box by box."""
import numpy as np
import pytest
import torch

import oracle
from helpers import compare_mesh
from paper_2408_05462_gb300 import batched, chr, synth
from paper_2408_05462_gb300 import build as chr_build

pytestmark = pytest.mark.gpu

CHR_ERR_OVERFLOW = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()


def _alone(h, level, k):
    R = h.reconstruct(level)
    cap = 5 * int(np.prod([s - 1 for s in R.shape])) + 16
    tris, counts, err = chr.isosurface_extract(R, [k], cap)
    torch.cuda.synchronize()
    n = int(counts[0])
    return R.cpu().numpy(), tris[0, :n].cpu().numpy()


@pytest.fixture(scope="module")
def small():
    # ragged sizes, a few smaller than one tile or brick, odd pitches
    sizes = [(9, 9, 9), (33, 17, 40), (70, 13, 21), (2, 5, 3), (64, 64, 8), (31, 45, 29), (41, 2, 19), (16, 70, 33),
             (50, 50, 50), (3, 3, 90), (17, 31, 9), (66, 35, 12)]
    items, fields = [], []
    for i, s in enumerate(sizes):
        f = synth.turbulence(s, seed=100 + i) if i % 2 else synth.gaussian_blobs(s, seed=200 + i)
        lo, hi = float(f.min()), float(f.max())
        k = float(np.float32(lo + (0.3 + 0.04 * i) * (hi - lo)))
        ebs = [1e-2 * (hi - lo), 1e-3 * (hi - lo)]
        h = chr.chr_compress(torch.from_numpy(f).cuda(), ebs, [k])
        items.append((h, i % 2, k))
        fields.append((f, ebs))
    return items, fields


def test_items_match_the_single_box_path(small):
    items, _ = small
    b = batched.make_batch(items)
    b.run()
    torch.cuda.synchronize()
    assert int(b.err.item()) == 0
    for i, (h, level, k) in enumerate(items):
        R, tris = _alone(h, level, k)
        F = b.field(i).cpu().numpy()
        assert np.array_equal(F.view(np.uint32), R.view(np.uint32)), i
        got = b.triangles(i).cpu().numpy()
        assert got.shape == tris.shape, (i, got.shape, tris.shape)
        assert np.array_equal(got.view(np.uint32), tris.view(np.uint32)), i


def test_items_match_the_oracle(small):
    items, fields = small
    b = batched.make_batch(items)
    b.run()
    for i in (1, 2, 5, 8, 11):
        h, level, k = items[i]
        f, ebs = fields[i]
        enc = oracle.encode(f, ebs, [k], fix=True)
        R = oracle.decode(enc, level)
        assert np.array_equal(b.field(i).cpu().numpy().view(np.uint32), R.view(np.uint32)), i
        nz, ny, nx = f.shape
        compare_mesh(b.triangles(i).cpu().numpy(), oracle.mc(R, k), (nx, ny, nz), "item %d" % i)


def test_graph_direct_and_tuned_agree(small):
    items, _ = small
    b = batched.make_batch(items)
    b.run()
    ref_t, ref_s = b.tris.clone(), b.box_start.clone()
    for cfg in ({"use_graph": 0}, {"count_blocks_per_sm": 1, "emit_blocks_per_sm": 1, "use_graph": 1},
                {"count_blocks_per_sm": 99, "emit_blocks_per_sm": 2, "use_graph": 0},
                {"decode_warps_per_block": 4, "use_graph": 1}, {"decode_warps_per_block": 4, "use_graph": 0}):
        b.config = cfg
        b.tris.zero_()
        b.run()
        assert torch.equal(b.box_start, ref_s)
        assert torch.equal(b.tris.view(torch.int32), ref_t.view(torch.int32))
    c = b.config
    assert 1 <= c["count_blocks_per_sm"] and 1 <= c["emit_blocks_per_sm"] and c["decode_warps_per_block"] == 4
    tuned = b.autotune(reps=2)
    assert tuned == b.config
    b.run()
    assert torch.equal(b.tris.view(torch.int32), ref_t.view(torch.int32))
    # a second batch of the same mix starts from the tuned configuration
    b2 = chr.Batch(items, 16)
    assert b2.config == tuned


def test_overflow_is_reported(small):
    items, _ = small
    full = batched.make_batch(items)
    full.run()
    total = int(full.box_start[-1].item())
    cap = total // 3
    b = chr.Batch(items, cap)
    b.run()
    torch.cuda.synchronize()
    assert int(b.err.item()) & (1 << CHR_ERR_OVERFLOW)
    assert torch.equal(b.box_start, full.box_start)
    assert torch.equal(b.tris[:cap].view(torch.int32), full.tris[:cap].view(torch.int32))


def test_bad_items_are_rejected(small):
    items, _ = small
    h = items[0][0]
    with pytest.raises(chr.ChrError):
        chr.Batch([(h, 5, 0.0)], 16)
    with pytest.raises(chr.ChrError):
        chr.Batch([], 16)


def test_full_workload_matches_per_box():
    specs = batched.make_specs(256, 256)
    items, fields = batched.build_items(specs)
    b = batched.make_batch(items)
    b.autotune(reps=2)
    b.run()
    torch.cuda.synchronize()
    assert int(b.err.item()) == 0
    bs = b.box_start.cpu().numpy()
    plain = batched.PlainPath(items, np.diff(bs))
    plain.run()
    torch.cuda.synchronize()
    assert np.array_equal(plain.counts.cpu().numpy(), np.diff(bs))
    for i in range(len(items)):
        n = int(bs[i + 1] - bs[i])
        assert torch.equal(b.tris[bs[i]:bs[i + 1]].view(torch.int32), plain.tris[i][0, :n].view(torch.int32)), i
    # the oracle on the smallest boxes of the batch
    small = sorted(range(len(specs)), key=lambda i: np.prod(specs[i].size))[:3]
    for i in small:
        h, level, k = items[i]
        f = fields[i]
        _, eb = batched.box_params(specs[i], f)
        R = oracle.decode(oracle.encode(f, [eb], [k], fix=True), 0)
        assert np.array_equal(b.field(i).cpu().numpy().view(np.uint32), R.view(np.uint32)), i
        nz, ny, nx = f.shape
        compare_mesh(b.triangles(i).cpu().numpy(), oracle.mc(R, k), (nx, ny, nz), "box %d" % i)

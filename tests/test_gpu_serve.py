"""The serving path on the GPU: chr_reconstruct_box against the crop of the
full reconstruction (bit-exact), chr_brick_range against the brick extrema
of the reconstruction, one served request against the oracle, and every
request's result identical when served alone and in a mix of concurrent
requests (counts and triangles bit for bit)."""
import numpy as np
import pytest
import torch

import oracle
from helpers import compare_mesh
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, serve, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()


def _field():
    return synth.turbulence((83, 70, 61), seed=31)  # ragged in every axis


@pytest.fixture(scope="module")
def handle():
    f = _field()
    rng = float(f.max() - f.min())
    h = chr.chr_compress(torch.from_numpy(f).cuda(), [r * rng for r in serve.LEVELS_REL], serve.FIX_ISOVALUES)
    return f, h


BOXES = [((0, 0, 0), (83, 70, 61)), ((0, 0, 0), (1, 1, 1)), ((82, 69, 60), (1, 1, 1)), ((3, 5, 7), (64, 33, 17)),
         ((8, 16, 24), (64, 32, 16)), ((9, 1, 2), (70, 69, 59)), ((40, 0, 30), (2, 70, 2)), ((77, 13, 0), (6, 9, 61))]


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_reconstruct_box_is_the_crop(handle, level):
    _, h = handle
    full = h.reconstruct(level).cpu().numpy()
    for (o, s) in BOXES:
        got = h.reconstruct_box(level, o, s).cpu().numpy()
        ref = full[o[2]:o[2] + s[2], o[1]:o[1] + s[1], o[0]:o[0] + s[0]]
        assert got.shape == ref.shape
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (level, o, s)


def test_reconstruct_box_rejects_bad_boxes(handle):
    _, h = handle
    for (o, s) in [((0, 0, 0), (84, 70, 61)), ((-1, 0, 0), (4, 4, 4)), ((0, 0, 60), (4, 4, 2)), ((0, 0, 0), (0, 4, 4))]:
        with pytest.raises((chr.ChrError, ValueError, RuntimeError)):
            h.reconstruct_box(0, o, s)
    with pytest.raises(chr.ChrError):
        h.reconstruct_box(4, (0, 0, 0), (8, 8, 8))


def test_brick_range_is_the_brick_extrema(handle):
    _, h = handle
    for level in range(4):
        R = h.reconstruct(level).cpu().numpy()
        got = h.brick_range(level).cpu().numpy()
        nz, ny, nx = R.shape
        assert got.shape == ((nz + 7) // 8, (ny + 7) // 8, (nx + 7) // 8, 2)
        for bz in range(got.shape[0]):
            for by in range(got.shape[1]):
                for bx in range(got.shape[2]):
                    blk = R[8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
                    assert got[bz, by, bx, 0] == blk.min() and got[bz, by, bx, 1] == blk.max()


def test_serve_request_equals_the_box_path(handle):
    # one call (pitched box field, tensor-map marching cubes) against
    # chr_reconstruct_box + isosurface_extract (dense box) of the same box
    _, h = handle
    result = torch.zeros(2, dtype=torch.int64, pin_memory=True)
    for (o, s), level, k in [(((3, 5, 7), (64, 33, 17)), 0, 0.1), (((9, 1, 2), (70, 69, 59)), 3, -0.4),
                             (((0, 0, 0), (83, 70, 61)), 2, 0.8), (((40, 0, 30), (2, 70, 2)), 1, 0.0),
                             (((77, 13, 0), (6, 9, 61)), 0, -1.0)]:
        box = h.reconstruct_box(level, o, s)
        cap = 5 * (s[0] - 1) * (s[1] - 1) * (s[2] - 1) + 8
        tris, counts, err = chr.isosurface_extract(box, [k], cap)
        mem = torch.empty(chr.chr_serve_request_bytes(s, cap), dtype=torch.uint8, device="cuda")
        chr.chr_serve_request(h, level, o, s, k, mem, cap, result)
        torch.cuda.synchronize()
        n = int(counts[0])
        assert int(result[0]) == n and int(result[1]) == 0 and int(err.item()) == 0
        got = mem[:36 * n].view(torch.int32)
        assert torch.equal(got, tris[0, :n].reshape(-1).view(torch.int32)), (o, s, level, k)
    with pytest.raises(chr.ChrError):
        chr.chr_serve_request(h, 0, (80, 0, 0), (8, 8, 8), 0.0, mem, 16, result)


def _server(f, slots):
    srv = serve.Server(budget_bytes=8 << 30, slots=slots, max_resident=2)
    fd = torch.from_numpy(f).cuda()
    srv.ingest(0, fd)
    srv.ingest(1, torch.roll(fd, shifts=(1, 2, 3), dims=(0, 1, 2)).contiguous())
    return srv


def test_served_request_matches_the_oracle():
    f = synth.turbulence((70, 66, 52), seed=32)
    srv = _server(f, 2)
    reqs = [serve.Request(0, 0.0, 0, 0.37, 1, (5, 9, 3), (61, 40, 44)),
            serve.Request(1, 0.0, 1, -0.8, 3, (0, 0, 0), (70, 66, 52))]
    res = srv.run(reqs, keep_results=True)
    rng = float(f.max() - f.min())
    for r, q in zip(res, reqs):
        src = f if q.step == 0 else np.roll(f, shift=(1, 2, 3), axis=(0, 1, 2))
        enc = oracle.encode(src, [e * rng for e in serve.LEVELS_REL], serve.FIX_ISOVALUES, fix=True)
        R = oracle.decode(enc, q.level)
        (x0, y0, z0), (bx, by, bz) = q.origin, q.size
        box = np.ascontiguousarray(R[z0:z0 + bz, y0:y0 + by, x0:x0 + bx])
        mesh = oracle.mc(box, q.k)
        assert r.ntris == mesh.ntri <= r.bound
        compare_mesh(r.tris.cpu().numpy(), mesh, (bx, by, bz), "request %d" % q.rid)


def test_results_identical_alone_and_in_the_mix():
    f = synth.turbulence(96, seed=33)
    srv = _server(f, 4)
    reqs = serve.make_requests(48, 0.0, (96, 96, 96), [0, 1], seed=5, side=(16, 96))
    mixed = srv.run(reqs, keep_results=True)
    # the same requests again, now arriving spread out so the overlap differs
    spread = [serve.Request(r.rid, 0.0005 * i, r.step, r.k, r.level, r.origin, r.size) for i, r in enumerate(reqs)]
    mixed2 = srv.run(spread, keep_results=True)
    alone_srv = srv.with_slots(1)
    for r, m, m2 in zip(reqs, mixed, mixed2):
        (a,) = alone_srv.run([serve.Request(r.rid, 0.0, r.step, r.k, r.level, r.origin, r.size)], keep_results=True)
        assert a.ntris == m.ntris == m2.ntris and a.ntris <= a.bound
        ta, tm, tm2 = (x.tris.cpu().numpy() for x in (a, m, m2))
        assert np.array_equal(ta.view(np.uint32), tm.view(np.uint32)), r.rid
        assert np.array_equal(ta.view(np.uint32), tm2.view(np.uint32)), r.rid
    assert sum(m.ntris for m in mixed) > 0


def test_admission_respects_the_budget():
    f = synth.turbulence(64, seed=34)
    srv = _server(f, 4)
    reqs = serve.make_requests(24, 0.0, (64, 64, 64), [0, 1], seed=9, side=(32, 64))
    need = [srv.request_bytes(r, srv.steps[r.step].tri_bound(r.level, r.k, r.origin, r.size)) for r in reqs]
    tight = srv.with_slots(4)
    tight.budget = max(need)  # one request at a time fits
    res = tight.run(reqs)
    # at every admission the requests then in flight fit the budget together
    for b in res:
        inflight = [a for a in res if a.admit_ms <= b.admit_ms < a.retire_ms]
        assert sum(a.nbytes for a in inflight) <= tight.budget
    assert max(len([a for a in res if a.admit_ms <= b.admit_ms < a.retire_ms]) for b in res) <= 4
    big = serve.Request(99, 0.0, 0, 0.0, 0, (0, 0, 0), (64, 64, 64))
    tight.budget = 1 << 20
    with pytest.raises(MemoryError):
        tight.run([big])

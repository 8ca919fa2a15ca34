"""Parity at the benchmark's full size and launch configuration: a 512^3
turbulence field (seed 512), isovalues {-1, -0.5, 0.5, 1}, bounds
{1e-2, 1e-3, 1e-4} x range, 3 levels, topology fix — exactly what bench.py
times.

The oracle is too slow for the whole grid, so it checks sampled 8^3 bricks
one by one (the codec and the marching cubes are brick-local), and properties
that hold at any size are checked over every vertex and cell:
prefix sums of the records, the strict error bound, sign agreement for every
candidate isovalue, and exact triangle totals."""
import math

import numpy as np
import pytest
import torch

import oracle
from helpers import vertex_tol
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, synth

pytestmark = pytest.mark.gpu

N_SIDE = 512
ISO = [-1.0, -0.5, 0.5, 1.0]
REL = [1e-2, 1e-3, 1e-4]


@pytest.fixture(scope="module")
def run():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()
    f = synth.turbulence(N_SIDE, seed=512)
    r = synth.value_range(f)
    eb = np.array([b * r for b in REL], np.float32)
    fd = torch.from_numpy(f).cuda()
    h = chr.chr_compress(fd, eb, ISO)
    R = h.reconstruct(2)
    _, counts, err = chr.isosurface_extract(R, ISO, 0)
    torch.cuda.synchronize()
    cap = int(counts.max().item()) + 16
    tris, counts, err = chr.isosurface_extract(R, ISO, cap)
    torch.cuda.synchronize()
    parsed = chr.parse_serialized(chr.chr_serialize(h))
    return dict(f=f, fd=fd, eb=eb, h=h, R=R, tris=tris, counts=counts.cpu().numpy(), err=int(err.item()),
                parsed=parsed)


def _sample_bricks(nb, count, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    picks = set(int(v) for v in g.integers(0, nb ** 3, size=count))
    picks |= {0, nb ** 3 - 1, nb - 1, nb * nb - 1}  # corners of the grid
    return sorted(picks)


def test_records_are_prefix_sums(run):
    for lv in run["parsed"]["levels"]:
        rec = lv["recs"].astype(np.int64)
        w = rec[:, 3] & 0xFF
        ne = rec[:, 3] >> 16
        assert np.array_equal(rec[:, 0], np.concatenate([[0], np.cumsum(w)[:-1]]))
        assert np.array_equal(rec[:, 1], np.concatenate([[0], np.cumsum(ne)[:-1]]))
        assert lv["words"].size == 16 * w.sum() and lv["exc_idx"].size == ne.sum()


def test_sampled_bricks_match_oracle(run):
    f, eb, parsed = run["f"], run["eb"], run["parsed"]
    nb = N_SIDE // 8
    for b in _sample_bricks(nb, 48, 1):
        bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
        sub = np.ascontiguousarray(f[8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8])
        enc = oracle.encode(sub, eb, ISO, fix=True)
        for l in range(3):
            lv = parsed["levels"][l]
            rec = lv["recs"][b]
            ref = enc.recs[l][0]
            assert np.array_equal(rec[2:], ref[2:]), (b, l)  # anchor, width | mode | count
            w = int(rec[3] & 0xFF)
            assert np.array_equal(lv["words"][16 * rec[0]:16 * rec[0] + 16 * w], enc.words[l]), (b, l)
            ne = int(rec[3] >> 16)
            assert np.array_equal(lv["exc_idx"][rec[1]:rec[1] + ne], enc.exc_idx[l]), (b, l)
            assert np.array_equal(lv["exc_val"][rec[1]:rec[1] + ne], enc.exc_val[l]), (b, l)
        dec = run["R"][8 * bz:8 * bz + 8, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8].cpu().numpy()
        assert np.array_equal(dec.view(np.uint32), enc.R[2].view(np.uint32)), b


def test_bound_and_signs_everywhere(run):
    fd, R, eb = run["fd"], run["R"], run["eb"]
    h = run["h"]
    for l in range(3):
        Rl = R if l == 2 else h.reconstruct(l)
        err = (Rl.double() - fd.double()).abs().max().item()
        assert err < float(eb[l]), (l, err)
        for k in ISO:
            assert torch.equal(Rl < k, fd < k), (l, k)


def _cell_cases(F, k):
    """Case byte of every cell (bit j = corner j below k), as uint8 on the GPU."""
    b = (F < k).to(torch.uint8)
    c = torch.zeros((F.shape[0] - 1, F.shape[1] - 1, F.shape[2] - 1), dtype=torch.uint8, device=F.device)
    for j in range(8):
        ox, oy, oz = j & 1, (j >> 1) & 1, (j >> 2) & 1
        c |= b[oz:oz + c.shape[0], oy:oy + c.shape[1], ox:ox + c.shape[2]] << j
    return c


def test_triangle_totals_and_sampled_triangles(run):
    R, tris, counts = run["R"], run["tris"], run["counts"]
    assert run["err"] == 0
    ntab = torch.tensor([oracle.cell_triangles(c).shape[0] for c in range(256)], dtype=torch.int64, device="cuda")
    Rh = R.cpu().numpy()
    nb = math.ceil((N_SIDE - 1) / 8)
    for j, k in enumerate(ISO):
        cases = _cell_cases(R, np.float32(k))
        per_cell = ntab[cases.long()]
        assert int(per_cell.sum().item()) == int(counts[j]), k
        # triangles per 8^3 cell brick, brick-major, for the offsets of sampled bricks
        pc = torch.nn.functional.pad(per_cell, (0, 8 * nb - per_cell.shape[2], 0, 8 * nb - per_cell.shape[1],
                                                0, 8 * nb - per_cell.shape[0]))
        per_brick = pc.view(nb, 8, nb, 8, nb, 8).sum(dim=(1, 3, 5)).flatten()
        start = torch.cumsum(per_brick, 0) - per_brick
        del cases, per_cell, pc
        for b in _sample_bricks(nb, 24, 2 + j):
            bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
            sub = np.ascontiguousarray(Rh[8 * bz:8 * bz + 9, 8 * by:8 * by + 9, 8 * bx:8 * bx + 9])
            mesh = oracle.mc(sub, k)
            n = int(per_brick[b].item())
            assert mesh.ntri == n, (k, b)
            if n == 0:
                continue
            s0 = int(start[b].item())
            got = tris[j, s0:s0 + n].cpu().numpy().astype(np.float64)
            ref = mesh.pos + np.array([8 * bx, 8 * by, 8 * bz], np.float64)
            assert np.all(np.abs(got - ref) <= vertex_tol(ref)), (k, b)


def test_translate_count_at_full_size(run):
    fd = run["fd"]
    eb, n = chr.chr_topo_translate(fd, ISO, 0.95)
    total = 0
    for k in ISO:
        for dim in range(3):
            a = fd.narrow(dim, 0, N_SIDE - 1)
            b = fd.narrow(dim, 1, N_SIDE - 1)
            lo, hi = torch.minimum(a, b), torch.maximum(a, b)
            total += 2 * int(((lo < k) & (k < hi)).sum().item())
    assert n == total
    assert 0.0 < eb < 1.0

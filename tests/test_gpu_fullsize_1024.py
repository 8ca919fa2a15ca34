"""Parity at the serving configuration's size: a 1024^3 turbulence timestep
(the GPU generator, seed 1024), 4 levels at {1e-2, 1e-3, 1e-4, 1e-5} x range,
the 4 candidate isovalues sign-fixed — the CHR the request loop serves and the
bench decodes and meshes whole.

As at 512^3, the oracle checks sampled 8^3 bricks one by one (codec and
marching cubes are brick-local) and properties that hold at any size are
checked over every vertex and cell on the GPU: the strict error bound and
sign agreement at every level, exact triangle totals per isovalue."""
import numpy as np
import pytest
import torch

import oracle
from helpers import vertex_tol
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, serve, synth
from test_gpu_fullsize import _cell_cases, _sample_bricks

pytestmark = pytest.mark.gpu

N_SIDE = 1024
ISO = list(serve.FIX_ISOVALUES)


@pytest.fixture(scope="module")
def run():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()
    fd = synth.turbulence_cuda(N_SIDE, seed=1024)
    lo, hi = torch.aminmax(fd)
    r = float(hi) - float(lo)
    eb = np.array([e * r for e in serve.LEVELS_REL], np.float32)
    h = chr.chr_compress(fd, eb, ISO)
    parsed = chr.parse_serialized(chr.chr_serialize(h))
    yield dict(fd=fd, eb=eb, h=h, parsed=parsed)
    h.free()


def test_bound_and_signs_everywhere(run):
    fd, eb, h = run["fd"], run["eb"], run["h"]
    for l in range(len(eb)):
        R = h.reconstruct(l)
        err = max((R[z:z + 128].double() - fd[z:z + 128].double()).abs().max().item() for z in range(0, N_SIDE, 128))
        assert err < float(eb[l]), (l, err)
        for k in ISO:
            assert torch.equal(R < k, fd < k), (l, k)
        del R


def test_sampled_bricks_match_oracle(run):
    fd, eb, parsed, h = run["fd"], run["eb"], run["parsed"], run["h"]
    nb = N_SIDE // 8
    R3 = h.reconstruct(3)
    for b in _sample_bricks(nb, 32, 11):
        bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
        sl = (slice(8 * bz, 8 * bz + 8), slice(8 * by, 8 * by + 8), slice(8 * bx, 8 * bx + 8))
        sub = np.ascontiguousarray(fd[sl].cpu().numpy())
        enc = oracle.encode(sub, eb, ISO, fix=True)
        for l in range(len(eb)):
            lv = parsed["levels"][l]
            rec = lv["recs"][b]
            assert np.array_equal(rec[2:], enc.recs[l][0][2:]), (b, l)
            w = int(rec[3] & 0xFF)
            assert np.array_equal(lv["words"][16 * rec[0]:16 * rec[0] + 16 * w], enc.words[l]), (b, l)
            ne = int(rec[3] >> 16)
            assert np.array_equal(lv["exc_idx"][rec[1]:rec[1] + ne], enc.exc_idx[l]), (b, l)
            assert np.array_equal(lv["exc_val"][rec[1]:rec[1] + ne], enc.exc_val[l]), (b, l)
        dec = R3[sl].cpu().numpy()
        assert np.array_equal(dec.view(np.uint32), enc.R[3].view(np.uint32)), b


def test_triangle_totals_and_sampled_triangles(run):
    h = run["h"]
    R = h.reconstruct(2)
    _, counts, err = chr.isosurface_extract(R, ISO, 0)
    torch.cuda.synchronize()
    cap = int(counts.max().item()) + 16
    tris, counts, err = chr.isosurface_extract(R, ISO, cap)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ntab = torch.tensor([oracle.cell_triangles(c).shape[0] for c in range(256)], dtype=torch.uint8, device="cuda")
    nb = (N_SIDE - 1 + 7) // 8
    for j, k in enumerate(ISO):
        cases = _cell_cases(R, np.float32(k))
        per_cell = ntab[cases.long()]
        del cases
        assert int(per_cell.sum(dtype=torch.int64).item()) == int(counts[j]), k
        pc = torch.nn.functional.pad(per_cell, (0, 8 * nb - per_cell.shape[2], 0, 8 * nb - per_cell.shape[1],
                                                0, 8 * nb - per_cell.shape[0]))
        del per_cell
        per_brick = pc.view(nb, 8, nb, 8, nb, 8).sum(dim=(1, 3, 5), dtype=torch.int64).flatten()
        del pc
        start = torch.cumsum(per_brick, 0) - per_brick
        for b in _sample_bricks(nb, 12, 20 + j):
            bx, by, bz = b % nb, (b // nb) % nb, b // (nb * nb)
            sub = np.ascontiguousarray(R[8 * bz:8 * bz + 9, 8 * by:8 * by + 9, 8 * bx:8 * bx + 9].cpu().numpy())
            mesh = oracle.mc(sub, k)
            n = int(per_brick[b].item())
            assert mesh.ntri == n, (k, b)
            if n == 0:
                continue
            s0 = int(start[b].item())
            got = tris[j, s0:s0 + n].cpu().numpy().astype(np.float64)
            ref = mesh.pos + np.array([8 * bx, 8 * by, 8 * bz], np.float64)
            assert np.all(np.abs(got - ref) <= vertex_tol(ref)), (k, b)

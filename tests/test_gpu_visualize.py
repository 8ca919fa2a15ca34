"""chr_isosurface: the visualization side's decode and marching cubes in one
call (Sec. 2) must equal chr_reconstruct followed by isosurface_extract, bit
for bit, whether the decoded field is kept or left in scratch, at every
level; the oracle's mesh of the decoded field; and overflow reported the way
isosurface_extract reports it."""
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


def test_one_call_equals_reconstruct_then_extract():
    f = synth.turbulence((45, 38, 70), seed=17)
    r = synth.value_range(f)
    K = [-0.5, 0.25, 0.9]
    h = chr.chr_compress(torch.from_numpy(f).cuda(), [1e-2 * r, 1e-3 * r], K)
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
    for level in range(2):
        R = h.reconstruct(level)
        t0, c0, e0 = chr.isosurface_extract(R, K, cap)
        keep = torch.full_like(R, float("nan"))
        t1, c1, e1 = chr.chr_isosurface(h, level, K, cap, field_out=keep)
        t2, c2, e2 = h.isosurface(level, K, cap)
        torch.cuda.synchronize()
        assert int(e0.item()) == 0
        assert torch.equal(_bits(keep), _bits(R))
        for t, c, e in ((t1, c1, e1), (t2, c2, e2)):
            assert int(e.item()) == 0
            assert torch.equal(c, c0)
            for j in range(len(K)):
                n = int(c0[j])
                assert torch.equal(_bits(t[j, :n]), _bits(t0[j, :n])), (level, j)
    # the sign fix keeps every case byte, so the counts are the original
    # field's; the positions are those of the decoded field
    Rh = h.reconstruct(1).cpu().numpy()
    t, c, e = chr.chr_isosurface(h, 1, K, cap)
    torch.cuda.synchronize()
    for j, k in enumerate(K):
        mesh = oracle.mc(Rh, k)
        assert int(c[j]) == mesh.ntri == oracle.mc_count(f, k)
        compare_mesh(t[j, :mesh.ntri].cpu().numpy(), mesh, (nx, ny, nz), f"k={k}")
    h.free()


def test_overflow_and_bad_arguments():
    f = synth.turbulence(32, seed=5)
    r = synth.value_range(f)
    h = chr.chr_compress(torch.from_numpy(f).cuda(), [1e-2 * r], [0.0])
    _, c, e = chr.chr_isosurface(h, 0, [0.0], 0)
    torch.cuda.synchronize()
    n = int(c[0])
    assert n > 0
    cap = n // 2
    t, c2, e2 = chr.chr_isosurface(h, 0, [0.0], cap)
    full, _, _ = chr.chr_isosurface(h, 0, [0.0], n)
    torch.cuda.synchronize()
    assert int(c2[0]) == n
    assert int(e2.item()) & chr.ERR_OVERFLOW_BIT
    assert torch.equal(_bits(t[0]), _bits(full[0, :cap]))
    with pytest.raises(chr.ChrError):
        chr.chr_isosurface(h, 1, [0.0], 10)  # one level only
    with pytest.raises(chr.ChrError):
        chr.chr_isosurface(h, 0, [float("nan")], 10)
    with pytest.raises(chr.ChrError):
        chr.chr_isosurface(h, 0, [], 10)
    h.free()

"""A wait that runs out, on the GPU, without a fault: the single-pass
extraction's look-back waits for the tiles before it to publish their
triangle counts.  The test-only variable CHR_TEST_UNPUBLISHED_TILE makes one
tile publish nothing; the tiles after it must give up after their bounded
spin (about a second), the call must report CHR_ERR_TIMEOUT in its error
word (every write still inside the output buffer), and the next call,
without the variable, must be right: the context stays usable."""
import time

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


@pytest.mark.parametrize("tile", [0, 3])
def test_lookback_wait_gives_up_and_the_context_stays_usable(monkeypatch, tile):
    f = synth.turbulence((130, 66, 34), seed=4)  # 5 x 9 x 5 = 225 tiles of 32x8x8 cells: the single pass
    fd = torch.from_numpy(f).cuda()
    isos = [-1.0, -0.5, 0.5, 1.0]
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
    guard = 1 << 12
    buf = torch.full((len(isos) * cap * 9 + guard,), 7.0, dtype=torch.float32, device="cuda")
    tris = buf[:len(isos) * cap * 9].view(len(isos), cap, 3, 3)
    monkeypatch.setenv("CHR_TEST_UNPUBLISHED_TILE", str(tile))
    t0 = time.perf_counter()
    _, _, err = chr.isosurface_extract(fd, isos, cap, tris=tris)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert int(err.item()) & chr.ERR_TIMEOUT_BIT
    assert waited < 60.0
    assert torch.all(buf[len(isos) * cap * 9:] == 7.0)  # nothing written past the buffer
    monkeypatch.delenv("CHR_TEST_UNPUBLISHED_TILE")
    tris2, counts, err2 = chr.isosurface_extract(fd, isos, cap)
    torch.cuda.synchronize()
    assert int(err2.item()) == 0
    t = tris2.cpu().numpy()
    for j, k in enumerate(isos):
        mesh = oracle.mc(f, k)
        assert int(counts[j]) == mesh.ntri, k
        compare_mesh(t[j, :mesh.ntri], mesh, (nx, ny, nz), f"after timeout k={k}")

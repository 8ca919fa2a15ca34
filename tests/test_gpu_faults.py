"""A wait that runs out, on the GPU, without a fault: the single-pass
extraction's look-back waits for the tiles before it to publish their
triangle counts.  In the checked build (the only one with this test hook),
chr_debug_unpublished_tile makes one tile publish nothing; the tiles after
it must give up after their bounded spin (about a second), the call must
report CHR_ERR_TIMEOUT in its error word (every write still inside the
output buffer), and the next call, with the hook cleared, must be right:
the context stays usable.  The release library refuses the hook.  Runs in
a process of its own (the checked library is loaded there)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys, time
root = sys.argv[1]
sys.path.insert(0, root)
sys.path.insert(0, os.path.join(root, "tests"))
import numpy as np
import torch
import oracle
from helpers import compare_mesh
from paper_2408_05462_gb300 import build, chr, synth

try:
    chr.chr_debug_unpublished_tile(3)
    raise SystemExit("the release library accepted the test hook")
except chr.ChrError:
    pass
chr.LIB_PATH = build.build(checked=True)
chr._lib = None
assert chr.chr_checked_build()

f = synth.turbulence((130, 66, 34), seed=4)  # 5 x 9 x 5 = 225 tiles of 32x8x8 cells: the single pass
fd = torch.from_numpy(f).cuda()
isos = [-1.0, -0.5, 0.5, 1.0]
nz, ny, nx = f.shape
cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
guard = 1 << 12
for tile in (0, 3):
    buf = torch.full((len(isos) * cap * 9 + guard,), 7.0, dtype=torch.float32, device="cuda")
    tris = buf[:len(isos) * cap * 9].view(len(isos), cap, 3, 3)
    chr.chr_debug_unpublished_tile(tile)
    t0 = time.perf_counter()
    _, _, err = chr.isosurface_extract(fd, isos, cap, tris=tris)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert int(err.item()) & chr.ERR_TIMEOUT_BIT, tile
    assert waited < 60.0
    assert torch.all(buf[len(isos) * cap * 9:] == 7.0)  # nothing written past the buffer
    chr.chr_debug_unpublished_tile(-1)
    tris2, counts, err2 = chr.isosurface_extract(fd, isos, cap)
    torch.cuda.synchronize()
    assert int(err2.item()) == 0
    t = tris2.cpu().numpy()
    for j, k in enumerate(isos):
        mesh = oracle.mc(f, k)
        assert int(counts[j]) == mesh.ntri, k
        compare_mesh(t[j, :mesh.ntri], mesh, (nx, ny, nz), f"after timeout k={k}")
print("timeout ok")
"""


def test_lookback_wait_gives_up_and_the_context_stays_usable():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "timeout ok" in r.stdout

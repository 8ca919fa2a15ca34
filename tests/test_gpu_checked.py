"""The bounds-checked library (build.build(checked=True): every
data-dependent shared-memory index and output range on the hot paths is
tested, and a failed test is recorded and the access skipped) runs the
codec at odd sizes with both topology modes, box and range decodes,
marching cubes for 1 to 6 isovalues with both workspaces, white noise that
overflows the shared active-cell pool, a grid past the two-pass threshold,
a batch of uneven boxes and the adjoint, in a process of its own; no index
may fail, and the results still match the oracle where checked."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
root = sys.argv[1]
sys.path.insert(0, root)
sys.path.insert(0, os.path.join(root, "tests"))
import numpy as np
import torch
import oracle
from paper_2408_05462_gb300 import batched, build, chr, synth

chr.LIB_PATH = build.build(checked=True)
chr._lib = None
assert chr.chr_checked_build()
chr.chr_debug_bounds_word(reset=True)

def dev(f):
    return torch.from_numpy(np.ascontiguousarray(f)).cuda()

# codec: odd sizes, FIX and TRANSLATE, every level, boxes and brick ranges
for shape, seed in (((37, 50, 65), 3), ((64, 48, 40), 5), ((2, 5, 3), 1), ((9, 33, 17), 7)):
    f = synth.turbulence(shape, seed=seed)
    r = synth.value_range(f)
    for topo in ("fix", "translate"):
        h = chr.chr_compress(dev(f), [1e-2 * r, 1e-3 * r, 1e-4 * r], [-0.5, 0.5, 1.0], topo=topo, accuracy=0.95)
        for l in range(3):
            R = h.reconstruct(l)
            chr.chr_brick_range(h, l)
        nx, ny, nz = shape
        chr.chr_reconstruct_box(h, 2, (nx // 3, ny // 4, nz // 5), (max(nx // 2, 1), max(ny // 2, 1), max(nz // 2, 1)))
        h2 = chr.chr_deserialize(chr.chr_serialize(h))
        h2.reconstruct(2)
        h2.free()
        h.free()

# marching cubes: 1..6 isovalues, both workspaces
f = synth.turbulence((70, 45, 33), seed=12)
fd = dev(f)
cap = 5 * 69 * 44 * 32
for isos in ([0.3], [-1.0, 0.5], [-1.0, -0.5, 0.5], [-1.0, -0.5, 0.5, 1.0], [-1.2, -0.6, 0.0, 0.2, 0.7, 1.1]):
    for size in (chr.isosurface_workspace_size, chr.isosurface_workspace_min_size):
        ws = torch.empty(size(f.shape, len(isos)), dtype=torch.uint8, device="cuda")
        t, c, e = chr.isosurface_extract(fd, isos, cap, workspace=ws)
        torch.cuda.synchronize()
        assert int(e.item()) == 0
        for j, k in enumerate(isos):
            assert int(c[j]) == oracle.mc(f, k).ntri, (isos, k)

# white noise at 4 isovalues: the slot-by-slot path
noise = synth.uniform_noise((20, 19, 70), 22)
t, c, e = chr.isosurface_extract(dev(noise), [-0.6, -0.2, 0.2, 0.6], 5 * 69 * 18 * 19)
torch.cuda.synchronize()
assert int(e.item()) == 0

# past the two-pass threshold at one isovalue
big = synth.turbulence((257, 129, 129), seed=31)
t, c, e = chr.isosurface_extract(dev(big), [0.3], 0)
torch.cuda.synchronize()
t, c, e = chr.isosurface_extract(dev(big), [0.3], int(c[0]) + 16)
torch.cuda.synchronize()
assert int(e.item()) == 0 and int(c[0]) == oracle.mc(big, 0.3).ntri

# a batch of uneven boxes
items, _ = batched.build_items(batched.make_specs(12, 7, 9, 70))
b = batched.make_batch(items)
b.run()
torch.cuda.synchronize()
assert int(b.err.item()) == 0

# the adjoint
g = torch.ones((1, cap, 3, 3), dtype=torch.float32, device="cuda")
chr.isosurface_backward(fd, [0.3], g, cap)
torch.cuda.synchronize()

w = chr.chr_debug_bounds_word()
assert w == 0, w
print("checked ok")
"""


def test_checked_build_sees_no_index_out_of_bounds():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout

"""The marching cubes' internal outputs against an oracle enumeration, bit for
bit, through the checked build's test outputs (in a process of its own):

* case bytes: the counting pass's case byte of every cell (chr_debug_cases)
  equals oracle.cases (paper Sec. 2.2: the case of each cell, which
  topology preservation keeps);
* active-cell lists: the cell of every emitted triangle, in output order
  (chr_debug_tri_cells), equals the oracle mesh's triangle cells reordered
  brick-major, and its run of distinct cells equals the oracle's active
  cells (case byte neither 0 nor 255) in the same order -- for the single
  pass, the two-pass form past its threshold, and chr_isosurface's forms.
"""
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
from helpers import brick_major_order
from paper_2408_05462_gb300 import build, chr, synth

chr.LIB_PATH = build.build(checked=True)
chr._lib = None
assert chr.chr_checked_build()

def dev(f):
    return torch.from_numpy(np.ascontiguousarray(f)).cuda()

def check_cells(cells, counts, fields, isos, dims, label):
    for j, k in enumerate(isos):
        mesh = oracle.mc(fields, k)
        n = int(counts[j])
        assert n == mesh.ntri, (label, k)
        got = cells[j, :n].cpu().numpy().astype(np.int64)
        want = mesh.cell[brick_major_order(mesh.cell, dims)]
        assert np.array_equal(got, want), (label, k)
        # the distinct cells in order: the oracle's active cells, brick-major
        c = oracle.cases(fields, k).reshape(-1)
        act = np.nonzero((c != 0) & (c != 255))[0]
        act = act[brick_major_order(act, dims)]
        runs = got[np.r_[True, got[1:] != got[:-1]]] if n else got
        assert np.array_equal(runs, act), (label, k)

for shape, seed, isos in (((37, 50, 65), 3, [-0.5, 0.5]), ((70, 45, 33), 12, [-1.0, -0.5, 0.5, 1.0, 0.1]),
                          ((9, 33, 17), 7, [0.0])):
    f = synth.turbulence(shape, seed=seed)
    fd = dev(f)
    nz, ny, nx = f.shape
    for k in isos:
        got = chr.chr_debug_cases(fd, k).cpu().numpy()
        assert np.array_equal(got, oracle.cases(f, k)), (shape, k)
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1)
    cells = torch.full((len(isos), cap), -1, dtype=torch.int32, device="cuda")
    chr.chr_debug_tri_cells(cells)
    _, counts, err = chr.isosurface_extract(fd, isos, cap)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    check_cells(cells, counts, f, isos, (nx, ny, nz), f"extract {shape}")
    # the forms of chr_isosurface on the decoded field
    r = synth.value_range(f)
    h = chr.chr_compress(fd, [1e-2 * r, 1e-3 * r], isos)
    R = h.reconstruct(1).cpu().numpy()
    for flags in (0, chr.ISO_INDEX, chr.ISO_FUSED | chr.ISO_INDEX):
        cells.fill_(-1)
        _, counts, err = chr.chr_isosurface(h, 1, isos, cap, flags=flags)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        check_cells(cells, counts, R, isos, (nx, ny, nz), f"chr_isosurface {shape} flags {flags}")
    h.free()
    chr.chr_debug_tri_cells(None)

# past the two-pass threshold (one isovalue, 9 x 16 x 16 tiles): the stored classification
big = synth.turbulence((257, 129, 129), seed=31)
bd = dev(big)
nz, ny, nx = big.shape
_, c, _ = chr.isosurface_extract(bd, [0.3], 0)
torch.cuda.synchronize()
cap = int(c[0]) + 16
cells = torch.full((1, cap), -1, dtype=torch.int32, device="cuda")
chr.chr_debug_tri_cells(cells)
_, counts, err = chr.isosurface_extract(bd, [0.3], cap)
torch.cuda.synchronize()
chr.chr_debug_tri_cells(None)
assert int(err.item()) == 0
check_cells(cells, counts, big, [0.3], (nx, ny, nz), "two-pass")
assert np.array_equal(chr.chr_debug_cases(bd, 0.3).cpu().numpy(), oracle.cases(big, 0.3))
print("debug outputs ok")
"""


def test_case_bytes_and_active_cells_match_the_oracle():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "debug outputs ok" in r.stdout


def test_release_build_refuses_the_test_outputs():
    r = subprocess.run([sys.executable, "-c", r'''
import sys
sys.path.insert(0, sys.argv[1])
from paper_2408_05462_gb300 import build, chr
import torch
build.build()
for fn in (lambda: chr.chr_debug_tri_cells(None), lambda: chr.chr_debug_unpublished_tile(1)):
    try:
        fn()
        raise SystemExit("accepted")
    except chr.ChrError:
        pass
print("refused")
''', ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "refused" in r.stdout

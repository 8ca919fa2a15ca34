"""The library from several host threads at once: in a fresh process, 8
threads on their own CUDA streams make their first marching-cubes calls
together (1 to 3 isovalues, so several per-device caches of kernel
attributes and resident-block counts are filled concurrently); every
result equals the same call made alone afterwards."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, threading
sys.path.insert(0, sys.argv[1])
import torch
from paper_2408_05462_gb300 import build, chr, synth
build.build()
f = torch.from_numpy(synth.turbulence((64, 48, 40), seed=3)).cuda()
torch.cuda.synchronize()
cap = 5 * 63 * 47 * 39
sets = [[0.0], [-0.5, 0.5], [-0.5, 0.0, 0.5]]
out = [None] * 8
start = threading.Barrier(8)

def work(i):
    s = torch.cuda.Stream()
    start.wait()
    with torch.cuda.stream(s):  # the outputs and the workspace belong to s as well
        t, c, e = chr.isosurface_extract(f, sets[i % 3], cap)
    s.synchronize()
    out[i] = (t.cpu(), c.cpu(), int(e.cpu().item()))

th = [threading.Thread(target=work, args=(i,)) for i in range(8)]
for x in th:
    x.start()
for x in th:
    x.join()
for i in range(8):
    t, c, e = chr.isosurface_extract(f, sets[i % 3], cap)
    torch.cuda.synchronize()
    assert e == 0 and out[i][2] == 0, (i, e, out[i][2])
    assert torch.equal(c.cpu(), out[i][1]), i
    for j in range(len(sets[i % 3])):
        n = int(c[j])
        assert torch.equal(t[j, :n].cpu().view(torch.int32), out[i][0][j, :n].view(torch.int32)), (i, j)
print("threads ok")
"""


def test_first_calls_from_several_threads_agree():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "threads ok" in r.stdout

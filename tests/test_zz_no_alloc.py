"""isosurface_extract_noalloc: marching cubes for callers that may not
allocate device memory (a host framework that owns all GPU memory, plugins
and callbacks that must not allocate, latency-bound loops).  It runs the same
kernels as isosurface_extract with the library's fixed device scratch in
place of a caller workspace, so its output must equal that entry point's.

This file is collected last on purpose: the fixed scratch keeps whatever the
previous call left in it, and the test must pass both alone in a fresh
process and after every other test."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import vertex_tol
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()
    chr.lib()


def _same(a_tris, a_counts, b_tris, b_counts):
    ca, cb = a_counts.cpu().numpy(), b_counts.cpu().numpy()
    assert np.array_equal(ca, cb)
    for j in range(ca.size):
        ref = a_tris[j, :ca[j]].cpu().numpy().astype(np.float64)
        got = b_tris[j, :cb[j]].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref) <= vertex_tol(ref))


@pytest.mark.parametrize("shape,isos", [((72, 80, 96), [-0.5, 0.5, 1.0]),
                                        ((41, 33, 60), [-1.5, -0.25, 0.0, 0.3, 0.9, 2.0])])
def test_noalloc_matches_workspace_entry_point(shape, isos):
    f = torch.from_numpy(synth.turbulence(shape, seed=sum(shape))).cuda()
    nz, ny, nx = f.shape
    cap = 5 * (nx - 1) * (ny - 1) * (nz - 1) // 4
    ref_tris, ref_counts, ref_err = chr.isosurface_extract(f, isos, cap)
    torch.cuda.synchronize()
    assert int(ref_err.item()) == 0
    tris = torch.empty_like(ref_tris)
    counts = torch.empty_like(ref_counts)
    err = torch.empty_like(ref_err)
    chr.isosurface_extract_noalloc(f, isos, cap, tris=tris, counts=counts, err=err)  # first call on the device
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the same scratch
        torch_bytes = torch.cuda.memory_allocated()
        free_bytes = torch.cuda.mem_get_info()[0]
        chr.isosurface_extract_noalloc(f, isos, cap, tris=tris, counts=counts, err=err)
        torch.cuda.synchronize()
        # the call itself allocated nothing: neither through torch nor from the device
        assert torch.cuda.memory_allocated() == torch_bytes
        assert torch.cuda.mem_get_info()[0] == free_bytes
        assert int(err.item()) == 0
        _same(ref_tris, ref_counts, tris, counts)


def test_noalloc_rejects_grids_beyond_its_scratch():
    L = chr.lib()
    iso = (ctypes.c_float * 1)(0.0)
    p = ctypes.c_void_p(0x1000)  # never dereferenced: the size check comes first
    st = L.isosurface_extract_noalloc(p, chr.ChrDims(1024, 1024, 1024), iso, 1, p, 10, p, None, None)
    assert st == 1
    assert b"scratch" in L.chr_last_error()

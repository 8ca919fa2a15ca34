"""The reports' reductions: per-brick sums of |g| (chr_brick_abs_sum, used
by autograd.brick_attribution) against a float64 sum of the same values, and
the count of cells whose case byte survives (chr_case_agreement, the
topology accuracy of Sec. 2.2 in the paper-shaped report) against the
oracle's case bytes, bit for bit."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    chr_build.build()
    chr.lib()


def _brick_sums64(g: np.ndarray) -> np.ndarray:
    nz, ny, nx = g.shape
    out = []
    for bz in range(0, nz, 8):
        for by in range(0, ny, 8):
            for bx in range(0, nx, 8):
                out.append(np.abs(g[bz:bz + 8, by:by + 8, bx:bx + 8].astype(np.float64)).sum())
    return np.array(out)


@pytest.mark.parametrize("shape", [(8, 8, 8), (19, 23, 37), (33, 9, 70)])
def test_brick_abs_sum(shape):
    rng = np.random.default_rng(sum(shape))
    g = rng.standard_normal(shape).astype(np.float32)
    g.ravel()[::7] *= -3.0
    d = torch.from_numpy(g).cuda()
    a = chr.chr_brick_abs_sum(d)
    b = chr.chr_brick_abs_sum(d)
    torch.cuda.synchronize()
    want = _brick_sums64(g)
    got = a.cpu().numpy().astype(np.float64)
    # float32 sums of at most 512 terms: within 512 ulp-scale of the float64 sum
    assert np.allclose(got, want, rtol=64 * 2.0 ** -23, atol=0.0)
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))  # a fixed order


def test_case_agreement_against_the_oracle():
    rng = np.random.default_rng(3)
    a = synth.turbulence((21, 26, 35), seed=4)
    b = (a + rng.normal(0, 0.05, a.shape)).astype(np.float32)
    b.ravel()[::97] = np.nan
    a.ravel()[5::131] = np.nan
    b.ravel()[11::173] = a.ravel()[11::173]
    K = [-0.5, 0.0, 0.25, 1.0]
    a.ravel()[::211] = 0.25  # vertices equal to an isovalue (outside)
    want = sum(int((oracle.cases(a, k) == oracle.cases(b, k)).sum()) for k in K)
    got = int(chr.chr_case_agreement(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), K).item())
    assert got == want
    same = int(chr.chr_case_agreement(torch.from_numpy(a).cuda(), torch.from_numpy(a).cuda(), K).item())
    assert same == len(K) * 20 * 25 * 34


def test_report_argument_errors():
    L = chr.lib()
    d = torch.zeros((9, 9, 9), device="cuda")
    dims = chr.ChrDims(9, 9, 9)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    iso = (ctypes.c_float * 17)(*([0.0] * 17))
    assert L.chr_brick_abs_sum(None, dims, d.data_ptr(), None) == 1
    assert L.chr_brick_abs_sum(d.data_ptr(), chr.ChrDims(1, 9, 9), d.data_ptr(), None) == 1
    assert L.chr_case_agreement(d.data_ptr(), d.data_ptr(), dims, iso, 0, cnt.data_ptr(), None) == 1
    assert L.chr_case_agreement(d.data_ptr(), d.data_ptr(), dims, iso, 17, cnt.data_ptr(), None) == 1
    nan = (ctypes.c_float * 1)(float("nan"))
    assert L.chr_case_agreement(d.data_ptr(), d.data_ptr(), dims, nan, 1, cnt.data_ptr(), None) == 1
    assert L.chr_case_agreement(d.data_ptr(), d.data_ptr(), dims, iso, 1, cnt.data_ptr() + 4, None) == 1

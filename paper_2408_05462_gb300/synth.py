"""Seeded synthetic input fields.

These stand in for the paper's Nyx temperature field (Sec. 3), which is not
available.  The module only draws and evaluates inputs; it holds none of the
method's arithmetic, so the CUDA path and the CPU oracle can both be fed from
it.  All fields are float32 arrays indexed [z, y, x] (x fastest in memory).

Recipes:
  gaussian_blobs(n, seed)   sum of 8 Gaussians on the unit cube; centres
                            U[0,1]^3, sigma U[0.05,0.2], amplitude U[0.5,1],
                            drawn in that order from PCG64(seed); evaluated in
                            float64 at p = index/(n-1), then cast.
  turbulence(n, seed)       random-phase spectral field with energy spectrum
                            E(k) ~ k^(-5/3): complex Gaussian Fourier
                            coefficients with amplitude |k|^(-11/6), zero mean
                            mode, inverse real FFT, normalised to mean 0 and
                            variance 1.  float64 FFT up to 256^3, float32 above.
"""
from __future__ import annotations

import os

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_blobs(n, seed: int = 64, nblobs: int = 8) -> np.ndarray:
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    g = _rng(seed)
    c = g.uniform(0.0, 1.0, size=(nblobs, 3))
    sigma = g.uniform(0.05, 0.2, size=nblobs)
    amp = g.uniform(0.5, 1.0, size=nblobs)
    x = np.arange(nx) / max(nx - 1, 1)
    y = np.arange(ny) / max(ny - 1, 1)
    z = np.arange(nz) / max(nz - 1, 1)
    f = np.zeros((nz, ny, nx), np.float64)
    for i in range(nblobs):
        gx = np.exp(-((x - c[i, 0]) ** 2) / (2 * sigma[i] ** 2))
        gy = np.exp(-((y - c[i, 1]) ** 2) / (2 * sigma[i] ** 2))
        gz = np.exp(-((z - c[i, 2]) ** 2) / (2 * sigma[i] ** 2))
        f += amp[i] * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return f.astype(np.float32)


def turbulence(n, seed: int = 512, slope: float = -5.0 / 3.0) -> np.ndarray:
    """Spectral random field, shell energy spectrum ~ k^slope (Kolmogorov -5/3)."""
    import scipy.fft as sfft

    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    big = nx * ny * nz > 256 ** 3
    ftype = np.float32 if big else np.float64
    g = _rng(seed)
    kz = np.fft.fftfreq(nz, 1.0 / nz).astype(ftype)
    ky = np.fft.fftfreq(ny, 1.0 / ny).astype(ftype)
    kx = np.fft.rfftfreq(nx, 1.0 / nx).astype(ftype)
    shape = (nz, ny, nx // 2 + 1)
    # amplitude |k|^((slope - 2)/2): shell energy 4 pi k^2 |u_k|^2 ~ k^slope
    expo = ftype((slope - 2.0) / 2.0)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2
    k2 = k2 + kx[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp = k2 ** (expo / 2)
    amp[0, 0, 0] = 0.0
    del k2
    re = g.standard_normal(size=shape, dtype=ftype)
    im = g.standard_normal(size=shape, dtype=ftype)
    spec = (re + 1j * im).astype(np.complex64 if big else np.complex128)
    del re, im
    spec *= amp
    del amp
    f = sfft.irfftn(spec, s=(nz, ny, nx), workers=os.cpu_count() or 1)
    del spec
    f -= f.mean(dtype=np.float64)
    f /= f.std(dtype=np.float64)
    return np.ascontiguousarray(f, dtype=np.float32)


def turbulence_cuda(n, seed: int = 1024, slope: float = -5.0 / 3.0):
    """The spectral field of `turbulence`, generated on the GPU in float32
    with torch's seeded CUDA generator (for grids too large for the host FFT;
    the random draws, hence the values, differ from `turbulence`).  Returns a
    [nz, ny, nx] float32 CUDA tensor with zero mean and unit variance."""
    import torch

    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    kz = torch.fft.fftfreq(nz, 1.0 / nz, device=dev)
    ky = torch.fft.fftfreq(ny, 1.0 / ny, device=dev)
    kx = torch.fft.rfftfreq(nx, 1.0 / nx, device=dev)
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp = k2.pow_((slope - 2.0) / 4.0)
    del k2
    amp[0, 0, 0] = 0.0
    shape = (nz, ny, nx // 2 + 1)
    spec = torch.complex(torch.randn(shape, generator=g, device=dev), torch.randn(shape, generator=g, device=dev))
    spec *= amp
    del amp
    f = torch.fft.irfftn(spec, s=(nz, ny, nx))
    del spec
    f -= f.mean(dtype=torch.float64).float()
    f /= f.double().std().float()
    return f.contiguous()


def sphere_distance(n, center, radius_unused=None) -> np.ndarray:
    """|p - c| in grid units (a sphere of radius r is its level set r)."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    return d.astype(np.float32)


def torus_field(n, center, R: float, r_unused=None) -> np.ndarray:
    """(sqrt(x^2 + y^2) - R)^2 + z^2 around center; level r^2 is a torus."""
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = x - center[0]
    y = y - center[1]
    z = z - center[2]
    return ((np.sqrt(x * x + y * y) - R) ** 2 + z * z).astype(np.float32)


def plane_field(n, normal=(0.0, 0.0, 1.0), offset: float = 0.0) -> np.ndarray:
    nx, ny, nz = (n, n, n) if np.isscalar(n) else n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (normal[0] * x + normal[1] * y + normal[2] * z - offset).astype(np.float32)


def uniform_noise(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    g = _rng(seed)
    return g.uniform(lo, hi, size=shape).astype(np.float32)


def value_range(f: np.ndarray) -> float:
    """max - min over finite values (for relative error bounds)."""
    ff = f[np.isfinite(f)]
    return float(ff.max() - ff.min()) if ff.size else 0.0

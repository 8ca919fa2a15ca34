"""Test-side helpers: comparing libchr outputs with the oracle's.

Nothing here computes the method: it reorders, parses and compares."""
from __future__ import annotations

import math

import numpy as np


def brick_major_order(cell: np.ndarray, dims) -> np.ndarray:
    """Stable permutation taking triangles in ascending cell order (the
    oracle's) to the library's output order: 8^3-cell bricks in x-fastest
    brick order, cells x-fastest inside a brick."""
    nx, ny, nz = dims
    cx, cy, cz = nx - 1, ny - 1, nz - 1
    x = cell % cx
    y = (cell // cx) % cy
    z = cell // (cx * cy)
    nbx = math.ceil(cx / 8)
    nby = math.ceil(cy / 8)
    key = (x // 8) + nbx * ((y // 8) + nby * (z // 8))
    return np.argsort(key, kind="stable")


def vertex_tol(ref: np.ndarray) -> np.ndarray:
    """1e-5 of a cell edge, plus one float32 ulp at the coordinate's
    magnitude (the output format cannot hold a vertex closer than that)."""
    mag = np.abs(ref).astype(np.float32)
    return 1e-5 + np.spacing(np.maximum(mag, np.float32(1.0))).astype(np.float64)


def compare_mesh(gpu_tris: np.ndarray, mesh, dims, label=""):
    """gpu_tris: (T, 3, 3) float32 from the library; mesh: oracle.Mesh."""
    T = mesh.ntri
    assert gpu_tris.shape[0] == T, f"{label}: {gpu_tris.shape[0]} vs {T} triangles"
    if T == 0:
        return 0.0
    order = brick_major_order(mesh.cell, dims)
    ref = mesh.pos[order]
    diff = np.abs(gpu_tris.astype(np.float64) - ref)
    tol = vertex_tol(ref)
    bad = diff > tol
    assert not bad.any(), f"{label}: {int(bad.sum())} coordinates off, worst {diff.max()}"
    return float(diff.max())

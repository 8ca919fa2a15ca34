"""CPU oracle for the CHR codec, the topology fix, error-bound translation and
marching cubes (arXiv 2408.05462, Sec. 2 and Sec. 2.2).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product library never does.  It is a
thin ctypes layer over ``chr_oracle.c`` (plain single-threaded C) and shares no
code with the CUDA path.

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
  encode / decode       pinned: strict bound in fp64, sign agreement, closed
                        forms for plane and constant fields, a hand-derived
                        dyadic worked example, exact round trips.
  cell_triangles / mc   pinned: hand-derived single-cell cases, closed
                        oriented 2-manifolds for all 256 cases, Euler
                        characteristic of sphere and torus, exact plane
                        surfaces, sphere volume.
  translate_D / _eb     pinned: closed-form ramps with known multiplicities,
                        downward rounding, the sign-preservation property.
  cases                 pinned: hand-set corners of single cells, the
                        triangle count of mc() as the sum of the cases'
                        triangle counts, complement symmetry.
  brick_index           pinned: brute force over tiny grids (no active cell
                        of mc() lies in a brick whose range excludes k, and
                        each bound is attained), hand-worked bricks at grid
                        edges, NaN as +inf, cell-less bricks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

BRICK = 8


def build(force: bool = False) -> str:
    """Compile chr_oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-frounding-math", "-fno-fast-math",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.orc_nbricks.restype = i64
        lib.orc_nbricks.argtypes = [i64, i64, i64]
        lib.orc_encode.restype = ctypes.c_int
        lib.orc_encode.argtypes = [P, i64, i64, i64, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int,
                                   P, P, P, P, P, P, P]
        lib.orc_decode.restype = ctypes.c_int
        lib.orc_decode.argtypes = [P, P, P, P, P, P, i64, i64, i64, P, ctypes.c_int, P]
        lib.orc_cell_triangles.restype = ctypes.c_int
        lib.orc_cell_triangles.argtypes = [ctypes.c_int, P]
        lib.orc_mc.restype = i64
        lib.orc_mc.argtypes = [P, i64, i64, i64, ctypes.c_float, P, P, P, i64]
        lib.orc_translate_D.restype = i64
        lib.orc_translate_D.argtypes = [P, i64, i64, i64, P, ctypes.c_int, P, i64]
        lib.orc_mc_backward.restype = i64
        lib.orc_mc_backward.argtypes = [P, i64, i64, i64, ctypes.c_float, P, P]
        lib.orc_dist_loss.restype = ctypes.c_double
        lib.orc_dist_loss.argtypes = [P, i64, i64, i64, ctypes.c_float, P, i64, P]
        lib.orc_cases.restype = None
        lib.orc_cases.argtypes = [P, i64, i64, i64, ctypes.c_float, P]
        lib.orc_brick_index.restype = None
        lib.orc_brick_index.argtypes = [P, i64, i64, i64, P, P]
        lib.orc_translate_eb.restype = ctypes.c_float
        lib.orc_translate_eb.argtypes = [P, i64, i64, i64, P, ctypes.c_int, ctypes.c_float, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _field(f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float32)
    if f.ndim != 3:
        raise ValueError("field must be 3-D, indexed [z, y, x]")
    return f


def nbricks(nx: int, ny: int, nz: int) -> int:
    return int(_load().orc_nbricks(nx, ny, nz))


@dataclass
class Encoded:
    """Oracle encoding.  Per level l: recs[l] (nbricks, 4) uint32 =
    (wsum, exc_off, anchor bits, w | mode<<8 | nexc<<16); words[l] uint32;
    exc_idx[l] uint16 slots; exc_val[l] uint32 value bits; R[l] float32 (the
    reconstruction the decoder must produce)."""
    dims: tuple
    eb: np.ndarray
    recs: list = field(default_factory=list)
    words: list = field(default_factory=list)
    exc_idx: list = field(default_factory=list)
    exc_val: list = field(default_factory=list)
    R: list = field(default_factory=list)

    @property
    def nlevels(self):
        return len(self.recs)

    def width(self, l):
        return (self.recs[l][:, 3] & 0xFF).astype(np.int64)

    def mode(self, l):
        return ((self.recs[l][:, 3] >> 8) & 0xFF).astype(np.int64)

    def nexc(self, l):
        return (self.recs[l][:, 3] >> 16).astype(np.int64)


def encode(f: np.ndarray, eb, isovalues=(), fix: bool = True) -> Encoded:
    """Encode field f[z, y, x] into len(eb) levels (Sec. 2, Sec. 2.2)."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    eb = np.ascontiguousarray(eb, dtype=np.float32)
    K = np.ascontiguousarray(isovalues, dtype=np.float32)
    if K.size == 0:
        K = np.zeros(1, np.float32)
        nK = 0
    else:
        nK = K.size
    L = eb.size
    N = nx * ny * nz
    nb = lib.orc_nbricks(nx, ny, nz)
    recs = np.zeros((L, nb, 4), np.uint32)
    words = np.zeros((L, nb * 512), np.uint32)
    exc_idx = np.zeros((L, N), np.uint16)
    exc_val = np.zeros((L, N), np.uint32)
    R = np.zeros((L, N), np.float32)
    nwords = np.zeros(L, np.int64)
    nexc = np.zeros(L, np.int64)
    rc = lib.orc_encode(_ptr(f), nx, ny, nz, L, _ptr(eb), _ptr(K), nK, int(bool(fix)), _ptr(recs), _ptr(words),
                        _ptr(exc_idx), _ptr(exc_val), _ptr(R), _ptr(nwords), _ptr(nexc))
    if rc != 0:
        raise ValueError("orc_encode failed")
    out = Encoded(dims=(nx, ny, nz), eb=eb.copy())
    for l in range(L):
        out.recs.append(recs[l].copy())
        out.words.append(words[l, :nwords[l]].copy())
        out.exc_idx.append(exc_idx[l, :nexc[l]].copy())
        out.exc_val.append(exc_val[l, :nexc[l]].copy())
        out.R.append(R[l].reshape(nz, ny, nx).copy())
    return out


def decode(enc: Encoded, level: int) -> np.ndarray:
    """Reconstruct level `level` from the oracle's own encoding."""
    lib = _load()
    nx, ny, nz = enc.dims
    L = enc.nlevels
    if not 0 <= level < L:
        raise ValueError("level out of range")
    recs = np.ascontiguousarray(np.stack(enc.recs), dtype=np.uint32)
    words = np.concatenate(enc.words + [np.zeros(1, np.uint32)]).astype(np.uint32)
    wbase = np.zeros(L, np.int64)
    wbase[1:] = np.cumsum([w.size for w in enc.words])[:-1]
    ei = np.concatenate(enc.exc_idx + [np.zeros(1, np.uint16)]).astype(np.uint16)
    ev = np.concatenate(enc.exc_val + [np.zeros(1, np.uint32)]).astype(np.uint32)
    ebase = np.zeros(L, np.int64)
    ebase[1:] = np.cumsum([e.size for e in enc.exc_idx])[:-1]
    out = np.zeros(nx * ny * nz, np.float32)
    lib.orc_decode(_ptr(recs), _ptr(words), _ptr(wbase), _ptr(ei), _ptr(ev), _ptr(ebase), nx, ny, nz,
                   _ptr(np.ascontiguousarray(enc.eb, np.float32)), level, _ptr(out))
    return out.reshape(nz, ny, nx)


def cell_triangles(caseb: int) -> np.ndarray:
    """Triangles (as edge-number triples) of one cell with inside bits `caseb`."""
    buf = np.zeros(36, np.int8)
    n = _load().orc_cell_triangles(int(caseb), _ptr(buf))
    return buf[:3 * n].reshape(n, 3).astype(np.int64)


@dataclass
class Mesh:
    pos: np.ndarray      # (T, 3, 3) float64, grid units, [tri, corner, xyz]
    cell: np.ndarray     # (T,) int64 cell index x + (nx-1)*(y + (ny-1)*z)
    edge_id: np.ndarray  # (T, 3) int64: 3*index(v0) + axis

    @property
    def ntri(self):
        return self.cell.size


def mc(f: np.ndarray, k: float) -> Mesh:
    """Marching cubes of f[z, y, x] at isovalue k, triangles in cell order."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    T = lib.orc_mc(_ptr(f), nx, ny, nz, ctypes.c_float(k), None, None, None, 0)
    pos = np.zeros((max(T, 1), 3, 3), np.float64)
    cell = np.zeros(max(T, 1), np.int64)
    eid = np.zeros((max(T, 1), 3), np.int64)
    lib.orc_mc(_ptr(f), nx, ny, nz, ctypes.c_float(k), _ptr(pos), _ptr(cell), _ptr(eid), T)
    return Mesh(pos[:T], cell[:T], eid[:T])


def mc_count(f: np.ndarray, k: float) -> int:
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    return int(lib.orc_mc(_ptr(f), nx, ny, nz, ctypes.c_float(k), None, None, None, 0))


def translate_D(f: np.ndarray, isovalues) -> np.ndarray:
    """The array D of Sec. 2.2 (edge order, d0 before d1)."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    K = np.ascontiguousarray(isovalues, dtype=np.float32)
    n = lib.orc_translate_D(_ptr(f), nx, ny, nz, _ptr(K), K.size, None, 0)
    D = np.zeros(max(n, 1), np.float32)
    lib.orc_translate_D(_ptr(f), nx, ny, nz, _ptr(K), K.size, _ptr(D), n)
    return D[:n]


def translate_eb(f: np.ndarray, isovalues, accuracy: float = 1.0):
    """(eb, |D|): the n-th smallest element of D, n = floor((1-accuracy)|D|)."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    K = np.ascontiguousarray(isovalues, dtype=np.float32)
    cnt = np.zeros(1, np.int64)
    eb = lib.orc_translate_eb(_ptr(f), nx, ny, nz, _ptr(K), K.size, ctypes.c_float(accuracy), _ptr(cnt))
    return float(np.float32(eb)), int(cnt[0])


def mc_backward(f: np.ndarray, k: float, grad_pos: np.ndarray) -> np.ndarray:
    """dL/df of L through the oracle's vertex positions (grad_pos: (T, 3, 3),
    in mc()'s order); float64."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    g = np.ascontiguousarray(grad_pos, dtype=np.float64)
    out = np.zeros(f.size, np.float64)
    T = lib.orc_mc_backward(_ptr(f), nx, ny, nz, ctypes.c_float(k), _ptr(g), _ptr(out))
    if T < 0 or T * 9 != g.size:
        raise ValueError("grad_pos does not match the mesh")
    return out.reshape(nz, ny, nx)


def dist_loss(f_orig: np.ndarray, k: float, pts: np.ndarray, with_grad: bool = True):
    """(mean |F(p)-k|/|grad F(p)| over the points, d/dp) in float64."""
    lib = _load()
    f = _field(f_orig)
    nz, ny, nx = f.shape
    P = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    g = np.zeros_like(P) if with_grad else None
    L = lib.orc_dist_loss(_ptr(f), nx, ny, nz, ctypes.c_float(k), _ptr(P), P.shape[0], _ptr(g) if with_grad else None)
    return float(L), (g.reshape(np.shape(pts)) if with_grad else None)


def cases(f: np.ndarray, k: float) -> np.ndarray:
    """Case byte of every cell, [z, y, x] over (nz-1, ny-1, nx-1) cells; bit j
    is corner (j&1, j>>1&1, j>>2&1) inside (v < k)."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    out = np.zeros((nz - 1) * (ny - 1) * (nx - 1), np.uint8)
    lib.orc_cases(_ptr(f), nx, ny, nz, ctypes.c_float(k), _ptr(out))
    return out.reshape(nz - 1, ny - 1, nx - 1)


def brick_index(f: np.ndarray):
    """(lo, hi) per 8^3 brick, [nbz, nby, nbx] float32: the range over the
    vertices of the brick's cells, NaN as +inf, (+inf, -inf) without cells."""
    lib = _load()
    f = _field(f)
    nz, ny, nx = f.shape
    nbx, nby, nbz = -(-nx // BRICK), -(-ny // BRICK), -(-nz // BRICK)
    lo = np.zeros(nbx * nby * nbz, np.float32)
    hi = np.zeros(nbx * nby * nbz, np.float32)
    lib.orc_brick_index(_ptr(f), nx, ny, nz, _ptr(lo), _ptr(hi))
    return lo.reshape(nbz, nby, nbx), hi.reshape(nbz, nby, nbx)

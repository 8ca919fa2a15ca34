"""ctypes binding of libchr.so (C ABI in include/chr.h).

Argument marshalling only: every step of compression, reconstruction,
error-bound translation and marching cubes runs in the library's CUDA
kernels.  torch provides device memory (through its caching allocator, handed
to the library as a chr_allocator) and the current CUDA stream.  There is no
CPU path: if libchr.so is missing or cannot load, every call raises.

Names follow the C ABI: chr_compress, chr_reconstruct, chr_reconstruct_box, chr_brick_range,
chr_serve_request, chr_serve_request_bytes, chr_box_tri_bound,
chr_topo_translate, chr_isosurface, chr_brick_index,
isosurface_extract, isosurface_workspace_size, isosurface_workspace_min_size, isosurface_extract_noalloc,
isosurface_backward, isosurface_distance_loss, chr_brick_abs_sum, chr_case_agreement,
chr_serialize, chr_deserialize,
chr_stats, chr_free, chr_pool_trim, chr_checked_build, chr_debug_bounds_word, and the chr_batch_*
calls (class Batch).
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_float, c_int, c_int64, c_size_t, c_uint32, c_uint64, c_void_p

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchr.so")

CHR_MAX_LEVELS = 8
CHR_MAX_ISO = 16
TOPO = {"none": 0, "fix": 1, "translate": 2}
STATUS = {0: "CHR_OK", 1: "CHR_ERR_INVALID", 2: "CHR_ERR_OOM", 3: "CHR_ERR_CUDA", 4: "CHR_ERR_OVERFLOW",
          5: "CHR_ERR_TIMEOUT", 6: "CHR_ERR_CORRUPT"}
ERR_OVERFLOW_BIT = 1 << 4
ERR_TIMEOUT_BIT = 1 << 5


class ChrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ChrDims(ctypes.Structure):
    _fields_ = [("nx", c_int64), ("ny", c_int64), ("nz", c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class ChrAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class ChrParams(ctypes.Structure):
    _fields_ = [("nlevels", c_uint32), ("error_bounds", POINTER(c_float)), ("isovalues", POINTER(c_float)),
                ("n_iso", c_uint32), ("topo_mode", c_uint32), ("topo_accuracy", c_float), ("flags", c_uint32)]


class ChrStats(ctypes.Structure):
    _fields_ = [("dims", ChrDims), ("nlevels", c_uint32), ("n_iso", c_uint32), ("topo_mode", c_uint32),
                ("reserved", c_uint32), ("nbricks", c_uint64), ("eb", c_float * CHR_MAX_LEVELS),
                ("eb_translated", c_float), ("topo_accuracy", c_float), ("translate_D_count", c_uint64),
                ("payload_words", c_uint64 * CHR_MAX_LEVELS), ("exceptions", c_uint64 * CHR_MAX_LEVELS),
                ("level_bytes", c_uint64 * CHR_MAX_LEVELS)]


_lib = None


class ChrBatchItem(ctypes.Structure):
    _fields_ = [("h", c_void_p), ("level", c_uint32), ("isovalue", c_float)]


class ChrBatchConfig(ctypes.Structure):
    _fields_ = [("count_blocks_per_sm", ctypes.c_int32), ("emit_blocks_per_sm", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("decode_warps_per_block", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    """The loaded libchr.so; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libchr.so not built ({LIB_PATH}); run paper_2408_05462_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        st = c_int
        L.chr_version.restype = c_int
        L.chr_last_error.restype = ctypes.c_char_p
        L.chr_compress.restype = st
        L.chr_compress.argtypes = [c_void_p, ChrDims, POINTER(ChrParams), POINTER(ChrAllocator), c_void_p,
                                   POINTER(c_void_p)]
        L.chr_reconstruct.restype = st
        L.chr_reconstruct.argtypes = [c_void_p, c_uint32, c_void_p, c_void_p]
        L.chr_reconstruct_box.restype = st
        L.chr_reconstruct_box.argtypes = [c_void_p, c_uint32, c_int64, c_int64, c_int64, ChrDims, c_void_p, c_void_p]
        L.chr_serve_request_bytes.restype = c_size_t
        L.chr_serve_request_bytes.argtypes = [ChrDims, c_uint64]
        L.chr_serve_request.restype = st
        L.chr_serve_request.argtypes = [c_void_p, c_uint32, c_int64, c_int64, c_int64, ChrDims, c_float, c_void_p,
                                        c_size_t, c_uint64, c_void_p, c_void_p]
        L.chr_box_tri_bound.restype = c_uint64
        L.chr_box_tri_bound.argtypes = [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int64, c_int64, c_int64,
                                        ChrDims, c_float]
        L.chr_brick_range.restype = st
        L.chr_brick_range.argtypes = [c_void_p, c_uint32, c_void_p, c_void_p]
        L.chr_topo_translate.restype = st
        L.chr_topo_translate.argtypes = [c_void_p, ChrDims, POINTER(c_float), c_uint32, c_float,
                                         POINTER(ChrAllocator), c_void_p, POINTER(c_float), POINTER(c_uint64)]
        L.isosurface_workspace_size.restype = c_size_t
        L.isosurface_workspace_size.argtypes = [ChrDims, c_uint32]
        L.isosurface_workspace_min_size.restype = c_size_t
        L.isosurface_workspace_min_size.argtypes = [ChrDims, c_uint32]
        L.isosurface_extract.restype = st
        L.isosurface_extract.argtypes = [c_void_p, ChrDims, POINTER(c_float), c_uint32, c_void_p, c_uint64, c_void_p,
                                         c_void_p, c_void_p, c_size_t, c_void_p]
        L.chr_isosurface.restype = st
        L.chr_isosurface.argtypes = [c_void_p, c_uint32, POINTER(c_float), c_uint32, c_void_p, c_void_p, c_uint64,
                                     c_void_p, c_void_p, c_uint32, POINTER(ChrAllocator), c_void_p]
        L.chr_brick_index.restype = st
        L.chr_brick_index.argtypes = [c_void_p, c_uint32, c_void_p, c_void_p]
        L.isosurface_extract_noalloc.restype = st
        L.isosurface_extract_noalloc.argtypes = [c_void_p, ChrDims, POINTER(c_float), c_uint32, c_void_p, c_uint64,
                                                 c_void_p, c_void_p, c_void_p]
        L.isosurface_backward_workspace_size.restype = c_size_t
        L.isosurface_backward_workspace_size.argtypes = [ChrDims, c_uint32]
        L.isosurface_backward.restype = st
        L.isosurface_backward.argtypes = [c_void_p, ChrDims, POINTER(c_float), c_uint32, c_void_p, c_uint64, c_void_p,
                                          c_void_p, c_size_t, c_void_p]
        L.isosurface_distance_loss_workspace_size.restype = c_size_t
        L.isosurface_distance_loss_workspace_size.argtypes = [c_uint64]
        L.isosurface_distance_loss.restype = st
        L.isosurface_distance_loss.argtypes = [c_void_p, ChrDims, c_float, c_void_p, c_uint64, c_void_p, c_void_p,
                                               c_void_p, c_size_t, c_void_p]
        L.chr_brick_abs_sum.restype = st
        L.chr_brick_abs_sum.argtypes = [c_void_p, ChrDims, c_void_p, c_void_p]
        L.chr_case_agreement.restype = st
        L.chr_case_agreement.argtypes = [c_void_p, c_void_p, ChrDims, POINTER(c_float), c_uint32, c_void_p, c_void_p]
        L.chr_serialize.restype = st
        L.chr_serialize.argtypes = [c_void_p, c_void_p, c_size_t, POINTER(c_size_t), c_void_p]
        L.chr_deserialize.restype = st
        L.chr_deserialize.argtypes = [c_void_p, c_size_t, POINTER(ChrAllocator), c_void_p, POINTER(c_void_p)]
        L.chr_stats.restype = st
        L.chr_stats.argtypes = [c_void_p, POINTER(ChrStats)]
        L.chr_free.restype = None
        L.chr_free.argtypes = [c_void_p]
        L.chr_pool_trim.restype = st
        L.chr_pool_trim.argtypes = [c_size_t]
        L.chr_checked_build.restype = c_int
        L.chr_debug_bounds_word.restype = st
        L.chr_debug_bounds_word.argtypes = [POINTER(c_uint32), c_int]
        L.chr_debug_unpublished_tile.restype = st
        L.chr_debug_unpublished_tile.argtypes = [c_int64]
        L.chr_debug_tri_cells.restype = st
        L.chr_debug_tri_cells.argtypes = [c_void_p]
        L.chr_debug_cases.restype = st
        L.chr_debug_cases.argtypes = [c_void_p, ChrDims, c_float, c_void_p, c_void_p, c_size_t, c_void_p]
        L.chr_batch_create.restype = st
        L.chr_batch_create.argtypes = [POINTER(ChrBatchItem), c_uint32, c_void_p, c_uint64, c_void_p, c_void_p,
                                       POINTER(ChrAllocator), c_void_p, POINTER(c_void_p)]
        L.chr_batch_run.restype = st
        L.chr_batch_run.argtypes = [c_void_p, c_void_p]
        L.chr_batch_autotune.restype = st
        L.chr_batch_autotune.argtypes = [c_void_p, c_uint32, c_void_p, POINTER(ChrBatchConfig)]
        L.chr_batch_get_config.restype = st
        L.chr_batch_get_config.argtypes = [c_void_p, POINTER(ChrBatchConfig)]
        L.chr_batch_set_config.restype = st
        L.chr_batch_set_config.argtypes = [c_void_p, POINTER(ChrBatchConfig)]
        L.chr_batch_field.restype = st
        L.chr_batch_field.argtypes = [c_void_p, c_uint32, POINTER(c_void_p), POINTER(ctypes.c_int64),
                                      POINTER(ctypes.c_int64)]
        L.chr_batch_field_copy.restype = st
        L.chr_batch_field_copy.argtypes = [c_void_p, c_uint32, c_void_p, c_void_p]
        L.chr_batch_free.restype = None
        L.chr_batch_free.argtypes = [c_void_p]
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise ChrError(status, lib().chr_last_error().decode(errors="replace"))


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


# torch caching allocator behind the chr_allocator vtable
def _torch_alloc(nbytes, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # reported to the library as NULL -> CHR_ERR_OOM
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    if ptr:
        torch.cuda.caching_allocator_delete(ptr)


_ALLOC_CB = ALLOC_FN(_torch_alloc)
_FREE_CB = FREE_FN(_torch_free)
TORCH_ALLOCATOR = ChrAllocator(_ALLOC_CB, _FREE_CB, None)


def _dims(field: torch.Tensor) -> ChrDims:
    if field.dim() != 3:
        raise ValueError("field must be a 3-D tensor indexed [z, y, x]")
    nz, ny, nx = field.shape
    return ChrDims(nx, ny, nz)


def _check_field(field: torch.Tensor):
    if not (field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()):
        raise ValueError("field must be a contiguous float32 CUDA tensor")


def _floats(vals):
    vals = [float(v) for v in vals]
    arr = (c_float * max(len(vals), 1))(*vals)
    return arr, len(vals)


class Chr:
    """A CHR handle (device buffers owned by the library, memory from torch)."""

    def __init__(self, ptr: int, shape):
        self._ptr = c_void_p(ptr)
        self.shape = tuple(shape)

    @property
    def ptr(self):
        return self._ptr

    def stats(self) -> dict:
        return chr_stats(self)

    def reconstruct(self, level: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        return chr_reconstruct(self, level, out, stream)

    def serialize(self, stream=None) -> bytes:
        return chr_serialize(self, stream)

    def reconstruct_box(self, level: int, origin, size, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        return chr_reconstruct_box(self, level, origin, size, out, stream)

    def brick_range(self, level: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        return chr_brick_range(self, level, out, stream)

    def isosurface(self, level: int, isovalues, cap: int, field_out: torch.Tensor | None = None, stream=None,
                   flags: int = 0):
        return chr_isosurface(self, level, isovalues, cap, field_out=field_out, stream=stream, flags=flags)

    def free(self):
        if self._ptr is not None and self._ptr.value:
            lib().chr_free(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def chr_compress(field: torch.Tensor, error_bounds, isovalues=(), topo: str = "fix", accuracy: float = 1.0,
                 stream=None, library_pool: bool = False) -> Chr:
    """Compress a [nz, ny, nx] float32 CUDA field into a CHR (chr.h: chr_compress).
    The CHR's buffers come from torch's caching allocator, or with
    library_pool=True from the library's own pool (a NULL chr_allocator)."""
    _check_field(field)
    eb, ne = _floats(error_bounds)
    iso, ni = _floats(isovalues)
    prm = ChrParams(ne, eb, iso, ni, TOPO[topo], float(accuracy), 0)
    out = c_void_p()
    alloc = None if library_pool else ctypes.byref(TORCH_ALLOCATOR)
    _check(lib().chr_compress(field.data_ptr(), _dims(field), ctypes.byref(prm), alloc, _stream(stream),
                              ctypes.byref(out)))
    return Chr(out.value, field.shape)


def chr_debug_unpublished_tile(tile: int) -> None:
    """Checked builds only: tile `tile` of later single-pass extractions
    publishes nothing (-1: none); see chr.h."""
    _check(lib().chr_debug_unpublished_tile(int(tile)))


def chr_debug_tri_cells(cells: torch.Tensor | None) -> None:
    """Checked builds only: later extractions also write each triangle's
    cell index into `cells` (int32 CUDA tensor laid out like the triangles,
    [n_iso, cap]); None stops it (chr.h: chr_debug_tri_cells)."""
    _check(lib().chr_debug_tri_cells(cells.data_ptr() if cells is not None else None))


def chr_debug_cases(field: torch.Tensor, isovalue: float, stream=None) -> torch.Tensor:
    """Checked builds only: the counting pass's case byte of every cell,
    [nz-1, ny-1, nx-1] uint8, corner (ox, oy, oz) at bit ox + 2 oy + 4 oz
    (chr.h: chr_debug_cases)."""
    _check_field(field)
    nz, ny, nx = field.shape
    out = torch.empty((nz - 1, ny - 1, nx - 1), dtype=torch.uint8, device="cuda")
    ws = torch.empty(isosurface_workspace_size(field.shape, 1), dtype=torch.uint8, device="cuda")
    _check(lib().chr_debug_cases(field.data_ptr(), _dims(field), float(isovalue), out.data_ptr(), ws.data_ptr(),
                                 ws.numel(), _stream(stream)))
    return out


def chr_checked_build() -> bool:
    """Whether the loaded library has the kernels' bounds tests compiled in
    (chr.h: chr_checked_build; build.build(checked=True) makes it)."""
    return bool(lib().chr_checked_build())


def chr_debug_bounds_word(reset: bool = False) -> int:
    """Kernel families that saw an index fail its bounds test in a checked
    build: bit 0 marching cubes, bit 1 codec (chr.h: chr_debug_bounds_word)."""
    w = c_uint32()
    _check(lib().chr_debug_bounds_word(ctypes.byref(w), int(bool(reset))))
    return int(w.value)


def chr_pool_trim(keep_bytes: int = 0) -> None:
    """Give the unused memory of the library's pool on the current device back
    to the driver, keeping `keep_bytes` (chr.h: chr_pool_trim)."""
    _check(lib().chr_pool_trim(int(keep_bytes)))


def chr_reconstruct(h: Chr, level: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Decode level `level` of a CHR into a float32 tensor (chr.h: chr_reconstruct)."""
    if out is None:
        out = torch.empty(h.shape, dtype=torch.float32, device="cuda")
    _check_field(out)
    if tuple(out.shape) != h.shape:
        raise ValueError("out has the wrong shape")
    _check(lib().chr_reconstruct(h.ptr, int(level), out.data_ptr(), _stream(stream)))
    return out


def chr_reconstruct_box(h: Chr, level: int, origin, size, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Decode the vertices origin .. origin+size (x, y, z) of level `level`
    into a [size_z, size_y, size_x] tensor (chr.h: chr_reconstruct_box)."""
    x0, y0, z0 = (int(v) for v in origin)
    bx, by, bz = (int(v) for v in size)
    if out is None:
        out = torch.empty((bz, by, bx), dtype=torch.float32, device="cuda")
    _check_field(out)
    if tuple(out.shape) != (bz, by, bx):
        raise ValueError("out has the wrong shape")
    _check(lib().chr_reconstruct_box(h.ptr, int(level), x0, y0, z0, ChrDims(bx, by, bz), out.data_ptr(),
                                     _stream(stream)))
    return out


def chr_serve_request_bytes(size, cap: int) -> int:
    """Device bytes chr_serve_request needs for a box of `size` (x, y, z) and
    room for `cap` triangles (chr.h: chr_serve_request_bytes)."""
    bx, by, bz = (int(v) for v in size)
    return int(lib().chr_serve_request_bytes(ChrDims(bx, by, bz), int(cap)))


def chr_serve_request(h: Chr, level: int, origin, size, isovalue: float, mem: torch.Tensor, cap: int,
                      result: torch.Tensor, stream=None):
    """Decode the box and mesh it at `isovalue` in one call (chr.h:
    chr_serve_request).  mem: uint8 CUDA tensor of chr_serve_request_bytes
    bytes whose first 36*cap bytes receive the triangles; result: int64 CPU
    tensor of 2 (pinned) that receives (count, error word)."""
    x0, y0, z0 = (int(v) for v in origin)
    bx, by, bz = (int(v) for v in size)
    if not (mem.is_cuda and mem.dtype == torch.uint8 and mem.is_contiguous()):
        raise ValueError("mem must be a contiguous uint8 CUDA tensor")
    if result.is_cuda or result.dtype != torch.int64 or result.numel() < 2 or not result.is_contiguous():
        raise ValueError("result must be a contiguous int64 CPU tensor of 2")
    _check(lib().chr_serve_request(h.ptr, int(level), x0, y0, z0, ChrDims(bx, by, bz), float(isovalue),
                                   mem.data_ptr(), mem.numel(), int(cap), result.data_ptr(), _stream(stream)))


def chr_box_tri_bound(mn, mx, origin, size, isovalue: float) -> int:
    """Triangle bound of a box from a host brick index (chr.h:
    chr_box_tri_bound); mn, mx: contiguous float32 numpy arrays [nbz, nby, nbx]."""
    nbz, nby, nbx = mn.shape
    x0, y0, z0 = (int(v) for v in origin)
    bx, by, bz = (int(v) for v in size)
    return int(lib().chr_box_tri_bound(mn.ctypes.data, mx.ctypes.data, nbx, nby, nbz, x0, y0, z0,
                                       ChrDims(bx, by, bz), float(isovalue)))


def chr_brick_range(h: Chr, level: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Per-brick (min, max) of level `level`, shape [nbz, nby, nbx, 2]
    (chr.h: chr_brick_range)."""
    nz, ny, nx = h.shape
    shape = ((nz + 7) // 8, (ny + 7) // 8, (nx + 7) // 8, 2)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
    if tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous float32 CUDA tensor of shape %s" % (shape,))
    _check(lib().chr_brick_range(h.ptr, int(level), out.data_ptr(), _stream(stream)))
    return out


def chr_topo_translate(field: torch.Tensor, isovalues, accuracy: float = 1.0, stream=None):
    """(eb, |D|): the Sec. 2.2 translated error bound (chr.h: chr_topo_translate)."""
    _check_field(field)
    iso, ni = _floats(isovalues)
    eb = c_float()
    cnt = c_uint64()
    _check(lib().chr_topo_translate(field.data_ptr(), _dims(field), iso, ni, float(accuracy),
                                    ctypes.byref(TORCH_ALLOCATOR), _stream(stream), ctypes.byref(eb),
                                    ctypes.byref(cnt)))
    return float(eb.value), int(cnt.value)


def isosurface_workspace_size(shape, n_iso: int) -> int:
    nz, ny, nx = shape
    return int(lib().isosurface_workspace_size(ChrDims(nx, ny, nz), int(n_iso)))


def isosurface_workspace_min_size(shape, n_iso: int) -> int:
    """Smallest workspace isosurface_extract accepts (chr.h: isosurface_workspace_min_size)."""
    nz, ny, nx = shape
    return int(lib().isosurface_workspace_min_size(ChrDims(nx, ny, nz), int(n_iso)))


def isosurface_extract(field: torch.Tensor, isovalues, cap: int, tris: torch.Tensor | None = None,
                       counts: torch.Tensor | None = None, err: torch.Tensor | None = None,
                       workspace: torch.Tensor | None = None, stream=None):
    """Marching cubes of `field` for each isovalue (chr.h: isosurface_extract).

    Returns (tris [n_iso, cap, 3, 3] float32, counts [n_iso] int64 true counts,
    err [1] int32 device error word).  Asynchronous: read counts/err after the
    stream finishes; counts[j] > cap means isovalue j overflowed."""
    _check_field(field)
    iso, ni = _floats(isovalues)
    if tris is None:
        tris = torch.empty((ni, max(int(cap), 0), 3, 3), dtype=torch.float32, device="cuda")
    if counts is None:
        counts = torch.empty(ni, dtype=torch.int64, device="cuda")
    if err is None:
        err = torch.empty(1, dtype=torch.int32, device="cuda")
    if workspace is None:
        workspace = torch.empty(isosurface_workspace_size(field.shape, ni), dtype=torch.uint8, device="cuda")
    elif workspace.numel() < isosurface_workspace_min_size(field.shape, ni):
        raise ValueError("workspace smaller than isosurface_workspace_min_size")
    if tris.numel() < ni * int(cap) * 9:
        raise ValueError("tris too small for n_iso * cap triangles")
    _check(lib().isosurface_extract(field.data_ptr(), _dims(field), iso, ni, tris.data_ptr() if cap > 0 else None,
                                    int(cap), counts.data_ptr(), err.data_ptr(), workspace.data_ptr(),
                                    workspace.numel(), _stream(stream)))
    return tris, counts, err


ISO_INDEX = 1
ISO_FUSED = 2


def chr_isosurface(h: Chr, level: int, isovalues, cap: int, field_out: torch.Tensor | None = None,
                   tris: torch.Tensor | None = None, counts: torch.Tensor | None = None,
                   err: torch.Tensor | None = None, stream=None, flags: int = 0):
    """Decode level `level` of a CHR and run marching cubes on it in one call
    (chr.h: chr_isosurface).  Returns (tris, counts, err) as isosurface_extract
    does; field_out, when given, receives the decoded field.  flags:
    ISO_INDEX (skip the bricks the value index rules out), ISO_FUSED (the
    one-launch form that decodes each tile in shared memory); same output.  Scratch comes from torch's caching allocator."""
    iso, ni = _floats(isovalues)
    if field_out is not None:
        _check_field(field_out)
        if tuple(field_out.shape) != h.shape:
            raise ValueError("field_out has the wrong shape")
    if tris is None:
        tris = torch.empty((ni, max(int(cap), 0), 3, 3), dtype=torch.float32, device="cuda")
    if counts is None:
        counts = torch.empty(ni, dtype=torch.int64, device="cuda")
    if err is None:
        err = torch.empty(1, dtype=torch.int32, device="cuda")
    if tris.numel() < ni * int(cap) * 9:
        raise ValueError("tris too small for n_iso * cap triangles")
    _check(lib().chr_isosurface(h.ptr, int(level), iso, ni, field_out.data_ptr() if field_out is not None else None,
                                tris.data_ptr() if cap > 0 else None, int(cap), counts.data_ptr(), err.data_ptr(),
                                int(flags), ctypes.byref(TORCH_ALLOCATOR), _stream(stream)))
    return tris, counts, err


def chr_brick_abs_sum(g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sum of |g| over every 8^3 brick, shape [nbz * nby * nbx] in x-fastest
    brick order (chr.h: chr_brick_abs_sum)."""
    _check_field(g)
    nz, ny, nx = g.shape
    nb = ((nz + 7) // 8) * ((ny + 7) // 8) * ((nx + 7) // 8)
    if out is None:
        out = torch.empty(nb, dtype=torch.float32, device=g.device)
    if out.numel() != nb or out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous float32 CUDA tensor of %d elements" % nb)
    _check(lib().chr_brick_abs_sum(g.data_ptr(), _dims(g), out.data_ptr(), _stream(stream)))
    return out


def chr_case_agreement(a: torch.Tensor, b: torch.Tensor, isovalues, count: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    """Number of cells whose case byte at each isovalue is the same in a and
    b, summed over the isovalues, as a one-element int64 CUDA tensor
    (chr.h: chr_case_agreement)."""
    _check_field(a)
    _check_field(b)
    if a.shape != b.shape:
        raise ValueError("a and b must have the same shape")
    iso, ni = _floats(isovalues)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=a.device)
    _check(lib().chr_case_agreement(a.data_ptr(), b.data_ptr(), _dims(a), iso, ni, count.data_ptr(), _stream(stream)))
    return count


def chr_brick_index(h: Chr, level: int, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The CHR's value index of level `level`: (min, max) over each brick's
    cell vertices, shape [nbz, nby, nbx, 2] (chr.h: chr_brick_index)."""
    nz, ny, nx = h.shape
    shape = ((nz + 7) // 8, (ny + 7) // 8, (nx + 7) // 8, 2)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
    if tuple(out.shape) != shape or out.dtype != torch.float32 or not out.is_contiguous() or not out.is_cuda:
        raise ValueError("out must be a contiguous float32 CUDA tensor of shape %s" % (shape,))
    _check(lib().chr_brick_index(h.ptr, int(level), out.data_ptr(), _stream(stream)))
    return out


def isosurface_extract_noalloc(field: torch.Tensor, isovalues, cap: int, tris: torch.Tensor | None = None,
                               counts: torch.Tensor | None = None, err: torch.Tensor | None = None, stream=None):
    """isosurface_extract without a workspace: the library's fixed device
    scratch is used, so the call itself allocates nothing (chr.h:
    isosurface_extract_noalloc).  Output tensors passed in are used as they
    are; tensors left as None are created here, for convenience."""
    _check_field(field)
    iso, ni = _floats(isovalues)
    if tris is None:
        tris = torch.empty((ni, max(int(cap), 0), 3, 3), dtype=torch.float32, device="cuda")
    if counts is None:
        counts = torch.empty(ni, dtype=torch.int64, device="cuda")
    if err is None:
        err = torch.empty(1, dtype=torch.int32, device="cuda")
    if tris.numel() < ni * int(cap) * 9:
        raise ValueError("tris too small for n_iso * cap triangles")
    _check(lib().isosurface_extract_noalloc(field.data_ptr(), _dims(field), iso, ni,
                                            tris.data_ptr() if cap > 0 else None, int(cap), counts.data_ptr(),
                                            err.data_ptr(), _stream(stream)))
    return tris, counts, err


def isosurface_backward(field: torch.Tensor, isovalues, grad_tris: torch.Tensor, cap: int,
                        grad_field: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """dL/dfield from dL/dtris in isosurface_extract's layout [n_iso, cap, 3, 3]
    (chr.h: isosurface_backward).  Deterministic."""
    _check_field(field)
    iso, ni = _floats(isovalues)
    if not (grad_tris.is_cuda and grad_tris.dtype == torch.float32 and grad_tris.is_contiguous()):
        raise ValueError("grad_tris must be a contiguous float32 CUDA tensor")
    if grad_tris.numel() < ni * int(cap) * 9:
        raise ValueError("grad_tris smaller than n_iso * cap triangles")
    if grad_field is None:
        grad_field = torch.empty_like(field)
    ws = torch.empty(int(lib().isosurface_backward_workspace_size(_dims(field), ni)), dtype=torch.uint8, device="cuda")
    _check(lib().isosurface_backward(field.data_ptr(), _dims(field), iso, ni, grad_tris.data_ptr() if cap > 0 else None,
                                     int(cap), grad_field.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)))
    return grad_field


def isosurface_distance_loss(orig_field: torch.Tensor, isovalue: float, points: torch.Tensor, with_grad: bool = True,
                             stream=None):
    """(mean distance of the points to orig_field's isovalue surface as a
    float64 device scalar, its gradient [npts, 3] or None) (chr.h:
    isosurface_distance_loss)."""
    _check_field(orig_field)
    pts = points.reshape(-1, 3)
    if not (pts.is_cuda and pts.dtype == torch.float32 and pts.is_contiguous()):
        raise ValueError("points must be a contiguous float32 CUDA tensor")
    n = pts.shape[0]
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    grad = torch.empty_like(pts) if with_grad else None
    ws = torch.empty(int(lib().isosurface_distance_loss_workspace_size(n)), dtype=torch.uint8, device="cuda")
    _check(lib().isosurface_distance_loss(orig_field.data_ptr(), _dims(orig_field), float(isovalue),
                                          pts.data_ptr() if n else None, n, loss.data_ptr(),
                                          grad.data_ptr() if with_grad else None, ws.data_ptr(), ws.numel(),
                                          _stream(stream)))
    return loss, grad


def chr_serialize(h: Chr, stream=None, out: torch.Tensor | None = None):
    """The CHR as bytes (chr.h: chr_serialize); with `out` (a CPU uint8
    tensor, e.g. pinned, of at least the size) the bytes go there and the
    used view of it is returned."""
    need = c_size_t()
    _check(lib().chr_serialize(h.ptr, None, 0, ctypes.byref(need), _stream(stream)))
    if out is not None:
        if out.dtype != torch.uint8 or out.is_cuda or not out.is_contiguous() or out.numel() < need.value:
            raise ValueError("out must be a contiguous CPU uint8 tensor of at least %d bytes" % need.value)
        _check(lib().chr_serialize(h.ptr, out.data_ptr(), need.value, ctypes.byref(need), _stream(stream)))
        return out[:need.value]
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().chr_serialize(h.ptr, buf, need.value, ctypes.byref(need), _stream(stream)))
    return buf.raw


def chr_serialized_size(h: Chr) -> int:
    need = c_size_t()
    _check(lib().chr_serialize(h.ptr, None, 0, ctypes.byref(need), None))
    return int(need.value)


def chr_deserialize(data, stream=None) -> Chr:
    """A handle from chr_serialize's bytes (chr.h: chr_deserialize): `data`
    is a bytes object or a CPU uint8 tensor (pinned memory uploads fastest)."""
    out = c_void_p()
    if isinstance(data, torch.Tensor):
        if data.dtype != torch.uint8 or data.is_cuda or not data.is_contiguous():
            raise ValueError("data must be a contiguous CPU uint8 tensor")
        ptr, n = c_void_p(data.data_ptr()), data.numel()
    else:
        ptr, n = data, len(data)
    _check(lib().chr_deserialize(ptr, n, ctypes.byref(TORCH_ALLOCATOR), _stream(stream), ctypes.byref(out)))
    h = Chr(out.value, (1, 1, 1))
    st = chr_stats(h)
    h.shape = (st["dims"][2], st["dims"][1], st["dims"][0])
    return h


def chr_stats(h: Chr) -> dict:
    s = ChrStats()
    _check(lib().chr_stats(h.ptr, ctypes.byref(s)))
    L = s.nlevels
    return {
        "dims": (s.dims.nx, s.dims.ny, s.dims.nz), "nlevels": L, "n_iso": s.n_iso, "topo_mode": s.topo_mode,
        "nbricks": s.nbricks, "eb": [s.eb[i] for i in range(L)], "eb_translated": s.eb_translated,
        "topo_accuracy": s.topo_accuracy, "translate_D_count": s.translate_D_count,
        "payload_words": [s.payload_words[i] for i in range(L)], "exceptions": [s.exceptions[i] for i in range(L)],
        "level_bytes": [s.level_bytes[i] for i in range(L)],
    }


def chr_free(h: Chr):
    h.free()


class Batch:
    """Many CHRs decoded and meshed by one captured launch sequence (chr.h:
    chr_batch_*).  items: (Chr, level, isovalue) triples; the handles must
    outlive the batch.  Outputs (tris [cap, 3, 3], box_start [n+1], err [1])
    are torch tensors owned here and rewritten by every run."""

    def __init__(self, items, cap: int, stream=None):
        self.items = list(items)
        n = len(self.items)
        arr = (ChrBatchItem * max(n, 1))(*[ChrBatchItem(h.ptr.value, int(l), float(k)) for h, l, k in self.items])
        self.cap = int(cap)
        self.tris = torch.empty((max(self.cap, 1), 3, 3), dtype=torch.float32, device="cuda")
        self.box_start = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        self.err = torch.zeros(1, dtype=torch.int32, device="cuda")
        out = c_void_p()
        _check(lib().chr_batch_create(arr, n, self.tris.data_ptr() if self.cap > 0 else None, self.cap,
                                      self.box_start.data_ptr(), self.err.data_ptr(), ctypes.byref(TORCH_ALLOCATOR),
                                      _stream(stream), ctypes.byref(out)))
        self._ptr = out

    def run(self, stream=None):
        _check(lib().chr_batch_run(self._ptr, _stream(stream)))

    def autotune(self, reps: int = 3, stream=None) -> dict:
        c = ChrBatchConfig()
        _check(lib().chr_batch_autotune(self._ptr, int(reps), _stream(stream), ctypes.byref(c)))
        return c.as_dict()

    @property
    def config(self) -> dict:
        c = ChrBatchConfig()
        _check(lib().chr_batch_get_config(self._ptr, ctypes.byref(c)))
        return c.as_dict()

    @config.setter
    def config(self, cfg: dict):
        c = ChrBatchConfig(int(cfg.get("count_blocks_per_sm", 0)), int(cfg.get("emit_blocks_per_sm", 0)),
                           int(cfg.get("use_graph", 1)), int(cfg.get("decode_warps_per_block", 0)))
        _check(lib().chr_batch_set_config(self._ptr, ctypes.byref(c)))

    def field(self, i: int, stream=None) -> torch.Tensor:
        """Item i's decoded field as a dense [nz, ny, nx] tensor (a copy)."""
        h = self.items[i][0]
        out = torch.empty(h.shape, dtype=torch.float32, device="cuda")
        _check(lib().chr_batch_field_copy(self._ptr, int(i), out.data_ptr(), _stream(stream)))
        return out

    def triangles(self, i: int) -> torch.Tensor:
        """Item i's triangles (a view; synchronises to read box_start)."""
        bs = self.box_start.cpu()
        a, b = int(bs[i]), min(int(bs[i + 1]), self.cap)
        return self.tris[a:max(a, b)]

    def free(self):
        if self._ptr is not None and self._ptr.value:
            lib().chr_batch_free(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def parse_serialized(data: bytes) -> dict:
    """Split a chr_serialize byte string into numpy arrays (format in chr.h)."""
    import numpy as np

    off = 0

    def take(dtype, n):
        nonlocal off
        a = np.frombuffer(data, dtype=dtype, count=n, offset=off)
        off += a.nbytes
        return a

    assert data[:4] == b"CHR1"
    off = 4
    version = int(take(np.uint32, 1)[0])
    nx, ny, nz = (int(v) for v in take(np.int64, 3))
    nlevels, n_iso, topo, flags = (int(v) for v in take(np.uint32, 4))
    acc, ebt = (float(v) for v in take(np.float32, 2))
    dcount = int(take(np.uint64, 1)[0])
    eb = take(np.float32, nlevels).copy()
    iso = take(np.float32, n_iso).copy()
    sizes = take(np.uint64, 2 * nlevels).reshape(nlevels, 2)
    nb = math.ceil(nx / 8) * math.ceil(ny / 8) * math.ceil(nz / 8)
    levels = []
    for l in range(nlevels):
        nw, ne = int(sizes[l, 0]), int(sizes[l, 1])
        recs = take(np.uint32, 4 * nb).reshape(nb, 4).copy()
        words = take(np.uint32, nw).copy()
        idx = take(np.uint16, ne).copy()
        off += ((2 * ne + 3) & ~3) - 2 * ne
        val = take(np.uint32, ne).copy()
        levels.append({"recs": recs, "words": words, "exc_idx": idx, "exc_val": val})
    if version >= 2:
        for l in range(nlevels):
            levels[l]["index"] = take(np.float32, 2 * nb).reshape(nb, 2).copy()
    return {"version": version, "dims": (nx, ny, nz), "nlevels": nlevels, "n_iso": n_iso, "topo_mode": topo,
            "flags": flags, "topo_accuracy": acc, "eb_translated": ebt, "translate_D_count": dcount, "eb": eb,
            "isovalues": iso, "levels": levels}

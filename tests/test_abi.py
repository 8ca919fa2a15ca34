"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every function include/chr.h declares, and rejects bad arguments and corrupt
serialized bytes before touching the device."""
import ctypes
import os
import re
import struct

import pytest

from paper_2408_05462_gb300 import build as chr_build
from paper_2408_05462_gb300 import chr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    chr_build.build()
    return chr.lib()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_function(L):
    names = _declared_functions()
    assert {"chr_compress", "chr_reconstruct", "isosurface_extract", "chr_topo_translate"} <= names
    for n in sorted(names):
        assert hasattr(L, n), f"libchr.so does not export {n}"
    assert L.chr_version() == 2


def _params(eb=(0.1,), iso=(0.5,), topo=1, acc=1.0, flags=0):
    ebs = (ctypes.c_float * max(len(eb), 1))(*eb)
    isos = (ctypes.c_float * max(len(iso), 1))(*iso)
    return chr.ChrParams(len(eb), ebs, isos, len(iso), topo, acc, flags), (ebs, isos)


@pytest.mark.parametrize("kw,dims", [
    (dict(eb=()), (8, 8, 8)),
    (dict(eb=(0.1, 0.2)), (8, 8, 8)),          # not decreasing
    (dict(eb=(0.0,)), (8, 8, 8)),
    (dict(eb=(float("nan"),)), (8, 8, 8)),
    (dict(eb=(float("inf"),)), (8, 8, 8)),
    (dict(iso=()), (8, 8, 8)),                  # FIX needs isovalues
    (dict(iso=tuple([0.0] * 17)), (8, 8, 8)),
    (dict(iso=(float("nan"),)), (8, 8, 8)),
    (dict(topo=3), (8, 8, 8)),
    (dict(topo=2, acc=0.0), (8, 8, 8)),
    (dict(topo=2, acc=1.5), (8, 8, 8)),
    (dict(flags=1), (8, 8, 8)),
    (dict(), (1, 8, 8)),
    (dict(), (8, 8, 0)),
    (dict(), (70000, 70000, 2)),
])
def test_compress_rejects_bad_arguments(L, kw, dims):
    prm, keep = _params(**kw)
    out = ctypes.c_void_p(1234)
    st = L.chr_compress(ctypes.c_void_p(0x1000), chr.ChrDims(*dims), ctypes.byref(prm), None, None,
                        ctypes.byref(out))
    assert st == 1, L.chr_last_error()
    assert out.value is None
    assert L.chr_last_error()


def test_other_calls_reject_bad_arguments(L):
    d = chr.ChrDims(8, 8, 8)
    iso = (ctypes.c_float * 1)(0.5)
    assert L.chr_reconstruct(None, 0, ctypes.c_void_p(0x1000), None) == 1
    assert L.isosurface_extract(None, d, iso, 1, None, 0, None, None, None, 0, None) == 1
    assert L.chr_isosurface(None, 0, iso, 1, None, None, 0, ctypes.c_void_p(0x1000), None, 0, None, None) == 1
    assert L.chr_brick_index(None, 0, ctypes.c_void_p(0x1000), None) == 1
    ws = L.isosurface_workspace_size(d, 1)
    ws_min = L.isosurface_workspace_min_size(d, 1)
    # the full workspace adds the stored classification of up to 4 isovalue slots to the tile arrays
    assert 0 < ws_min < ws < L.isosurface_workspace_size(d, 2) < L.isosurface_workspace_size(d, 4)
    assert L.isosurface_workspace_size(d, 4) == L.isosurface_workspace_size(d, 16)
    assert L.isosurface_workspace_min_size(d, 16) == ws_min
    # too small a workspace, zero or too many isovalues, non-finite isovalue
    p = ctypes.c_void_p(0x1000)
    assert L.isosurface_extract(p, d, iso, 1, p, 10, p, None, p, ws_min - 1, None) == 1
    assert L.isosurface_extract(p, d, iso, 0, p, 10, p, None, p, ws, None) == 1
    assert L.isosurface_extract(p, d, iso, 17, p, 10, p, None, p, ws, None) == 1
    bad = (ctypes.c_float * 1)(float("inf"))
    assert L.isosurface_extract(p, d, bad, 1, p, 10, p, None, p, ws, None) == 1
    assert L.isosurface_extract(p, d, iso, 1, None, 10, p, None, p, ws, None) == 1
    eb = ctypes.c_float()
    assert L.chr_topo_translate(p, d, iso, 1, 0.0, None, None, ctypes.byref(eb), None) == 1
    assert L.chr_topo_translate(p, d, iso, 0, 1.0, None, None, ctypes.byref(eb), None) == 1
    assert L.chr_stats(None, None) == 1
    L.chr_free(None)


def _header(nx=8, ny=8, nz=8, nlevels=1, n_iso=0, topo=0, nwords=0, nexc=0):
    b = b"CHR1" + struct.pack("<I", 1) + struct.pack("<qqq", nx, ny, nz)
    b += struct.pack("<IIII", nlevels, n_iso, topo, 0) + struct.pack("<ff", 1.0, float("inf")) + struct.pack("<Q", 0)
    b += struct.pack("<f", 0.1) * nlevels + struct.pack("<f", 0.5) * n_iso
    b += struct.pack("<QQ", nwords, nexc) * nlevels
    return b


def test_deserialize_rejects_corrupt_bytes(L):
    out = ctypes.c_void_p()

    def des(b):
        return L.chr_deserialize(b, len(b), None, None, ctypes.byref(out))

    assert des(b"XXXX" + b"\0" * 100) == 6
    assert des(b"CHR1" + struct.pack("<I", 3) + b"\0" * 100) == 6   # unknown version
    assert des(_header()[:30]) == 6                      # truncated header
    assert des(_header(nlevels=9)) == 6
    assert des(_header()) == 6                           # header without the level data
    rec = struct.pack("<IIiI", 0, 0, 0, 33)              # width 33 > 32
    assert des(_header(nwords=16 * 33) + rec + b"\0" * (4 * 16 * 33)) == 6
    rec = struct.pack("<IIiI", 5, 0, 0, 1)               # wsum of brick 0 must be 0
    assert des(_header(nwords=16) + rec + b"\0" * 64) == 6
    rec = struct.pack("<IIiI", 0, 0, 0, 1 | (1 << 16))    # one exception at slot 600
    assert des(_header(nwords=16, nexc=1) + rec + b"\0" * 64 + struct.pack("<H", 600) + b"\0\0" +
               b"\0" * 4) == 6
    rec = struct.pack("<IIiI", 0, 0, 0, 1 | (2 << 16))    # slots not ascending
    assert des(_header(nwords=16, nexc=2) + rec + b"\0" * 64 + struct.pack("<HH", 5, 3) + b"\0" * 8) == 6
    rec = struct.pack("<IIiI", 0, 0, 0, 0 | (1 << 16))    # slot outside a 4x8x8 grid
    assert des(_header(nx=4, nwords=0, nexc=1) + rec + struct.pack("<H", 7) + b"\0\0" + b"\0" * 4) == 6
    assert out.value is None


def test_deserialize_reports_a_failing_allocator(L):
    # a valid one-brick, one-level CHR; the allocator returns NULL for the
    # handle's record block, so the call fails with CHR_ERR_OOM before any
    # device work and leaves no handle
    blob = _header(nx=8, ny=8, nz=8, nlevels=1) + struct.pack("<IIiI", 0, 0, 0, 0)
    calls = []

    def alloc(n, s, c):
        calls.append(n)
        return None

    fail = chr.ChrAllocator(chr.ALLOC_FN(alloc), chr.FREE_FN(lambda p, n, s, c: None), None)
    out = ctypes.c_void_p()
    assert L.chr_deserialize(blob, len(blob), ctypes.byref(fail), None, ctypes.byref(out)) == 2
    assert out.value is None and len(calls) == 1


def test_deserialize_reports_corruption_ahead_of_a_failing_allocator(L):
    # the copies are issued before the records are checked, so an allocation
    # can fail first; a string that is also corrupt is still reported as
    # corrupt, and no handle is left
    rec = struct.pack("<IIiI", 5, 0, 0, 1)  # wsum of brick 0 must be 0
    blob = _header(nwords=16) + rec + b"\0" * 64

    def alloc(n, s, c):
        return None

    fail = chr.ChrAllocator(chr.ALLOC_FN(alloc), chr.FREE_FN(lambda p, n, s, c: None), None)
    out = ctypes.c_void_p()
    assert L.chr_deserialize(blob, len(blob), ctypes.byref(fail), None, ctypes.byref(out)) == 6
    assert out.value is None


def test_checked_build_is_a_separate_library():
    # build(checked=True) makes libchr_checked.so with the kernels' bounds
    # tests compiled in; the normal library reports none (no GPU needed)
    normal = ctypes.CDLL(chr_build.build())
    checked = ctypes.CDLL(chr_build.build(checked=True))
    assert normal.chr_checked_build() == 0
    assert checked.chr_checked_build() == 1

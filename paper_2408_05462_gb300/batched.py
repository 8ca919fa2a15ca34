"""Many boxes of uneven size, each with its own isovalue and error bound,
through one batched launch sequence (chr.h: chr_batch_*), against the plain
path that decodes and meshes the boxes one by one.

The boxes stand for the output of the paper's block merging (Sec. 2):
rectangular regions of different shapes, each compressed on its own.  The
workload: n boxes (default 256), sides drawn independently from U{32..192},
half Gaussian-blob and half k^-5/3 turbulence fields, isovalue k drawn
uniformly inside the box's (min, max), error bound drawn log-uniformly from
[1e-4, 1e-2] times the box's value range; one CHR level per box with the
box's k sign-fixed.
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import chr, synth


@dataclass
class BoxSpec:
    index: int
    size: tuple   # (nx, ny, nz)
    kind: str     # "blobs" | "turbulence"
    seed: int
    u_k: float    # position of k inside (min, max)
    u_e: float    # position of log10(eb/range) inside [-4, -2]


def make_specs(n: int = 256, seed: int = 256, lo: int = 32, hi: int = 192):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        size = tuple(int(g.integers(lo, hi + 1)) for _ in range(3))
        kind = "blobs" if g.uniform() < 0.5 else "turbulence"
        out.append(BoxSpec(i, size, kind, int(g.integers(1, 2 ** 31 - 1)), float(g.uniform()), float(g.uniform())))
    return out


def box_field(spec: BoxSpec) -> np.ndarray:
    if spec.kind == "blobs":
        return synth.gaussian_blobs(spec.size, seed=spec.seed)
    return synth.turbulence(spec.size, seed=spec.seed)


def box_params(spec: BoxSpec, f: np.ndarray):
    """(isovalue, error bound) of a box from its field's value range."""
    lo, hi = float(f.min()), float(f.max())
    k = float(np.float32(lo + spec.u_k * (hi - lo)))
    eb = 10.0 ** (-4.0 + 2.0 * spec.u_e) * (hi - lo)
    return k, eb


def build_items(specs):
    """Compress every box (one level, its own k fixed): [(Chr, 0, k)], fields."""
    items, fields = [], []
    for sp in specs:
        f = box_field(sp)
        k, eb = box_params(sp, f)
        h = chr.chr_compress(torch.from_numpy(f).cuda(), [eb], [k])
        items.append((h, 0, k))
        fields.append(f)
    return items, fields


def make_batch(items, stream=None) -> chr.Batch:
    """A batch with exactly enough triangle room (one sizing run first)."""
    probe = chr.Batch(items, 0, stream)
    probe.run(stream)
    total = int(probe.box_start[-1].item())
    probe.free()
    return chr.Batch(items, max(total, 1), stream)


class PlainPath:
    """The same work one box at a time: chr_reconstruct + isosurface_extract
    per box, into buffers allocated up front."""

    def __init__(self, items, counts):
        self.items = items
        self.fields = [torch.empty(h.shape, dtype=torch.float32, device="cuda") for h, _, _ in items]
        self.tris = [torch.empty((1, max(int(c), 1), 3, 3), dtype=torch.float32, device="cuda") for c in counts]
        self.caps = [int(c) for c in counts]
        self.counts = torch.zeros(len(items), dtype=torch.int64, device="cuda")
        self.err = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.ws = torch.empty(max(chr.isosurface_workspace_size(h.shape, 1) for h, _, _ in items), dtype=torch.uint8,
                              device="cuda")

    def run(self, stream=None):
        for i, (h, level, k) in enumerate(self.items):
            chr.chr_reconstruct(h, level, out=self.fields[i], stream=stream)
            chr.isosurface_extract(self.fields[i], [k], self.caps[i], tris=self.tris[i], counts=self.counts[i:i + 1],
                                   err=self.err, workspace=self.ws, stream=stream)


def _time(fn, reps: int, warmup: int = 3) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure(n: int = 256, seed: int = 256, reps: int = 20):
    specs = make_specs(n, seed)
    t0 = time.perf_counter()
    items, fields = build_items(specs)
    t_build = time.perf_counter() - t0
    batch = make_batch(items)
    default_cfg = batch.config
    t_default = _time(batch.run, reps)
    tuned = batch.autotune(reps=5)
    t_tuned = _time(batch.run, reps)
    cfg = dict(tuned)
    cfg["use_graph"] = 0
    batch.config = cfg
    t_nograph = _time(batch.run, reps)
    cfg["use_graph"] = 1
    batch.config = cfg
    batch.run()
    torch.cuda.synchronize()
    bs = batch.box_start.cpu().numpy()
    counts = np.diff(bs)
    plain = PlainPath(items, counts)
    t_plain = _time(plain.run, reps)
    vertices = sum(int(np.prod(sp.size)) for sp in specs)
    total = int(bs[-1])
    comp = sum(int(h.stats()["level_bytes"][0]) for h, _, _ in items)
    # decode reads the compressed stream and writes the field; marching cubes
    # reads the field and writes 36 B per triangle
    alg = comp + 8.0 * vertices + 36.0 * total
    return {
        "workload": "%d boxes, sides U{32..192}, blobs/turbulence, own k and eb in [1e-4,1e-2] x range, seed %d"
                    % (n, seed),
        "vertices": vertices, "triangles": total, "build_s": t_build,
        "batched_ms": t_tuned, "batched_default_cfg_ms": t_default, "batched_no_graph_ms": t_nograph,
        "per_box_ms": t_plain, "speedup_vs_per_box": t_plain / t_tuned,
        "batched_field_GBps": 4.0 * vertices / (t_tuned * 1e-3) / 1e9,
        "per_box_field_GBps": 4.0 * vertices / (t_plain * 1e-3) / 1e9,
        "tuned_config": tuned, "default_config": default_cfg,
        "launches_batched": 7, "launches_per_box": 6 * n,
        "compressed_bytes": comp, "algorithmic_bytes": alg,
        "batched_algorithmic_GBps": alg / (t_tuned * 1e-3) / 1e9,
    }


if __name__ == "__main__":
    from . import build

    build.build()
    print(json.dumps(measure()))

"""The paper's end-to-end experiment (Sec. 3, Fig. 4), reshaped for synthetic
data on one GB300: the in-transit workflow is compress at the source, stream
the bytes over a 1 Gbps WAN (modelled as bytes * 8 / 1e9 seconds, as the
paper simulates it), reconstruct and extract the isosurfaces at the
visualization side; the baseline streams the raw field and extracts directly.

Modes: topology fix (every case byte preserved) and the paper's error-bound
translation at 100 / 99 / 95 / 80 % topology accuracy (the n-th smallest of
D), each at one level with a user bound of 1e-2 x range.  For every mode the
measured fraction of cells whose case is unchanged (over all isovalues) is
reported beside the speedup.  GPU stages are timed with CUDA events; the
field (synthetic k^-5/3 turbulence, standing in for the paper's Nyx data) is
resident on the device.

Usage: python -m paper_2408_05462_gb300.paper_e2e [--size 512] [--reps 5]
Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import chr, synth

WAN_BITS_PER_S = 1e9
ISOVALUES = [-1.0, -0.5, 0.5, 1.0]


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run(size: int = 512, reps: int = 5, seed: int = 512) -> dict:
    f = torch.from_numpy(synth.turbulence(size, seed=seed)).cuda()
    N = f.numel()
    rng = float(f.max() - f.min())
    eb = [1e-2 * rng]
    R = torch.empty_like(f)
    _, counts, err = chr.isosurface_extract(f, ISOVALUES, 0)
    torch.cuda.synchronize()
    cap = int(counts.max().item() * 1.05) + 4096
    tris = torch.empty((len(ISOVALUES), cap, 3, 3), dtype=torch.float32, device="cuda")
    ws = torch.empty(chr.isosurface_workspace_size(f.shape, len(ISOVALUES)), dtype=torch.uint8, device="cuda")

    def extract(F):
        chr.isosurface_extract(F, ISOVALUES, cap, tris=tris, counts=counts, err=err, workspace=ws)

    t_mc_raw = _time(lambda: extract(f), reps)
    raw_s = 4.0 * N * 8 / WAN_BITS_PER_S
    base_ms = raw_s * 1e3 + t_mc_raw
    n_cells = len(ISOVALUES) * (f.shape[0] - 1) * (f.shape[1] - 1) * (f.shape[2] - 1)
    out = {"size": size, "isovalues": ISOVALUES, "wan_gbps": WAN_BITS_PER_S / 1e9,
           "baseline": {"stream_ms": raw_s * 1e3, "extract_ms": t_mc_raw, "total_ms": base_ms, "bytes": 4 * N},
           "modes": {}}
    modes = [("fix", "fix", 1.0)] + [(f"translate_{int(a * 100)}", "translate", a) for a in (1.0, 0.99, 0.95, 0.8)]
    for name, topo, acc in modes:
        holder = {}

        def comp():
            holder["h"] = chr.chr_compress(f, eb, ISOVALUES, topo=topo, accuracy=acc)

        t_comp = _time(comp, reps)
        h = holder["h"]
        st = h.stats()
        nbytes = sum(st["level_bytes"])
        t_dec = _time(lambda: h.reconstruct(0, R), reps)
        t_mc = _time(lambda: extract(R), reps)
        same = int(chr.chr_case_agreement(f, R, ISOVALUES).item())  # cells whose case survives, every isovalue
        stream_ms = nbytes * 8 / WAN_BITS_PER_S * 1e3
        total = t_comp + stream_ms + t_dec + t_mc
        out["modes"][name] = {
            "error_bound": st["eb"][0], "compressed_bytes": nbytes, "ratio": 4.0 * N / nbytes,
            "exceptions": st["exceptions"][0], "topology_accuracy": same / n_cells,
            "compress_ms": t_comp, "stream_ms": stream_ms, "reconstruct_ms": t_dec, "extract_ms": t_mc,
            "total_ms": total, "speedup_vs_raw": base_ms / total,
        }
        del h, holder
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps(run(a.size, a.reps)))


if __name__ == "__main__":
    main()

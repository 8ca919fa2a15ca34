"""Benchmark of the visualization side's hot path (paper Sec. 2): decode a
CHR level, its exact vertices (the topology fix), and marching cubes for 4
isovalues, in one chr_isosurface call, on a seeded 1024^3 float32 turbulence
field (energy spectrum k^-5/3, unit variance, generated on the GPU),
isovalues {-1,-0.5,0.5,1}, CHR levels at relative bounds 1e-2/1e-3/1e-4 with
the topology fix, level 2 requested.

One step = one chr_isosurface call over the whole field.  `value` is field
GB/s (4*N bytes of field per step / step time), timed with CUDA events over
K steps after W warm-up steps, inputs resident in HBM (the 2 GB CHR, the
4.3 GB decoded field and the 32 GB mesh are far larger than L2).  The
compression (chr_compress, the data source's side) is timed separately
(stages).  `e2e` is the same call through the public API with the CHR's
bytes in pinned host memory: chr_deserialize (host validation and upload),
chr_isosurface and the read-back of the triangle counts in the timed region,
the mesh consumed on the device (e2e.mesh_d2h adds the mesh's copy back).

--impl reference times the CPU oracle (test infrastructure) on every host
core, each on its own sub-box of the same field; it is the baseline, not
the target.  Under torchrun every rank runs its own replica on its own field
(weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ISOVALUES = [-1.0, -0.5, 0.5, 1.0]
REL_BOUNDS = [1e-2, 1e-3, 1e-4]


LEVEL = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="chr", choices=["chr", "reference"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--sample", type=int, default=160, help="edge of each oracle process's sub-box")
    ap.add_argument("--no-forms", action="store_true", help="skip timing the other chr_isosurface forms")
    ap.add_argument("--no-side", action="store_true", help="skip the 512^3 configuration")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-loop measurement")
    ap.add_argument("--serve-size", type=int, default=1024, help="grid side of the served timesteps")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-box batched measurement")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profiled_traffic(name="chr_isosurface_turb1024.md"):
    """DRAM bytes per step of the headline call from the committed ncu
    summary, or None when a source it depends on has changed since."""
    import hashlib
    import re

    summary = os.path.join(ROOT, "profiles", name)
    try:
        text = open(summary).read()
        traffic = float(re.search(r"traffic_per_step_bytes: ([0-9.e+]+)", text).group(1))
        for src, sha in re.findall(r"source: (\S+) sha256 ([0-9a-f]{64})", text):
            if hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest() != sha:
                return None
        return traffic
    except (OSError, AttributeError, ValueError):
        return None


def aggregate_ranks(total_ms, world, n_per_rank, reduce_max=None):
    """Whole-job field GB/s: the time is the maximum over ranks (reduce_max
    maps a local time to the global maximum), every rank processed its own
    field of n_per_rank vertices."""
    t = reduce_max(total_ms) if (reduce_max and world > 1) else total_ms
    return t, world * 4.0 * n_per_rank / (t * 1e-3) / 1e9


def workload_config(n, args, extra=None):
    cfg = {"workload": f"turbulence {n}^3 float32, k^-5/3, unit variance, GPU generator seed {args.seed}; "
                       f"3-level CHR at {REL_BOUNDS} x range with the topology fix for isovalues {ISOVALUES}; "
                       f"chr_isosurface of level {LEVEL} at those 4 isovalues",
           "field_shape": [n, n, n], "isovalues": ISOVALUES, "levels": 3, "level": LEVEL, "topo": "fix",
           "step": f"chr_isosurface(level {LEVEL}, 4 isovalues): decode + exact vertices + marching cubes; "
                   "chr_compress timed separately (stages.chr_compress)",
           "l2": "inputs larger than L2 (CHR about 2 GB, decoded field 4.3 GB, mesh 32 GB); no flush",
           "mesh": "consumed on the device; e2e.mesh_d2h adds its copy to the host"}
    if extra:
        cfg.update(extra)
    return cfg


def host_info():
    """(threads this process may use, CPU model)."""
    try:
        ncores = len(os.sched_getaffinity(0))
    except AttributeError:
        ncores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return ncores, (model or "unknown") + " (%s)" % os.uname().machine


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, enabled, index=0):
        self.enabled = enabled
        self.proc = None
        self.path = None
        self.index = index

    def __enter__(self):
        if not self.enabled:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        mx = max(r[1] for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[2:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(rows)}


def _oracle_worker(conn, sub, eb):
    """One oracle process (test infrastructure: the CPU baseline): encode its
    sub-box once (untimed), then on every "run" decode level LEVEL and count
    the marching-cubes triangles of the 4 isovalues, and send (seconds,
    triangles) back."""
    sys.path.insert(0, ROOT)
    import oracle

    enc = oracle.encode(sub, eb, ISOVALUES, fix=True)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg != "run":
            break
        t0 = time.perf_counter()
        R = oracle.decode(enc, LEVEL)
        tris = sum(oracle.mc_count(R, k) for k in ISOVALUES)
        conn.send((time.perf_counter() - t0, tris))
    conn.close()


class OraclePool:
    """One spawned process per sub-box (each pinned to nothing: the OS
    spreads them over the host cores); run() times one round of decode +
    marching cubes in every process at once."""

    def __init__(self, subs, eb):
        import multiprocessing as mp

        import oracle

        oracle.build()
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for sub in subs:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, sub, eb), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"
        self.vertices = sum(int(sub.size) for sub in subs)

    def run(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("run")
        res = [c.recv() for c in self.conns]
        return time.perf_counter() - t0, sum(r[1] for r in res)

    def close(self):
        for c in self.conns:
            c.send("stop")
        for p in self.procs:
            p.join(timeout=30)


def sub_boxes(field, count, s):
    """`count` sub-boxes of s^3 vertices of a [n, n, n] field (torch, CUDA or
    CPU), at distinct positions, copied to host numpy."""
    n = field.shape[0]
    s = min(s, n)
    per = max(n // s, 1)
    out = []
    for i in range(count):
        z, y, x = (i % per) * s, ((i // per) % per) * s, ((i // (per * per)) % per) * s
        out.append(np.ascontiguousarray(field[z:z + s, y:y + s, x:x + s].cpu().numpy()))
    return out


def reference_field(n, seed):
    """The bench's field: on the GPU when there is one, else the same
    recipe on the host at no more than 256^3 (a smaller sample)."""
    import torch

    from paper_2408_05462_gb300 import synth

    if torch.cuda.is_available():
        torch.cuda.set_device(0)
        return synth.turbulence_cuda(n, seed=seed), n
    m = min(n, 256)
    return torch.from_numpy(synth.turbulence(m, seed=seed)), m


def run_reference(args):
    """The CPU oracle (as it stands) on every host core: each process
    decodes level LEVEL of its own oracle-encoded s^3 sub-box of the field
    and counts the marching-cubes triangles of the 4 isovalues; one step is
    one such round in every process at once."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    ncores, model = host_info()
    f, n = reference_field(args.size, args.seed)
    r = float(f.max() - f.min())
    eb = np.array([b * r for b in REL_BOUNDS], np.float32)
    subs = sub_boxes(f, ncores, args.sample)
    del f
    pool = OraclePool(subs, eb)
    try:
        for _ in range(args.warmup):
            pool.run()
        t = 0.0
        for _ in range(args.steps):
            t += pool.run()[0]
    finally:
        pool.close()
    dt = t / args.steps
    gbs = 4.0 * pool.vertices / dt / 1e9
    s = subs[0].shape[0]
    sample = (f"{len(subs)} processes, each an {s}^3 sub-box of the {n}^3 field: oracle decode of level {LEVEL} "
              f"(3-level CHR, fix) + marching-cubes count x4, encode untimed; host: {model}")
    print(json.dumps({
        "impl": "reference", "metric": "field GB/s (decode+fix+marching cubes), % HBM roofline; serve p50/p99 ms",
        "value": gbs, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": workload_config(n, args, {"sample": sample}),
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": len(subs), "kind": "oracle", "sample": sample,
                         "nproc": ncores, "cpu_model": model},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def cpu_baseline(subs, eb):
    """The oracle on 1 core (one process, one sub-box) and on every host core
    (one process per sub-box), field GB/s of decode + marching cubes."""
    ncores, model = host_info()
    one = OraclePool(subs[:1], eb)
    try:
        one.run()
        t1, _ = one.run()
    finally:
        one.close()
    v1 = 4.0 * one.vertices / t1 / 1e9
    pool = OraclePool(subs, eb)
    try:
        pool.run()
        tn, tris = pool.run()
    finally:
        pool.close()
    vn = 4.0 * pool.vertices / tn / 1e9
    s = subs[0].shape[0]
    return {"value": vn, "unit": "GB/s", "cores": len(subs), "kind": "oracle",
            "sample": f"{len(subs)} processes at once, each an {s}^3 sub-box of the field: oracle decode of level "
                      f"{LEVEL} + marching-cubes count x4 ({tris} triangles) in {tn:.2f} s; encode untimed",
            "one_core": {"value": v1, "unit": "GB/s", "cores": 1, "seconds": t1},
            "nproc": ncores, "cpu_model": model}


def adjoint_timing(n=256, seed=256256, reps=10):
    """The differentiation workload (256^3 k^-5/3 turbulence, k = 0, error
    bound 1e-3): isosurface_backward of the vertex positions and the
    distance loss to the original surface, each timed alone with CUDA events
    after warm-up."""
    import torch

    from paper_2408_05462_gb300 import chr, synth

    f0 = torch.from_numpy(synth.turbulence(n, seed=seed)).cuda()
    h = chr.chr_compress(f0, [1e-3], [0.0])
    R = h.reconstruct(0)
    cap = 12 * n ** 3 // 10
    tris, counts, _ = chr.isosurface_extract(R, [0.0], cap)
    torch.cuda.synchronize()
    T = int(counts[0])
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    G = torch.randn(tris.shape, generator=g, device="cuda")
    pts = tris[0, :T].reshape(-1, 3).contiguous()
    out = {"workload": "turbulence k^-5/3 %d^3, k=0, eb=1e-3" % n, "triangles": T}

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    gf = torch.empty_like(R)
    ms = timed(lambda: chr.isosurface_backward(R, [0.0], G, cap, grad_field=gf))
    # two walks over the field and the incoming gradients, the fixed-point
    # accumulator written and read, the gradient field written
    nb = 2 * (4.0 * n ** 3 + 36.0 * T) + 16.0 * n ** 3 + 4.0 * n ** 3
    out["isosurface_backward"] = {"ms": ms, "algorithmic_bytes": nb, "GBps": nb / (ms * 1e-3) / 1e9}
    ms = timed(lambda: chr.isosurface_distance_loss(f0, 0.0, pts))
    nb = 2 * 12.0 * 3 * T
    out["isosurface_distance_loss"] = {"ms": ms, "points": 3 * T, "points_per_s": 3 * T / (ms * 1e-3)}
    peak, peak_kind = measured_peaks()
    gbps = out["isosurface_backward"]["GBps"]
    out["roofline"] = {"kernel": "isosurface_backward", "bound": "hbm", "achieved": gbps, "peak": peak,
                       "unit": "GB/s", "frac": gbps / peak, "peak_kind": peak_kind}
    del f0, R, tris, G, pts, gf
    h.free()
    return out


def adjoint_cpu_baseline(n=64, seed=256256):
    """The oracle's adjoints (single thread) on an n^3 sample of the
    differentiation field: marching cubes, the position adjoint and the
    distance loss with its gradient."""
    import oracle
    from paper_2408_05462_gb300 import synth

    oracle.build()
    f = synth.turbulence(n, seed=seed)
    t0 = time.perf_counter()
    m = oracle.mc(f, 0.0)
    L, gp = oracle.dist_loss(f, 0.0, m.pos.reshape(-1, 3))
    oracle.mc_backward(f, 0.0, gp.reshape(m.pos.shape))
    dt = time.perf_counter() - t0
    return {"value": m.ntri / dt, "unit": "triangles/s", "cores": 1, "kind": "oracle",
            "sample": "%d^3 turbulence, k=0: oracle mc + distance loss + position adjoint, %d triangles, single "
                      "thread, %.2f s" % (n, m.ntri, dt)}


def batched_cpu_baseline(n_boxes=12):
    """The oracle (single thread) on the smallest boxes of the 256-box
    workload: encode with the box's bound and k fixed, decode, marching cubes
    at k; field GB/s over those boxes."""
    import oracle
    from paper_2408_05462_gb300 import batched

    specs = sorted(batched.make_specs(256, 256), key=lambda sp: int(np.prod(sp.size)))[:n_boxes]
    oracle.build()
    vox = 0
    t0 = time.perf_counter()
    for sp in specs:
        f = batched.box_field(sp)
        k, eb = batched.box_params(sp, f)
        R = oracle.decode(oracle.encode(f, [eb], [k], fix=True), 0)
        oracle.mc_count(R, k)
        vox += f.size
    dt = time.perf_counter() - t0
    return {"value": 4.0 * vox / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%d smallest boxes of the workload (%d vertices), oracle encode + decode + marching-cubes "
                      "count, single thread, %.1f s" % (len(specs), vox, dt)}


def serve_measurement(args):
    """The request loop over resident CHRs of two advected turbulence
    timesteps (4 accuracy levels each): capacity with all requests queued,
    the same requests one at a time on one stream (the plain path), and
    Poisson arrivals at 0.25, 0.5 and 0.8 of capacity with p50/p99."""
    import torch

    from paper_2408_05462_gb300 import serve, synth

    n = args.serve_size
    srv = serve.Server(budget_bytes=96 << 30, slots=4, max_resident=2)
    f = synth.turbulence_cuda(n, seed=1024)
    srv.ingest(0, f)
    f = torch.roll(f, shifts=(1, 2, 3), dims=(0, 1, 2))  # advected by (3, 2, 1) voxels in (x, y, z)
    srv.ingest(1, f)
    del f
    torch.cuda.empty_cache()
    out = serve.measure(srv, (n, n, n), [0, 1], args.serve_requests)
    out.update({"workload": "turbulence k^-5/3 %d^3 (GPU generator, seed 1024), 2 timesteps advected by (3,2,1), "
                            "levels 1e-2..1e-5 x range, requests: k~U[-1,1], level~U{0..3}, sides~U{64..512}, "
                            "seed 5" % n,
                "resident_gib": srv.resident_bytes / 2 ** 30,
                "latency": "arrival to triangles and count ready (device event), results left on the device"})
    for ts in list(srv.steps.values()):
        ts.handle.free()
    return out


def fused_bytes(st, level, T):
    """Algorithmic bytes of chr_isosurface at `level` (the bytes a fused decode and marching cubes moves):
    every brick's record (16 B), the packed words and the exceptions (6 B
    each) of levels 0..level, and 36 B per triangle written."""
    nb = st["nbricks"]
    return sum(16.0 * nb + 4.0 * st["payload_words"][l] + 6.0 * st["exceptions"][l] for l in range(level + 1)) + 36.0 * T


def time_events(fn, reps, warm=2):
    import torch

    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def side_512(args):
    """The 512^3 configuration (host-generated turbulence, seed 512): compress,
    chr_isosurface of level 2, each timed with CUDA events."""
    import torch

    from paper_2408_05462_gb300 import chr, synth

    f = torch.from_numpy(synth.turbulence(512, seed=512)).cuda()
    r = synth.value_range(f.cpu().numpy())
    eb = [b * r for b in REL_BOUNDS]
    t_c = time_events(lambda: chr.chr_compress(f, eb, ISOVALUES).free(), 5)
    h = chr.chr_compress(f, eb, ISOVALUES)
    _, c, _ = chr.chr_isosurface(h, LEVEL, ISOVALUES, 0)
    torch.cuda.synchronize()
    cap = int(c.max()) + 1024
    tris = torch.empty((len(ISOVALUES), cap, 3, 3), dtype=torch.float32, device="cuda")
    t_i = time_events(lambda: chr.chr_isosurface(h, LEVEL, ISOVALUES, cap, tris=tris, counts=c), 10)
    st = h.stats()
    T = int(c.sum())
    peak, _ = measured_peaks()
    fb = fused_bytes(st, LEVEL, T)
    N = 512 ** 3
    # the error-bound translation (the other topology mode): min D is one
    # walk over the edges, an n-th smallest two walks and two small passes
    translate = {}
    for kk, tag in ((ISOVALUES, "4iso"), ([0.5], "1iso")):
        for acc in (1.0, 0.95):
            chr.chr_topo_translate(f, kk, acc)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(5):
                eb_t, nD = chr.chr_topo_translate(f, kk, acc)
            t_ms = (time.perf_counter() - t0) / 5 * 1e3
            translate[f"{tag}_accuracy_{acc}"] = {"ms": t_ms, "eb": eb_t, "D": nD}
    out = {"workload": "turbulence 512^3 (host generator, seed 512), same levels and isovalues",
           "chr_compress_ms": t_c, "chr_isosurface_ms": t_i, "field_GBps": 4.0 * N / (t_i * 1e-3) / 1e9,
           "triangles": T, "fused_algorithmic_bytes": fb, "frac_of_measured_hbm": fb / (t_i * 1e-3) / 1e9 / peak,
           "compressed_bytes": sum(st["level_bytes"]), "translate": translate}
    h.free()
    del f, tris
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__

    __graft_entry__.build()
    from paper_2408_05462_gb300 import chr, synth

    n = args.size
    N = n ** 3
    stream = torch.cuda.current_stream()
    f = synth.turbulence_cuda(n, seed=args.seed + rank)
    r = float(f.max() - f.min())
    eb = [b * r for b in REL_BOUNDS]
    ncores, _ = host_info()
    subs = sub_boxes(f, ncores, args.sample) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    # the data source's side, timed on its own
    t_comp = time_events(lambda: chr.chr_compress(f, eb, ISOVALUES).free(), 3, warm=1)
    h = chr.chr_compress(f, eb, ISOVALUES)
    del f
    torch.cuda.empty_cache()
    st = h.stats()
    comp_bytes = sum(st["level_bytes"])

    # size the triangle buffers from one untimed call
    _, counts, err = chr.chr_isosurface(h, LEVEL, ISOVALUES, 0)
    torch.cuda.synchronize()
    cap = int(counts.max().item() * 1.02) + 1024
    tris = torch.empty((len(ISOVALUES), cap, 3, 3), dtype=torch.float32, device="cuda")

    def step():
        chr.chr_isosurface(h, LEVEL, ISOVALUES, cap, tris=tris, counts=counts, err=err)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ntri = [int(c) for c in counts.cpu().tolist()]
    assert int(err.item()) == 0, "overflow or timeout during warm-up"
    T = sum(ntri)

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with Clocks(not args.no_clocks and rank == 0, local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = start.elapsed_time(end)

    def _max_over_ranks(v):
        t = torch.tensor([v], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    total_ms, _ = aggregate_ranks(total_ms, world, N, _max_over_ranks if world > 1 else None)
    ms_step = total_ms / args.steps
    _, value = aggregate_ranks(ms_step, 1, world * N)
    peak, peak_kind = measured_peaks()

    # the two kernels the default form runs, each timed on its own, and the
    # other forms of the call (same output)
    stages = {"chr_compress": {"ms": t_comp, "algorithmic_bytes": 4.0 * N + comp_bytes}}
    forms = {}
    if not args.no_forms:
        R = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
        ws = torch.empty(chr.isosurface_workspace_size(R.shape, len(ISOVALUES)), dtype=torch.uint8, device="cuda")
        t_dec = time_events(lambda: chr.chr_reconstruct(h, LEVEL, R), 5)
        t_mc = time_events(lambda: chr.isosurface_extract(R, ISOVALUES, cap, tris=tris, counts=counts, workspace=ws), 5)
        dec_bytes = sum(16.0 * st["nbricks"] + 4.0 * st["payload_words"][l] + 6.0 * st["exceptions"][l]
                        for l in range(LEVEL + 1)) + 4.0 * N
        stages["chr_reconstruct"] = {"ms": t_dec, "algorithmic_bytes": dec_bytes}
        stages["isosurface_extract"] = {"ms": t_mc, "algorithmic_bytes": 4.0 * N + 36.0 * T}
        del R, ws
        torch.cuda.empty_cache()
        for name, flags in (("index", chr.ISO_INDEX), ("fused_kernel", chr.ISO_FUSED),
                            ("fused_kernel_index", chr.ISO_FUSED | chr.ISO_INDEX)):
            ms = time_events(lambda: chr.chr_isosurface(h, LEVEL, ISOVALUES, cap, tris=tris, counts=counts,
                                                        err=err, flags=flags), 3, warm=1)
            forms[name] = {"ms": ms, "field_GBps": 4.0 * N / (ms * 1e-3) / 1e9}
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        # what the value index lets the index forms skip: (cell brick,
        # isovalue) pairs whose range does not straddle the isovalue, and
        # whole tiles (4 bricks along x) with no straddling pair
        idx = chr.chr_brick_index(h, LEVEL).cpu().numpy()
        act = np.stack([(idx[..., 0] < k) & (k <= idx[..., 1]) for k in ISOVALUES])
        pad = (-act.shape[-1]) % 4
        tiles = np.pad(act, [(0, 0)] * 3 + [(0, pad)]).reshape(act.shape[:3] + (-1, 4)).any(axis=(0, 4))
        forms["index"]["skipped_brick_isovalue_frac"] = float(1.0 - act.mean())
        forms["index"]["skipped_tile_frac"] = float(1.0 - tiles.mean())
    for v in stages.values():
        v["GBps"] = v["algorithmic_bytes"] / (v["ms"] * 1e-3) / 1e9
        v["frac_of_measured_hbm"] = v["GBps"] / peak

    # the roofline of the step (one chr_isosurface call: k_decode, then
    # k_mc_count, three scan kernels and k_mc_emit_stored) on the fused
    # algorithmic bytes: what the method must move, levels 0..2 of the CHR
    # read once and the mesh written once
    fb = fused_bytes(st, LEVEL, T)
    achieved = fb / (ms_step * 1e-3) / 1e9
    traffic = profiled_traffic()
    roofline = {"bound": "hbm", "kernel": "chr_isosurface (k_decode + k_mc_count + scans + k_mc_emit_stored)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": fb,
                "traffic_note": "DRAM read+write bytes of one call from the committed ncu capture "
                                "(profiles/chr_isosurface_turb1024.md); null when its sources changed since"}

    # end to end through the public API from pinned host memory: every step
    # uploads the CHR's bytes (chr_deserialize: host validation, upload),
    # runs chr_isosurface and reads the triangle counts back
    e2e = None
    if not args.no_e2e:
        blob = torch.empty(chr.chr_serialized_size(h), dtype=torch.uint8).pin_memory()
        blob = chr.chr_serialize(h, out=blob)
        counts_host = torch.empty(len(ISOVALUES), dtype=torch.int64).pin_memory()

        def e2e_step(mesh_host=None):
            h2 = chr.chr_deserialize(blob)
            chr.chr_isosurface(h2, LEVEL, ISOVALUES, cap, tris=tris, counts=counts, err=err)
            counts_host.copy_(counts, non_blocking=True)
            if mesh_host is not None:
                for j, t in enumerate(ntri):
                    mesh_host[j].copy_(tris[j, :t].reshape(-1), non_blocking=True)
            torch.cuda.synchronize()
            h2.free()

        e2e_step()
        ke = min(args.steps, 5)
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        e2e_ms = (time.perf_counter() - t0) / ke * 1e3
        e2e = {"value": world * 4.0 * N / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": int(blob.numel()), "d2h_bytes_per_step": 8 * len(ISOVALUES),
               "steps": ke, "clock": "host wall clock (chr_deserialize synchronizes)",
               "mesh": "consumed on the device"}
        try:
            mesh_host = [torch.empty(9 * t, dtype=torch.float32).pin_memory() for t in ntri]
            e2e_step(mesh_host)
            t0 = time.perf_counter()
            for _ in range(2):
                e2e_step(mesh_host)
            m_ms = (time.perf_counter() - t0) / 2 * 1e3
            e2e["mesh_d2h"] = {"value": world * 4.0 * N / (m_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": m_ms,
                               "d2h_bytes_per_step": 36 * T + 8 * len(ISOVALUES), "steps": 2}
            del mesh_host
        except RuntimeError as ex:
            e2e["mesh_d2h"] = {"unavailable": str(ex).splitlines()[0][:200]}
        del blob

    del tris
    h.free()
    torch.cuda.empty_cache()

    side = None if args.no_side or world > 1 else side_512(args)
    adjoint = None if args.no_adjoint or world > 1 else adjoint_timing()
    if adjoint is not None and not args.no_cpu_baseline:
        adjoint["cpu_baseline"] = adjoint_cpu_baseline()
    batch = None
    if not args.no_batched and world == 1:
        from paper_2408_05462_gb300 import batched

        batch = batched.measure(256, 256, reps=20)
        batch["roofline"] = {"bound": "hbm", "achieved": batch["batched_algorithmic_GBps"], "peak": peak,
                             "unit": "GB/s", "frac": batch["batched_algorithmic_GBps"] / peak, "peak_kind": peak_kind}
        if not args.no_cpu_baseline:
            batch["cpu_baseline"] = batched_cpu_baseline()
    serving = None if args.no_serve or world > 1 else serve_measurement(args)

    ntiles = ((n - 1 + 31) // 32) * ((n - 1 + 7) // 8) ** 2
    per_step = 1 + (5 if ntiles >= 2048 * 64 else 1)  # decoder, then count + 3 scans + emit, or the single pass
    out = {
        "metric": "field GB/s (decode+fix+marching cubes), % HBM roofline; serve p50/p99 ms",
        "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(n, args, {"parallelism": "replicas" if world > 1 else "single"}),
        "roofline": roofline,
        "tris_per_s": T / (ms_step * 1e-3),
        "stages": stages, "forms": forms,
        "triangles": ntri, "compressed_bytes": comp_bytes, "compression_ratio": 4.0 * N / comp_bytes,
        "exceptions": st["exceptions"],
        "gpu_launches": per_step * args.steps,
        "e2e": e2e,
    }
    if side is not None:
        out["turb512"] = side
    if adjoint is not None:
        out["adjoint"] = adjoint
    if batch is not None:
        out["batched"] = batch
    if serving is not None:
        out["serve"] = serving
    if rank == 0:
        clk_s = clk.summary()
        if clk_s:
            out["clocks"] = clk_s
        if subs is not None:
            out["cpu_baseline"] = cpu_baseline(subs, np.array(eb, np.float32))
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

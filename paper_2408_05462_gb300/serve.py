"""Request loop of the visualization side: CHR timesteps stay resident on the
device, and requests for (timestep, isovalue, accuracy level, subvolume)
arrive over time (Sec. 2: the analysis side asks for the data it needs at
the accuracy it needs; Sec. 1, in-transit visualization).

Every request is one chr_serve_request call (decode only the bricks of its
box at its level into a pitched box field, marching cubes of the box, the
count copied back) on one of a few CUDA streams ("slots").  Scheduling is continuous: whenever a request
finishes, its slot and memory are released and the next waiting requests are
admitted in arrival order, so new work starts while older work is still on the
device.  Admission is by a device-memory budget: a request holds its box
field, its workspace and room for an upper bound on its triangles, taken from
the CHR's stored value index (chr_brick_index, Sec. 2.1): a brick's cells
can only be active for k if the range over the vertices they touch
straddles k, and a cell has at most 5 triangles.  With the bound as capacity
no request can overflow.  (dilate_range builds a looser index from
chr_brick_range's per-brick extrema, for handles without a stored one.)

Results are triangles in box-local grid coordinates, left on the device (for
the renderer), plus the count copied to the host.  A request's result does
not depend on what else is in flight: every kernel writes only its own
request's buffers, and the kernels are deterministic.
"""
from __future__ import annotations

import argparse
import json
import time
from collections import OrderedDict, deque
from dataclasses import dataclass

import numpy as np
import torch

from . import chr

# accuracy levels of a served timestep (relative to the value range) and the
# isovalues whose case bytes the encoder fixes (Sec. 2.2)
LEVELS_REL = (1e-2, 1e-3, 1e-4, 1e-5)
FIX_ISOVALUES = (-1.0, -0.5, 0.5, 1.0)
MAX_TRIS_PER_CELL = 5


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the run
    step: int       # timestep id
    k: float
    level: int
    origin: tuple   # (x0, y0, z0) grid vertex
    size: tuple     # (nx, ny, nz) vertices


@dataclass
class Result:
    rid: int
    ntris: int
    bound: int
    admit_ms: float   # host time of admission, ms after start
    done_ms: float    # device completion, ms after start
    latency_ms: float
    retire_ms: float  # host time the loop saw it finish and released its memory
    nbytes: int       # device memory it held while in flight
    tris: torch.Tensor | None = None  # [ntris, 3, 3] float32 on the device (keep_results)


def dilate_range(rng: np.ndarray):
    """(min, max) per brick over the brick and its +x, +y, +z neighbours (the
    vertices a brick's cells touch).  rng: [nbz, nby, nbx, 2]."""
    mn = rng[..., 0].copy()
    mx = rng[..., 1].copy()
    for axis in range(3):
        n = mn.shape[axis]
        if n < 2:
            continue
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        mn[lo] = np.minimum(mn[lo], mn[hi])
        mx[lo] = np.maximum(mx[lo], mx[hi])
    return mn, mx


@dataclass
class Timestep:
    step: int
    handle: chr.Chr
    shape: tuple           # (nz, ny, nx)
    index: list            # per level: (min, max) over each brick's cell vertices, [nbz, nby, nbx]
    resident_bytes: int

    def tri_bound(self, level: int, k: float, origin, size) -> int:
        mn, mx = self.index[level]
        return chr.chr_box_tri_bound(mn, mx, origin, size, k)


@dataclass
class _Flight:
    req: Request
    slot: int
    block: tuple  # (offset, bytes) in the arena; the triangles come first
    bound: int
    admit_ms: float
    done: torch.cuda.Event
    count_host: torch.Tensor  # pinned (triangle count, error word)
    keep_results: bool


class FreeList:
    """First-fit allocation of byte ranges in 256-byte units, with freed
    ranges merged back into their neighbours."""

    def __init__(self, size: int):
        self.size = int(size)
        self.free = [(0, self.size)]  # (offset, bytes), sorted by offset, coalesced

    def alloc(self, nbytes: int):
        n = (int(nbytes) + 255) & ~255
        for i, (off, size) in enumerate(self.free):
            if size >= n:
                if size == n:
                    del self.free[i]
                else:
                    self.free[i] = (off + n, size - n)
                return off, n
        return None

    def release(self, off: int, n: int):
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        self.free.insert(i, (off, n))
        if i + 1 < len(self.free) and off + n == self.free[i + 1][0]:  # merge with the next range
            self.free[i] = (off, n + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:  # and the previous one
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]


class Arena(FreeList):
    """The requests' device memory: one allocation made once and handed out
    by the free list, so serving never calls the device allocator."""

    def __init__(self, nbytes: int):
        super().__init__(nbytes)
        self.buf = torch.empty(self.size, dtype=torch.uint8, device="cuda")

    def view(self, off: int, n: int) -> torch.Tensor:
        return self.buf[off:off + n]


class Server:
    """Resident CHR timesteps and a continuous-batching request loop.

    budget_bytes bounds the device memory of the requests in flight (box
    fields, workspaces and triangle capacity): it is the size of the arena the
    requests' memory comes from, allocated at the first run.  The resident
    CHRs are counted in `resident_bytes` and limited by max_resident
    timesteps."""

    def __init__(self, budget_bytes: int = 96 << 30, slots: int = 4, max_resident: int = 2,
                 levels_rel=LEVELS_REL, fix_isovalues=FIX_ISOVALUES):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.budget = int(budget_bytes)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.max_resident = int(max_resident)
        self.levels_rel = tuple(levels_rel)
        self.fix_isovalues = tuple(fix_isovalues)
        self.steps: OrderedDict[int, Timestep] = OrderedDict()
        self._slot_bufs = []
        self.arena = None
        self.host_ms = 0.0  # host time spent on admission and launches in the last run

    def _bufs(self, slot: int):
        """Per-slot pinned host words (triangle count, error word), reused
        request after request (a slot runs one request at a time)."""
        while len(self._slot_bufs) <= slot:
            self._slot_bufs.append(torch.zeros(2, dtype=torch.int64, pin_memory=True))
        return self._slot_bufs[slot]

    def with_slots(self, slots: int) -> "Server":
        """A server over the same resident timesteps with `slots` streams (1:
        the plain path, one request after another)."""
        other = object.__new__(Server)
        other.__dict__.update(self.__dict__)
        other.streams = self.streams[:slots] if slots <= len(self.streams) else \
            self.streams + [torch.cuda.Stream() for _ in range(slots - len(self.streams))]
        other._slot_bufs = []
        other.arena = None
        return other

    @property
    def resident_bytes(self) -> int:
        return sum(t.resident_bytes for t in self.steps.values())

    # ---- timesteps ------------------------------------------------------
    def ingest(self, step: int, field: torch.Tensor) -> Timestep:
        """Compress a timestep into a resident CHR with one level per entry
        of levels_rel and build its brick index; evicts the oldest timestep
        beyond max_resident.  Not to be called while `run` is serving."""
        lo, hi = torch.aminmax(field)
        vrange = float(hi) - float(lo)
        ebs = [r * vrange for r in self.levels_rel]
        h = chr.chr_compress(field, ebs, self.fix_isovalues, "fix")
        # the CHR's stored value index: each brick's range over its cell
        # vertices, exactly the vertices its cells touch (no decoder pass)
        index = []
        for l in range(len(ebs)):
            ix = chr.chr_brick_index(h, l).cpu().numpy()
            index.append((np.ascontiguousarray(ix[..., 0]), np.ascontiguousarray(ix[..., 1])))
        st = h.stats()
        ts = Timestep(step, h, tuple(field.shape), index, int(sum(st["level_bytes"])))
        self.steps[step] = ts
        while len(self.steps) > self.max_resident:
            _, old = self.steps.popitem(last=False)
            old.handle.free()
        return ts

    # ---- one request ------------------------------------------------------
    def request_bytes(self, req: Request, bound: int) -> int:
        return chr.chr_serve_request_bytes(req.size, max(bound, 1))

    def _launch(self, req: Request, slot: int, bound: int, block, t0: float, keep_results: bool) -> _Flight:
        ts = self.steps[req.step]
        s = self.streams[slot]
        result = self._bufs(slot)
        mem = self.arena.view(*block)
        with torch.cuda.stream(s):
            chr.chr_serve_request(ts.handle, req.level, req.origin, req.size, req.k, mem, bound, result, stream=s)
            done = torch.cuda.Event(enable_timing=True)
            done.record(s)
        admit_ms = (time.perf_counter() - t0) * 1e3
        return _Flight(req, slot, block, bound, admit_ms, done, result, keep_results)

    # ---- the loop ---------------------------------------------------------
    def run(self, requests, keep_results: bool = False, poll_s: float = 20e-6):
        """Serve `requests` (arrival times in seconds from now) in real time.
        Returns the results in request order."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in reqs:
            if r.step not in self.steps:
                raise KeyError("timestep %d is not resident" % r.step)
            nz, ny, nx = self.steps[r.step].shape
            if not (0 <= r.level < len(self.levels_rel)):
                raise ValueError("request %d: level out of range" % r.rid)
            if min(r.size) < 2 or any(o < 0 for o in r.origin) or r.origin[0] + r.size[0] > nx or \
                    r.origin[1] + r.size[1] > ny or r.origin[2] + r.size[2] > nz:
                raise ValueError("request %d: box outside the grid" % r.rid)
        if self.arena is None or self.arena.size != self.budget:
            self.arena = None
            self.arena = Arena(self.budget)
        pending = deque(reqs)
        waiting: deque = deque()
        flights: dict[int, _Flight] = {}
        free_slots = list(range(len(self.streams)))[::-1]
        results: dict[int, Result] = {}
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        start.record(torch.cuda.current_stream())
        host = 0.0
        while pending or waiting or flights:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append([pending.popleft(), None, None])
            progressed = False
            for slot, fl in list(flights.items()):
                if fl.done.query():
                    n, e = int(fl.count_host[0]), int(fl.count_host[1])
                    if e != 0 or n > fl.bound:
                        raise RuntimeError("request %d: device error %d, %d triangles for capacity %d"
                                           % (fl.req.rid, e, n, fl.bound))
                    done_ms = start.elapsed_time(fl.done)
                    tris = None
                    if fl.keep_results:  # copied out before the block goes back to the arena
                        tris = self.arena.view(fl.block[0], 36 * n).clone().view(torch.float32).view(n, 3, 3)
                    results[fl.req.rid] = Result(fl.req.rid, n, fl.bound, fl.admit_ms, done_ms,
                                                 done_ms - 1e3 * fl.req.arrival,
                                                 (time.perf_counter() - t0) * 1e3, fl.block[1], tris)
                    self.arena.release(*fl.block)
                    free_slots.append(slot)
                    del flights[slot]
                    progressed = True
            while waiting and free_slots:
                ta = time.perf_counter()
                head = waiting[0]
                if head[1] is None:  # the triangle bound, once a slot could take the request
                    r = head[0]
                    head[1] = self.steps[r.step].tri_bound(r.level, r.k, r.origin, r.size)
                    head[2] = self.request_bytes(r, head[1])
                    if head[2] > self.budget:
                        raise MemoryError("request %d needs %d bytes, above the budget" % (r.rid, head[2]))
                block = self.arena.alloc(head[2])
                if block is None:  # no room until a request in flight retires
                    host += time.perf_counter() - ta
                    break
                r, b, _ = waiting.popleft()
                slot = free_slots.pop()
                flights[slot] = self._launch(r, slot, b, block, t0, keep_results)
                progressed = True
                host += time.perf_counter() - ta
            if not progressed:
                if pending and not waiting and not flights:
                    time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 1e-3)))
                elif poll_s > 0:
                    time.sleep(poll_s)
        self.host_ms = host * 1e3
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]


def make_requests(n: int, rate: float, grid, steps, seed: int = 5, side=(64, 512), levels: int = 4):
    """n requests with Poisson arrivals at `rate` per second (rate <= 0: all
    at time 0), k ~ U[-1, 1], level ~ U{0..levels-1}, each box side ~
    U{side[0]..side[1]} (clipped to the grid) at a uniform offset, timestep
    uniform over `steps`.  grid = (nx, ny, nz)."""
    g = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(g.exponential(1.0 / rate, size=n)) if rate > 0 else np.zeros(n)
    out = []
    for i in range(n):
        size = tuple(int(min(g.integers(side[0], side[1] + 1), grid[a])) for a in range(3))
        origin = tuple(int(g.integers(0, grid[a] - size[a] + 1)) for a in range(3))
        out.append(Request(i, float(t[i]), int(steps[int(g.integers(0, len(steps)))]), float(g.uniform(-1.0, 1.0)),
                           int(g.integers(0, levels)), origin, size))
    return out


def percentiles(lat_ms):
    a = np.asarray(lat_ms, np.float64)
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max())}


def field_bytes(reqs) -> int:
    return sum(4 * r.size[0] * r.size[1] * r.size[2] for r in reqs)


def measure(server: Server, grid, steps, n_req: int = 200, rates=(0.25, 0.5, 0.8), seed: int = 5, slots_plain=1):
    """Capacity (all requests at t=0), then Poisson runs at fractions of it;
    the same burst through a one-slot server is the plain sequential path."""
    burst = make_requests(n_req, 0.0, grid, steps, seed)
    server.run(burst)  # warm the allocator and the kernels
    res = server.run(burst)
    span_s = max(r.done_ms for r in res) / 1e3
    capacity = n_req / span_s
    out = {"requests": n_req, "slots": len(server.streams), "budget_gib": server.budget / 2 ** 30,
           "capacity_req_s": capacity, "burst_field_gbs": field_bytes(burst) / span_s / 1e9,
           "burst_tris_per_s": sum(r.ntris for r in res) / span_s,
           "host_ms_per_request": server.host_ms / n_req,
           "tris_over_bound": sum(r.ntris for r in res) / max(1, sum(r.bound for r in res))}
    plain = server.with_slots(slots_plain)
    plain.run(burst)
    res1 = plain.run(burst)
    span1 = max(r.done_ms for r in res1) / 1e3
    out["plain_one_stream_req_s"] = n_req / span1
    out["rates"] = []
    for frac in rates:
        reqs = make_requests(n_req, frac * capacity, grid, steps, seed + 1)
        rr = server.run(reqs)
        span = max(r.done_ms for r in rr) / 1e3
        d = {"load": frac, "rate_req_s": frac * capacity, "throughput_req_s": n_req / span}
        d.update(percentiles([r.latency_ms for r in rr]))
        out["rates"].append(d)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="serve (isovalue, level, subvolume) requests over resident CHRs")
    ap.add_argument("--n", type=int, default=1024, help="grid side of a timestep")
    ap.add_argument("--timesteps", type=int, default=2)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--budget-gib", type=float, default=96.0)
    ap.add_argument("--seed", type=int, default=1024)
    args = ap.parse_args(argv)
    from . import build, synth

    build.build()
    srv = Server(int(args.budget_gib * 2 ** 30), args.slots, max_resident=args.timesteps)
    f = synth.turbulence_cuda(args.n, args.seed)
    for t in range(args.timesteps):
        if t:
            f = torch.roll(f, shifts=(1, 2, 3), dims=(0, 1, 2))  # advect by (3, 2, 1) voxels (x, y, z)
        srv.ingest(t, f)
    del f
    grid = (args.n, args.n, args.n)
    out = measure(srv, grid, list(range(args.timesteps)), args.requests)
    out["grid"] = args.n
    out["resident_gib"] = srv.resident_bytes / 2 ** 30
    print(json.dumps(out))


if __name__ == "__main__":
    main()

"""Continuous-batching reconstruction server.

Each request carries a geometry (2D fan or 3D cone beam), measured projections and a
number of NAG iterations on the Tikhonov objective (Section "Numerical Experiments",
Eq. (exp_tikh)).  Requests of one shape bucket -- geometry, iterations, power iterations,
lambda -- share W, its norm and therefore every projector call, so the server batches them:

* A *slot batch* per bucket holds the NAG state of up to C requests (``NAGSlots``) on its
  own CUDA stream.  One iteration of all its occupied slots is captured once per occupancy
  n into a CUDA graph and replayed; each slot runs its own momentum sequence (its iteration
  counter lives on the device), so requests join a running batch at any iteration boundary
  (continuous batching, as in LLM serving) and leave when their iterations are done: the
  host queues the copy of their result and moves the last occupied slot into the freed one.
  Every projector call of a replay serves all the batch's requests at once (the kernels
  share the geometry of an entry among the batch items).
* Requests are admitted in arrival order: into a free slot of a batch of their bucket, else
  into a new batch while its memory (C request footprints) fits the budget (120 GB by
  default) and a batch slot of the request's cost class is free.  A request waiting for
  memory holds back all later ones (none starves); one whose class is full does not hold
  back cheaper ones.  Batch streams are prioritised by cost class (cheapest highest), so a
  small request's blocks start before the remaining blocks of a large one, and the costlier
  a class the fewer of its batches run at once (16, 4, 2, 1 for four classes).
* ||W|| comes from a power iteration on the device, once per geometry (start vector seeded
  by the geometry); a batch that empties stays idle with its graphs for later requests of
  its bucket and is released, oldest first, when memory is needed.
* The host keeps at most two iterations of a batch in flight, so that admissions and
  read-outs are not queued behind many iterations; it polls events and returns results with
  their latency.  A request that cannot run (refused geometry, projections of the wrong
  size, more memory than the whole budget, a failed set-up) comes back with `error` set.

Every device step is a library kernel (projectors, csm_dot / csm_axpby / csm_fista_coeffs).
A request's result does not depend on the other requests of its batch beyond rounding: each
batch item's arithmetic is its own (the 2D kernels and the reductions in a fixed order,
bit-identical; the 3D kernels per item in a fixed order, equal to rounding across batch
sizes).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from ._capi import CsmError
from .projector import Projector
from .sched import admit_order, geometry_key, geometry_seed
from .solvers import NAG, NAGSlots, power_norm2_device


@dataclasses.dataclass
class Request:
    id: int
    geom: dict
    sino: np.ndarray                 # measured projections, [n_views, (nv,) nu]
    arrival: float = 0.0             # seconds after the start of serving
    iters: int = 20
    lam: float = 1e-4
    power_iters: int = 20
    seed: int = 0                    # caller's tag (the power iteration is seeded by the geometry)
    result: np.ndarray | None = None
    t_admit: float | None = None
    t_done: float | None = None
    error: str | None = None         # why the request could not run (then result is None)

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def cost_estimate(geom: dict, iters: int, power_iters: int) -> float:
    """Relative device work of a request: projector calls x views x voxels x the entries per
    voxel and view (about 2.5 elements in 2D, 6 elements in 3D)."""
    nvox = geom["nx"] * geom["ny"] * geom.get("nz", 1)
    per = 6.0 if geom.get("dim", 2) == 3 else 2.5
    return 2.0 * (iters + power_iters + 1) * geom["n_views"] * nvox * per


def priority_range():
    """(lowest, highest) stream priority of the device (a lower number is a higher priority)."""
    fn = getattr(torch.cuda.Stream, "priority_range", None)
    if fn is not None:
        lo, hi = fn()
        return int(lo), int(hi)
    return 0, -1


def footprint_bytes(geom: dict, elem: int = 4) -> int:
    """Device memory one request holds: NAG state u, y, g (3 volumes), residual and data
    (2 sinograms), power-iteration vectors (2 volumes, 1 sinogram), the projector's
    workspaces (2 volumes, 1 sinogram; the back projection's differenced sinogram counts
    as four) and its geometry table."""
    nvox = geom["nx"] * geom["ny"] * geom["nz"]
    nsino = geom["n_views"] * geom.get("nv", 1) * geom["nu"]
    table = geom["n_views"] * (geom["nu"] + 1) * 48 + geom["n_views"] * (geom.get("nv", 1) + 1) * 48
    return elem * (7 * nvox + 7 * nsino) + table + (1 << 20)


def bucket_of(req: Request):
    return (geometry_key(req.geom), int(req.iters), int(req.power_iters), float(req.lam))


class _Batch:
    """A slot batch of one bucket: projector, slot solver, graphs per occupancy, stream."""

    def __init__(self, bucket, P, nag, stream, lv, plv, capacity, nbytes, dim):
        self.bucket, self.P, self.nag, self.stream = bucket, P, nag, stream
        self.lv, self.plv, self.C, self.nbytes, self.dim = lv, plv, capacity, nbytes, dim
        self.slots = []            # [request, iterations issued, pinned result buffer]
        self.graphs = {}
        self.inflight = []         # events of issued iterations
        self.pending_out = []      # (request, pinned buffer, event) read-outs queued


class ReconServer:
    """budget_bytes: device memory the admitted batches may hold; max_active: batches on the
    GPU at once; max_slots: requests per batch (2D, 3D); use_graphs: replay captured
    iterations (else launch them one by one); priorities: order streams by request cost;
    cost_edges: cost thresholds between priority levels (default: decades of
    ``cost_estimate`` from 1e10, the cheapest level highest); level_caps: batches of each
    level (highest first) that may run at once; max_idle: emptied batches kept for reuse."""

    def __init__(self, device="cuda:0", budget_bytes: int = 120 << 30, max_active: int = 16,
                 use_graphs: bool = True, priorities: bool = True, cost_edges=None, level_caps=None,
                 max_idle: int = 4, max_slots=(8, 4), inflight: int = 2):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.use_graphs = use_graphs
        self.max_slots = tuple(int(v) for v in max_slots)
        self.inflight = max(1, int(inflight))
        lo, hi = priority_range() if priorities else (0, 0)
        hi = max(hi, lo - 3)                                  # at most four levels
        self.levels = list(range(hi, lo + 1))               # highest priority first
        self.cost_edges = list(cost_edges) if cost_edges is not None else \
            [10.0 ** e for e in range(10, 10 + len(self.levels) - 1)]
        self.pool = {lv: [torch.cuda.Stream(device=self.device, priority=lv) for _ in range(self.max_active)]
                     for lv in self.levels}
        if level_caps is None:
            level_caps = [self.max_active, 4, 2, 1][:len(self.levels)]
            if len(self.levels) > 1:
                level_caps[-1] = 1
        self.caps = {lv: max(1, min(int(c), self.max_active)) for lv, c in zip(self.levels, level_caps)}
        self.running = {lv: 0 for lv in self.levels}      # batches (with requests) per level
        self.sigma_cache = {}        # (geometry key, power iterations) -> (||W||^2 on the device, event)
        self.sigma_hits = 0
        self.max_idle = int(max_idle)
        self.batches = []            # batches holding requests
        self.idle = []               # emptied batches kept for reuse, oldest first
        self.joined = 0              # requests that joined a batch already holding requests
        self.batch_hits = 0          # batches reused from the idle list
        self.max_occupancy = 0
        self.slots = self.max_active
        self._deferred = []          # projectors released once the device is idle

    def level_of(self, req: Request) -> int:
        c = cost_estimate(req.geom, req.iters, req.power_iters)
        i = sum(1 for e in self.cost_edges if c >= e)
        return self.levels[min(i, len(self.levels) - 1)]

    def capacity_of(self, req: Request) -> int:
        """Slots of a new batch for this request: the per-dimension maximum, fewer when the
        budget holds fewer request footprints (at least one)."""
        top = self.max_slots[1] if req.geom.get("dim", 2) == 3 else self.max_slots[0]
        return max(1, min(top, self.budget // max(footprint_bytes(req.geom), 1)))

    def batch_bytes(self, req: Request) -> int:
        return self.capacity_of(req) * footprint_bytes(req.geom)

    # -----------------------------------------------------------------------------------
    def _sigma2(self, P, req, s):
        key = (geometry_key(req.geom), req.power_iters)
        hit = self.sigma_cache.get(key)
        if hit is None:
            gen = torch.Generator(device=self.device)
            gen.manual_seed(geometry_seed(req.geom))
            start = torch.randn((1,) + tuple(P.vol_shape), generator=gen, device=self.device, dtype=torch.float32)
            sig2 = power_norm2_device(P, iters=req.power_iters, start=start)
            ev = torch.cuda.Event()
            ev.record(s)
            self.sigma_cache[key] = (sig2, ev)
            return sig2
        sig2, ev = hit
        s.wait_event(ev)
        sig2.record_stream(s)
        self.sigma_hits += 1
        return sig2

    def _new_batch(self, req: Request) -> _Batch:
        lv = self.level_of(req)
        s = self.pool[lv].pop()
        try:
            with torch.cuda.device(self.device), torch.cuda.stream(s):
                P = Projector(req.geom, device=self.device)
                sig2 = self._sigma2(P, req, s)
                C = self.capacity_of(req)
                nag = NAGSlots(P, C, req.iters, req.lam, sig2, sigma_scale=1.01)
                nag.reserve()
        except Exception:
            self.pool[lv].append(s)
            raise
        return _Batch(bucket_of(req), P, nag, s, lv, lv, C, self.batch_bytes(req), req.geom.get("dim", 2))

    def _join(self, b: _Batch, req: Request, now: float):
        data = torch.from_numpy(np.ascontiguousarray(req.sino, dtype=np.float32))
        if data.numel() != b.nag.p[0].numel():
            raise ValueError("projections of %d values for a geometry of %d" % (data.numel(), b.nag.p[0].numel()))
        with torch.cuda.device(self.device), torch.cuda.stream(b.stream):
            b.nag.load(len(b.slots), data.pin_memory().to(self.device, non_blocking=True))
        b.slots.append([req, 0, torch.empty(tuple(b.P.vol_shape), dtype=torch.float32).pin_memory()])
        req.t_admit = now
        self.max_occupancy = max(self.max_occupancy, len(b.slots))

    def _issue(self, b: _Batch):
        """One iteration of the batch's occupied slots; read-out and compaction of the slots
        that finish with it."""
        n = len(b.slots)
        with torch.cuda.device(self.device), torch.cuda.stream(b.stream):
            if self.use_graphs:
                gr = b.graphs.get(n)
                if gr is None:
                    gr = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(gr, stream=b.stream):
                        b.nag.step(n)
                    b.graphs[n] = gr
                    # capturing does not run the work: run it once
                gr.replay()
            else:
                b.nag.step(n)
            ev = torch.cuda.Event()
            ev.record(b.stream)
            b.inflight.append(ev)
            for sl in b.slots:
                sl[1] += 1
            for i in reversed(range(n)):
                req, k, buf = b.slots[i]
                if k >= req.iters:
                    buf.copy_(b.nag.u[i], non_blocking=True)
                    done = torch.cuda.Event()
                    done.record(b.stream)
                    b.pending_out.append((req, buf, done))
                    last = len(b.slots) - 1
                    if i != last:
                        b.nag.move(last, i)
                        b.slots[i] = b.slots[last]
                    b.slots.pop()

    def _memory_blocked(self, pending, now, used) -> bool:
        for r in pending:
            if r.arrival > now:
                return False
            if any(b.bucket == bucket_of(r) and len(b.slots) < b.C for b in self.batches):
                return False
            lv = self.level_of(r)
            if self.running[lv] >= self.caps[lv]:
                continue
            return used + self.batch_bytes(r) > self.budget
        return False

    def _drop(self, b: _Batch):
        self._deferred.append(b.P)
        b.graphs = {}
        b.nag = None

    def _release_deferred(self):
        for P in self._deferred:
            P.close()
        self._deferred = []

    # -----------------------------------------------------------------------------------
    def serve(self, requests, realtime: bool = True, poll_s: float = 2e-4):
        """Serve `requests`.  With realtime, arrivals follow the wall clock from the start of
        the call; otherwise every request is available at once.  Returns the requests with
        result, t_admit, t_done filled in (seconds)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        if not realtime:
            for r in pending:
                r.arrival = 0.0
        for r in [r for r in pending if footprint_bytes(r.geom) > self.budget]:
            r.error = "needs %d bytes of device memory, more than the budget of %d" % (footprint_bytes(r.geom),
                                                                                       self.budget)
            r.t_done = r.arrival
            pending.remove(r)
        used = 0
        t0 = time.perf_counter()
        while pending or self.batches:
            now = time.perf_counter() - t0
            # admissions in arrival order: a free slot of the bucket's batch, else a new batch
            i = 0
            while i < len(pending) and pending[i].arrival <= now:
                req = pending[i]
                bk = bucket_of(req)
                target = next((b for b in self.batches if b.bucket == bk and len(b.slots) < b.C), None)
                try:
                    if target is not None:
                        self._join(target, req, now)
                        self.joined += 1
                        pending.pop(i)
                        continue
                    reuse = next((j for j, b in enumerate(self.idle) if b.bucket == bk), None)
                    lv = self.level_of(req)
                    if self.slots <= 0 or self.running[lv] >= self.caps[lv]:
                        i += 1
                        continue
                    need = 0 if reuse is not None else self.batch_bytes(req)
                    while (reuse is None and self.idle and
                           used + self.idle_bytes() + need > self.budget):
                        self._drop(self.idle.pop(0))
                    if used + self.idle_bytes() + need > self.budget:
                        break                                   # waits for memory; later ones wait too
                    if reuse is not None:
                        b = self.idle.pop(reuse)
                        self.batch_hits += 1
                        b.stream = self.pool[b.lv].pop()
                    else:
                        b = self._new_batch(req)
                    used += b.nbytes
                    self.slots -= 1
                    self.running[b.lv] += 1
                    self.batches.append(b)
                    self._join(b, req, now)
                    pending.pop(i)
                except (CsmError, ValueError, RuntimeError) as e:   # this request cannot run
                    req.error = "%s: %s" % (type(e).__name__, e)
                    req.t_done = time.perf_counter() - t0
                    pending.pop(i)
            # iterations: at most `inflight` per batch queued on the GPU
            issued = False
            for b in self.batches:
                b.inflight = [e for e in b.inflight if not e.query()]
                if b.slots and len(b.inflight) < self.inflight:
                    self._issue(b)
                    issued = True
            # results
            still = []
            for b in self.batches:
                keep = []
                for req, buf, done in b.pending_out:
                    if done.query():
                        req.result = buf.numpy().copy()
                        req.t_done = time.perf_counter() - t0
                    else:
                        keep.append((req, buf, done))
                b.pending_out = keep
                if not b.slots and not b.pending_out:
                    b.inflight = []
                    self.pool[b.lv].append(b.stream)
                    self.slots += 1
                    self.running[b.lv] -= 1
                    used -= b.nbytes
                    if self.use_graphs and self.max_idle > 0:
                        self.idle.append(b)
                        while len(self.idle) > self.max_idle:
                            self._drop(self.idle.pop(0))
                    else:
                        self._drop(b)
                else:
                    still.append(b)
            self.batches = still
            if not self.batches and self._deferred:
                self._release_deferred()
            if not issued and (self.batches or pending):
                time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        self._release_deferred()
        return requests

    def idle_bytes(self) -> int:
        return sum(b.nbytes for b in self.idle)

    def close(self):
        """Release the idle batches and their geometry tables."""
        while self.idle:
            self._drop(self.idle.pop(0))
        torch.cuda.synchronize(self.device)
        self._release_deferred()


def solve_alone(req: Request, device="cuda:0") -> np.ndarray:
    """The same reconstruction with plain, unbatched calls on the default stream (the
    reference the serving results are compared with)."""
    dev = torch.device(device)
    P = Projector(req.geom, device=dev)
    p = torch.from_numpy(np.ascontiguousarray(req.sino, dtype=np.float32)).to(dev).reshape((1,) + tuple(P.sino_shape))
    gen = torch.Generator(device=dev)
    gen.manual_seed(geometry_seed(req.geom))
    start = torch.randn((1,) + tuple(P.vol_shape), generator=gen, device=dev, dtype=torch.float32)
    sig2 = power_norm2_device(P, iters=req.power_iters, start=start)
    nag = NAG(P, 1, lam=req.lam, sigma2_device=sig2, sigma_scale=1.01)
    u = nag.run(p, iters=req.iters)
    out = u[0].cpu().numpy().copy()
    P.close()
    return out


def serve_unbatched(requests, device="cuda:0", realtime: bool = True):
    """The unbatched reference server, run for real: requests one at a time in arrival order
    with plain calls (solve_alone), waiting for each arrival on the wall clock.  Fills result,
    t_admit and t_done like ReconServer.serve."""
    pending = sorted(requests, key=lambda r: r.arrival)
    if not realtime:
        for r in pending:
            r.arrival = 0.0
    t0 = time.perf_counter()
    for r in pending:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.t_admit = time.perf_counter() - t0
        try:
            r.result = solve_alone(r, device=device)
        except (CsmError, ValueError, RuntimeError) as e:
            r.error = "%s: %s" % (type(e).__name__, e)
        torch.cuda.synchronize(torch.device(device))
        r.t_done = time.perf_counter() - t0
    return requests


def latency_stats(lat):
    lat = np.sort(np.asarray(lat, dtype=np.float64))
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def fifo_latencies(arrivals, service):
    """Latencies of a single server taking requests one at a time in arrival order."""
    t = 0.0
    out = []
    for a, s in sorted(zip(arrivals, service)):
        t = max(t, a) + s
        out.append(t - a)
    return out

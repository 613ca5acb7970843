"""Continuous-batching reconstruction server.

Each request carries a geometry (2D fan or 3D cone beam), measured projections and a
number of NAG iterations on the Tikhonov objective (Section "Numerical Experiments",
Eq. (exp_tikh)).  The server

* admits requests in arrival order while their device-memory footprint fits a budget
  (120 GB by default) and a slot of their cost class is free; requests that arrive while
  others run are admitted as soon as memory and slots free up (a request waiting for a slot
  of its class does not hold back cheaper ones; one waiting for memory holds back all later
  ones, so that none starves);
* runs every admitted request on its own CUDA stream, so the projections of different
  requests overlap on the GPU; the stream's priority follows the request's estimated cost
  (cheapest requests highest), so the block scheduler starts the blocks of short requests
  before the remaining blocks of long ones: a small request does not wait for a large one to
  drain, which is what a FIFO of whole requests would make it do.  The costlier a class, the
  fewer of its requests run at once (16, 4, 2, 1 for the four classes by default): one large
  3D solve already fills the GPU, and large requests sharing it would all finish late.  A
  request that has already waited longer than its own estimated service time (its cost
  times the smallest time per cost seen on completed requests) gets a stream one level
  higher, so that the requests that waited longest are not also the slowest to run;
* estimates ||W|| by power iteration on the device (the scalar never leaves the GPU) once
  per geometry: the start vector is seeded by the geometry, so the estimate is a function of
  the geometry alone and later requests of the same geometry reuse it (after an event on the
  stream that computed it); then captures the request's NAG iterations once into a CUDA
  graph and replays it: the whole solve is a single launch.  A finished solve (projector,
  solver state, graph) is kept per shape bucket -- geometry, iterations, lambda -- and a
  later request of the same bucket loads its projections into it, resets the iterate and
  replays the graph, with no new allocation or capture; idle solves count against the memory
  budget and are released, oldest first, when an admission needs the memory;
* polls completion events and returns results with their latency.  A request that cannot
  run (its geometry is refused, its projections have the wrong size, it needs more memory
  than the whole budget, or its set-up fails with an out-of-memory error) is returned with
  `error` set and no result; the others are served as usual.

All device work is in the library's kernels; the server only orders it.  Results do not
depend on which other requests run at the same time beyond rounding: every kernel sees only
its own request's data, the 2D kernels and all reductions have a fixed order (bit-identical
results), and the 3D forward adds the entries of one detector row through shared-memory
atomics of one warp, whose order can change the last bits of an FP32 sum.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from ._capi import CsmError
from .projector import Projector
from .sched import admit_order, aged_level, geometry_key, geometry_seed
from .solvers import NAG, power_norm2_device


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
    """Device memory a request holds: NAG state u, y, g (3 volumes), residual and data
    (2 sinograms), power-iteration vectors (2 volumes, 1 sinogram), the projector's
    workspaces (2 volumes, 1 sinogram) and its geometry table."""
    nvox = geom["nx"] * geom["ny"] * geom["nz"]
    nsino = geom["n_views"] * geom.get("nv", 1) * geom["nu"]
    table = geom["n_views"] * (geom["nu"] + 1) * 48 + geom["n_views"] * (geom.get("nv", 1) + 1) * 48
    return elem * (7 * nvox + 4 * nsino) + table + (1 << 20)


class _Solve:
    """A request's device state: projector, NAG state, the captured graph of its iterations,
    the buffers the graph starts from and the one it leaves the iterate in."""

    def __init__(self, key, P, nag, graph, u0, y0, u_out, nbytes):
        self.key, self.P, self.nag, self.graph = key, P, nag, graph
        self.u0, self.y0, self.u_out, self.nbytes = u0, y0, u_out, nbytes


class _Active:
    def __init__(self, req, stream, solve, out_host, done, nbytes):
        self.req, self.stream, self.solve = req, stream, solve
        self.out_host, self.done, self.nbytes = out_host, done, nbytes


class ReconServer:
    """budget_bytes: device memory the admitted requests may hold; max_active: requests on
    the GPU at once; priorities: order streams by request cost (else all at one priority);
    cost_edges: cost thresholds between priority levels (default: decades of
    ``cost_estimate`` from 1e10, the cheapest level highest); level_caps: requests of each
    level (highest first) that may run at once; aging: promote requests that waited longer
    than their estimated service time by one priority level; max_idle: finished solves kept
    for reuse by later requests of their shape bucket."""

    def __init__(self, device="cuda:0", budget_bytes: int = 120 << 30, max_active: int = 16,
                 use_graphs: bool = True, priorities: bool = True, cost_edges=None, level_caps=None,
                 aging: bool = True, max_idle: int = 4):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.use_graphs = use_graphs
        lo, hi = priority_range() if priorities else (0, 0)
        hi = max(hi, lo - 3)                                  # at most four levels
        self.levels = list(range(hi, lo + 1))               # highest priority first
        self.cost_edges = list(cost_edges) if cost_edges is not None else \
            [10.0 ** e for e in range(10, 10 + len(self.levels) - 1)]
        # one stream per slot and level, created up front so that no two admitted requests
        # ever share a stream
        self.pool = {lv: [torch.cuda.Stream(device=self.device, priority=lv) for _ in range(self.max_active)]
                     for lv in self.levels}
        if level_caps is None:
            level_caps = [self.max_active, 4, 2, 1][:len(self.levels)]
            if len(self.levels) > 1:
                level_caps[-1] = 1
        self.caps = {lv: max(1, min(int(c), self.max_active)) for lv, c in zip(self.levels, level_caps)}
        self.running = {lv: 0 for lv in self.levels}
        self.aging = aging
        self.sec_per_cost = None     # smallest (completion - admission) / cost seen so far
        self.sigma_cache = {}        # (geometry key, power iterations) -> (||W||^2 on the device, event)
        self.sigma_hits = 0
        self.max_idle = int(max_idle) if use_graphs else 0
        self.idle = []               # finished solves kept for reuse, oldest first
        self.graph_hits = 0
        self.slots = self.max_active
        self._deferred = []          # projectors released once the device is idle

    def level_of(self, req: Request) -> int:
        c = cost_estimate(req.geom, req.iters, req.power_iters)
        i = sum(1 for e in self.cost_edges if c >= e)
        return self.levels[min(i, len(self.levels) - 1)]

    def stream_level(self, req: Request, now: float) -> int:
        """Priority of the request's stream: its class level, one level higher when it has
        waited longer than its estimated service time."""
        lv = self.level_of(req)
        if not self.aging or self.sec_per_cost is None:
            return lv
        est = self.sec_per_cost * cost_estimate(req.geom, req.iters, req.power_iters)
        return self.levels[aged_level(self.levels.index(lv), now - req.arrival, est)]

    # -----------------------------------------------------------------------------------
    def _launch(self, req: Request, now: float) -> _Active:
        lv = self.level_of(req)
        plv = self.stream_level(req, now)
        s = self.pool[plv].pop()
        self.slots -= 1
        self.running[lv] += 1
        try:
            return self._start(req, now, lv, plv, s)
        except Exception:
            self.slots += 1
            self.running[lv] -= 1
            self.pool[plv].append(s)
            raise

    def _start(self, req: Request, now: float, lv: int, plv: int, s) -> _Active:
        g = req.geom
        bucket = (geometry_key(g), req.iters, req.power_iters, float(req.lam))
        sv = None
        for i, cand in enumerate(self.idle):
            if cand.key == bucket:
                sv = self.idle.pop(i)
                break
        with torch.cuda.device(self.device), torch.cuda.stream(s):
            data = torch.from_numpy(np.ascontiguousarray(req.sino, dtype=np.float32)).pin_memory()
            if sv is not None:
                # same shape bucket: load the data, reset the iterate, replay the graph
                if data.numel() != sv.nag.p.numel():
                    raise ValueError("projections of %d values for a geometry of %d" % (data.numel(), sv.nag.p.numel()))
                sv.nag.p.copy_(data.reshape(sv.nag.p.shape), non_blocking=True)
                sv.u0.zero_()
                sv.y0.zero_()
                sv.graph.replay()
                self.graph_hits += 1
            else:
                sv = self._new_solve(req, bucket, data, s)
            out_host = torch.empty(tuple(sv.P.vol_shape), dtype=torch.float32).pin_memory()
            out_host.copy_(sv.u_out[0], non_blocking=True)
            done = torch.cuda.Event()
            done.record(s)
        req.t_admit = now
        return _Active(req, (lv, plv, s), sv, out_host, done, footprint_bytes(g))

    def _new_solve(self, req: Request, bucket, data, s) -> _Solve:
        g = req.geom
        P = Projector(g, device=self.device)
        p = data.to(self.device, non_blocking=True).reshape((1,) + tuple(P.sino_shape))
        key = (geometry_key(g), req.power_iters)
        hit = self.sigma_cache.get(key)
        if hit is None:
            gen = torch.Generator(device=self.device)
            gen.manual_seed(geometry_seed(g))
            start = torch.randn((1,) + tuple(P.vol_shape), generator=gen, device=self.device, dtype=torch.float32)
            sig2 = power_norm2_device(P, iters=req.power_iters, start=start)
            ev = torch.cuda.Event()
            ev.record(s)
            self.sigma_cache[key] = (sig2, ev)
        else:
            sig2, ev = hit
            s.wait_event(ev)
            sig2.record_stream(s)         # read on this stream too
            self.sigma_hits += 1
        # an estimated norm: a 1% margin keeps the step 1 / (1 + lam) below 1 / L
        nag = NAG(P, 1, lam=req.lam, sigma2_device=sig2, sigma_scale=1.01)
        nag.start(p)
        u0, y0 = nag.u, nag.y
        graph = None
        if self.use_graphs:
            graph = torch.cuda.CUDAGraph()
            graph.capture_begin()
            for _ in range(req.iters):
                nag.step()
            graph.capture_end()
            graph.replay()
        else:
            for _ in range(req.iters):
                nag.step()
        return _Solve(bucket, P, nag, graph, u0, y0, nag.u, footprint_bytes(g))

    def _finish(self, act: _Active, now: float):
        act.req.result = act.out_host.numpy().copy()
        act.req.t_done = now
        self.slots += 1
        lv, plv, s = act.stream
        self.pool[plv].append(s)
        self.running[lv] -= 1
        spc = (now - act.req.t_admit) / cost_estimate(act.req.geom, act.req.iters, act.req.power_iters)
        self.sec_per_cost = spc if self.sec_per_cost is None else min(self.sec_per_cost, spc)
        sv = act.solve
        act.solve = None
        if self.max_idle > 0 and sv.graph is not None:
            self.idle.append(sv)
            while len(self.idle) > self.max_idle:
                self._drop(self.idle.pop(0))
        else:
            self._drop(sv)

    def _drop(self, sv: _Solve):
        self._deferred.append(sv.P)
        sv.graph = None
        sv.nag = None

    def idle_bytes(self) -> int:
        return sum(sv.nbytes for sv in self.idle)

    def _memory_blocked(self, pending, now, used) -> bool:
        """Whether the next request admission would take (the first arrived one whose class
        has a free slot) waits for memory."""
        for r in pending:
            if r.arrival > now:
                return False
            lv = self.level_of(r)
            if self.running[lv] >= self.caps[lv]:
                continue
            return used + self.idle_bytes() + footprint_bytes(r.geom) > self.budget
        return False

    def _release_deferred(self):
        # freeing a geometry table synchronises the device; done only when it is idle
        for P in self._deferred:
            P.close()
        self._deferred = []

    # -----------------------------------------------------------------------------------
    def serve(self, requests, realtime: bool = True, poll_s: float = 2e-4):
        """Serve `requests` (sorted by arrival).  With realtime, arrivals follow the wall
        clock from the start of the call; otherwise every request is available at once.
        Returns the requests with result, t_admit, t_done filled in (seconds)."""
        pending = sorted(requests, key=lambda r: r.arrival)
        if not realtime:
            for r in pending:
                r.arrival = 0.0
        for r in [r for r in pending if footprint_bytes(r.geom) > self.budget]:
            r.error = "needs %d bytes of device memory, more than the budget of %d" % (footprint_bytes(r.geom),
                                                                                       self.budget)
            r.t_done = r.arrival
            pending.remove(r)
        active = []
        used = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            # admit in arrival order while memory and a slot of the request's class are free; idle
            # solves hold memory too and are released, oldest first, when a request needs it
            idx = admit_order(pending, now, self.slots, self.running, self.caps, used + self.idle_bytes(),
                              self.budget, self.level_of, lambda r: footprint_bytes(r.geom))
            while not idx and self.idle and self.slots > 0 and self._memory_blocked(pending, now, used):
                self._drop(self.idle.pop(0))
                idx = admit_order(pending, now, self.slots, self.running, self.caps, used + self.idle_bytes(),
                                  self.budget, self.level_of, lambda r: footprint_bytes(r.geom))
            for i in idx:
                req = pending[i]
                try:
                    active.append(self._launch(req, time.perf_counter() - t0))
                    used += footprint_bytes(req.geom)
                except (CsmError, ValueError, RuntimeError) as e:   # this request cannot run
                    req.error = "%s: %s" % (type(e).__name__, e)
                    req.t_done = time.perf_counter() - t0
            for i in reversed(idx):
                pending.pop(i)
            # completions
            still = []
            for act in active:
                if act.done.query():
                    self._finish(act, time.perf_counter() - t0)
                    used -= act.nbytes
                else:
                    still.append(act)
            active = still
            if not active and self._deferred:
                self._release_deferred()
            if active or pending:
                time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        self._release_deferred()
        return requests

    def close(self):
        """Release the idle solves and their geometry tables."""
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

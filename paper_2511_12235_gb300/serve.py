"""Continuous-batching reconstruction server.

Each request carries a geometry (2D fan or 3D cone beam), measured projections and a
number of NAG iterations on the Tikhonov objective (Section "Numerical Experiments",
Eq. (exp_tikh)).  The server

* admits requests in arrival order while their device-memory footprint fits a budget
  (120 GB by default) and a slot is free; requests that arrive while others run are admitted
  as soon as memory and slots free up;
* runs every admitted request on its own CUDA stream, so the projections of different
  requests overlap on the GPU;
* estimates ||W|| by power iteration on the device (the scalar never leaves the GPU), then
  captures the request's NAG iterations once into a CUDA graph and replays it: the whole
  solve is a single launch;
* polls completion events and returns results with their latency.

All device work is in the library's kernels; the server only orders it.  Results do not
depend on which other requests run at the same time: every kernel has a fixed reduction
order and no atomics.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from .projector import Projector
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
    seed: int = 0
    result: np.ndarray | None = None
    t_admit: float | None = None
    t_done: float | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def footprint_bytes(geom: dict, elem: int = 4) -> int:
    """Device memory a request holds: NAG state u, y, g (3 volumes), residual and data
    (2 sinograms), power-iteration vectors (2 volumes, 1 sinogram), the projector's
    workspaces (2 volumes, 1 sinogram) and its geometry table."""
    nvox = geom["nx"] * geom["ny"] * geom["nz"]
    nsino = geom["n_views"] * geom.get("nv", 1) * geom["nu"]
    table = geom["n_views"] * (geom["nu"] + 1) * 48 + geom["n_views"] * (geom.get("nv", 1) + 1) * 48
    return elem * (7 * nvox + 4 * nsino) + table + (1 << 20)


class _Active:
    def __init__(self, req, stream, P, nag, graph, out_host, done, nbytes):
        self.req, self.stream, self.P, self.nag, self.graph = req, stream, P, nag, graph
        self.out_host, self.done, self.nbytes = out_host, done, nbytes


class ReconServer:
    def __init__(self, device="cuda:0", budget_bytes: int = 120 << 30, max_active: int = 16,
                 use_graphs: bool = True):
        self.device = torch.device(device)
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.use_graphs = use_graphs
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.max_active)]
        self.free_streams = list(range(self.max_active))
        self._deferred = []          # projectors released once the device is idle

    # -----------------------------------------------------------------------------------
    def _launch(self, req: Request, now: float) -> _Active:
        si = self.free_streams.pop()
        s = self.streams[si]
        g = req.geom
        with torch.cuda.device(self.device), torch.cuda.stream(s):
            P = Projector(g, device=self.device)
            data = torch.from_numpy(np.ascontiguousarray(req.sino, dtype=np.float32)).pin_memory()
            p = data.to(self.device, non_blocking=True).reshape((1,) + tuple(P.sino_shape))
            gen = torch.Generator(device=self.device)
            gen.manual_seed(req.seed)
            start = torch.randn((1,) + tuple(P.vol_shape), generator=gen, device=self.device, dtype=torch.float32)
            sig2 = power_norm2_device(P, iters=req.power_iters, start=start)
            # an estimated norm: a 1% margin keeps the step 1 / (1 + lam) below 1 / L
            nag = NAG(P, 1, lam=req.lam, sigma2_device=sig2, sigma_scale=1.01)
            nag.start(p)
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
            out_host = torch.empty(tuple(P.vol_shape), dtype=torch.float32).pin_memory()
            out_host.copy_(nag.u[0], non_blocking=True)
            done = torch.cuda.Event()
            done.record(s)
        req.t_admit = now
        act = _Active(req, si, P, nag, graph, out_host, done, footprint_bytes(g))
        return act

    def _finish(self, act: _Active, now: float):
        act.req.result = act.out_host.numpy().copy()
        act.req.t_done = now
        self.free_streams.append(act.stream)
        self._deferred.append(act.P)
        act.graph = None
        act.nag = None

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
        active = []
        used = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            # admit in arrival order while memory and a slot are free
            while pending and pending[0].arrival <= now and self.free_streams:
                need = footprint_bytes(pending[0].geom)
                if need > self.budget:
                    raise ValueError("request %d needs %d bytes, more than the budget" % (pending[0].id, need))
                if used + need > self.budget:
                    break
                req = pending.pop(0)
                active.append(self._launch(req, now))
                used += need
                now = time.perf_counter() - t0
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


def solve_alone(req: Request, device="cuda:0") -> np.ndarray:
    """The same reconstruction with plain, unbatched calls on the default stream (the
    reference the serving results are compared with)."""
    dev = torch.device(device)
    P = Projector(req.geom, device=dev)
    p = torch.from_numpy(np.ascontiguousarray(req.sino, dtype=np.float32)).to(dev).reshape((1,) + tuple(P.sino_shape))
    gen = torch.Generator(device=dev)
    gen.manual_seed(req.seed)
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

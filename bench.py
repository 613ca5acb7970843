#!/usr/bin/env python3
"""Benchmark: cone-beam forward + back projection with the consistent system matrix.

Default workload (one step): 3D circular cone beam, 512^3 unit voxels, 360 views over
360 deg, 768 x 768 detector of unit elements, source-isocentre 1000, source-detector 1500;
one seeded random-ellipsoid phantom in FP32; one step = p = W x over all views, then
x' = W^T p.  Metric: G voxel-ray updates per second, an update being one nonzero W_ij
applied to one batch item, counted 2 nnz(W) B per step (forward + back).  ``--workload``
selects the other workloads (fan2d_512: 512^2, 720 views, 768 elements, batch 16;
fan2d_64; cone3d_128) and ``serving`` the reconstruction-serving mix.

Runs one rank per GPU (torchrun for N > 1); every rank projects its own phantoms
(independent problems: weak scaling, no data-path collective).  ``--impl reference``
times the FP64 CPU oracle instead (rank 0 only), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+back projector Gvoxel-ray updates/s vs FP64 oracle; served recon p50/p99"
UNIT = "Gupdates/s"
WORKLOAD = "cone3d_512"
# other workloads (not the default line): batch and storage dtype
WORKLOADS = {
    "fan2d_512": dict(batch=16, dtype="f32"),
    "fan2d_64": dict(batch=1, dtype="f64"),
    "cone3d_128": dict(batch=1, dtype="f32"),
    "cone3d_512": dict(batch=1, dtype="f32"),
}
# Algorithmic FP operations (add / sub / mul 1, FMA 2, divide 1) of the kernels as implemented, per
# nonzero entry of W, as (geometry part, part per batch item).  2D: two cell atoms and their
# difference per entry, one multiply-add per item.  3D: counted per event of the fast forms
# (face corrections, planes inside a voxel, first plane above; plane rows and cells of the
# forward) and divided by the entries, with the event counts of the 512^3 workload:
#   back    93 flops per (voxel, view) = 75 + 18 per item, 7.85 entries per (voxel, view)
#   forward 59 flops per plane row = 33 + 26 per item, 0.10 plane rows per entry on the phantom
#           (rows outside the column's nonzero voxels are skipped), plus 1390 per cell set-up
# The same rate counted per entry of the direct closed form (every entry's Phi differences
# formed and applied one by one, as the paper's per-voxel procedure does): 2D two cell atoms
# and their difference (12 flops); 3D one Phi (two relu integrals over a top-view atom, shared
# by four entries) and the double difference (40 flops); one multiply-add per batch item.
DIRECT_FLOPS = {2: (12.0, 2.0), 3: (40.0, 2.0)}
ALG_FLOPS = {(2, "forward"): (12.0, 2.0), (2, "back"): (12.0, 2.0),
             (3, "back"): (9.6, 2.3), (3, "forward"): (4.35, 2.6)}
L2_FLUSH_BYTES = 512 << 20
# the reference arm (the oracle) is sized so that all its steps take about this long
REFERENCE_TOTAL_S = 120.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--requests", type=int, default=200, help="serving: number of requests")
    ap.add_argument("--load", type=float, default=0.7, help="serving: arrival rate / measured capacity")
    ap.add_argument("--sweep", type=str, default="",
                    help="serving: further loads to run after --load, comma separated (e.g. 0.5,0.9)")
    ap.add_argument("--dtype", default=None, choices=["f32", "f64", "bf16", "f16"],
                    help="storage dtype of volume and sinogram (default per workload)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_seeds(rank: int, batch: int):
    """Phantom seeds of one rank: every rank projects its own independent batch."""
    return list(range(rank * batch, (rank + 1) * batch))


def max_over_ranks(values, world: int, device="cpu"):
    """Element-wise maximum of per-rank timings (the job finishes with its slowest rank)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def kernel_source_hash() -> str:
    """sha256 over the CUDA sources and the C header (sorted by name) with comments and
    whitespace removed, so that only a change of the code itself changes it."""
    import glob
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2511_12235_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")))
    files.append(os.path.join(ROOT, "include", "csm.h"))
    h = hashlib.sha256()
    for f in files:
        with open(f) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)       # block comments
        text = re.sub(r"//[^\n]*", " ", text)                    # line comments
        h.update(os.path.basename(f).encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def dram_traffic(workload: str, kernel: str):
    """DRAM bytes (read + write) per call of `kernel` ("forward" / "back") on `workload`
    from the committed ncu capture (profiles/dram_traffic.json), or None when there is none
    or the kernel sources changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_sha256") != kernel_source_hash():
        return None
    v = d.get(workload, {}).get(kernel)
    return float(v) if v is not None else None


def measure_alu_peak(dev, clocks_gpu: int):
    """FP32 (and FP64) fused multiply-add rate of this GPU from the library's FMA-chain
    kernel (csm_fma_rate): a burst (one launch of ~10 ms, for a kernel timed alone) and a
    sustained figure (back-to-back launches for ~3 s, the last 2 s timed, for a kernel timed
    inside a long step), with the SM clocks sampled meanwhile.  TFLOP/s."""
    import torch
    from paper_2511_12235_gb300 import _capi as capi
    stream = torch.cuda.current_stream(dev).cuda_stream
    capi.csm_fma_rate(capi.CSM_F32, 1000, 8, 1, stream)                       # warm-up
    f, t = capi.csm_fma_rate(capi.CSM_F32, 10000, 8, 1, stream)
    burst = f / t / 1e12
    iters = max(1000, int(10000 * 0.05 / max(t, 1e-6)))                       # ~50 ms launches
    capi.csm_fma_rate(capi.CSM_F32, iters, 8, 20, stream)                     # ~1 s to settle
    clk = ClockSampler(clocks_gpu)
    clk.start()
    f, t = capi.csm_fma_rate(capi.CSM_F32, iters, 8, 40, stream)
    c = clk.stop()
    sustained = f / t / 1e12
    f, t = capi.csm_fma_rate(capi.CSM_F64, 500, 8, 1, stream)
    fp64 = f / t / 1e12
    return {"fp32_burst_tflops": burst, "fp32_sustained_tflops": sustained, "fp64_burst_tflops": fp64,
            "sustained_sm_mhz": c.get("sm_mhz"), "sustained_reasons": c.get("reasons"),
            "how": "csm_fma_rate: 8 blocks x 256 threads per SM, 8 independent FMA chains per thread; "
                   "burst = one ~10 ms launch, sustained = 40 back-to-back ~50 ms launches after 1 s"}


# ---------------------------------------------------------------------------------------
# CPU baselines: the FP64 oracle as it stands, on the host cores, on a bounded sample.
def cpu_oracle_leg(steps: int, target_s: float = 15.0):
    """2D sample: forward + back of one phantom over a subset of views, sized so that one
    step takes about target_s / steps.  Returns (geometry, phantom, views, threads)."""
    import numpy as np
    import oracle
    import synth
    g = synth.config("fan2d_512")
    x = synth.ellipse_phantom(512, 0)
    per_step = max(1.0, target_s / max(steps, 1))
    v_try = [0, 180, 360, 540]
    p = oracle.forward_2d(g, x, views=v_try[:1])   # thread-pool start-up, not timed
    t0 = time.perf_counter()
    p = oracle.forward_2d(g, x, views=v_try)
    oracle.back_2d(g, p, views=v_try)
    t_view = (time.perf_counter() - t0) / len(v_try)
    n_views = int(max(2, min(720, per_step / max(t_view, 1e-6))))
    views = (np.arange(n_views) * (720 // n_views if n_views <= 720 else 1)) % 720
    return g, x, views, oracle.num_threads()


def cpu_slab_sample(g, target_s: float):
    """3D sample: the oracle's back projection W^T p of one view (view 0) over a z-slab of the
    volume, p a seeded uniform [1][nv][nu] sinogram; the slab (centred in z) is sized so that
    one evaluation takes about target_s.  Returns (p, iz0, iz1)."""
    import numpy as np
    import oracle
    p = np.random.default_rng(2).uniform(size=(1, g["nv"], g["nu"]))
    mid = g["nz"] // 2
    oracle.back_slab_3d(g, p, mid, mid + 1, views=[0])             # thread-pool start-up
    t0 = time.perf_counter()
    oracle.back_slab_3d(g, p, mid - 2, mid + 2, views=[0])
    t4 = max(time.perf_counter() - t0, 1e-4) / 4
    h = int(max(2, min(g["nz"], target_s / t4)))
    iz0 = max(0, mid - h // 2)
    return p, iz0, min(g["nz"], iz0 + h)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    import synth
    wl = getattr(args, "workload", WORKLOAD)
    if wl not in WORKLOADS:
        wl = WORKLOAD
    g = synth.config(wl)
    if g["dim"] == 3:
        # each step: the oracle's back projection of one view over a z-slab (bounded sample)
        per_step = max(0.05, REFERENCE_TOTAL_S / max(args.steps + args.warmup, 1))
        p, iz0, iz1 = cpu_slab_sample(g, per_step)
        for _ in range(args.warmup):
            oracle.back_slab_3d(g, p, iz0, iz1, views=[0])
        n_upd = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, n = oracle.back_slab_3d(g, p, iz0, iz1, views=[0])
            n_upd += n
        dt = time.perf_counter() - t0
        value = n_upd / dt / 1e9
        sample = ("oracle FP64 back projection W^T p of view 0 over voxel slices %d..%d of %d (%d nonzero "
                  "entries per step)" % (iz0, iz1 - 1, g["nz"], n_upd // max(args.steps, 1)))
        cfg = {"workload": wl + " (sampled: one view, z-slab)", "batch": 1, "views": 1, "slab": [iz0, iz1]}
    else:
        g, x, views, _ = cpu_oracle_leg(args.steps)
        nnz_sample = oracle.count_2d(g, views=views)
        for _ in range(args.warmup):
            p = oracle.forward_2d(g, x, views=views)
            oracle.back_2d(g, p, views=views)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            p = oracle.forward_2d(g, x, views=views)
            oracle.back_2d(g, p, views=views)
        dt = time.perf_counter() - t0
        value = 2.0 * nnz_sample * args.steps / dt / 1e9
        sample = "oracle FP64 fwd+back of 1 phantom over %d of 720 views (%d nonzero entries)" % (len(views),
                                                                                               nnz_sample)
        cfg = {"workload": "fan2d_512 (sampled views)", "batch": 1, "views": int(len(views))}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def elementwise_rel(got, want):
    """Largest |got - want| / (|want| + 0.1 max|want|) over the samples: the relative error
    of every sample, floored at a tenth of the largest value, so that a bound b on it reads
    |got - want| <= b |want| + 0.1 b max|want| (elements with almost no weight are compared
    on the scale of their projection)."""
    import numpy as np
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    scale = np.abs(want) + 0.1 * np.max(np.abs(want))
    return float(np.max(np.abs(got - want) / scale))


def sample_elements(g, n, seed):
    """(view, k, l) detector elements spread over views, columns and rows (every row window)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    v = rng.integers(0, g["n_views"], n)
    k = rng.integers(g["nu"] // 6, g["nu"] - g["nu"] // 6, n)
    l = (np.arange(n) * (g["nv"] - 1)) // max(n - 1, 1)
    return [(int(a), int(b), int(c)) for a, b, c in zip(v, k, l)]


def cpu_baseline_3d(g, x_host, p_gpu_item0, P, dev, target_s=12.0):
    """The oracle on the host cores on a sample of the 3D workload, and the parity of the
    timed kernels on it: the oracle's back projection of one view over a z-slab (timed:
    updates/s), the GPU back projection of the same synthetic view against it, and sampled
    detector elements of the timed forward (batch item 0) against the oracle's."""
    import numpy as np
    import torch
    import oracle
    import paper_2511_12235_gb300 as csm
    p, iz0, iz1 = cpu_slab_sample(g, target_s)
    t0 = time.perf_counter()
    xs, n_upd = oracle.back_slab_3d(g, p, iz0, iz1, views=[0])
    dt = time.perf_counter() - t0
    g1 = dict(g)
    g1["angles"] = g["angles"][:1].copy()
    g1["n_views"] = 1
    P1 = csm.Projector(g1, device=dev)
    b = P1.back(torch.from_numpy(p).float().to(dev))[iz0:iz1].double().cpu().numpy()
    P1.close()
    back_err = elementwise_rel(b, xs)
    els = sample_elements(g, 24, seed=3)
    want = np.array([oracle.forward_element_3d(g, x_host, v, k, l) for v, k, l in els])
    got = np.array([float(p_gpu_item0[v, l, k]) for v, k, l in els])
    fwd_err = elementwise_rel(got, want)
    return {"value": n_upd / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "FP64 oracle back projection W^T p of view 0 over voxel slices %d..%d of %d "
                      "(%d nonzero entries, %.1f s), p seeded uniform" % (iz0, iz1 - 1, g["nz"], n_upd, dt),
            "back_parity_max_rel": back_err,
            "forward_parity_max_rel": fwd_err,
            "parity_note": "per sample |gpu - oracle| / (|oracle| + 0.1 max|oracle|): the back over the "
                           "slab's %d voxels, the timed forward on %d sampled detector elements"
                           % (xs.size, len(els))}


def cpu_baseline_2d(P, x):
    import numpy as np
    import oracle
    gq, xq, views, cores = cpu_oracle_leg(1, target_s=12.0)
    n_sample = oracle.count_2d(gq, views=views)
    t0 = time.perf_counter()
    pq = oracle.forward_2d(gq, xq, views=views)
    oracle.back_2d(gq, pq, views=views)
    dt = time.perf_counter() - t0
    # parity of the timed forward (batch item 0, the same phantom) on the sampled views
    p_gpu = P.forward(x)[0].double().cpu().numpy()[views]
    num = np.linalg.norm(p_gpu - pq, axis=1)
    den = np.linalg.norm(pq, axis=1)
    rel = float(np.max(num[den > 0] / den[den > 0]))
    return {"value": 2.0 * n_sample / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle fwd+back of 1 phantom over %d of 720 views (%d entries), %.1f s"
                      % (len(views), n_sample, dt),
            "forward_parity_max_rel_l2_per_view": rel}


# ---------------------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    try:
        import paper_2511_12235_gb300 as csm
        from paper_2511_12235_gb300 import _capi  # noqa: F401  (loads the library)
    except ImportError:
        from paper_2511_12235_gb300 import build
        build.build()
        import paper_2511_12235_gb300 as csm
    import synth

    wl = args.workload
    batch = WORKLOADS[wl]["batch"]
    sdt = args.dtype or WORKLOADS[wl]["dtype"]
    tdt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16, "f16": torch.float16}[sdt]
    g = synth.config(wl)
    seeds = rank_seeds(rank, batch)
    if g["dim"] == 2:
        xs_host = np.stack([synth.ellipse_phantom(g["nx"], s) for s in seeds]).astype(np.float32)
    else:
        xs_host = np.stack([synth.ellipsoid_phantom(g["nx"], s, dtype=np.float32, slab=8,
                                                    workers=os.cpu_count() or 1) for s in seeds])
    x_zero_fraction = float((xs_host == 0).mean())
    x = torch.from_numpy(xs_host).to(dev).to(tdt)
    # the same phantoms with no zero voxel: every entry of W contributes to the forward
    x_dense = (torch.from_numpy(xs_host).to(dev) + 0.05).to(tdt)
    peak = measure_alu_peak(dev, local)
    P = csm.Projector(g, device=dev)
    nnz = P.nnz()
    stream = torch.cuda.current_stream(dev)
    p = torch.empty((batch,) + P.sino_shape, dtype=tdt, device=dev)
    xb = torch.empty((batch,) + P.vol_shape, dtype=tdt, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        P.forward(x, out=p)
        P.back(p, out=xb)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2511_12235_gb300 import _capi as capi
    clocks = ClockSampler(local)
    # --- timed region: K steps, L2 flushed before each (flush not timed) ---------------
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    clocks.start()
    n_launch0 = capi.csm_launch_count()
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    n_launches = capi.csm_launch_count() - n_launch0   # the library's kernels in the timed steps
    barrier()
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in evs)
    p_item0 = p[0].float().cpu().numpy() if g["dim"] == 3 else None

    # --- per-kernel timing for the roofline: forward alone, back alone ------------------
    n_op = 3 if g["dim"] == 3 else 5

    def time_op(fn, n=n_op):
        es = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for i in range(n):
            flush.fill_(float(i))
            es[i][0].record(stream)
            fn()
            es[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in es) / n

    t_fwd = time_op(lambda: P.forward(x, out=p))
    t_back = time_op(lambda: P.back(p, out=xb))
    p_dense = torch.empty_like(p)
    t_fwd_dense = time_op(lambda: P.forward(x_dense, out=p_dense))

    # --- end to end through the public API with host buffers ----------------------------
    # Every step copies its input from pinned host memory, projects forward and back and
    # copies the result to pinned host memory.  The copies run on a second stream, pipelined:
    # step i + 1's input is uploaded while step i computes, step i's result is downloaded
    # while step i + 1 computes (two device buffers each); the L2 flush stays in every step.
    k_e2e = min(args.steps, 5)
    x_pin = x.cpu().pin_memory()
    out_pin = [torch.empty((batch,) + P.vol_shape, dtype=tdt).pin_memory() for _ in range(2)]
    x_e = [torch.empty_like(x) for _ in range(2)]
    p_e = [torch.empty_like(p) for _ in range(2)]
    r_e = [torch.empty_like(xb) for _ in range(2)]
    s_copy = torch.cuda.Stream(dev)
    h2d = [torch.cuda.Event() for _ in range(k_e2e)]
    comp = [torch.cuda.Event() for _ in range(k_e2e)]
    d2h = [torch.cuda.Event() for _ in range(k_e2e)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    s_copy.wait_stream(stream)
    e_start.record(s_copy)
    with torch.cuda.stream(s_copy):
        x_e[0].copy_(x_pin, non_blocking=True)
    h2d[0].record(s_copy)
    for i in range(k_e2e):
        b = i % 2
        stream.wait_event(h2d[i])
        if i >= 2:
            stream.wait_event(d2h[i - 2])          # r_e[b] downloaded: free again
        flush.fill_(float(i))
        P.forward(x_e[b], out=p_e[b])
        P.back(p_e[b], out=r_e[b])
        comp[i].record(stream)
        with torch.cuda.stream(s_copy):
            if i + 1 < k_e2e:
                if i >= 1:
                    s_copy.wait_event(comp[i - 1])  # x_e[1 - b] read by step i - 1: free again
                x_e[1 - b].copy_(x_pin, non_blocking=True)
                h2d[i + 1].record(s_copy)
            s_copy.wait_event(comp[i])
            out_pin[b].copy_(r_e[b], non_blocking=True)
            d2h[i].record(s_copy)
    e_end.record(s_copy)
    barrier()
    t_e2e = e_start.elapsed_time(e_end)
    out_pin = out_pin[0]

    t_ms, t_e2e, t_fwd, t_back, t_fwd_dense = max_over_ranks([t_ms, t_e2e, t_fwd, t_back, t_fwd_dense], world, dev)

    updates_per_step = 2.0 * nnz * batch * world
    value = updates_per_step * args.steps / (t_ms / 1e3) / 1e9
    # (voxel, view) pairs visited by the two projections, per second
    voxel_views = 2.0 * g["nx"] * g["ny"] * g["nz"] * g["n_views"] * batch * world * args.steps / (t_ms / 1e3) / 1e9
    e2e_value = updates_per_step * k_e2e / (t_e2e / 1e3) / 1e9
    dense_value = updates_per_step / ((t_fwd_dense + t_back) / 1e3) / 1e9

    # roofline of the dominant kernel (ALU bound: algorithmic flops / launch time)
    dom, t_dom = ("forward", t_fwd) if t_fwd >= t_back else ("back", t_back)
    fpe, fpb = ALG_FLOPS[(g["dim"], dom)]
    dfe, dfb = DIRECT_FLOPS[g["dim"]]
    direct = nnz * (dfe + dfb * batch) / (t_dom / 1e3) / 1e12
    flops = nnz * (fpe + fpb * batch)
    achieved = flops / (t_dom / 1e3) / 1e12
    fp64 = tdt == torch.float64
    long_kernel = t_dom > 100.0
    if fp64:
        pk, which = peak["fp64_burst_tflops"], "FP64 FMA burst"
    elif long_kernel:
        pk, which = peak["fp32_sustained_tflops"], "FP32 FMA sustained"
    else:
        pk, which = peak["fp32_burst_tflops"], "FP32 FMA burst"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": sdt, "data": "synthetic",
        "config": {"workload": wl, "grid": [g["nx"], g["ny"]] + ([g["nz"]] if g["dim"] == 3 else []),
                   "views": g["n_views"], "detector": [g["nu"]] + ([g["nv"]] if g["dim"] == 3 else []),
                   "s": g["s"], "sdd": g["sdd"],
                   "batch": batch, "nnz_per_item": nnz, "x_zero_fraction": round(x_zero_fraction, 4),
                   "l2": "flushed before every timed step (512 MiB write, untimed); inputs larger than L2"
                         if g["dim"] == 3 else "flushed before every timed step (512 MiB write, untimed)",
                   "step": "forward over all views + back projection of the batch"},
        "gpu_launches": n_launches,
        "gpu_launches_note": "kernels of the library launched in the timed steps, counted by the library "
                             "(csm_launch_count) at every launch site",
        "gvoxel_views_per_s": voxel_views,
        "kernels_ms": {"forward": t_fwd, "back": t_back, "forward_dense_input": t_fwd_dense},
        "dense_input": {"value": dense_value, "unit": UNIT, "x_zero_fraction": 0.0,
                        "note": "the same rate with the forward of the phantoms plus 0.05 (no zero voxel: "
                                "every entry of W is evaluated and applied) and the timed back projection"},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                     "frac": achieved / pk, "traffic": dram_traffic(wl, dom),
                     "traffic_unit": "bytes per call of the kernel (ncu dram__bytes_read.sum + dram__bytes_write.sum; "
                                     "the back projection's launches over its view groups summed, like its time)",
                     "peak_note": "%s rate measured in this run by csm_fma_rate (of measured); algorithmic "
                                  "flops = nnz x (%.2f + %.2f x batch), the FP operations of the kernel as "
                                  "implemented per entry" % (which, fpe, fpb),
                     "direct_form": {"flops_per_entry": "%.0f + %.0f x batch" % DIRECT_FLOPS[g["dim"]],
                                     "achieved": direct, "frac": direct / pk,
                                     "note": "the same kernel time counted with the flops of the direct "
                                             "per-entry closed form, which the fast forms replace"}},
        "alu_peak_measured": peak,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x_pin.numel() * x_pin.element_size()),
                "d2h_bytes_per_step": int(out_pin.numel() * out_pin.element_size()), "steps": k_e2e,
                "note": "Projector.forward/back from pinned host input to pinned host output, every step's "
                        "H2D and D2H inside the timed region, pipelined on a copy stream (the next step's "
                        "upload and the previous step's download overlap the current step's kernels)"},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and wl in ("cone3d_512", "fan2d_512"):
        try:
            if g["dim"] == 3:
                line["cpu_baseline"] = cpu_baseline_3d(g, xs_host[0].astype(np.float64), p_item0, P, dev)
            else:
                line["cpu_baseline"] = cpu_baseline_2d(P, x)
        except Exception as e:  # the baseline is reported, not required
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                                    "sample": "failed: %s" % e}
    if rank == 0:
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serving(args, rank, world, local):
    """Serving mix: Poisson arrivals of reconstruction requests (60% 2D, 40% 3D on fixed scanner
    protocols, 20 NAG iterations each), served by the continuous-batching server, against
    the same requests run for real one at a time with plain calls.  Rank 0 only (one server
    per GPU)."""
    import numpy as np
    import torch
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import synth
    import paper_2511_12235_gb300 as csm
    from paper_2511_12235_gb300.serve import ReconServer, Request, latency_stats, serve_unbatched
    specs = synth.serving_requests(args.requests, seed=0, rate_per_s=1.0)
    base = []
    for sp in specs:      # measured data: projections of a seeded phantom with Poisson noise
        g = sp["geom"]
        P = csm.Projector(g, device=dev)
        if g["dim"] == 2:
            x = torch.from_numpy(synth.ellipse_phantom(g["nx"], sp["seed"])).float().to(dev)
        else:
            x = synth.ellipsoid_phantom_torch(g["nx"], sp["seed"], dev)
        p = P.forward(x).double().cpu().numpy()
        P.close()
        pn, _ = synth.poisson_sinogram(p, seed=sp["seed"])
        base.append(dict(id=sp["id"], geom=g, sino=pn.astype(np.float32), iters=20, power_iters=20, seed=sp["seed"]))
    torch.cuda.synchronize()
    n = len(base)
    fresh = lambda: [Request(**b) for b in base]
    kinds = np.array([b["geom"]["dim"] for b in base])
    # unbatched plain calls, one at a time, all waiting: the service time of every request
    serve_unbatched(fresh()[:1], device=dev, realtime=False)          # warm-up
    alone = serve_unbatched(fresh(), device=dev, realtime=False)
    service = np.array([r.t_done - r.t_admit for r in alone])
    unb_makespan = max(r.t_done for r in alone)
    # throughput: every request waiting at t = 0
    srv = ReconServer(device=dev, budget_bytes=120 << 30, use_graphs=True)
    t0 = time.perf_counter()
    sat = srv.serve(fresh(), realtime=False)
    makespan = time.perf_counter() - t0
    stats_sat = dict(joined=srv.joined, max_occupancy=srv.max_occupancy, batch_hits=srv.batch_hits)
    srv.close()
    worst = 0.0
    for r, a in zip(sorted(sat, key=lambda r: r.id), sorted(alone, key=lambda r: r.id)):
        worst = max(worst, float(np.linalg.norm(r.result - a.result) / max(np.linalg.norm(a.result), 1e-30)))
    # latency: Poisson arrivals at `load` times the unbatched capacity, both servers run for real
    cap = 1.0 / float(np.mean(service))

    def latency_run(load, seed):
        rate = load * cap
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
        reqs = fresh()
        for r, t in zip(reqs, arrivals):
            r.arrival = float(t)
        srv = ReconServer(device=dev, budget_bytes=120 << 30, use_graphs=True)
        done = srv.serve(reqs, realtime=True)
        st_run = dict(joined=srv.joined, max_occupancy=srv.max_occupancy)
        srv.close()
        lat = np.array([r.latency for r in sorted(done, key=lambda r: r.id)])
        ub = fresh()
        for r, t in zip(ub, arrivals):
            r.arrival = float(t)
        serve_unbatched(ub, device=dev, realtime=True)
        base_lat = np.array([r.latency for r in sorted(ub, key=lambda r: r.id)])
        st, bst = latency_stats(lat), latency_stats(base_lat)
        med = lambda a_, k: float(np.median(a_[kinds == k])) if (kinds == k).any() else None
        return rate, dict({"load_vs_capacity": load, "arrival_rate_per_s": rate,
                           "p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"],
                           "p50_2d_s": med(lat, 2), "p50_3d_s": med(lat, 3),
                           "unbatched": {"p50_s": bst["p50_s"], "p99_s": bst["p99_s"], "mean_s": bst["mean_s"],
                                         "p50_2d_s": med(base_lat, 2), "p50_3d_s": med(base_lat, 3)}}, **st_run)

    rate, main_run = latency_run(args.load, 1)
    sweep = [latency_run(float(ld), 2 + i)[1] for i, ld in enumerate(x for x in args.sweep.split(",") if x)]
    line = {
        "metric": METRIC, "value": n / makespan, "unit": "requests/s", "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "requests": n, "share_2d": float((kinds == 2).mean()),
                   "protocols_2d": [list(p) for p in synth.SERVING_PROTOCOLS_2D],
                   "protocols_3d": [list(p) for p in synth.SERVING_PROTOCOLS_3D],
                   "nag_iterations": 20, "power_iterations": 20, "budget_gb": 120,
                   "slots_per_batch": {"2d": 8, "3d": 4}, "arrival_rate_per_s": rate, "load_vs_capacity": args.load},
        "throughput": {"served_requests_per_s": n / makespan, "unbatched_requests_per_s": n / unb_makespan,
                       "served_makespan_s": makespan, "unbatched_makespan_s": unb_makespan,
                       "note": "all requests waiting at t = 0", **stats_sat},
        "p50_s": main_run["p50_s"], "p99_s": main_run["p99_s"], "mean_s": main_run["mean_s"],
        "p50_2d_s": main_run["p50_2d_s"], "p50_3d_s": main_run["p50_3d_s"],
        "unbatched": dict(main_run["unbatched"], mean_service_s=float(np.mean(service)),
                          note="the same requests and arrivals served for real one at a time with plain "
                               "csm_forward/csm_back calls (FIFO)"),
        "joined_running_batches": main_run["joined"], "max_occupancy": main_run["max_occupancy"],
        "load_sweep": sweep,
        "served_vs_alone_max_rel_l2": worst,
        "service_s": [round(float(x), 4) for x in service],
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()

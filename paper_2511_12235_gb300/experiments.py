"""The paper's synthetic checkerboard experiments (Section "Numerical Experiments", "Synthetic
Data" in 2D and 3D), run on the library: a 4 x 4 (x 4) black / white checkerboard on N^d
unit voxels, projections generated with the consistent (area / volume) system matrix plus
Gaussian noise, and reconstructions by NAG on the Tikhonov objective (Eq. (exp_tikh)) with the
consistent matrix and with the line-based comparators (Siddon, Joseph), each divided by its
spectral norm from 100 power iterations.  Reports the mean squared error to the ground truth
per grid size and method.

Parameters as printed: 60 views equidistant in [0, 2 pi), 60 detector elements (60 x 60 in
3D) of width 0.75, unit voxels, lambda = sigma = 1e-4, at most 1000 NAG iterations (500 in 3D)
or until ||grad F||^2 < 1e-9.  Readings: the distances read "s = d = 250" (source-isocentre
250, source-detector 500); the data p are divided by the spectral norm of the matrix that
generated them, so that every method's normalised matrix reconstructs the image itself.

    python -m paper_2511_12235_gb300.experiments [--sizes 16,32,48,64] [--dims 2,3]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from .projector import Projector
from .solvers import NAG, power_norm


class LineOperator:
    """A line-based comparator model behind the interface the solvers use (forward / back with
    out=, shapes, device)."""

    def __init__(self, P: Projector, model: str, lines: int = 1):
        self.P, self.model, self.lines = P, model, lines
        self.device, self.vol_shape, self.sino_shape = P.device, P.vol_shape, P.sino_shape

    def forward(self, x, out=None):
        return self.P.forward_line(x, self.model, self.lines, out=out)

    def back(self, p, out=None):
        return self.P.back_line(p, self.model, self.lines, out=out)


def checkerboard(n: int, dim: int, blocks: int = 4) -> np.ndarray:
    """blocks^dim alternating blocks of 0 and 1 on an n^dim grid ([z][y][x] or [y][x])."""
    idx = (np.arange(n) * blocks) // n
    if dim == 2:
        return ((idx[:, None] + idx[None, :]) % 2).astype(np.float64)
    return ((idx[:, None, None] + idx[None, :, None] + idx[None, None, :]) % 2).astype(np.float64)


def geometry(n: int, dim: int) -> dict:
    import synth
    if dim == 2:
        return synth.geometry(n, n, 1, n_views=60, s=250.0, sdd=500.0, nu=60, du=0.75)
    g = synth.geometry(n, n, n, n_views=60, s=250.0, sdd=500.0, nu=60, nv=60, du=0.75, dv=0.75)
    g["dim"] = 3
    return g


def run_case(n: int, dim: int, lam: float = 1e-4, noise: float = 1e-4, seed: int = 0, max_iters=None,
             lines_models=("siddon", "joseph"), device="cuda"):
    """MSE and iterations of every method on one grid size."""
    g = geometry(n, dim)
    P = Projector(g, device=device)
    u_true = torch.from_numpy(checkerboard(n, dim)).to(P.device)
    iters = max_iters or (1000 if dim == 2 else 500)
    p = P.forward(u_true)
    gen = torch.Generator(device=P.device)
    gen.manual_seed(seed)
    p = p + noise * torch.randn(p.shape, generator=gen, device=P.device, dtype=p.dtype)
    sig_area = power_norm(P, iters=100, dtype=torch.float64)
    data = p / sig_area
    out = {}
    ops = [("area" if dim == 2 else "volume", P, sig_area)]
    for m in lines_models:
        L = LineOperator(P, m)
        ops.append(("line_" + m, L, power_norm(L, iters=100, dtype=torch.float64)))
    for name, op, sig in ops:
        t0 = time.perf_counter()
        nag = NAG(op, 1, lam=lam, sigma=sig, dtype=torch.float64)
        u = nag.run(data[None], iters=iters, tol=1e-9, check_every=10)
        torch.cuda.synchronize(P.device)
        mse = float(((u[0] - u_true) ** 2).mean())
        out[name] = {"mse": mse, "seconds": time.perf_counter() - t0, "spectral_norm": sig}
    P.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--sizes", default="16,32,48,64")
    ap.add_argument("--dims", default="2,3")
    args = ap.parse_args(argv)
    res = {}
    for dim in (int(d) for d in args.dims.split(",") if d):
        for n in (int(s) for s in args.sizes.split(",") if s):
            res["%dD_%d" % (dim, n)] = run_case(n, dim)
            print(json.dumps({"case": "%dD %d" % (dim, n), **res["%dD_%d" % (dim, n)]}), flush=True)
    return res


if __name__ == "__main__":
    main()

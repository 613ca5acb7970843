"""Reconstruction solvers on the device: power iteration for ||W||, Nesterov's accelerated
gradient (NAG) on the Tikhonov objective, CG least squares (CGLS).

The paper reconstructs by minimising F(u) = 1/2 ||W u - p||^2 + lam/2 ||u||^2 with NAG,
W normalised by its spectral norm from 100 power iterations, iterating to 1000 steps or
||grad F||^2 < 1e-9 (Section "Numerical Experiments", Eq. (exp_tikh)); it also names the
conjugate-gradient method there.  Every step runs in the library's kernels: projections
(csm_forward / csm_back) and the batched vector kernels (csm_dot / csm_axpby), whose
scalars stay on the device, so an iteration issues no host synchronisation and can be
captured in a CUDA graph.  All functions work on batches [B, ...] of independent problems.
"""
from __future__ import annotations

import math

import torch

from . import _capi as capi
from .projector import Projector, _dt, nvtx_range


class VecOps:
    """Batched inner products and axpby on tensors of shape [B, ...]."""

    def __init__(self, device, batch: int):
        self.device = torch.device(device)
        self.batch = batch
        self.ws = torch.empty(capi.csm_dot_workspace_bytes(batch), dtype=torch.uint8, device=self.device)

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def dot(self, a: torch.Tensor, b: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """out[i] = <a[i], b[i]> (FP64, fixed order); out: float64 [B] (or a view of it)."""
        assert a.is_contiguous() and b.is_contiguous() and a.dtype == b.dtype and out.dtype == torch.float64
        B = a.shape[0]
        n = a.numel() // B
        capi.csm_dot(a.data_ptr(), b.data_ptr(), n, B, _dt(a.dtype), out.data_ptr(), self.ws.data_ptr(),
                     self.ws.numel(), self._stream())
        return out

    def axpby(self, a_c: float, x: torch.Tensor | None, b_c: float, y: torch.Tensor, *, a_num=None, a_den=None,
              b_num=None, b_den=None, flags: int = 0) -> torch.Tensor:
        """y = A x + B y per batch item with A = a_c a_num / a_den, B = b_c b_num / b_den
        (num / den: float64 device tensors [B] or None)."""
        B = y.shape[0]
        n = y.numel() // B
        ptr = lambda t: None if t is None else t.data_ptr()
        capi.csm_axpby(n, B, _dt(y.dtype), float(a_c), ptr(a_num), ptr(a_den), ptr(x), float(b_c), ptr(b_num),
                       ptr(b_den), y.data_ptr(), flags, self._stream())
        return y


def power_norm(P: Projector, iters: int = 100, start: torch.Tensor | None = None,
               dtype: torch.dtype = torch.float32, seed: int = 0) -> float:
    """Spectral norm ||W||_2 by `iters` power iterations on W^T W (Section "Numerical
    Experiments": W is divided by its spectral norm, 100 power iterations)."""
    return math.sqrt(float(power_norm2_device(P, iters, start, dtype, seed).item()))


def power_norm2_device(P: Projector, iters: int = 100, start: torch.Tensor | None = None,
                       dtype: torch.dtype = torch.float32, seed: int = 0) -> torch.Tensor:
    """The same estimate of ||W||_2^2, left on the device (float64 tensor [1]) so that the
    caller does not wait for it."""
    dev = P.device
    if start is None:
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        start = torch.randn((1,) + tuple(P.vol_shape), generator=g, device=dev, dtype=dtype)
    b = start.reshape((1,) + tuple(P.vol_shape)).to(device=dev, dtype=dtype).contiguous().clone()
    ops = VecOps(dev, 1)
    nrm = torch.zeros(2, dtype=torch.float64, device=dev)
    ops.dot(b, b, nrm[0:1])
    ops.axpby(1.0, b, 0.0, b, a_den=nrm[0:1], flags=1)         # b / ||b||
    p = torch.empty((1,) + tuple(P.sino_shape), dtype=dtype, device=dev)
    z = torch.empty_like(b)
    for _ in range(iters):
        P.forward(b, out=p)
        P.back(p, out=z)
        ops.dot(z, z, nrm[0:1])
        ops.axpby(1.0, z, 0.0, b, a_den=nrm[0:1], flags=1)     # b = W^T W b / ||W^T W b||
    P.forward(b, out=p)
    ops.dot(p, p, nrm[1:2])                                  # Rayleigh quotient ||W b||^2
    return nrm[1:2]


class CGLS:
    """Conjugate-gradient least squares for min ||W x - p||^2 on a batch.

    ``run(p, iters)`` returns (x, res2) with res2[k, i] = ||p_i - W x_i^{(k)}||^2 for
    k = 0..iters (float64, on the device)."""

    def __init__(self, P: Projector, batch: int, dtype: torch.dtype = torch.float32):
        self.P, self.B, self.dtype = P, batch, dtype
        dev = P.device
        vs, ss = (batch,) + tuple(P.vol_shape), (batch,) + tuple(P.sino_shape)
        self.x = torch.zeros(vs, dtype=dtype, device=dev)
        self.d = torch.empty(vs, dtype=dtype, device=dev)
        self.s = torch.empty(vs, dtype=dtype, device=dev)
        self.r = torch.empty(ss, dtype=dtype, device=dev)
        self.q = torch.empty(ss, dtype=dtype, device=dev)
        self.gam = torch.zeros(2, batch, dtype=torch.float64, device=dev)
        self.qq = torch.zeros(batch, dtype=torch.float64, device=dev)
        self.ops = VecOps(dev, batch)

    def start(self, p: torch.Tensor, x0: torch.Tensor | None = None):
        P, ops = self.P, self.ops
        if x0 is None:
            self.x.zero_()
            self.r.copy_(p.reshape(self.r.shape))
        else:
            self.x.copy_(x0.reshape(self.x.shape))
            P.forward(self.x, out=self.r)
            ops.axpby(1.0, p.reshape(self.r.shape).contiguous(), -1.0, self.r)   # r = p - W x0
        P.back(self.r, out=self.s)
        self.d.copy_(self.s)
        ops.dot(self.s, self.s, self.gam[0])
        self.cur = 0

    def step(self, res2_out: torch.Tensor | None = None):
        with nvtx_range("cgls_step"):
            self._step(res2_out)

    def _step(self, res2_out):
        P, ops = self.P, self.ops
        g_old, g_new = self.gam[self.cur], self.gam[1 - self.cur]
        P.forward(self.d, out=self.q)
        ops.dot(self.q, self.q, self.qq)
        ops.axpby(1.0, self.d, 1.0, self.x, a_num=g_old, a_den=self.qq)      # x += alpha d
        ops.axpby(-1.0, self.q, 1.0, self.r, a_num=g_old, a_den=self.qq)     # r -= alpha q
        P.back(self.r, out=self.s)
        ops.dot(self.s, self.s, g_new)
        ops.axpby(1.0, self.s, 1.0, self.d, b_num=g_new, b_den=g_old)         # d = s + beta d
        self.cur = 1 - self.cur
        if res2_out is not None:
            ops.dot(self.r, self.r, res2_out)

    def run(self, p: torch.Tensor, iters: int = 50, x0=None):
        res2 = torch.zeros(iters + 1, self.B, dtype=torch.float64, device=self.P.device)
        self.start(p, x0)
        self.ops.dot(self.r, self.r, res2[0])
        for k in range(iters):
            self.step(res2[k + 1])
        return self.x, res2


class NAG:
    """Nesterov's accelerated gradient (FISTA momentum) on the Tikhonov objective with W
    normalised by its spectral norm sigma:

        F(u) = 1/2 || (W / sigma) u - p ||^2 + lam / 2 ||u||^2,   step 1 / (1 + lam),
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,  y = u_{k+1} + (t_k - 1) / t_{k+1} (u_{k+1} - u_k).

    ``run`` returns u (the paper's variable); u / sigma is the image in the units of W."""

    def __init__(self, P: Projector, batch: int, lam: float = 1e-4, sigma: float | None = None,
                 dtype: torch.dtype = torch.float32, sigma2_device: torch.Tensor | None = None,
                 sigma_scale: float = 1.0):
        """sigma: ||W|| as a number; or sigma2_device: ||W||^2 as a float64 device tensor of
        one element per batch item (or one shared), read by the kernels without a host wait.
        sigma_scale multiplies sigma (a safety margin for an estimated norm)."""
        self.P, self.B, self.lam, self.dtype = P, batch, float(lam), dtype
        dev = P.device
        if sigma2_device is not None:
            s2 = sigma2_device.to(device=dev, dtype=torch.float64).reshape(-1)
            self.sig2 = (s2.expand(batch) if s2.numel() == 1 else s2).contiguous()
            self.sigma = None
            self.inv_c = 1.0 / sigma_scale
        else:
            self.sigma = float(sigma) if sigma is not None else power_norm(P, dtype=dtype)
            self.sig2 = None
            self.inv_c = 1.0 / (sigma_scale * self.sigma)
        vs, ss = (batch,) + tuple(P.vol_shape), (batch,) + tuple(P.sino_shape)
        self.u = torch.zeros(vs, dtype=dtype, device=dev)
        self.y = torch.zeros(vs, dtype=dtype, device=dev)
        self.g = torch.empty(vs, dtype=dtype, device=dev)
        self.r = torch.empty(ss, dtype=dtype, device=dev)
        self.p = torch.empty(ss, dtype=dtype, device=dev)
        self.ops = VecOps(dev, batch)
        self.t = 1.0

    def start(self, p: torch.Tensor, u0: torch.Tensor | None = None):
        self.p.copy_(p.reshape(self.p.shape))
        if u0 is None:
            self.u.zero_()
        else:
            self.u.copy_(u0.reshape(self.u.shape))
        self.y.copy_(self.u)
        self.t = 1.0

    def gradient(self, y: torch.Tensor, out: torch.Tensor):
        """out = grad F(y) = W^T (W y / sigma - p) / sigma + lam y."""
        P, ops, inv = self.P, self.ops, self.inv_c
        sd, fl = self.sig2, (2 if self.sig2 is not None else 0)   # B = inv / sqrt(sigma^2)
        P.forward(y, out=self.r)
        ops.axpby(-1.0, self.p, inv, self.r, b_den=sd, flags=fl)    # r = W y / sigma - p
        P.back(self.r, out=out)
        ops.axpby(self.lam, y, inv, out, b_den=sd, flags=fl)        # g = W^T r / sigma + lam y
        return out

    def step(self):
        with nvtx_range("nag_step"):
            self._step()

    def _step(self):
        ops = self.ops
        step = 1.0 / (1.0 + self.lam)
        self.gradient(self.y, self.g)
        ops.axpby(1.0, self.y, -step, self.g)           # g := u_new = y - step grad
        t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * self.t * self.t))
        theta = (self.t - 1.0) / t_new
        ops.axpby(1.0 + theta, self.g, -theta, self.u)  # u-buffer := y_new = u_new + theta (u_new - u)
        self.u, self.y, self.g = self.g, self.u, self.y  # rotate buffers: u <- u_new, y <- y_new
        self.t = t_new

    def run(self, p: torch.Tensor, iters: int = 20, u0=None, tol: float | None = None, check_every: int = 10):
        """`iters` NAG steps; with ``tol`` stop once ||grad F(u)||^2 < tol for every batch
        item (checked on the host every ``check_every`` steps)."""
        self.start(p, u0)
        gn = torch.zeros(self.B, dtype=torch.float64, device=self.P.device)
        for k in range(iters):
            self.step()
            if tol is not None and (k + 1) % check_every == 0:
                self.gradient(self.u, self.g)
                self.ops.dot(self.g, self.g, gn)
                if float(gn.max().item()) < tol:
                    break
        return self.u


def fista_thetas(iters: int):
    """theta_k = (t_k - 1) / t_{k+1} for k = 0 .. iters - 1, t_0 = 1 (the momentum sequence of
    NAG.step, in the same FP64 arithmetic)."""
    t, out = 1.0, []
    for _ in range(iters):
        t_new = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        out.append((t - 1.0) / t_new)
        t = t_new
    return out


class NAGSlots:
    """NAG (as ``NAG``) on a batch of slots whose problems share W, lambda and sigma but are at
    different iterations: slot b runs its own momentum sequence (csm_fista_coeffs reads its
    iteration counter on the device).  ``step(n)`` advances slots 0 .. n - 1 by one iteration
    in fixed buffers (no host values enter it), so it can be captured once per n in a CUDA
    graph and replayed while problems are loaded into free slots and finished ones are read
    out and compacted.  A slot's iterates equal those of ``NAG`` on its problem alone."""

    def __init__(self, P: Projector, capacity: int, iters: int, lam: float, sigma2_device: torch.Tensor,
                 sigma_scale: float = 1.0, dtype: torch.dtype = torch.float32):
        self.P, self.C, self.iters, self.lam, self.dtype = P, capacity, iters, float(lam), dtype
        dev = P.device
        vs, ss = (capacity,) + tuple(P.vol_shape), (capacity,) + tuple(P.sino_shape)
        self.u = torch.zeros(vs, dtype=dtype, device=dev)
        self.y = torch.zeros(vs, dtype=dtype, device=dev)
        self.g = torch.zeros(vs, dtype=dtype, device=dev)
        self.r = torch.zeros(ss, dtype=dtype, device=dev)
        self.p = torch.zeros(ss, dtype=dtype, device=dev)
        self.k = torch.zeros(capacity, dtype=torch.int32, device=dev)
        self.opt = torch.zeros(capacity, dtype=torch.float64, device=dev)
        self.th = torch.zeros(capacity, dtype=torch.float64, device=dev)
        self.table = torch.tensor(fista_thetas(iters), dtype=torch.float64, device=dev)
        s2 = sigma2_device.to(device=dev, dtype=torch.float64).reshape(-1)
        self.sig2 = (s2.expand(capacity) if s2.numel() == 1 else s2).contiguous()
        self.inv_c = 1.0 / sigma_scale
        self.ops = VecOps(dev, capacity)

    def reserve(self):
        """Allocates the projector workspaces of every batch size up front (before capture)."""
        self.P.workspace(0, self.C, self.dtype)
        self.P.workspace(1, self.C, self.dtype)

    def load(self, slot: int, p: torch.Tensor):
        """Puts a problem (its projections) into a free slot, iterate zero, iteration 0."""
        self.p[slot].copy_(p.reshape(self.p.shape[1:]), non_blocking=True)
        self.u[slot].zero_()
        self.y[slot].zero_()
        self.k[slot:slot + 1].zero_()

    def move(self, src: int, dst: int):
        """Moves a slot's problem and state to another slot (compaction)."""
        for t in (self.u, self.y, self.p, self.k):
            t[dst].copy_(t[src])

    def step(self, n: int):
        with nvtx_range("nag_slots_step"):
            P, ops, inv = self.P, self.ops, self.inv_c
            u, y, g, r, p = self.u[:n], self.y[:n], self.g[:n], self.r[:n], self.p[:n]
            sd = self.sig2[:n]
            step = 1.0 / (1.0 + self.lam)
            P.forward(y, out=r)
            ops.axpby(-1.0, p, inv, r, b_den=sd, flags=2)             # r = W y / sigma - p
            P.back(r, out=g)
            ops.axpby(self.lam, y, inv, g, b_den=sd, flags=2)         # g = grad F(y)
            ops.axpby(1.0, y, -step, g)                               # g = u_new = y - step grad
            capi.csm_fista_coeffs(n, self.table.data_ptr(), self.table.numel(), self.k.data_ptr(),
                                  self.opt.data_ptr(), self.th.data_ptr(),
                                  torch.cuda.current_stream(P.device).cuda_stream)
            ops.axpby(1.0, u, 0.0, y)                                 # y = u_old
            ops.axpby(1.0, g, -1.0, y, a_num=self.opt, b_num=self.th)  # y = (1 + theta) u_new - theta u_old
            ops.axpby(1.0, g, 0.0, u)                                 # u = u_new

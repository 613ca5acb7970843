"""PyTorch front end of the C ABI: geometry handles, forward / back on CUDA tensors.

PyTorch supplies device memory and the current stream only; every step of the projection
runs in the library's CUDA kernels (``_capi``).  With the environment variable CSM_NVTX=1 the
calls are wrapped in NVTX ranges ("csm_forward", "csm_back") for timeline profilers.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import math
import os

import numpy as np
import torch

from . import _capi as capi

_NVTX = os.environ.get("CSM_NVTX", "") == "1"


def nvtx_range(name: str):
    """An NVTX range around a block when CSM_NVTX=1, else nothing."""
    return torch.cuda.nvtx.range(name) if _NVTX else contextlib.nullcontext()


_DT = {torch.float32: capi.CSM_F32, torch.float64: capi.CSM_F64,
       torch.bfloat16: capi.CSM_BF16, torch.float16: capi.CSM_F16}


_LINE = {"siddon": capi.CSM_LINE_SIDDON, "joseph": capi.CSM_LINE_JOSEPH}


def _dt(t: torch.dtype) -> int:
    try:
        return _DT[t]
    except KeyError:
        raise TypeError("unsupported dtype %s (float32, float64, bfloat16, float16)" % t)


class Projector:
    """Matrix-free consistent system matrix W for one geometry on one CUDA device.

    ``geom`` is a dict with keys nx, ny, nz, a, b, c, n_views, angles, s, sdd, nu, nv, du,
    dv, u_off, v_off (see ``synth.geometry``); ``dim`` 2 selects the fan-beam model (nz = nv
    = 1), 3 the cone-beam model.
    """

    def __init__(self, geom: dict, device=None):
        self.geom = dict(geom)
        self.dim = int(geom.get("dim", 3 if (geom.get("nz", 1) > 1 or geom.get("nv", 1) > 1) else 2))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.type != "cuda":
            raise ValueError("Projector needs a CUDA device")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        ang = np.ascontiguousarray(np.asarray(geom["angles"], dtype=np.float64))
        self._angles = ang
        aptr = ang.ctypes.data_as(C.POINTER(C.c_double))
        with torch.cuda.device(self.device):
            if self.dim == 2:
                d = capi.csm_geom2d_desc(geom["nx"], geom["ny"], geom["a"], geom["b"], geom["n_views"], aptr,
                                         geom["s"], geom["sdd"], geom["nu"], geom["du"], geom.get("u_off", 0.0))
                self.handle = capi.csm_geom_create_2d(d)
            else:
                d = capi.csm_geom3d_desc(geom["nx"], geom["ny"], geom["nz"], geom["a"], geom["b"], geom["c"],
                                         geom["n_views"], aptr, geom["s"], geom["sdd"], geom["nu"], geom["nv"],
                                         geom["du"], geom["dv"], geom.get("u_off", 0.0), geom.get("v_off", 0.0))
                self.handle = capi.csm_geom_create_3d(d)
        g = self.geom
        self.vol_shape = (g["ny"], g["nx"]) if self.dim == 2 else (g["nz"], g["ny"], g["nx"])
        self.sino_shape = (g["n_views"], g["nu"]) if self.dim == 2 else (g["n_views"], g["nv"], g["nu"])
        self._ws = {}

    # ---------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            capi.csm_geom_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, op: int, batch: int, compute: torch.dtype) -> torch.Tensor:
        n = capi.csm_workspace_bytes(self.handle, op, batch, _dt(compute))
        # the back projection's two sizes (op 3 = op 1 and a copy of x) share one buffer
        key = (1 if op == 3 else op, compute)
        buf = self._ws.get(key)
        if buf is None or buf.numel() < n:
            buf = torch.empty(max(n, 256), dtype=torch.uint8, device=self.device)
            self._ws[key] = buf
        return buf

    def _batched(self, t: torch.Tensor, shape) -> tuple[torch.Tensor, bool]:
        if tuple(t.shape) == tuple(shape):
            return t.unsqueeze(0), True
        if tuple(t.shape[1:]) != tuple(shape):
            raise ValueError("expected shape [B, %s] or %s, got %s" % (list(shape), list(shape), list(t.shape)))
        return t, False

    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None, *, flags: int = 0,
                out_dtype: torch.dtype | None = None, variant: str | None = None) -> torch.Tensor:
        """p = W x.  x: [B, *vol_shape] or vol_shape on this device.

        variant: "ray" (ray-driven gather, the default) or "voxel" (voxel-driven scatter with
        shared-memory partial sums and atomics, the form of the paper's Algorithm 1)."""
        if variant is None:
            variant = "ray"
        if variant == "voxel":
            flags |= capi.CSM_VOXEL_DRIVEN
        elif variant != "ray":
            raise ValueError("variant must be 'ray' or 'voxel'")
        xb, single = self._batched(x, self.vol_shape)
        if not xb.is_contiguous():
            xb = xb.contiguous()
        B = xb.shape[0]
        odt = out_dtype or x.dtype
        if out is None:
            out = torch.empty((B,) + tuple(self.sino_shape), dtype=odt, device=self.device)
            if flags & capi.CSM_ACCUMULATE:
                out.zero_()
        else:
            out = out.view((B,) + tuple(self.sino_shape))
            assert out.is_contiguous() and out.device == self.device
        compute = torch.float64 if torch.float64 in (xb.dtype, out.dtype) else torch.float32
        ws = self.workspace(2 if flags & capi.CSM_VOXEL_DRIVEN else 0, B, compute)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        with nvtx_range("csm_forward"):
            capi.csm_forward(self.handle, xb.data_ptr(), out.data_ptr(), B, _dt(xb.dtype), _dt(out.dtype), flags,
                             ws.data_ptr(), ws.numel(), stream)
        return out[0] if single else out

    def back(self, p: torch.Tensor, out: torch.Tensor | None = None, *, flags: int = 0,
             out_dtype: torch.dtype | None = None) -> torch.Tensor:
        """x = W^T p.  p: [B, *sino_shape] or sino_shape on this device."""
        pb, single = self._batched(p, self.sino_shape)
        if not pb.is_contiguous():
            pb = pb.contiguous()
        B = pb.shape[0]
        odt = out_dtype or p.dtype
        if out is None:
            out = torch.empty((B,) + tuple(self.vol_shape), dtype=odt, device=self.device)
            if flags & capi.CSM_ACCUMULATE:
                out.zero_()
        else:
            out = out.view((B,) + tuple(self.vol_shape))
        compute = torch.float64 if torch.float64 in (pb.dtype, out.dtype) else torch.float32
        # x stored in another type: the workspace with room for the sums in the arithmetic type
        ws = self.workspace(1 if out.dtype == compute else 3, B, compute)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        with nvtx_range("csm_back"):
            capi.csm_back(self.handle, pb.data_ptr(), out.data_ptr(), B, _dt(pb.dtype), _dt(out.dtype), flags,
                          ws.data_ptr(), ws.numel(), stream)
        return out[0] if single else out

    def set_element_weights(self, weights) -> None:
        """Per-element detector sensitivity weights (array of sino_shape, or None for all 1):
        forward returns w * (W x), back projects w * p."""
        if weights is None:
            capi.csm_geom_set_element_weights(self.handle, None)
            return
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(self.sino_shape))
        capi.csm_geom_set_element_weights(self.handle, w.ctypes.data)

    def forward_line(self, x: torch.Tensor, model: str = "siddon", lines: int = 1,
                     out: torch.Tensor | None = None) -> torch.Tensor:
        """p = W_line x for a line-based comparator model ("siddon" or "joseph"), the mean over
        `lines` rays per detector element (lines x lines in 3D)."""
        xb, single = self._batched(x, self.vol_shape)
        xb = xb.contiguous()
        B = xb.shape[0]
        if out is None:
            out = torch.empty((B,) + tuple(self.sino_shape), dtype=x.dtype, device=self.device)
        else:
            out = out.view((B,) + tuple(self.sino_shape))
        capi.csm_forward_line(self.handle, _LINE[model], lines, xb.data_ptr(), out.data_ptr(), B, _dt(xb.dtype),
                              _dt(out.dtype), 0, torch.cuda.current_stream(self.device).cuda_stream)
        return out[0] if single else out

    def back_line(self, p: torch.Tensor, model: str = "siddon", lines: int = 1,
                  out: torch.Tensor | None = None) -> torch.Tensor:
        """x = W_line^T p, the exact adjoint of forward_line (float32 / float64 output)."""
        pb, single = self._batched(p, self.sino_shape)
        pb = pb.contiguous()
        B = pb.shape[0]
        if out is None:
            odt = pb.dtype if pb.dtype in (torch.float32, torch.float64) else torch.float32
            out = torch.empty((B,) + tuple(self.vol_shape), dtype=odt, device=self.device)
        else:
            out = out.view((B,) + tuple(self.vol_shape))
        capi.csm_back_line(self.handle, _LINE[model], lines, pb.data_ptr(), out.data_ptr(), B, _dt(pb.dtype),
                           _dt(out.dtype), 0, torch.cuda.current_stream(self.device).cuda_stream)
        return out[0] if single else out

    def nnz(self) -> int:
        """Number of nonzero entries of W (cached after the first call)."""
        return capi.csm_nnz(self.handle, torch.cuda.current_stream(self.device).cuda_stream)

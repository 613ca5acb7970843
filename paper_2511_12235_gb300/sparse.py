"""The system matrix W as explicit CSR matrices on the device, and SART on them.

For problems small enough to store W, ``SparseW`` exports W and W^T (csm_export_csr) from the
same closed-form entries the projectors evaluate on the fly; ``matvec`` / ``rmatvec`` apply
them with the library's CSR kernel (csm_csr_spmv).  ``sart`` runs the simultaneous
algebraic reconstruction technique, one of the algebraic methods the paper lists for
p = W u (Introduction, Eq. (ip)):
    x <- x + lam C^{-1} W^T R^{-1} (p - W x),   R = diag(W 1), C = diag(W^T 1),
with W R^{-1}-normalised by rows and W^T by the column sums of W (csm_csr_normalize_rows),
so that an iteration is two CSR products.
"""
from __future__ import annotations

import torch

from . import _capi as capi
from .projector import Projector, _dt
from .solvers import VecOps


class CSR:
    """One CSR matrix on the device (row_ptr int64, col int32, val float32/float64)."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, n_cols: int):
        self.row_ptr, self.col, self.val, self.n_cols = row_ptr, col, val, n_cols
        self.n_rows = row_ptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.val.numel()

    def mv(self, x: torch.Tensor, out: torch.Tensor | None = None, alpha: float = 1.0, beta: float = 0.0):
        """out = alpha A x + beta out."""
        x = x.reshape(-1).contiguous()
        assert x.numel() == self.n_cols and x.dtype == self.val.dtype
        if out is None:
            out = torch.zeros(self.n_rows, dtype=self.val.dtype, device=self.val.device)
        capi.csm_csr_spmv(self.n_rows, self.row_ptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr(),
                          _dt(self.val.dtype), alpha, x.data_ptr(), beta, out.data_ptr(),
                          torch.cuda.current_stream(self.val.device).cuda_stream)
        return out

    def normalized_rows(self):
        """(a copy with every row divided by its sum, the row sums)."""
        val = self.val.clone()
        sums = torch.empty(self.n_rows, dtype=val.dtype, device=val.device)
        capi.csm_csr_normalize_rows(self.n_rows, self.row_ptr.data_ptr(), val.data_ptr(), _dt(val.dtype),
                                    sums.data_ptr(), torch.cuda.current_stream(val.device).cuda_stream)
        return CSR(self.row_ptr, self.col, val, self.n_cols), sums

    def to_torch(self) -> torch.Tensor:
        return torch.sparse_csr_tensor(self.row_ptr, self.col, self.val, size=(self.n_rows, self.n_cols))


def export(P: Projector, transpose: bool = False, dtype: torch.dtype = torch.float64, relative: bool = False) -> CSR:
    """W (rows: detector elements) or W^T (rows: voxels) of the projector's geometry."""
    flags = (capi.CSM_EXPORT_TRANSPOSE if transpose else 0) | (capi.CSM_RELATIVE_WEIGHTS if relative else 0)
    dev = P.device
    nvox = 1
    for d in P.vol_shape:
        nvox *= d
    nel = 1
    for d in P.sino_shape:
        nel *= d
    n_rows, n_cols = (nvox, nel) if transpose else (nel, nvox)
    ws = torch.empty(max(capi.csm_export_workspace_bytes(P.handle, flags), 256), dtype=torch.uint8, device=dev)
    row_ptr = torch.empty(n_rows + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    vdt = _dt(dtype)
    nnz = capi.csm_export_csr(P.handle, flags, vdt, row_ptr.data_ptr(), None, None, 0, ws.data_ptr(), ws.numel(),
                              stream)
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz, 1), dtype=dtype, device=dev)
    capi.csm_export_csr(P.handle, flags, vdt, row_ptr.data_ptr(), col.data_ptr(), val.data_ptr(), nnz,
                        ws.data_ptr(), ws.numel(), stream)
    return CSR(row_ptr, col[:nnz], val[:nnz], n_cols)


class SparseW:
    """W and W^T of one geometry as CSR matrices (float64 by default)."""

    def __init__(self, P: Projector, dtype: torch.dtype = torch.float64, relative: bool = False):
        self.P = P
        self.W = export(P, False, dtype, relative)
        self.WT = export(P, True, dtype, relative)

    def matvec(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        return self.W.mv(x, out)

    def rmatvec(self, p: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        return self.WT.mv(p, out)


def sart(S: SparseW, p: torch.Tensor, iters: int, lam: float = 1.0, x0: torch.Tensor | None = None,
         residuals: bool = True):
    """SART iterations on measured projections p (one problem).  Returns (x, [||p - W x_k||^2
    for k = 0..iters] (float64 on the host; empty when residuals is False))."""
    M, rsum = S.W.normalized_rows()          # R^{-1} W
    N, _ = S.WT.normalized_rows()            # C^{-1} W^T
    dt = S.W.val.dtype
    dev = S.W.val.device
    stream = torch.cuda.current_stream(dev).cuda_stream
    pv = p.reshape(-1).to(dev, dt).contiguous()
    pt = torch.empty_like(pv)
    capi.csm_ediv(pv.numel(), _dt(dt), pv.data_ptr(), rsum.data_ptr(), pt.data_ptr(), stream)   # R^{-1} p
    x = (torch.zeros(S.W.n_cols, dtype=dt, device=dev) if x0 is None
         else x0.reshape(-1).to(dev, dt).contiguous().clone())
    t = torch.empty_like(pt)
    res = torch.empty(S.W.n_rows, dtype=dt, device=dev)
    r2 = torch.zeros(1, dtype=torch.float64, device=dev)
    ops = VecOps(dev, 1)
    hist = []

    def resid():
        res.copy_(pv)
        S.W.mv(x, res, alpha=-1.0, beta=1.0)
        ops.dot(res[None], res[None], r2)
        hist.append(float(r2.item()))

    if residuals:
        resid()
    for _ in range(iters):
        t.copy_(pt)
        M.mv(x, t, alpha=-1.0, beta=1.0)      # R^{-1} p - R^{-1} W x
        N.mv(t, x, alpha=lam, beta=1.0)       # x + lam C^{-1} W^T (...)
        if residuals:
            resid()
    return x.reshape(S.P.vol_shape), hist

"""ctypes binding of the C ABI in include/csm.h (argument marshalling only).

The functions keep the C names.  Importing this module loads ``_build/libcsm.so`` and
raises ImportError when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcsm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libcsm.so is not built (expected at %s); run `python -c \"import __graft_entry__ as g; g.build()\"`"
        % LIB_PATH)

lib = C.CDLL(LIB_PATH)

CSM_OK, CSM_EINVAL, CSM_EGEOM, CSM_ENOMEM, CSM_ECUDA, CSM_EUNSUPPORTED, CSM_ETIMEOUT = range(7)
CSM_F32, CSM_F64, CSM_BF16, CSM_F16 = range(4)
CSM_ACCUMULATE = 1
CSM_RELATIVE_WEIGHTS = 2
CSM_VOXEL_DRIVEN = 4
CSM_EXPORT_TRANSPOSE = 8
CSM_LINE_SIDDON = 1
CSM_LINE_JOSEPH = 2


class csm_geom2d_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("a", C.c_double), ("b", C.c_double),
                ("n_views", C.c_int), ("angles", C.POINTER(C.c_double)),
                ("s", C.c_double), ("sdd", C.c_double), ("nu", C.c_int),
                ("du", C.c_double), ("u_off", C.c_double)]


class csm_geom3d_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("a", C.c_double), ("b", C.c_double), ("c", C.c_double),
                ("n_views", C.c_int), ("angles", C.POINTER(C.c_double)),
                ("s", C.c_double), ("sdd", C.c_double), ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double), ("u_off", C.c_double), ("v_off", C.c_double)]


csm_geom_t = C.c_void_p
_st = C.c_int

lib.csm_geom_create_2d.argtypes = [C.POINTER(csm_geom2d_desc), C.POINTER(csm_geom_t)]
lib.csm_geom_create_2d.restype = _st
lib.csm_geom_create_3d.argtypes = [C.POINTER(csm_geom3d_desc), C.POINTER(csm_geom_t)]
lib.csm_geom_create_3d.restype = _st
lib.csm_geom_set_element_weights.argtypes = [csm_geom_t, C.c_void_p]
lib.csm_geom_set_element_weights.restype = _st
lib.csm_geom_free.argtypes = [csm_geom_t]
lib.csm_geom_free.restype = None
lib.csm_workspace_bytes.argtypes = [csm_geom_t, C.c_int, C.c_int64, C.c_int, C.POINTER(C.c_size_t)]
lib.csm_workspace_bytes.restype = _st
lib.csm_forward.argtypes = [csm_geom_t, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                            C.c_void_p, C.c_size_t, C.c_void_p]
lib.csm_forward.restype = _st
lib.csm_back.argtypes = [csm_geom_t, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                         C.c_void_p, C.c_size_t, C.c_void_p]
lib.csm_back.restype = _st
lib.csm_nnz.argtypes = [csm_geom_t, C.POINTER(C.c_int64), C.c_void_p]
lib.csm_nnz.restype = _st
lib.csm_dot_workspace_bytes.argtypes = [C.c_int64, C.POINTER(C.c_size_t)]
lib.csm_dot_workspace_bytes.restype = _st
lib.csm_dot.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_size_t,
                        C.c_void_p]
lib.csm_dot.restype = _st
lib.csm_axpby.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
lib.csm_axpby.restype = _st
lib.csm_dot_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]
lib.csm_dot_noalloc.restype = _st
lib.csm_fma_rate.argtypes = [C.c_int, C.c_int64, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                             C.c_void_p]
lib.csm_fma_rate.restype = _st
lib.csm_launch_count.argtypes = [C.POINTER(C.c_uint64)]
lib.csm_launch_count.restype = _st
lib.csm_forward_line.argtypes = [csm_geom_t, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                                 C.c_int, C.c_void_p]
lib.csm_forward_line.restype = _st
lib.csm_back_line.argtypes = [csm_geom_t, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                              C.c_int, C.c_void_p]
lib.csm_back_line.restype = _st
lib.csm_export_workspace_bytes.argtypes = [csm_geom_t, C.c_int, C.POINTER(C.c_size_t)]
lib.csm_export_workspace_bytes.restype = _st
lib.csm_export_csr.argtypes = [csm_geom_t, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                               C.POINTER(C.c_int64), C.c_void_p, C.c_size_t, C.c_void_p]
lib.csm_export_csr.restype = _st
lib.csm_csr_spmv.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                             C.c_double, C.c_void_p, C.c_void_p]
lib.csm_csr_spmv.restype = _st
lib.csm_csr_normalize_rows.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
lib.csm_csr_normalize_rows.restype = _st
lib.csm_fista_coeffs.argtypes = [C.c_int64, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
lib.csm_fista_coeffs.restype = _st
lib.csm_ediv.argtypes = [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
lib.csm_ediv.restype = _st
lib.csm_sync_status.argtypes = [C.c_void_p]
lib.csm_sync_status.restype = _st
lib.csm_status_string.argtypes = [_st]
lib.csm_status_string.restype = C.c_char_p
lib.csm_last_cuda_error.argtypes = []
lib.csm_last_cuda_error.restype = C.c_char_p

EXPORTED = [
    "csm_geom_create_2d", "csm_geom_create_3d", "csm_geom_free", "csm_workspace_bytes",
    "csm_forward", "csm_back", "csm_nnz", "csm_sync_status", "csm_status_string",
    "csm_last_cuda_error", "csm_dot_workspace_bytes", "csm_dot", "csm_axpby", "csm_dot_noalloc",
    "csm_fma_rate", "csm_launch_count", "csm_export_workspace_bytes", "csm_export_csr", "csm_csr_spmv",
    "csm_csr_normalize_rows",
    "csm_ediv", "csm_fista_coeffs", "csm_forward_line", "csm_back_line", "csm_geom_set_element_weights",
]
CSM_DOT_NOALLOC_MAX_BATCH = 64


class CsmError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = "%s: %s" % (what, lib.csm_status_string(status).decode())
        if status == CSM_ECUDA:
            msg += " (" + lib.csm_last_cuda_error().decode() + ")"
        super().__init__(msg)
        self.status = status


def check(status: int, what: str) -> None:
    if status != CSM_OK:
        raise CsmError(status, what)


# Same-named thin wrappers -----------------------------------------------------------------
def csm_geom_create_2d(desc: csm_geom2d_desc) -> int:
    h = csm_geom_t()
    check(lib.csm_geom_create_2d(C.byref(desc), C.byref(h)), "csm_geom_create_2d")
    return h.value


def csm_geom_create_3d(desc: csm_geom3d_desc) -> int:
    h = csm_geom_t()
    check(lib.csm_geom_create_3d(C.byref(desc), C.byref(h)), "csm_geom_create_3d")
    return h.value


def csm_geom_free(h: int) -> None:
    lib.csm_geom_free(h)


def csm_workspace_bytes(h: int, op: int, batch: int, compute: int) -> int:
    n = C.c_size_t()
    check(lib.csm_workspace_bytes(h, op, batch, compute, C.byref(n)), "csm_workspace_bytes")
    return n.value


def csm_forward(h, x_ptr, p_ptr, batch, x_dt, p_dt, flags, ws_ptr, ws_bytes, stream) -> None:
    check(lib.csm_forward(h, x_ptr, p_ptr, batch, x_dt, p_dt, flags, ws_ptr, ws_bytes, stream), "csm_forward")


def csm_back(h, p_ptr, x_ptr, batch, p_dt, x_dt, flags, ws_ptr, ws_bytes, stream) -> None:
    check(lib.csm_back(h, p_ptr, x_ptr, batch, p_dt, x_dt, flags, ws_ptr, ws_bytes, stream), "csm_back")


def csm_nnz(h, stream) -> int:
    n = C.c_int64()
    check(lib.csm_nnz(h, C.byref(n), stream), "csm_nnz")
    return n.value


def csm_sync_status(stream) -> None:
    check(lib.csm_sync_status(stream), "csm_sync_status")


def csm_dot_workspace_bytes(batch: int) -> int:
    n = C.c_size_t()
    check(lib.csm_dot_workspace_bytes(batch, C.byref(n)), "csm_dot_workspace_bytes")
    return n.value


def csm_dot(a_ptr, c_ptr, n, batch, dt, out_ptr, ws_ptr, ws_bytes, stream) -> None:
    check(lib.csm_dot(a_ptr, c_ptr, n, batch, dt, out_ptr, ws_ptr, ws_bytes, stream), "csm_dot")


def csm_axpby(n, batch, dt, a_c, a_num, a_den, x_ptr, b_c, b_num, b_den, y_ptr, flags, stream) -> None:
    check(lib.csm_axpby(n, batch, dt, a_c, a_num, a_den, x_ptr, b_c, b_num, b_den, y_ptr, flags, stream),
          "csm_axpby")


def csm_dot_noalloc(a_ptr, c_ptr, n, batch, dt, out_ptr, stream) -> None:
    check(lib.csm_dot_noalloc(a_ptr, c_ptr, n, batch, dt, out_ptr, stream), "csm_dot_noalloc")


def csm_fma_rate(dt, iters, blocks_per_sm, launches, stream) -> tuple[float, float]:
    """(flops, seconds) of the FMA-chain kernel on the current device."""
    f, t = C.c_double(), C.c_double()
    check(lib.csm_fma_rate(dt, iters, blocks_per_sm, launches, C.byref(f), C.byref(t), stream), "csm_fma_rate")
    return f.value, t.value


def csm_launch_count() -> int:
    """Kernels the library has launched from the host so far (all devices and streams)."""
    n = C.c_uint64()
    check(lib.csm_launch_count(C.byref(n)), "csm_launch_count")
    return n.value


def csm_export_workspace_bytes(h, flags) -> int:
    n = C.c_size_t()
    check(lib.csm_export_workspace_bytes(h, flags, C.byref(n)), "csm_export_workspace_bytes")
    return n.value


def csm_export_csr(h, flags, val_dt, row_ptr, col_idx, val, capacity, ws_ptr, ws_bytes, stream) -> int:
    """Writes the CSR arrays (col_idx / val may be None for the count only); returns nnz."""
    n = C.c_int64()
    st = lib.csm_export_csr(h, flags, val_dt, row_ptr, col_idx, val, capacity, C.byref(n), ws_ptr, ws_bytes, stream)
    if st == CSM_EINVAL and col_idx and capacity < n.value:
        raise CsmError(st, "csm_export_csr (capacity %d < nnz %d)" % (capacity, n.value))
    check(st, "csm_export_csr")
    return n.value


def csm_csr_spmv(n_rows, row_ptr, col_idx, val, dt, alpha, x, beta, y, stream) -> None:
    check(lib.csm_csr_spmv(n_rows, row_ptr, col_idx, val, dt, alpha, x, beta, y, stream), "csm_csr_spmv")


def csm_csr_normalize_rows(n_rows, row_ptr, val, dt, row_sums, stream) -> None:
    check(lib.csm_csr_normalize_rows(n_rows, row_ptr, val, dt, row_sums, stream), "csm_csr_normalize_rows")


def csm_ediv(n, dt, num, den, out, stream) -> None:
    check(lib.csm_ediv(n, dt, num, den, out, stream), "csm_ediv")


def csm_fista_coeffs(batch, table, n_table, k, one_plus, theta, stream) -> None:
    check(lib.csm_fista_coeffs(batch, table, n_table, k, one_plus, theta, stream), "csm_fista_coeffs")


def csm_forward_line(h, model, lines, x_ptr, p_ptr, batch, x_dt, p_dt, flags, stream) -> None:
    check(lib.csm_forward_line(h, model, lines, x_ptr, p_ptr, batch, x_dt, p_dt, flags, stream), "csm_forward_line")


def csm_back_line(h, model, lines, p_ptr, x_ptr, batch, p_dt, x_dt, flags, stream) -> None:
    check(lib.csm_back_line(h, model, lines, p_ptr, x_ptr, batch, p_dt, x_dt, flags, stream), "csm_back_line")


def csm_geom_set_element_weights(h, weights_ptr) -> None:
    check(lib.csm_geom_set_element_weights(h, weights_ptr), "csm_geom_set_element_weights")

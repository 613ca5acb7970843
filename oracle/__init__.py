"""FP64 CPU oracle for the consistent cone-beam system matrix (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It computes every entry W_ij as the plain area/volume of the
intersection of voxel j with the cone of detector element i (Introduction, Eq. (ip);
Notation and Setup, Eq. (z rotation)), by polygon / polyhedron clipping in C
(``csm_oracle.c``), and builds p = W x and x = W^T p from those entries.  It shares no
code with the CUDA path.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (Monte Carlo, the paper's closed-form atoms, partition and
column-sum invariants, closed-form fan/pyramid volumes, scaling and symmetry); the COO
export, the entry counts and the z-slab back projection are pinned against the projections
they must reproduce (``tests/test_oracle_coo.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcsm_oracle.so")
_lock = threading.Lock()
_lib = None


class _Geom(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("a", C.c_double), ("b", C.c_double), ("c", C.c_double),
        ("n_views", C.c_int), ("angles", C.POINTER(C.c_double)),
        ("s", C.c_double), ("sdd", C.c_double),
        ("nu", C.c_int), ("nv", C.c_int),
        ("du", C.c_double), ("dv", C.c_double),
        ("u_off", C.c_double), ("v_off", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP) into oracle/_build/libcsm_oracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        gp = C.POINTER(_Geom)
        lib.orc_clip_area_2d.argtypes = [C.c_double] * 4 + [dp, C.c_int]
        lib.orc_clip_area_2d.restype = C.c_double
        lib.orc_clip_volume_3d.argtypes = [C.c_double] * 6 + [dp, C.c_int]
        lib.orc_clip_volume_3d.restype = C.c_double
        lib.orc2d_entries.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, ip, dp, C.c_int]
        lib.orc2d_entries.restype = C.c_int
        lib.orc3d_entries.argtypes = [gp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip, dp, C.c_int]
        lib.orc3d_entries.restype = C.c_int
        lib.orc2d_forward.argtypes = [gp, dp, dp, ip, C.c_int]
        lib.orc2d_back.argtypes = [gp, dp, dp, ip, C.c_int]
        lib.orc2d_forward_element.argtypes = [gp, dp, C.c_int, C.c_int]
        lib.orc2d_forward_element.restype = C.c_double
        lib.orc3d_forward.argtypes = [gp, dp, dp, ip, C.c_int]
        lib.orc3d_back.argtypes = [gp, dp, dp, ip, C.c_int]
        lib.orc3d_back_voxel.argtypes = [gp, dp, ip, C.c_int, C.c_int, C.c_int, C.c_int]
        lib.orc3d_back_voxel.restype = C.c_double
        lib.orc3d_forward_element.argtypes = [gp, dp, C.c_int, C.c_int, C.c_int]
        lib.orc3d_forward_element.restype = C.c_double
        lib.orc2d_coo.argtypes = [gp, ip, C.c_int, ip, ip, dp, C.c_long]
        lib.orc2d_coo.restype = C.c_long
        lib.orc3d_coo.argtypes = [gp, ip, C.c_int, ip, ip, dp, C.c_long]
        lib.orc3d_coo.restype = C.c_long
        lib.orc3d_back_slab.argtypes = [gp, dp, dp, ip, C.c_int, C.c_int, C.c_int]
        lib.orc3d_back_slab.restype = C.c_long
        lib.orc_line_forward.argtypes = [gp, C.c_int, C.c_int, dp, dp, ip, C.c_int]
        lib.orc_line_back.argtypes = [gp, C.c_int, C.c_int, dp, dp, ip, C.c_int]
        lib.orc2d_count.argtypes = [gp, ip, C.c_int]
        lib.orc2d_count.restype = C.c_long
        lib.orc_num_threads.restype = C.c_int
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int))


class _GeomHolder:
    """Keeps the angle array alive while the C struct points at it."""

    def __init__(self, g: dict):
        self.angles = np.ascontiguousarray(np.asarray(g["angles"], dtype=np.float64))
        self.s = _Geom(g["nx"], g["ny"], g["nz"], g["a"], g["b"], g["c"], g["n_views"],
                       _dptr(self.angles), g["s"], g["sdd"], g["nu"], g["nv"], g["du"],
                       g["dv"], g["u_off"], g["v_off"])

    @property
    def ref(self):
        return C.byref(self.s)


def _views(g, views):
    if views is None:
        views = np.arange(g["n_views"])
    return np.ascontiguousarray(np.asarray(views, dtype=np.int32))


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------------------------------
# Primitive clips (exposed so the tests can pin them on their own).
# ---------------------------------------------------------------------------------------
def clip_area_2d(box, planes) -> float:
    """Area of the box [x0,x1]x[y0,y1] inside all half-planes c0 x + c1 y + c3 >= 0."""
    pl = np.ascontiguousarray(np.asarray(planes, dtype=np.float64).reshape(-1, 4))
    return float(_load().orc_clip_area_2d(*map(float, box), _dptr(pl), pl.shape[0]))


def clip_volume_3d(box, planes) -> float:
    """Volume of the box [x0,x1]x[y0,y1]x[z0,z1] inside all half-spaces n.P + c >= 0."""
    pl = np.ascontiguousarray(np.asarray(planes, dtype=np.float64).reshape(-1, 4))
    return float(_load().orc_clip_volume_3d(*map(float, box), _dptr(pl), pl.shape[0]))


# ---------------------------------------------------------------------------------------
# Entries, projections.
# ---------------------------------------------------------------------------------------
def entries_2d(g: dict, view: int, ix: int, iy: int, all_elements: bool = False):
    """Nonzero W entries of pixel (ix, iy) in one view: (element indices, areas)."""
    h = _GeomHolder(g)
    ks = np.zeros(256, np.int32)
    ws = np.zeros(256, np.float64)
    n = _load().orc2d_entries(h.ref, int(view), int(ix), int(iy), int(all_elements),
                              _iptr(ks), _dptr(ws), 256)
    return ks[:n].copy(), ws[:n].copy()


def entries_3d(g: dict, view: int, ix: int, iy: int, iz: int, all_elements: bool = False):
    """Nonzero W entries of voxel (ix,iy,iz) in one view: ((k, l) pairs, volumes)."""
    h = _GeomHolder(g)
    kl = np.zeros(4096, np.int32)
    ws = np.zeros(4096, np.float64)
    n = _load().orc3d_entries(h.ref, int(view), int(ix), int(iy), int(iz), int(all_elements),
                              _iptr(kl), _dptr(ws), 4096)
    kl = kl[:n]
    return np.stack([kl % g["nu"], kl // g["nu"]], axis=1), ws[:n].copy()


def forward_2d(g: dict, x: np.ndarray, views=None) -> np.ndarray:
    """p[view][nu] = W x for one image x[ny][nx] (float64)."""
    h = _GeomHolder(g)
    v = _views(g, views)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (g["ny"], g["nx"])
    p = np.zeros((len(v), g["nu"]), np.float64)
    _load().orc2d_forward(h.ref, _dptr(x), _dptr(p), _iptr(v), len(v))
    return p


def back_2d(g: dict, p: np.ndarray, views=None) -> np.ndarray:
    """x[ny][nx] = W^T p over the given views (p is [len(views)][nu])."""
    h = _GeomHolder(g)
    v = _views(g, views)
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert p.shape == (len(v), g["nu"])
    x = np.zeros((g["ny"], g["nx"]), np.float64)
    _load().orc2d_back(h.ref, _dptr(p), _dptr(x), _iptr(v), len(v))
    return x


def forward_element_2d(g: dict, x: np.ndarray, view: int, k: int) -> float:
    h = _GeomHolder(g)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().orc2d_forward_element(h.ref, _dptr(x), int(view), int(k)))


def forward_3d(g: dict, x: np.ndarray, views=None) -> np.ndarray:
    """p[view][nv][nu] = W x for one volume x[nz][ny][nx] (float64)."""
    h = _GeomHolder(g)
    v = _views(g, views)
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (g["nz"], g["ny"], g["nx"])
    p = np.zeros((len(v), g["nv"], g["nu"]), np.float64)
    _load().orc3d_forward(h.ref, _dptr(x), _dptr(p), _iptr(v), len(v))
    return p


def back_3d(g: dict, p: np.ndarray, views=None) -> np.ndarray:
    """x[nz][ny][nx] = W^T p over the given views (p is [len(views)][nv][nu])."""
    h = _GeomHolder(g)
    v = _views(g, views)
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert p.shape == (len(v), g["nv"], g["nu"])
    x = np.zeros((g["nz"], g["ny"], g["nx"]), np.float64)
    _load().orc3d_back(h.ref, _dptr(p), _dptr(x), _iptr(v), len(v))
    return x


def back_slab_3d(g: dict, p: np.ndarray, iz0: int, iz1: int, views=None):
    """x[iz0:iz1] of W^T p over the given views (p is [len(views)][nv][nu]), and the number of
    nonzero entries that went into it.  Returns (x [iz1 - iz0][ny][nx], count)."""
    h = _GeomHolder(g)
    v = _views(g, views)
    p = np.ascontiguousarray(p, dtype=np.float64)
    assert p.shape == (len(v), g["nv"], g["nu"]) and 0 <= iz0 <= iz1 <= g["nz"]
    x = np.zeros((iz1 - iz0, g["ny"], g["nx"]), np.float64)
    n = _load().orc3d_back_slab(h.ref, _dptr(p), _dptr(x), _iptr(v), len(v), int(iz0), int(iz1))
    return x, int(n)


def forward_element_3d(g: dict, x: np.ndarray, view: int, k: int, l: int) -> float:
    """One detector value p[view][l][k], computed on its own."""
    h = _GeomHolder(g)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().orc3d_forward_element(h.ref, _dptr(x), int(view), int(k), int(l)))


def back_voxel_3d(g: dict, p: np.ndarray, ix: int, iy: int, iz: int, views=None) -> float:
    """One back-projected value x[iz][iy][ix] over the given views (p is [len(views)][nv][nu])."""
    h = _GeomHolder(g)
    v = _views(g, views)
    p = np.ascontiguousarray(p, dtype=np.float64)
    return float(_load().orc3d_back_voxel(h.ref, _dptr(p), _iptr(v), len(v), int(ix), int(iy), int(iz)))


def count_2d(g: dict, views=None) -> int:
    """Number of nonzero 2D entries over the given views."""
    h = _GeomHolder(g)
    v = _views(g, views)
    return int(_load().orc2d_count(h.ref, _iptr(v), len(v)))


def coo(g: dict, views=None, cap: int | None = None):
    """Explicit sparse W (rows over the selected views, columns over voxels) as COO arrays."""
    h = _GeomHolder(g)
    v = _views(g, views)
    nvox = g["nx"] * g["ny"] * g["nz"]
    if cap is None:
        cap = int(nvox * len(v) * (64 if g.get("dim", 2) == 3 else 8)) + 1024
    rows = np.zeros(cap, np.int32)
    cols = np.zeros(cap, np.int32)
    vals = np.zeros(cap, np.float64)
    fn = _load().orc3d_coo if g.get("dim", 2) == 3 else _load().orc2d_coo
    n = fn(h.ref, _iptr(v), len(v), _iptr(rows), _iptr(cols), _dptr(vals), cap)
    if n < 0:
        raise RuntimeError("COO capacity too small")
    return rows[:n].copy(), cols[:n].copy(), vals[:n].copy()


LINE_MODELS = {"siddon": 1, "joseph": 2}


def line_forward(g: dict, x: np.ndarray, model: str = "siddon", lines: int = 1, views=None) -> np.ndarray:
    """Line-based comparator projections (Siddon: lengths in voxels; Joseph: interpolation
    per slice), the mean over `lines` rays per element (lines x lines in 3D).  Returns
    [views][nu] (2D) or [views][nv][nu] (3D)."""
    h = _GeomHolder(g)
    v = _views(g, views)
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.zeros((len(v), g["nv"], g["nu"]), np.float64)
    _load().orc_line_forward(h.ref, LINE_MODELS[model], int(lines), _dptr(x), _dptr(p), _iptr(v), len(v))
    return p if g.get("dim", 2) == 3 else p[:, 0, :]


def line_back(g: dict, p: np.ndarray, model: str = "siddon", lines: int = 1, views=None) -> np.ndarray:
    """The adjoint of line_forward (same rays and weights)."""
    h = _GeomHolder(g)
    v = _views(g, views)
    p = np.ascontiguousarray(np.asarray(p, np.float64).reshape(len(v), g["nv"], g["nu"]))
    x = np.zeros((g["nz"], g["ny"], g["nx"]), np.float64)
    _load().orc_line_back(h.ref, LINE_MODELS[model], int(lines), _dptr(p), _dptr(x), _iptr(v), len(v))
    return x if g.get("dim", 2) == 3 else x[0]

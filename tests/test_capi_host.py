"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol that
include/csm.h declares, and rejects bad arguments on the host before touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2511_12235_gb300 import build
    build.build()
    from paper_2511_12235_gb300 import _capi
    return _capi


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "csm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(csm_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(capi):
    syms = _declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(capi.lib, s), s
    assert set(capi.EXPORTED) == set(syms)


def test_launch_count_on_host(capi):
    """The launch counter reads without a GPU and never goes down; a NULL pointer is refused."""
    a = capi.csm_launch_count()
    assert a >= 0 and capi.csm_launch_count() >= a
    assert capi.lib.csm_launch_count(None) == capi.CSM_EINVAL


def test_status_strings(capi):
    for s in range(7):
        assert capi.lib.csm_status_string(s)


def _desc2d(capi, **kw):
    ang = np.linspace(0, 6, 8)
    base = dict(nx=16, ny=16, a=1.0, b=1.0, n_views=8, s=40.0, sdd=70.0, nu=24, du=1.0, u_off=0.0)
    base.update(kw)
    d = capi.csm_geom2d_desc(base["nx"], base["ny"], base["a"], base["b"], base["n_views"],
                             ang.ctypes.data_as(C.POINTER(C.c_double)), base["s"], base["sdd"], base["nu"],
                             base["du"], base["u_off"])
    return d, ang


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=0), 1), (dict(nu=-1), 1), (dict(a=0.0), 1), (dict(du=float("nan")), 1),
    (dict(s=5.0), 2),            # source inside the grid's circumcircle
    (dict(sdd=30.0), 2),         # detector in front of the source
])
def test_geometry_validation_on_host(capi, kw, expect):
    d, ang = _desc2d(capi, **kw)
    h = capi.csm_geom_t()
    assert capi.lib.csm_geom_create_2d(C.byref(d), C.byref(h)) == expect
    assert not h.value


def test_null_arguments(capi):
    h = capi.csm_geom_t()
    assert capi.lib.csm_geom_create_2d(None, C.byref(h)) == capi.CSM_EINVAL
    assert capi.lib.csm_forward(None, None, None, 1, 0, 0, 0, None, 0, None) == capi.CSM_EINVAL
    assert capi.lib.csm_back(None, None, None, 1, 0, 0, 0, None, 0, None) == capi.CSM_EINVAL
    n = C.c_size_t()
    assert capi.lib.csm_workspace_bytes(None, 0, 1, 0, C.byref(n)) == capi.CSM_EINVAL
    capi.lib.csm_geom_free(None)

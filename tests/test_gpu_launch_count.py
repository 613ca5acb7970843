"""The library's own launch counter (csm_launch_count) against the launches each projector
call is known to make: 2D forward / back one layout kernel and one projector kernel per chunk
of 16 batch items; 3D forward the volume layout kernel, the columns' nonzero ranges and one
projector kernel; 3D back the differenced-sinogram kernel and one projector launch per group
of views."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _count(fn):
    from paper_2511_12235_gb300 import _capi as capi
    torch.cuda.synchronize()
    a = capi.csm_launch_count()
    fn()
    torch.cuda.synchronize()
    return capi.csm_launch_count() - a


def test_launches_per_call_2d():
    from paper_2511_12235_gb300 import Projector
    g = synth.config("fan2d_64")
    P = Projector(g)
    x = torch.rand((20, g["ny"], g["nx"]), dtype=torch.float32, device="cuda")
    p = P.forward(x)
    xb = P.back(p)
    assert _count(lambda: P.forward(x, out=p)) == 2 * 2      # two chunks: 16 + 4 items
    assert _count(lambda: P.back(p, out=xb)) == 2 * 2
    assert _count(lambda: P.forward(x[:1], out=p[:1])) == 2
    P.close()


def test_launches_per_call_3d():
    from paper_2511_12235_gb300 import Projector
    g = synth.config("cone3d_128")
    P = Projector(g)
    x = torch.from_numpy(synth.ellipsoid_phantom(g["nx"], 0)).float().cuda()[None]
    p = P.forward(x)
    xb = P.back(p)
    assert _count(lambda: P.forward(x, out=p)) == 3   # layouts, nonzero ranges, projector
    # views in groups whose slices of the differenced sinogram (FP32, batch 1) fit in 64 MiB
    slice_bytes = (g["nu"] + 1) * (g["nv"] + 2) * 4 * 4
    group = max(1, min(g["n_views"], (64 << 20) // slice_bytes))
    assert _count(lambda: P.back(p, out=xb)) == 1 + -(-g["n_views"] // group)
    P.close()

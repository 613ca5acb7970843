"""The voxel-driven forward variant (CSM_VOXEL_DRIVEN, the scatter form of the paper's
Algorithm 1) against the oracle and the ray-driven gather: FP64 within 1e-11 relative of the
oracle, FP32 within 1e-5 per view, BF16 output within the storage bound; flags and batches."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _per_view(p, ref):
    p = np.asarray(p, np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(p - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)))


def _g3():
    ang = np.concatenate([synth.uniform_angles(10), [0.0, math.pi / 2, math.pi / 4]])
    g = synth.geometry(9, 8, 11, a=1.2, b=0.9, c=1.1, n_views=len(ang), angles=ang, s=14.0 * 1.6, sdd=23.0 * 1.6,
                       nu=21, nv=19, du=1.3, dv=1.1, u_off=0.2, v_off=-0.35)
    g["dim"] = 3
    return g


@pytest.mark.parametrize("dim", [2, 3])
def test_voxel_driven_forward_matches_oracle(dim):
    from paper_2511_12235_gb300 import Projector
    g = synth.config("fan2d_64") if dim == 2 else _g3()
    P = Projector(g)
    rng = np.random.default_rng(30 + dim)
    x = rng.uniform(size=(2,) + P.vol_shape)
    x[1][x[1] < 0.5] = 0.0                                 # zero voxels / columns are skipped
    for i in range(2):
        ref = oracle.forward_2d(g, x[i]) if dim == 2 else oracle.forward_3d(g, x[i])
        p64 = P.forward(torch.from_numpy(x[i]).cuda(), variant="voxel").cpu().numpy()
        assert np.max(np.abs(p64 - ref)) <= 1e-11 * np.max(np.abs(ref))
    xt = torch.from_numpy(x).float().cuda()
    p32 = P.forward(xt, variant="voxel").cpu().numpy()
    pr = P.forward(xt).cpu().numpy()
    for i in range(2):
        ref = oracle.forward_2d(g, x[i]) if dim == 2 else oracle.forward_3d(g, x[i])
        assert _per_view(p32[i], ref) < 1e-5
        assert _per_view(pr[i], ref) < 1e-5
    # storage types and flags
    pb = P.forward(xt.to(torch.bfloat16), variant="voxel").float().cpu().numpy()
    ref0 = oracle.forward_2d(g, x[0]) if dim == 2 else oracle.forward_3d(g, x[0])
    assert _per_view(pb[0], ref0) < 2 * 2 ** -9 + 1e-5
    from paper_2511_12235_gb300 import _capi as capi
    out = P.forward(xt[0], variant="voxel").clone()
    P.forward(xt[0], out=out, variant="voxel", flags=capi.CSM_ACCUMULATE)
    assert _per_view(out.cpu().numpy() / 2, ref0) < 1e-5
    rel = P.forward(xt[0], variant="voxel", flags=capi.CSM_RELATIVE_WEIGHTS).cpu().numpy()
    meas = g["a"] * g["b"] * (g["c"] if dim == 3 else 1.0)
    assert _per_view(rel * meas, ref0) < 1e-5
    P.close()

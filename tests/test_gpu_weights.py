"""Per-element detector sensitivity weights: the forward returns w * (W x), the back projection
projects w * p (the adjoint of the weighted forward), the exported matrix is diag(w) W, and
removing the weights restores W; checked against the unweighted kernels and the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _geom(dim):
    if dim == 2:
        return synth.config("fan2d_64")
    ang = synth.uniform_angles(12)
    g = synth.geometry(10, 9, 8, n_views=12, angles=ang, s=30.0, sdd=50.0, nu=18, nv=15, du=1.1, dv=0.9)
    g["dim"] = 3
    return g


@pytest.mark.parametrize("dim", [2, 3])
def test_weighted_forward_back_export(dim):
    from paper_2511_12235_gb300 import Projector, sparse
    g = _geom(dim)
    P = Projector(g)
    rng = np.random.default_rng(dim)
    w = rng.uniform(0.5, 1.5, size=P.sino_shape)
    x = rng.uniform(size=P.vol_shape)
    y = rng.uniform(size=P.sino_shape)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    p0 = P.forward(xt).cpu().numpy()
    b0 = P.back(torch.from_numpy(w * y).cuda()).cpu().numpy()
    P.set_element_weights(w)
    p1 = P.forward(xt).cpu().numpy()
    b1 = P.back(yt).cpu().numpy()
    assert np.allclose(p1, w * p0, rtol=1e-13, atol=1e-13 * np.abs(p0).max())
    assert np.allclose(b1, b0, rtol=1e-13, atol=1e-13 * np.abs(b0).max())
    # against the oracle's unweighted W
    pref = oracle.forward_2d(g, x) if dim == 2 else oracle.forward_3d(g, x)
    assert np.max(np.abs(p1 - w * pref)) <= 1e-11 * np.abs(pref).max()
    # FP32 path too
    p32 = P.forward(xt.float()).double().cpu().numpy()
    assert np.linalg.norm(p32 - w * pref) <= 1e-5 * np.linalg.norm(w * pref)
    # adjoint of the weighted pair
    lhs = float(np.sum(p1 * y))
    rhs = float(np.sum(x * b1))
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(p1) * np.linalg.norm(y)
    # the export is diag(w) W
    Wc = sparse.export(P, dtype=torch.float64)
    assert torch.allclose(Wc.mv(xt), torch.from_numpy(p1).cuda().reshape(-1), rtol=1e-11,
                          atol=1e-11 * float(np.abs(p1).max()))
    P.set_element_weights(None)
    assert np.array_equal(P.forward(xt).cpu().numpy(), p0)
    P.close()

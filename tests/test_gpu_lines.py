"""GPU line-based comparator projectors (csm_forward_line / csm_back_line) against the
oracle's Siddon and Joseph projections: FP64 within 1e-11 relative, FP32 within 1e-5 relative
per view, the back projection the adjoint of the forward."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csm():
    import paper_2511_12235_gb300 as m
    return m


def _geom(dim):
    if dim == 2:
        ang = np.concatenate([synth.uniform_angles(8), [0.0, math.pi / 2, math.pi / 4]])
        return synth.geometry(20, 17, 1, a=1.1, b=0.8, n_views=len(ang), angles=ang, s=40.0, sdd=70.0, nu=31,
                              du=1.1, u_off=0.2)
    ang = np.concatenate([synth.uniform_angles(5), [0.0, math.pi / 2]])
    g = synth.geometry(9, 8, 10, a=1.2, b=0.9, c=1.1, n_views=len(ang), angles=ang, s=25.0, sdd=40.0, nu=17, nv=15,
                       du=1.4, dv=1.2, u_off=0.3, v_off=-0.2)
    g["dim"] = 3
    return g


def _rel_per_view(p, ref):
    p = np.asarray(p, np.float64).reshape(ref.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return float(np.max(np.linalg.norm(p - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)))


@pytest.mark.parametrize("model", ["siddon", "joseph"])
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lines", [1, 3])
def test_line_projectors_match_oracle(csm, model, dim, lines):
    g = _geom(dim)
    P = csm.Projector(g)
    rng = np.random.default_rng(dim * 10 + lines)
    x = rng.uniform(size=P.vol_shape)
    ref = oracle.line_forward(g, x, model, lines=lines)
    p64 = P.forward_line(torch.from_numpy(x).cuda(), model, lines).cpu().numpy()
    assert _rel_per_view(p64, ref) < 1e-11
    p32 = P.forward_line(torch.from_numpy(x).float().cuda(), model, lines).cpu().numpy()
    assert _rel_per_view(p32, ref) < 1e-5
    y = rng.uniform(size=P.sino_shape)
    bref = oracle.line_back(g, y, model, lines=lines)
    b64 = P.back_line(torch.from_numpy(y).cuda(), model, lines).cpu().numpy()
    assert np.linalg.norm(b64 - bref) <= 1e-11 * np.linalg.norm(bref)
    b32 = P.back_line(torch.from_numpy(y).float().cuda(), model, lines).cpu().numpy()
    assert np.linalg.norm(b32 - bref) <= 1e-5 * np.linalg.norm(bref)
    P.close()


@pytest.mark.parametrize("model", ["siddon", "joseph"])
def test_line_adjoint_and_batch(csm, model):
    g = _geom(3)
    P = csm.Projector(g)
    rng = np.random.default_rng(2)
    x = torch.from_numpy(rng.normal(size=(2,) + P.vol_shape)).cuda()
    y = torch.from_numpy(rng.normal(size=(2,) + P.sino_shape)).cuda()
    px = P.forward_line(x, model, 2)
    by = P.back_line(y, model, 2)
    for i in range(2):
        lhs = float((px[i] * y[i]).sum())
        rhs = float((x[i] * by[i]).sum())
        assert abs(lhs - rhs) <= 1e-12 * float(px[i].norm()) * float(y[i].norm())
        assert torch.allclose(px[i], P.forward_line(x[i], model, 2), rtol=0, atol=0)
    P.close()

"""GPU parity of the 2D fan-beam projectors against the FP64 clipping oracle.

Bar: FP64 path within 1e-12 relative (rounding order only); FP32 path within 1e-5 relative
L2 per projection (per view for the forward, per image for the back), as stated for the
projector in FP32; BF16/F16 storage within the bound derived from the input and output
rounding (2 * 2^-9 + 1e-5 for BF16, 2 * 2^-11 + 1e-5 for F16).
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def csm():
    import paper_2511_12235_gb300 as m
    return m


def per_view_rel(p, ref):
    p = np.asarray(p, np.float64).reshape(ref.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    num = np.linalg.norm(p - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    ok = den > 0
    return float(np.max(num[ok] / den[ok])) if ok.any() else float(np.max(num))


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_fan64_fp64_forward_back_full(csm):
    g = synth.config("fan2d_64")
    x = synth.ellipse_phantom(64, 0)
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    p_ref = oracle.forward_2d(g, x)
    assert per_view_rel(p, p_ref) < FP64_TOL
    y = np.random.default_rng(1).uniform(size=p_ref.shape)
    b = P.back(torch.from_numpy(y).cuda()).cpu().numpy()
    b_ref = oracle.back_2d(g, y)
    assert rel(b, b_ref) < FP64_TOL
    assert np.max(np.abs(b - b_ref)) < 1e-11 * np.max(np.abs(b_ref))


def test_element_pairs_odd_detector_fp64(csm):
    """Enough views and elements that the forward runs one thread per element pair, with an
    odd element count (the last pair has one element): FP64 against the oracle."""
    ang = synth.uniform_angles(512)
    g = synth.geometry(24, 20, 1, n_views=512, angles=ang, s=60.0, sdd=100.0, nu=257, du=0.18, u_off=0.1)
    assert (g["nu"] // 2) * g["n_views"] >= 65536
    rng = np.random.default_rng(3)
    x = rng.uniform(size=(2, 20, 24))
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    for i in range(2):
        ref = oracle.forward_2d(g, x[i])
        assert per_view_rel(p[i], ref) < FP64_TOL
        assert np.count_nonzero(ref[:, -1]) > 0          # the unpaired last element carries weight


def test_fan64_fp32(csm):
    g = synth.config("fan2d_64")
    x = synth.ellipse_phantom(64, 0)
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).float().cuda()).cpu().numpy()
    p_ref = oracle.forward_2d(g, x)
    assert per_view_rel(p, p_ref) < FP32_TOL
    b = P.back(torch.from_numpy(p_ref).float().cuda()).cpu().numpy()
    assert rel(b, oracle.back_2d(g, p_ref)) < FP32_TOL


@pytest.mark.parametrize("nx,ny,nu,u_off,a,b,batch", [
    (13, 7, 31, 0.37, 1.3, 0.8, 1),     # odd / ragged sizes, shifted detector
    (40, 33, 50, -1.1, 0.6, 0.9, 3),    # ragged batch chunk
    (5, 64, 40, 0.0, 1.0, 1.0, 17),     # two batch chunks, elongated grid
    (1, 1, 1, 0.2, 1.0, 1.0, 2),        # a single pixel and a single element
])
def test_ragged_shapes_fp64(csm, nx, ny, nu, u_off, a, b, batch):
    ang = np.concatenate([synth.uniform_angles(12), [0.0, math.pi / 2, math.pi, -math.pi / 2, 0.7853981633974483]])
    g = synth.geometry(nx, ny, 1, a=a, b=b, n_views=len(ang), angles=ang, s=max(nx * a, ny * b) * 1.5 + 5,
                       sdd=max(nx * a, ny * b) * 2.5 + 9, nu=nu, du=1.1, u_off=u_off)
    rng = np.random.default_rng(nx * 100 + ny)
    x = rng.uniform(size=(batch, ny, nx))
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    for bi in range(batch):
        ref = oracle.forward_2d(g, x[bi])
        assert np.max(np.abs(p[bi] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    y = rng.uniform(size=(batch, len(ang), nu))
    bx = P.back(torch.from_numpy(y).cuda()).cpu().numpy()
    for bi in range(batch):
        ref = oracle.back_2d(g, y[bi])
        assert np.max(np.abs(bx[bi] - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_flags_accumulate_relative(csm):
    g = synth.geometry(20, 20, 1, a=1.5, b=0.5, n_views=9, s=60.0, sdd=100.0, nu=33, du=0.9)
    x = np.random.default_rng(3).uniform(size=(20, 20))
    P = csm.Projector(g)
    xt = torch.from_numpy(x).cuda()
    p_abs = P.forward(xt)
    p_rel = P.forward(xt, flags=2)
    assert torch.allclose(p_abs, p_rel * 0.75, rtol=1e-13, atol=0)
    acc = p_abs.clone()
    P.forward(xt, out=acc, flags=1)
    assert torch.allclose(acc, 2 * p_abs, rtol=1e-13, atol=0)
    b1 = P.back(p_abs)
    b2 = b1.clone()
    P.back(p_abs, out=b2, flags=1)
    assert torch.allclose(b2, 2 * b1, rtol=1e-13, atol=0)


def test_adjoint_fp64_and_fp32(csm):
    g = synth.config("fan2d_64")
    P = csm.Projector(g)
    rng = np.random.default_rng(5)
    for dt, tol in ((torch.float64, 1e-14), (torch.float32, 1e-6)):
        x = torch.from_numpy(rng.normal(size=(64, 64))).to(dt).cuda()
        y = torch.from_numpy(rng.normal(size=(90, 96))).to(dt).cuda()
        lhs = float((P.forward(x).double() * y.double()).sum())
        rhs = float((x.double() * P.back(y).double()).sum())
        assert abs(lhs - rhs) <= tol * (float(P.forward(x).double().norm()) * float(y.double().norm()))


@pytest.mark.parametrize("dt,bound", [(torch.bfloat16, 2 * 2 ** -9 + 1e-5), (torch.float16, 2 * 2 ** -11 + 1e-5)])
def test_half_storage(csm, dt, bound):
    g = synth.config("fan2d_64")
    x = synth.ellipse_phantom(64, 1)
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).to(dt).cuda()).float().cpu().numpy()
    p_ref = oracle.forward_2d(g, x)
    err = per_view_rel(p, p_ref)
    assert err < bound, err
    b = P.back(torch.from_numpy(p_ref).to(dt).cuda()).float().cpu().numpy()
    assert rel(b, oracle.back_2d(g, p_ref)) < bound


def test_nnz_matches_oracle(csm):
    """nnz counts entries above 1e-6 of the pixel area, evaluated in FP32 (error ~1e-7 of
    a pixel): it lies between the oracle's counts above 1.5e-6 and above 0.5e-6."""
    g = synth.config("fan2d_64")
    rows, cols, vals = oracle.coo(g)
    n = csm.Projector(g).nnz()
    assert int(np.sum(vals > 1.5e-6)) <= n <= int(np.sum(vals > 0.5e-6)), (n, len(vals))


def test_fan512_batch16_sampled_views(csm):
    """The 512^2 / 720-view / batch-16 workload in the benchmark's launch configuration:
    forward over all views; 36 evenly spaced views of 4 phantoms against the oracle."""
    g = synth.config("fan2d_512")
    xs = np.stack([synth.ellipse_phantom(512, s) for s in range(16)])
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(xs).float().cuda()).cpu().numpy()
    views = np.arange(0, 720, 20)
    worst = 0.0
    for bi in (0, 5, 10, 15):
        ref = oracle.forward_2d(g, xs[bi], views=views)
        worst = max(worst, per_view_rel(p[bi, views], ref))
    assert worst < FP32_TOL, worst
    # back over the same 36 views: a geometry holding only those angles
    gs = dict(g)
    gs["angles"] = g["angles"][views].copy()
    gs["n_views"] = len(views)
    Ps = csm.Projector(gs)
    ref_p = oracle.forward_2d(g, xs[3], views=views)
    bx = Ps.back(torch.from_numpy(ref_p).float().cuda()).cpu().numpy()
    assert rel(bx, oracle.back_2d(gs, ref_p)) < FP32_TOL


def assert_elementwise(got, want, tol, what=""):
    """Every sample: |got - want| <= tol |want| + 0.1 tol max|want| (relative error per
    element, floored at a tenth of the largest value for elements of almost no weight)."""
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    bound = tol * (np.abs(want) + 0.1 * np.max(np.abs(want)))
    bad = np.abs(got - want) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - want) / bound)) * tol)


def test_fan512_back_all_views_elementwise(csm):
    """The back projection over all 720 views in the benchmark's launch configuration
    (batch 16), pixel by pixel against the oracle, for two batch items; and the forward of
    the whole sinogram element by element on 24 views of one phantom."""
    g = synth.config("fan2d_512")
    rng = np.random.default_rng(21)
    ps = rng.uniform(size=(16, 720, 768))
    P = csm.Projector(g)
    b = P.back(torch.from_numpy(ps).float().cuda()).cpu().numpy()
    for bi in (0, 13):
        assert_elementwise(b[bi], oracle.back_2d(g, ps[bi]), FP32_TOL, "back item %d" % bi)
    xs = np.stack([synth.ellipse_phantom(512, s) for s in range(16)])
    p = P.forward(torch.from_numpy(xs).float().cuda()).cpu().numpy()
    views = np.arange(7, 720, 30)
    ref = oracle.forward_2d(g, xs[9], views=views)
    for i, v in enumerate(views):
        assert_elementwise(p[9, v], ref[i], FP32_TOL, "forward view %d" % v)


def test_batch_invariance(csm):
    """A batch item's projections do not depend on the other items of its batch or on the
    batch size (the 16-, 8-, 2- and 1-item kernels give bit-identical results)."""
    g = synth.config("fan2d_512")
    xs = np.stack([synth.ellipse_phantom(512, s) for s in range(16)]).astype(np.float32)
    P = csm.Projector(g)
    x = torch.from_numpy(xs).cuda()
    p16 = P.forward(x).cpu().numpy()
    for b in (1, 2, 11):
        assert np.array_equal(P.forward(x[:b]).cpu().numpy(), p16[:b]), b
    y = torch.from_numpy(p16[:, :, :]).cuda()
    b16 = P.back(y).cpu().numpy()
    for b in (1, 2, 11):
        assert np.array_equal(P.back(y[:b]).cpu().numpy(), b16[:b]), b


def test_empty_and_zero_inputs(csm):
    """A batch of zero items returns empty outputs without launching; zero inputs give exact
    zeros (2D and 3D, both directions)."""
    g2 = synth.config("fan2d_64")
    g3 = synth.geometry(6, 5, 7, n_views=5, s=14.0, sdd=23.0, nu=14, nv=12, a=1.2, b=0.9, c=1.1)
    g3["dim"] = 3
    for g in (g2, g3):
        P = csm.Projector(g)
        for dt in (torch.float32, torch.float64):
            x0 = torch.zeros((0,) + P.vol_shape, dtype=dt, device="cuda")
            p0 = torch.zeros((0,) + P.sino_shape, dtype=dt, device="cuda")
            assert P.forward(x0).shape == (0,) + P.sino_shape
            assert P.back(p0).shape == (0,) + P.vol_shape
            z = torch.zeros((2,) + P.vol_shape, dtype=dt, device="cuda")
            assert int(torch.count_nonzero(P.forward(z))) == 0
            zp = torch.zeros((2,) + P.sino_shape, dtype=dt, device="cuda")
            assert int(torch.count_nonzero(P.back(zp))) == 0
        torch.cuda.synchronize()

"""Solvers and autograd on the GPU against FP64 references built from the oracle's explicit
sparse W (scipy), and against finite differences."""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import paper_2511_12235_gb300 as csm
    from paper_2511_12235_gb300 import autograd, solvers
    return csm, solvers, autograd


def sparse_W(g, views=None):
    rows, cols, vals = oracle.coo(g, views=views)
    nv = len(g["angles"]) if views is None else len(views)
    m = nv * g["nu"] * g.get("nv", 1)
    n = g["nx"] * g["ny"] * g["nz"]
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, n))


def test_power_norm_matches_sparse(mods):
    csm, solvers, _ = mods
    g = synth.config("fan2d_64")
    W = sparse_W(g)
    P = csm.Projector(g)
    start = np.random.default_rng(0).normal(size=(1, 64, 64))
    sig = solvers.power_norm(P, iters=100, start=torch.from_numpy(start), dtype=torch.float64)
    # the same iteration on the explicit matrix
    b = start.ravel() / np.linalg.norm(start)
    for _ in range(100):
        z = W.T @ (W @ b)
        b = z / np.linalg.norm(z)
    ref = np.linalg.norm(W @ b)
    assert abs(sig - ref) < 1e-10 * ref
    smax = sp.linalg.svds(W, k=1, return_singular_vectors=False)[0]
    assert abs(sig - smax) < 1e-3 * smax


def _cgls_ref(W, b, iters):
    """Plain FP64 CGLS on an explicit matrix: iterates and squared residuals per iteration."""
    x = np.zeros(W.shape[1]); r = b.copy(); s = W.T @ r; d = s.copy(); gam = s @ s
    xs, hist = [x.copy()], [r @ r]
    for _ in range(iters):
        q = W @ d; al = gam / (q @ q); x = x + al * d; r = r - al * q; s = W.T @ r
        gn = s @ s; d = s + (gn / gam) * d; gam = gn
        xs.append(x.copy()); hist.append(r @ r)
    return np.array(xs), np.array(hist)


def test_cgls_matches_fp64_reference(mods):
    """50 CGLS iterations on the 64^2 fan-beam problem against a plain FP64 CGLS on the
    oracle's explicit W.

    CG on these noisy, ill-posed problems amplifies rounding erratically: perturbing W by a
    relative 1e-15 moves the reference's own iterate by up to ~1e-3 at some iterations and
    by ~1e-9 at others, and single residuals by up to a few percent.  So the test measures
    that spread itself (three references with W perturbed by +-1e-15) and compares the GPU
    iterate tightly (1e-6) at every iteration where the reference is insensitive (spread
    below 1e-8); the first nine residuals within 1e-8; the residual never grows; the final
    residual within 5 %."""
    csm, solvers, _ = mods
    g = synth.config("fan2d_64")
    W = sparse_W(g)
    x_true = np.stack([synth.ellipse_phantom(64, s) for s in (0, 1)])
    p = np.stack([(W @ xt.ravel()).reshape(90, 96) for xt in x_true])
    p_noisy = np.stack([synth.poisson_sinogram(pi, seed=i)[0] for i, pi in enumerate(p)])
    P = csm.Projector(g)
    cg = solvers.CGLS(P, 2, dtype=torch.float64)
    iters = 50
    res2 = torch.zeros(iters + 1, 2, dtype=torch.float64, device="cuda")
    cg.start(torch.from_numpy(p_noisy).cuda())
    cg.ops.dot(cg.r, cg.r, res2[0])
    xs_gpu = [cg.x.cpu().numpy().reshape(2, -1)]
    for k in range(iters):
        cg.step(res2[k + 1])
        xs_gpu.append(cg.x.cpu().numpy().reshape(2, -1))
    xs_gpu, res2 = np.stack(xs_gpu), res2.cpu().numpy()
    rng = np.random.default_rng(0)
    coo = W.tocoo()
    for i in range(2):
        b = p_noisy[i].ravel()
        xr, hist = _cgls_ref(W, b, iters)
        spread = np.zeros(iters + 1)
        for _ in range(3):
            Wp = sp.csr_matrix((coo.data * (1 + 1e-15 * rng.choice([-1.0, 1.0], size=coo.nnz)), (coo.row, coo.col)),
                               shape=W.shape)
            xp, _ = _cgls_ref(Wp, b, iters)
            spread = np.maximum(spread, np.linalg.norm(xp - xr, axis=1) / np.maximum(np.linalg.norm(xr, axis=1), 1e-300))
        quiet = [k for k in range(1, iters + 1) if spread[k] < 1e-8]
        assert len(quiet) >= 10, quiet
        for k in quiet:
            d = np.linalg.norm(xs_gpu[k, i] - xr[k]) / np.linalg.norm(xr[k])
            assert d < 1e-6, (i, k, d)
        assert np.max(np.abs(res2[:9, i] - hist[:9]) / hist[:9]) < 1e-8
        assert np.all(np.diff(res2[:, i]) <= 1e-9 * res2[:-1, i])
        assert abs(res2[iters, i] - hist[iters]) <= 0.05 * hist[iters]


def test_cgls_fp32_fan512_sinograms(mods):
    """50 CGLS iterations in FP32 on a batch of noisy 512^2 / 720-view sinograms: the residual
    decreases monotonically and the first iterations agree with FP64."""
    csm, solvers, _ = mods
    g = synth.config("fan2d_512")
    P = csm.Projector(g)
    xs = torch.from_numpy(np.stack([synth.ellipse_phantom(512, s) for s in range(4)])).float().cuda()
    p = P.forward(xs).double().cpu().numpy()
    pn = np.stack([synth.poisson_sinogram(pi, seed=i)[0] for i, pi in enumerate(p)])
    cg = solvers.CGLS(P, 4, dtype=torch.float32)
    x, res2 = cg.run(torch.from_numpy(pn).float().cuda(), iters=50)
    r = res2.cpu().numpy()
    assert np.all(np.diff(r, axis=0) <= 1e-6 * r[:-1])
    cg64 = solvers.CGLS(P, 4, dtype=torch.float64)
    _, r64 = cg64.run(torch.from_numpy(pn).cuda(), iters=5)
    assert np.max(np.abs(r[:6] - r64.cpu().numpy()) / r64.cpu().numpy()) < 1e-4


def test_nag_matches_fp64_reference(mods):
    csm, solvers, _ = mods
    g = synth.config("fan2d_64")
    W = sparse_W(g)
    x_true = synth.ellipse_phantom(64, 3)
    p = (W @ x_true.ravel()).reshape(1, 90, 96)
    P = csm.Projector(g)
    sigma = sp.linalg.svds(W, k=1, return_singular_vectors=False)[0]
    lam = 1e-4
    nag = solvers.NAG(P, 1, lam=lam, sigma=sigma, dtype=torch.float64)
    u = nag.run(torch.from_numpy(p).cuda(), iters=40).cpu().numpy().ravel()
    Wn = W / sigma
    uu = np.zeros(W.shape[1]); y = uu.copy(); t = 1.0; b = p.ravel()
    for _ in range(40):
        grad = Wn.T @ (Wn @ y - b) + lam * y
        un = y - grad / (1 + lam)
        tn = 0.5 * (1 + math.sqrt(1 + 4 * t * t))
        y = un + (t - 1) / tn * (un - uu)
        uu, t = un, tn
    assert np.linalg.norm(u - uu) < 1e-10 * np.linalg.norm(uu)


def test_autograd_gradcheck_and_oracle_WT(mods):
    """16^3 crop of the 128^3 cone-beam geometry, 18 views: gradcheck (finite differences,
    first and second order) and the backward against the oracle's explicit W^T."""
    csm, _, ag = mods
    base = synth.config("cone3d_128")
    views = np.arange(0, 180, 10)
    g = synth.geometry(16, 16, 16, n_views=len(views), angles=base["angles"][views], s=400.0, sdd=800.0,
                       nu=192, nv=192)
    g["dim"] = 3
    P = csm.Projector(g)
    x = torch.randn(1, 16, 16, 16, dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda t: ag.project(t, P)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-7, fast_mode=True)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-6, atol=1e-7, fast_mode=True)
    y = torch.randn(1, len(views), 192, 192, dtype=torch.float64, device="cuda")
    (gx,) = torch.autograd.grad(f(x), x, grad_outputs=y)
    W = sparse_W(g)
    ref = W.T @ y.cpu().numpy().ravel()
    got = gx.cpu().numpy().ravel()
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)

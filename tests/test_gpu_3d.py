"""GPU parity of the 3D cone-beam projectors against the FP64 clipping oracle.

Bar: FP64 within 1e-11 relative (rounding order); FP32 within 1e-5 relative L2 per
projection (view) for the forward and per volume for the back; BF16 storage within
2 * 2^-9 + 1e-5.  Full-size workloads (128^3 and 512^3) are checked on views / detector
elements / voxels the oracle computes one by one, in the launch configuration the benchmark
uses.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


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
    return float(np.max(num[ok] / den[ok]))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


SMALL = dict(a=1.2, b=0.9, c=1.1, s=14.0, sdd=23.0, du=1.3, dv=1.1, u_off=0.2, v_off=-0.35)


def small_geom(nx=6, ny=5, nz=7, nu=14, nv=12, angles=None, **kw):
    if angles is None:
        angles = np.concatenate([synth.uniform_angles(10), [0.0, math.pi / 2, math.pi, 0.25 * math.pi]])
    g = synth.geometry(nx, ny, nz, n_views=len(angles), angles=angles, nu=nu, nv=nv, **dict(SMALL, **kw))
    g["dim"] = 3
    return g


@pytest.mark.parametrize("shape", [(6, 5, 7, 14, 12), (3, 4, 1, 9, 5), (1, 1, 1, 4, 3), (9, 8, 6, 17, 11),
                                   (20, 3, 37, 15, 40)])
def test_small_fp64_forward_back(csm, shape):
    nx, ny, nz, nu, nv = shape
    # the tall grid needs the source farther out (rows per voxel stay within the kernels' bound)
    g = small_geom(nx, ny, nz, nu, nv, **({"s": 60.0, "sdd": 100.0} if nz > 20 else {}))
    rng = np.random.default_rng(sum(shape))
    x = rng.uniform(size=(nz, ny, nx))
    P = csm.Projector(g)
    ref = oracle.forward_3d(g, x)
    p = P.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.max(np.abs(p - ref)) <= 1e-11 * np.max(np.abs(ref)), np.max(np.abs(p - ref))
    y = rng.uniform(size=ref.shape)
    b = P.back(torch.from_numpy(y).cuda()).cpu().numpy()
    bref = oracle.back_3d(g, y)
    assert np.max(np.abs(b - bref)) <= 1e-11 * np.max(np.abs(bref))


def test_small_fp32_and_batch(csm):
    g = small_geom(9, 8, 6, 17, 11)
    rng = np.random.default_rng(4)
    xs = rng.uniform(size=(3, 6, 8, 9))
    P = csm.Projector(g)
    refs = [oracle.forward_3d(g, xs[i]) for i in range(3)]
    p = P.forward(torch.from_numpy(xs).float().cuda()).cpu().numpy()
    for i in range(3):
        assert per_view_rel(p[i], refs[i]) < FP32_TOL
    ys = rng.uniform(size=(3,) + p.shape[1:])
    b = P.back(torch.from_numpy(ys).float().cuda()).cpu().numpy()
    for i in range(3):
        assert rel(b[i], oracle.back_3d(g, ys[i])) < FP32_TOL


def test_row_windows_batch4(csm):
    """A tall detector (200 rows) and a batch of 4: the forward splits the rows into windows
    (96 rows per warp at four batch items); every window and batch item against the oracle."""
    ang = synth.uniform_angles(6)
    g = synth.geometry(8, 8, 40, n_views=6, angles=ang, nu=24, nv=200, s=60.0, sdd=100.0, du=1.0, dv=0.6)
    g["dim"] = 3
    rng = np.random.default_rng(9)
    xs = rng.uniform(size=(4, 40, 8, 8))
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(xs).float().cuda()).cpu().numpy()
    for i in range(4):
        ref = oracle.forward_3d(g, xs[i])
        assert per_view_rel(p[i], ref) < FP32_TOL
        assert np.count_nonzero(ref[:, 96:, :]) > 0          # rows beyond the first window carry weight
    ys = rng.uniform(size=(4,) + p.shape[1:])
    b = P.back(torch.from_numpy(ys).float().cuda()).cpu().numpy()
    for i in range(4):
        assert rel(b[i], oracle.back_3d(g, ys[i])) < FP32_TOL


def test_adjoint_3d(csm):
    ang = synth.uniform_angles(12)
    g = synth.geometry(8, 8, 8, n_views=12, angles=ang, nu=16, nv=14, **dict(SMALL, s=20.0, sdd=33.0))
    g["dim"] = 3
    P = csm.Projector(g)
    rng = np.random.default_rng(6)
    for dt, tol in ((torch.float64, 1e-14), (torch.float32, 2e-6)):
        x = torch.from_numpy(rng.normal(size=(8, 8, 8))).to(dt).cuda()
        y = torch.from_numpy(rng.normal(size=(12, 14, 16))).to(dt).cuda()
        px = P.forward(x).double()
        lhs = float((px * y.double()).sum())
        rhs = float((x.double() * P.back(y).double()).sum())
        assert abs(lhs - rhs) <= tol * float(px.norm()) * float(y.double().norm())


def test_nnz_3d(csm):
    """nnz counts entries above 1e-6 of the voxel volume, evaluated in FP32."""
    g = small_geom(6, 5, 7, 14, 12)
    rows, cols, vals = oracle.coo(g)
    vol = g["a"] * g["b"] * g["c"]
    n = csm.Projector(g).nnz()
    assert int(np.sum(vals > 1.5e-6 * vol)) <= n <= int(np.sum(vals > 0.5e-6 * vol)), (n, len(vals))


def test_cone128_views_and_crop(csm):
    """128^3 / 180 views / 192^2: forward on 3 views (all rows) and back over those views."""
    g = synth.config("cone3d_128")
    x = synth.ellipsoid_phantom(128, 0)
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).float().cuda()).cpu().numpy()
    views = [0, 37, 113]
    ref = oracle.forward_3d(g, x, views=views)
    assert per_view_rel(p[views], ref) < FP32_TOL
    gs = dict(g)
    gs["angles"] = g["angles"][views].copy()
    gs["n_views"] = len(views)
    b = csm.Projector(gs).back(torch.from_numpy(ref).float().cuda()).cpu().numpy()
    # sampled voxels (the oracle's full back over 128^3 is slow): 300 random voxels
    rng = np.random.default_rng(0)
    idx = rng.integers(0, 128, size=(300, 3))
    got = np.array([b[iz, iy, ix] for ix, iy, iz in idx])
    want = np.array([oracle.back_voxel_3d(gs, ref, ix, iy, iz) for ix, iy, iz in idx])
    assert rel(got, want) < FP32_TOL


def test_cone512_sampled_fp32_and_bf16(csm):
    """512^3 / 360 views / 768^2 in the launch configuration of a full projection: sampled
    detector elements and voxels against the oracle; BF16 storage error stated."""
    g = synth.config("cone3d_512")
    x = synth.ellipsoid_phantom(512, 0, dtype=np.float32)
    P = csm.Projector(g)
    xt = torch.from_numpy(x).cuda()
    p = P.forward(xt)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    samples = [(int(v), int(k), int(l)) for v, k, l in zip(rng.integers(0, 360, 24), rng.integers(64, 704, 24),
                                                         rng.integers(64, 704, 24))]
    samples += [(0, 384, 384), (90, 300, 760), (180, 767, 400), (45, 10, 5)]
    x64 = x.astype(np.float64)
    got = np.array([float(p[v, l, k]) for v, k, l in samples])
    want = np.array([oracle.forward_element_3d(g, x64, v, k, l) for v, k, l in samples])
    err = rel(got, want)
    assert err < FP32_TOL, err
    # BF16 storage of volume and sinogram, FP32 accumulation
    pb = P.forward(xt.to(torch.bfloat16))
    got_b = np.array([float(pb[v, l, k]) for v, k, l in samples])
    assert rel(got_b, want) < 2 * 2 ** -9 + 1e-5
    # back projection of the computed sinogram, sampled voxels
    bx = P.back(p)
    vox = [(int(a), int(b_), int(c)) for a, b_, c in rng.integers(100, 412, size=(6, 3))]
    pn = p.double().cpu().numpy()
    got = np.array([float(bx[iz, iy, ix]) for ix, iy, iz in vox])
    want = np.array([oracle.back_voxel_3d(g, pn, ix, iy, iz) for ix, iy, iz in vox])
    assert rel(got, want) < FP32_TOL


def test_batch_invariance_3d(csm):
    """A batch item's projections do not depend on its batch mates: the back projection is
    bit-identical for batch sizes 1, 2 and 3 (fixed summation order); the forward, which adds
    a row's entries with shared-memory atomics, agrees to FP32 rounding."""
    g = small_geom(9, 8, 6, 17, 11)
    rng = np.random.default_rng(12)
    xs = torch.from_numpy(rng.uniform(size=(3, 6, 8, 9))).float().cuda()
    P = csm.Projector(g)
    p3 = P.forward(xs).cpu().numpy()
    for b in (1, 2):
        assert rel(P.forward(xs[:b]).cpu().numpy(), p3[:b]) < 1e-6
    y = torch.from_numpy(p3).cuda()
    b3 = P.back(y).cpu().numpy()
    for b in (1, 2):
        assert np.array_equal(P.back(y[:b]).cpu().numpy(), b3[:b]), b

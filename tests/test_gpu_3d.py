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
    (128 rows per warp at four batch items); every window and batch item against the oracle."""
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
        assert np.count_nonzero(ref[:, 128:, :]) > 0         # rows beyond the first window carry weight
    ys = rng.uniform(size=(4,) + p.shape[1:])
    b = P.back(torch.from_numpy(ys).float().cuda()).cpu().numpy()
    for i in range(4):
        assert rel(b[i], oracle.back_3d(g, ys[i])) < FP32_TOL


def test_sparse_columns_fp64(csm):
    """The forward skips the columns without a nonzero voxel and limits the planes of the
    others to their range of nonzero voxels: one nonzero voxel, a zero volume, two nonzero
    voxels at the ends of one column (zeros between them), and a batch whose items are nonzero
    in different columns, in FP64 against the oracle (a zero volume projects to exact zeros)."""
    g = small_geom(9, 8, 6, 17, 11)
    P = csm.Projector(g)
    one = np.zeros((6, 8, 9))
    one[3, 4, 5] = 1.0
    ends = np.zeros((6, 8, 9))
    ends[0, 2, 2], ends[5, 2, 2] = 0.7, 1.3
    for x in (one, ends):
        ref = oracle.forward_3d(g, x)
        p = P.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.count_nonzero(ref) > 0
        assert np.max(np.abs(p - ref)) <= 1e-11 * np.max(np.abs(ref))
    p0 = P.forward(torch.zeros((6, 8, 9), dtype=torch.float64, device="cuda")).cpu().numpy()
    assert not np.any(p0)
    xs = np.zeros((2, 6, 8, 9))
    xs[0, 1, 3, 4] = 1.0
    xs[1, 4, 6, 7] = 2.0
    p = P.forward(torch.from_numpy(xs).cuda()).cpu().numpy()
    for i in range(2):
        ref = oracle.forward_3d(g, xs[i])
        assert np.max(np.abs(p[i] - ref)) <= 1e-11 * np.max(np.abs(ref))


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


def assert_elementwise(got, want, tol, what=""):
    """Every sample: |got - want| <= tol |want| + 0.1 tol max|want| (relative error per
    element, floored at a tenth of the largest value for elements of almost no weight)."""
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    bound = tol * (np.abs(want) + 0.1 * np.max(np.abs(want)))
    bad = np.abs(got - want) > bound
    assert not bad.any(), (what, int(bad.sum()), float(np.max(np.abs(got - want) / bound)) * tol)


def _elements_512(n, seed):
    """Detector elements of the 512^3 workload: every row from the bottom to the top edge (so
    every row window of the forward), columns over the detector's middle two thirds, random
    views, plus the centre and the views along the axes."""
    rng = np.random.default_rng(seed)
    rows = (np.arange(n) * 767) // (n - 1)
    cols = rng.integers(128, 640, n)
    views = rng.integers(0, 360, n)
    els = [(int(v), int(k), int(l)) for v, k, l in zip(views, cols, rows)]
    els += [(0, 384, 384), (90, 383, 384), (180, 384, 383), (270, 300, 500), (45, 600, 200)]
    return els


@pytest.fixture(scope="module")
def cone512(csm):
    g = synth.config("cone3d_512")
    x = synth.ellipsoid_phantom(512, 0, dtype=np.float32, slab=8, workers=8)
    P = csm.Projector(g)
    yield g, x, P
    P.close()


def test_cone512_forward_elementwise_fp32_bf16(cone512):
    """512^3 / 360 views / 768^2 in the benchmark's launch configuration: 205 detector
    elements spanning every row (every row window) against the oracle one by one, for FP32
    and for BF16 storage of volume and sinogram (bound 2 * 2^-9 + 1e-5: one rounding of the
    input and one of the output)."""
    g, x, P = cone512
    xt = torch.from_numpy(x).cuda()
    p = P.forward(xt)
    pb = P.forward(xt.to(torch.bfloat16))
    torch.cuda.synchronize()
    els = _elements_512(200, 1)
    x64 = x.astype(np.float64)
    want = np.array([oracle.forward_element_3d(g, x64, v, k, l) for v, k, l in els])
    assert np.count_nonzero(want) > 150
    got = np.array([float(p[v, l, k]) for v, k, l in els])
    assert_elementwise(got, want, FP32_TOL, "fp32 forward")
    got_b = np.array([float(pb[v, l, k]) for v, k, l in els])
    assert_elementwise(got_b, want, 2 * 2 ** -9 + 1e-5, "bf16 forward")


def test_cone512_back_elementwise_window_edges(cone512):
    """The back projection of a seeded sinogram over all 360 views: 208 voxels against the
    oracle one by one, on the z-window boundaries (iz = 0, 127/128, 255/256, 383/384, 511)
    and at random places; the oracle and the kernel read the same seeded input."""
    g, x, P = cone512
    rng = np.random.default_rng(5)
    ps = rng.random((360, 768, 768), dtype=np.float32)
    b = P.back(torch.from_numpy(ps).cuda())
    torch.cuda.synchronize()
    zs = [0, 1, 127, 128, 255, 256, 383, 384, 510, 511]
    vox = [(int(ix), int(iy), z) for z in zs for ix, iy in rng.integers(40, 472, size=(16, 2))]
    vox += [(int(a), int(b_), int(c)) for a, b_, c in rng.integers(0, 512, size=(48, 3))]
    p64 = ps.astype(np.float64)
    want = np.array([oracle.back_voxel_3d(g, p64, ix, iy, iz) for ix, iy, iz in vox])
    got = np.array([float(b[iz, iy, ix]) for ix, iy, iz in vox])
    assert np.count_nonzero(want) > 150
    assert_elementwise(got, want, FP32_TOL, "fp32 back")


def test_cone128_f16_storage(csm):
    """F16 storage of volume and sinogram in 3D (FP32 arithmetic): forward on three full views
    and back on sampled voxels within 2 * 2^-11 + 1e-5 of the oracle."""
    g = synth.config("cone3d_128")
    x = synth.ellipsoid_phantom(128, 3)
    P = csm.Projector(g)
    p = P.forward(torch.from_numpy(x).half().cuda()).float().cpu().numpy()
    views = [5, 50, 140]
    ref = oracle.forward_3d(g, x, views=views)
    bound = 2 * 2 ** -11 + 1e-5
    assert per_view_rel(p[views], ref) < bound
    rng = np.random.default_rng(8)
    y = rng.uniform(size=(180, 192, 192))
    b = P.back(torch.from_numpy(y).half().cuda()).float().cpu().numpy()
    vox = [tuple(int(t) for t in r) for r in rng.integers(10, 118, size=(40, 3))]
    want = np.array([oracle.back_voxel_3d(g, y, ix, iy, iz) for ix, iy, iz in vox])
    got = np.array([b[iz, iy, ix] for ix, iy, iz in vox])
    assert_elementwise(got, want, bound, "f16 back")


def test_back_half_storage_view_groups(csm):
    """Back projection into BF16 / F16 x with the workspace that holds an FP32 copy of x (op 3):
    the view groups add their sums into that copy in the same order as the FP32 path adds them
    into an FP32 x, and x is rounded once, so the result is the FP32 result rounded to BF16 /
    F16 bit for bit (also with CSM_ACCUMULATE).  With op 1's workspace the back projection
    runs in one launch over all views: within one rounding step of the same values."""
    from paper_2511_12235_gb300 import _capi as capi
    g = synth.config("cone3d_128")
    P = csm.Projector(g)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    y = torch.rand((1,) + tuple(P.sino_shape), generator=gen, device="cuda")
    b32 = P.back(y)
    for dt in (torch.bfloat16, torch.float16):
        bh = P.back(y, out_dtype=dt)
        assert torch.equal(bh, b32.to(dt))
        x0 = torch.rand(b32.shape, generator=gen, device="cuda").to(dt)
        acc = P.back(y, out=x0.clone(), flags=capi.CSM_ACCUMULATE)
        assert torch.equal(acc, (x0.float() + b32).to(dt))
        n1 = capi.csm_workspace_bytes(P.handle, 1, 1, capi.CSM_F32)     # no room for the copy of x
        ws1 = torch.empty(n1, dtype=torch.uint8, device="cuda")
        one = torch.empty(b32.shape, dtype=dt, device="cuda")
        capi.csm_back(P.handle, y.data_ptr(), one.data_ptr(), 1, capi.CSM_F32,
                      capi.CSM_BF16 if dt == torch.bfloat16 else capi.CSM_F16, 0, ws1.data_ptr(), n1,
                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        step = 2.0 ** -7 if dt == torch.bfloat16 else 2.0 ** -10       # one rounding step, relative
        diff = (one.float() - bh.float()).abs()
        assert bool((diff <= step * b32.abs() + 1e-30).all())
        assert bool((diff > 0).any())       # the single launch sums in another order
    P.close()


def test_back_half_storage_batches(csm):
    """The FP32 / FP64 copy of x with chunks of batch items: a batch of 3 (chunks of 2 and 1)
    into BF16 x equals the FP32 batch rounded to BF16, and FP32 x under FP64 arithmetic (FP64
    projections) equals the FP64 result rounded to FP32."""
    g = small_geom(9, 8, 6, 17, 11)
    P = csm.Projector(g)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)
    y = torch.rand((3,) + tuple(P.sino_shape), generator=gen, device="cuda")
    b32 = P.back(y)
    assert torch.equal(P.back(y, out_dtype=torch.bfloat16), b32.to(torch.bfloat16))
    y64 = y.double()
    b64 = P.back(y64)
    assert torch.equal(P.back(y64, out_dtype=torch.float32), b64.float())
    P.close()


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

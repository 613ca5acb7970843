"""The explicit sparse W (csm_export_csr) against the oracle's COO export, its CSR products
against the matrix-free projectors, and SART on it against a plain FP64 SART on the oracle's
matrix.

Bar: FP64 values within 1e-12 relative of the oracle's (rounding order of the closed forms);
FP32 within 1e-5 of max(|w|, a tenth of the voxel measure); the stored pattern equals the
oracle's entries above the storage threshold (1e-12 / 1e-6 of the voxel measure), entries
of the oracle near the threshold being allowed either way.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import paper_2511_12235_gb300 as csm
    from paper_2511_12235_gb300 import sparse
    return csm, sparse


def _geom2d():
    return synth.config("fan2d_64")


def _geom3d():
    ang = np.concatenate([synth.uniform_angles(6), [0.0, math.pi / 2]])
    g = synth.geometry(6, 5, 7, a=1.2, b=0.9, c=1.1, n_views=len(ang), angles=ang, s=14.0, sdd=23.0, nu=14, nv=12,
                       du=1.3, dv=1.1, u_off=0.2, v_off=-0.35)
    g["dim"] = 3
    return g


def _dense_from_csr(C):
    rp = C.row_ptr.cpu().numpy()
    col = C.col.cpu().numpy()
    val = C.val.double().cpu().numpy()
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(val)
    for r in range(len(rp) - 1):                       # columns sorted within every row
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)
    return sp.csr_matrix((val, col, rp), shape=(len(rp) - 1, C.n_cols))


def _at(M, r, c):
    return np.asarray(M[r, c]).ravel() if len(r) else np.zeros(0)


def _compare_with_oracle(g, C, thr, tol, meas):
    rows, cols, vals = oracle.coo(g)
    ref = sp.csr_matrix((vals, (rows, cols)), shape=(C.n_rows, C.n_cols))
    got = _dense_from_csr(C)
    # pattern: every oracle entry clearly above the threshold is stored, every stored entry is
    # clearly nonzero for the oracle
    big = vals > 2 * thr
    assert np.all(_at(got, rows[big], cols[big]) != 0)
    gc = got.tocoo()
    assert np.all(_at(ref, gc.row, gc.col) > 0.5 * thr)
    # values
    want = _at(ref, gc.row, gc.col)
    scale = np.maximum(np.abs(want), 0.1 * meas)
    assert np.all(np.abs(gc.data - want) <= tol * scale), np.max(np.abs(gc.data - want) / scale)


@pytest.mark.parametrize("dim", [2, 3])
def test_export_matches_oracle_fp64_and_fp32(m, dim):
    csm, sparse = m
    g = _geom2d() if dim == 2 else _geom3d()
    P = csm.Projector(g)
    meas = g["a"] * g["b"] * (g["c"] if dim == 3 else 1.0)
    W64 = sparse.export(P, dtype=torch.float64)
    _compare_with_oracle(g, W64, 1e-12 * meas, 1e-11, meas)
    W32 = sparse.export(P, dtype=torch.float32)
    _compare_with_oracle(g, W32, 1e-6 * meas, 1e-5, meas)
    # the CSR of W^T is the transpose of the CSR of W, entry for entry
    WT64 = sparse.export(P, transpose=True, dtype=torch.float64)
    a = _dense_from_csr(W64).T.tocsr()
    b = _dense_from_csr(WT64)
    assert (a != b).count_nonzero() == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_csr_products_equal_projectors(m, dim):
    csm, sparse = m
    g = _geom2d() if dim == 2 else _geom3d()
    P = csm.Projector(g)
    S = sparse.SparseW(P)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.uniform(size=P.vol_shape)).cuda()
    p = torch.from_numpy(rng.uniform(size=P.sino_shape)).cuda()
    fx = P.forward(x).reshape(-1)
    bp = P.back(p).reshape(-1)
    assert torch.allclose(S.matvec(x), fx, rtol=1e-11, atol=1e-11 * float(fx.abs().max()))
    assert torch.allclose(S.rmatvec(p), bp, rtol=1e-11, atol=1e-11 * float(bp.abs().max()))


def test_sart_fan64_against_plain_sart(m):
    """SART on the 64^2 / 90-view workload from noisy projections: the residual decreases at
    every iteration, and the iterates equal a plain FP64 SART on the oracle's COO matrix."""
    csm, sparse = m
    g = _geom2d()
    P = csm.Projector(g)
    S = sparse.SparseW(P)
    x_true = synth.ellipse_phantom(64, 0)
    p_clean = oracle.forward_2d(g, x_true)
    p_noisy, _ = synth.poisson_sinogram(p_clean, seed=0)
    iters = 15
    x, hist = sparse.sart(S, torch.from_numpy(p_noisy).cuda(), iters, lam=1.0)
    assert all(b < a for a, b in zip(hist, hist[1:])), hist
    rows, cols, vals = oracle.coo(g)
    W = sp.csr_matrix((vals, (rows, cols)), shape=(g["n_views"] * g["nu"], 64 * 64))
    R = np.asarray(W.sum(axis=1)).ravel()
    Cs = np.asarray(W.sum(axis=0)).ravel()
    Rinv = np.where(R > 0, 1.0 / np.where(R > 0, R, 1), 0.0)
    Cinv = np.where(Cs > 0, 1.0 / np.where(Cs > 0, Cs, 1), 0.0)
    xr = np.zeros(64 * 64)
    pv = p_noisy.ravel()
    for _ in range(iters):
        xr = xr + Cinv * (W.T @ (Rinv * (pv - W @ xr)))
    got = x.cpu().numpy().ravel()
    assert np.max(np.abs(got - xr)) <= 1e-9 * np.max(np.abs(xr))
    err0 = np.linalg.norm(x_true.ravel())
    assert np.linalg.norm(got - x_true.ravel()) < 0.5 * err0

"""Pins of the oracle's explicit-matrix and counting functions (coo, count_2d, back_slab_3d).

The sparse matrix the oracle exports must be the operator its projections apply: assembled
from ``coo()``, W x equals ``forward_2d/3d`` and W^T p equals ``back_2d/3d`` element by
element (these are pinned on their own by the sweep integrators, Monte Carlo, the paper's
atoms and the invariants in test_oracle_2d.py / test_oracle_3d.py), so a wrong row or column
index in the export (e.g. a transposed (k, l) or a dropped view offset) fails here.  The
counts that the benchmark divides by equal the number of exported entries.
"""
import math

import numpy as np
import pytest

import oracle
import synth

sp = pytest.importorskip("scipy.sparse")


def _geom2d():
    ang = np.concatenate([synth.uniform_angles(7), [0.0, math.pi / 2, 0.3]])
    return synth.geometry(11, 9, 1, a=1.1, b=0.8, n_views=len(ang), angles=ang, s=30.0, sdd=52.0, nu=21,
                          du=0.9, u_off=0.35)


def _geom3d():
    ang = np.concatenate([synth.uniform_angles(5), [0.0, math.pi / 2, 0.7]])
    g = synth.geometry(6, 5, 7, a=1.2, b=0.9, c=1.1, n_views=len(ang), angles=ang, s=14.0, sdd=23.0, nu=14, nv=12,
                       du=1.3, dv=1.1, u_off=0.2, v_off=-0.35)
    g["dim"] = 3
    return g


def _matrix(g, views=None):
    rows, cols, vals = oracle.coo(g, views=views)
    nsel = g["n_views"] if views is None else len(views)
    nrow = nsel * g["nu"] * g["nv"]
    ncol = g["nx"] * g["ny"] * g["nz"]
    assert rows.min() >= 0 and rows.max() < nrow and cols.min() >= 0 and cols.max() < ncol
    assert np.all(vals > 0)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nrow, ncol)), len(vals)


def _close(a, b, rtol=1e-13):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    assert np.all(np.abs(a - b) <= rtol * (np.abs(b) + np.max(np.abs(b)) * 1e-3)), np.max(np.abs(a - b))


def test_coo_2d_is_the_operator_of_forward_and_back():
    g = _geom2d()
    rng = np.random.default_rng(3)
    x = rng.uniform(size=(g["ny"], g["nx"]))
    W, n = _matrix(g)
    _close(W @ x.ravel(), oracle.forward_2d(g, x))
    p = rng.uniform(size=(g["n_views"], g["nu"]))
    _close(W.T @ p.ravel(), oracle.back_2d(g, p))
    # no duplicate (row, column) pairs: every entry is one intersection
    rows, cols, _ = oracle.coo(g)
    assert len(set(zip(rows.tolist(), cols.tolist()))) == n


def test_coo_2d_view_subset_rows_follow_the_selection():
    g = _geom2d()
    views = [8, 2, 5]
    x = np.random.default_rng(4).uniform(size=(g["ny"], g["nx"]))
    W, _ = _matrix(g, views)
    _close(W @ x.ravel(), oracle.forward_2d(g, x, views=views))


def test_coo_3d_is_the_operator_of_forward_and_back():
    g = _geom3d()
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(g["nz"], g["ny"], g["nx"]))
    W, n = _matrix(g)
    _close(W @ x.ravel(), oracle.forward_3d(g, x))
    p = rng.uniform(size=(g["n_views"], g["nv"], g["nu"]))
    _close(W.T @ p.ravel(), oracle.back_3d(g, p))
    rows, cols, _ = oracle.coo(g)
    assert len(set(zip(rows.tolist(), cols.tolist()))) == n


def test_coo_3d_row_index_is_view_row_column():
    """Row index (v * nv + l) * nu + k: the entries of row (v, l, k) are the voxels that
    forward_element_3d sums for that element."""
    g = _geom3d()
    x = np.random.default_rng(6).uniform(size=(g["nz"], g["ny"], g["nx"]))
    W, _ = _matrix(g)
    Wx = W @ x.ravel()
    for v, k, l in [(0, 3, 2), (6, 7, 9), (2, 10, 5), (5, 0, 11)]:
        r = (v * g["nv"] + l) * g["nu"] + k
        want = oracle.forward_element_3d(g, x, v, k, l)
        assert abs(Wx[r] - want) <= 1e-13 * max(abs(want), 1.0)


def test_count_2d_equals_the_exported_entries():
    g = _geom2d()
    _, n = _matrix(g)
    assert oracle.count_2d(g) == n
    views = [1, 4, 9]
    _, n_sel = _matrix(g, views)
    assert oracle.count_2d(g, views=views) == n_sel
    per_pixel = sum(len(oracle.entries_2d(g, v, ix, iy)[0]) for v in views
                    for iy in range(g["ny"]) for ix in range(g["nx"]))
    assert per_pixel == n_sel


def test_back_slab_3d_is_a_slice_of_back_and_counts_its_entries():
    g = _geom3d()
    p = np.random.default_rng(7).uniform(size=(3, g["nv"], g["nu"]))
    views = [0, 4, 6]
    full = oracle.back_3d(g, p, views=views)
    rows, cols, _ = oracle.coo(g, views=views)
    nvx = g["nx"] * g["ny"]
    for iz0, iz1 in [(0, g["nz"]), (2, 5), (6, 7), (3, 3)]:
        xs, n = oracle.back_slab_3d(g, p, iz0, iz1, views=views)
        assert np.array_equal(xs, full[iz0:iz1])
        assert n == int(np.sum((cols >= iz0 * nvx) & (cols < iz1 * nvx)))

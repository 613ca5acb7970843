"""Pins of the oracle's line-based comparator projections (Siddon, Joseph, multi-line mean).

Siddon's value is the line integral of the piecewise-constant image: for the constant image
it is the length of the ray inside the grid box (one slab intersection, computed here on its
own), and for any image it is the limit of fine sampling along the ray.  Joseph's
interpolation is linear between voxel centres across the ray, so for an image linear in that
direction its per-slice midpoint sum is the exact integral of the linear function.  The mean
over several lines per element equals the single-line values of the subdivided detector.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _g2d(views=None, nu=21, du=1.3, u_off=0.2):
    ang = np.asarray(views if views is not None else [0.0, 0.4, 1.3, math.pi / 2, 2.5, 4.0])
    return synth.geometry(12, 9, 1, a=1.1, b=0.8, n_views=len(ang), angles=ang, s=40.0, sdd=70.0, nu=nu, du=du,
                          u_off=u_off)


def _g3d(nu=9, nv=8, du=1.4, dv=1.2, u_off=0.3, v_off=-0.2, views=None):
    ang = np.asarray(views if views is not None else [0.0, 0.7, math.pi / 2, 3.9])
    g = synth.geometry(6, 5, 7, a=1.2, b=0.9, c=1.1, n_views=len(ang), angles=ang, s=25.0, sdd=40.0, nu=nu, nv=nv,
                       du=du, dv=dv, u_off=u_off, v_off=v_off)
    g["dim"] = 3
    return g


def _rays(g, view, k, l=0):
    c, s = math.cos(g["angles"][view]), math.sin(g["angles"][view])
    u = (k + 0.5 - 0.5 * g["nu"]) * g["du"] + g["u_off"]
    w = (l + 0.5 - 0.5 * g["nv"]) * g["dv"] + g["v_off"] if g.get("dim", 2) == 3 else 0.0
    S = np.array([g["s"] * c, g["s"] * s, 0.0])
    d = np.array([-g["sdd"] * c - u * s, -g["sdd"] * s + u * c, w])
    return S, d


def _box(g):
    lo = np.array([-0.5 * g["nx"] * g["a"], -0.5 * g["ny"] * g["b"], -0.5 * g["nz"] * g["c"]])
    return lo, -lo


def _chord(g, S, d, dims):
    lo, hi = _box(g)
    t0, t1 = 0.0, 1.0
    for a in range(dims):
        if d[a] == 0:
            if not lo[a] <= S[a] <= hi[a]:
                return 0.0
            continue
        ta, tb = sorted(((lo[a] - S[a]) / d[a], (hi[a] - S[a]) / d[a]))
        t0, t1 = max(t0, ta), min(t1, tb)
    return max(t1 - t0, 0.0) * float(np.linalg.norm(d[:dims]))


@pytest.mark.parametrize("dim", [2, 3])
def test_siddon_constant_image_is_the_chord_length(dim):
    g = _g2d() if dim == 2 else _g3d()
    shape = (g["ny"], g["nx"]) if dim == 2 else (g["nz"], g["ny"], g["nx"])
    p = oracle.line_forward(g, np.ones(shape), "siddon")
    for v in range(g["n_views"]):
        for l in range(g["nv"] if dim == 3 else 1):
            for k in range(g["nu"]):
                S, d = _rays(g, v, k, l)
                want = _chord(g, S, d, dim)
                got = p[v, l, k] if dim == 3 else p[v, k]
                assert abs(got - want) <= 1e-12 * max(want, 1.0), (v, l, k, got, want)


@pytest.mark.parametrize("dim", [2, 3])
def test_siddon_is_the_limit_of_fine_sampling(dim):
    g = _g2d() if dim == 2 else _g3d()
    rng = np.random.default_rng(7)
    shape = (g["ny"], g["nx"]) if dim == 2 else (g["nz"], g["ny"], g["nx"])
    x = rng.uniform(size=shape)
    p = oracle.line_forward(g, x, "siddon")
    lo, hi = _box(g)
    h = np.array([g["a"], g["b"], g["c"]])
    n = np.array([g["nx"], g["ny"], g["nz"]])
    N = 400000
    t = (np.arange(N) + 0.5) / N
    for v, k, l in [(0, 10, 3), (1, 4, 0), (3, 15, 5), (5, 7, 2)]:
        if dim == 2:
            l = 0
        if k >= g["nu"] or v >= g["n_views"]:
            continue
        S, d = _rays(g, v, k, l)
        P = S[None, :] + t[:, None] * d[None, :]
        idx = np.floor((P - lo) / h).astype(int)
        inside = np.all((idx[:, :dim] >= 0) & (idx[:, :dim] < n[:dim]), axis=1)
        vals = np.zeros(N)
        if dim == 2:
            vals[inside] = x[idx[inside, 1], idx[inside, 0]]
        else:
            vals[inside] = x[idx[inside, 2], idx[inside, 1], idx[inside, 0]]
        want = vals.mean() * np.linalg.norm(d[:dim])
        got = p[v, l, k] if dim == 3 else p[v, k]
        assert abs(got - want) <= 2e-4 * max(abs(want), 1.0), (v, k, got, want)


def test_joseph_is_exact_for_images_linear_across_the_ray():
    """View 0 (source on the +x axis): rays step along x; with x(i, j) = alpha + beta y_j the
    interpolated value is exact wherever the ray stays between the outer pixel centres, and the
    per-column midpoint sum equals the integral of the linear function over the grid's x-range."""
    g = _g2d(views=[0.0, math.pi, 0.05])
    alpha, beta = 0.7, -0.3
    yc = (np.arange(g["ny"]) + 0.5 - 0.5 * g["ny"]) * g["b"]
    x = np.tile((alpha + beta * yc)[:, None], (1, g["nx"]))
    p = oracle.line_forward(g, x, "joseph")
    X0, X1 = -0.5 * g["nx"] * g["a"], 0.5 * g["nx"] * g["a"]
    checked = 0
    for v in range(g["n_views"]):
        for k in range(g["nu"]):
            S, d = _rays(g, v, k)
            ys = [S[1] + (X - S[0]) / d[0] * d[1] for X in (X0, X1)]
            if not all(yc[0] <= y <= yc[-1] for y in ys):
                continue
            # integral over X in [X0, X1] of (alpha + beta y(X)) ds, ds = |d| / |d_x| dX
            ym = 0.5 * (ys[0] + ys[1])
            want = (alpha + beta * ym) * (X1 - X0) * np.linalg.norm(d[:2]) / abs(d[0])
            assert abs(p[v, k] - want) <= 1e-12 * abs(want), (v, k, p[v, k], want)
            checked += 1
    assert checked >= 10


@pytest.mark.parametrize("model", ["siddon", "joseph"])
@pytest.mark.parametrize("dim", [2, 3])
def test_multi_line_mean_equals_the_subdivided_detector(model, dim):
    L = 3
    if dim == 2:
        g = _g2d()
        fine = _g2d(nu=g["nu"] * L, du=g["du"] / L, u_off=g["u_off"])
    else:
        g = _g3d()
        fine = _g3d(nu=g["nu"] * L, nv=g["nv"] * L, du=g["du"] / L, dv=g["dv"] / L)
    rng = np.random.default_rng(11)
    shape = (g["ny"], g["nx"]) if dim == 2 else (g["nz"], g["ny"], g["nx"])
    x = rng.uniform(size=shape)
    p = oracle.line_forward(g, x, model, lines=L)
    pf = oracle.line_forward(fine, x, model, lines=1)
    if dim == 2:
        want = pf.reshape(g["n_views"], g["nu"], L).mean(axis=2)
    else:
        want = pf.reshape(g["n_views"], g["nv"], L, g["nu"], L).mean(axis=(2, 4))
    assert np.allclose(p, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("model", ["siddon", "joseph"])
@pytest.mark.parametrize("dim", [2, 3])
def test_line_back_is_the_adjoint(model, dim):
    g = _g2d() if dim == 2 else _g3d()
    rng = np.random.default_rng(5)
    shape = (g["ny"], g["nx"]) if dim == 2 else (g["nz"], g["ny"], g["nx"])
    x = rng.normal(size=shape)
    p = oracle.line_forward(g, x, model, lines=2)
    y = rng.normal(size=p.shape)
    b = oracle.line_back(g, y, model, lines=2)
    assert abs(float(np.sum(p * y)) - float(np.sum(x * b))) <= 1e-12 * np.linalg.norm(p) * np.linalg.norm(y)

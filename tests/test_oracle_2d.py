"""Pins of the 2D oracle against things other than itself.

* every entry of the 64x64 workload against an independent exact x/y-sweep integrator;
* Monte Carlo with the detector hit computed from the paper's ray parametrisation
  (Eq. (z rotation)) by a linear solve;
* the paper's triangle / trapezoid atoms (Sections 'Triangle', 'Trapezoid') and the worked
  composition Eq. (2d procedure) on configurations where they apply;
* invariants: partition of the fan, closed-form fan area through the grid, similarity
  scaling, mirror symmetry, adjointness of the oracle's forward and back.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import paper_formulas as pf
from tests import sweep


def _corner_u(g, k):
    return (k - g["nu"] / 2.0) * g["du"] + g["u_off"]


def _grid(g, i, axis):
    n, h = (g["nx"], g["a"]) if axis == 0 else (g["ny"], g["b"])
    return (i - n / 2.0) * h


# ----------------------------------------------------------------------------------------
def test_every_entry_of_64_grid_matches_sweep():
    """P2: the full W of the 64x64 / 90-view workload against the exact sweep (every entry,
    and no entry missing: every element whose sweep area is positive is reported)."""
    g = synth.config("fan2d_64")
    rng = np.random.default_rng(0)
    worst = 0.0
    n_checked = 0
    for v in range(g["n_views"]):
        phi = g["angles"][v]
        pix = [(ix, iy) for ix in range(g["nx"]) for iy in range(g["ny"])]
        # all pixels on a few views, a random subset on the rest
        if v % 15 != 0:
            pix = [pix[i] for i in rng.choice(len(pix), 120, replace=False)]
        for ix, iy in pix:
            ks, ws = oracle.entries_2d(g, v, ix, iy)
            got = dict(zip(ks.tolist(), ws.tolist()))
            x0, x1 = _grid(g, ix, 0), _grid(g, ix + 1, 0)
            y0, y1 = _grid(g, iy, 1), _grid(g, iy + 1, 1)
            us = [pf.gamma(phi, g["s"], X, Y) for X in (x0, x1) for Y in (y0, y1)]
            umin = math.tan(min(us)) * g["sdd"]
            umax = math.tan(max(us)) * g["sdd"]
            k0 = max(0, int(math.floor((umin - _corner_u(g, 0)) / g["du"])) - 1)
            k1 = min(g["nu"] - 1, int(math.floor((umax - _corner_u(g, 0)) / g["du"])) + 1)
            for k in range(k0, k1 + 1):
                ref = sweep.element_area_sweep_any(phi, g["s"], g["sdd"], _corner_u(g, k),
                                                   _corner_u(g, k + 1), x0, x1, y0, y1)
                err = abs(got.get(k, 0.0) - ref)
                worst = max(worst, err)
                n_checked += 1
    assert n_checked > 50000
    assert worst < 1e-11, worst


def _mc_u(phi, s, sdd, P):
    """Detector coordinate of points P (N x 2) from Eq. (z rotation): solve
    P - S = lam * (s+d)(cos, sin) + mu * (sin, -cos) for (lam, mu); the ray through P meets
    the detector at corner coordinate m d_y = mu / lam (lam = -1 is the detector)."""
    c, sn = math.cos(phi), math.sin(phi)
    M = np.array([[sdd * c, sn], [sdd * sn, -c]])
    rhs = (P - np.array([s * c, s * sn])).T
    lam, mu = np.linalg.solve(M, rhs)
    return mu / lam


def test_monte_carlo_entries():
    """P3: entries against Monte Carlo estimates (within 5 sigma)."""
    g = synth.geometry(6, 5, 1, a=1.3, b=0.9, n_views=7, s=9.0, sdd=16.0, nu=12, du=0.7,
                       u_off=0.15)
    rng = np.random.default_rng(3)
    N = 400_000
    for v in range(g["n_views"]):
        for ix, iy in [(0, 0), (2, 3), (5, 4), (3, 1)]:
            x0, x1 = _grid(g, ix, 0), _grid(g, ix + 1, 0)
            y0, y1 = _grid(g, iy, 1), _grid(g, iy + 1, 1)
            P = np.stack([rng.uniform(x0, x1, N), rng.uniform(y0, y1, N)], 1)
            u = _mc_u(g["angles"][v], g["s"], g["sdd"], P)
            k = np.floor((u - g["u_off"]) / g["du"] + g["nu"] / 2.0).astype(int)
            area = (x1 - x0) * (y1 - y0)
            ks, ws = oracle.entries_2d(g, v, ix, iy)
            got = dict(zip(ks.tolist(), ws.tolist()))
            for kk in range(g["nu"]):
                p = np.mean(k == kk)
                est = area * p
                sig = area * math.sqrt(max(p * (1 - p), 1.0 / N) / N)
                assert abs(got.get(kk, 0.0) - est) <= 5 * sig + 1e-12, (v, ix, iy, kk)


# ----------------------------------------------------------------------------------------
def _half_plane_u(phi, s, sdd, u, keep_below):
    """u(P) <= u (keep_below) or u(P) >= u as  c0 x + c1 y + c3 >= 0."""
    c, sn = math.cos(phi), math.sin(phi)
    pl = np.array([-sdd * sn + u * c, sdd * c + u * sn, 0.0, -u * s])
    return -pl if keep_below else pl


def test_triangle_atom_A3():
    """The triangle atom: area cut off at V_{n,2} = ((n_x+1)a, n_y b) by one ray that meets
    the two edges at that vertex equals ab * A_3(phi, gamma_2, gamma_1, beta)."""
    rng = np.random.default_rng(7)
    s, sdd, a, b = 12.0, 20.0, 1.7, 1.1
    hits = 0
    while hits < 200:
        phi = rng.uniform(-math.pi, math.pi)
        nx, ny = int(rng.integers(-3, 3)), int(rng.integers(-3, 3))
        V = {1: (nx * a, ny * b), 2: ((nx + 1) * a, ny * b),
             3: ((nx + 1) * a, (ny + 1) * b), 4: (nx * a, (ny + 1) * b)}
        gam = {i: pf.gamma(phi, s, *V[i]) for i in V}
        others = [gam[i] for i in (1, 3, 4)]
        lo = gam[2] < min(others)
        hi = gam[2] > max(others)
        if not (lo or hi):
            continue
        edge = min(others) if lo else max(others)
        bm = gam[2] + rng.uniform(0.05, 0.95) * (edge - gam[2])
        u = math.tan(bm) * sdd
        area = oracle.clip_area_2d((nx * a, (nx + 1) * a, ny * b, (ny + 1) * b),
                                   [_half_plane_u(phi, s, sdd, u, keep_below=lo)])
        ref = a * b * pf.A3(phi, gam[2], gam[1], bm, a, b)
        assert abs(area - ref) < 1e-10 * max(1.0, ref), (area, ref)
        hits += 1


def test_trapezoid_atom_A4():
    """Two rays that both cross the faces x = n_x a and x = (n_x+1) a bound a trapezoid of
    area ab * A_4 (Eq. (area trapezoid rel))."""
    rng = np.random.default_rng(11)
    s, sdd, a, b = 15.0, 25.0, 0.8, 1.9
    hits = 0
    while hits < 200:
        phi = rng.uniform(-math.pi, math.pi)
        if abs(math.cos(phi)) < 0.3:
            continue
        nx, ny = int(rng.integers(-4, 4)), int(rng.integers(-4, 4))
        x0, x1, y0, y1 = nx * a, (nx + 1) * a, ny * b, (ny + 1) * b
        # pick two rays through points on the face x = x0 and check they cross x = x1 inside
        ys = np.sort(rng.uniform(y0, y1, 2))
        bms = [pf.gamma(phi, s, x0, yy) for yy in ys]
        ok = True
        for bm in bms:
            yc = s * math.sin(phi) - (s * math.cos(phi) - x1) * math.tan(phi - bm)  # Eq. (y expression)
            ok &= (y0 < yc < y1)
        if not ok:
            continue
        u0, u1 = sorted(math.tan(bm) * sdd for bm in bms)
        area = oracle.clip_area_2d((x0, x1, y0, y1), [_half_plane_u(phi, s, sdd, u0, False),
                                                      _half_plane_u(phi, s, sdd, u1, True)])
        ref = a * b * pf.A4(phi, nx, bms[0], bms[1], a, b, s)
        assert abs(area - ref) < 1e-10, (area, ref)
        hits += 1


def _load_composition():
    path = os.path.join(os.path.dirname(__file__), "golden", "composition_2d.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return np.array(rows, dtype=float)


def test_worked_composition_example():
    """Eq. (2d procedure): for the order Gamma_1 < beta_{m0} < Gamma_2 < beta_{m0+1} < Gamma_3
    < beta_{m0+2} < beta_{m0+3} < Gamma_4 (the paper's m0 = -3) the five element weights
    are the printed 7x7 matrix times the atom vector.  Searched on the figure's geometry
    (s = d = 5, d_y = 0.8, pixel side 1.8); the oracle's entries must match."""
    Mx = _load_composition()
    s, sdd, dy, a = 5.0, 10.0, 0.8, 1.8
    found = 0
    for phi in np.linspace(-math.pi, math.pi, 721)[:-1]:
        for nx in range(-3, 3):
            for ny in range(-3, 3):
                V = {1: (nx * a, ny * a), 2: ((nx + 1) * a, ny * a),
                     3: ((nx + 1) * a, (ny + 1) * a), 4: (nx * a, (ny + 1) * a)}
                gam = {i: pf.gamma(phi, s, *V[i]) for i in V}
                order = sorted(gam, key=gam.get)
                G = [gam[i] for i in order]
                # the middle trapezoid must cross the x-faces: {V(1), V(2)} is a y-edge
                if {order[0], order[1]} not in ({1, 2}, {3, 4}):
                    continue
                m0 = math.floor(math.tan(G[0]) * sdd / dy) + 1
                B = {m: pf.beta(m * dy, sdd) for m in range(m0 - 1, m0 + 5)}
                if not (B[m0 - 1] < G[0] < B[m0] < G[1] < B[m0 + 1] < G[2] < B[m0 + 2]
                        < B[m0 + 3] < G[3] < B[m0 + 4]):
                    continue
                A3 = lambda gt, ga, bb: pf.A3(phi, gt, ga, bb, a, a)
                A4 = lambda b0, b1: pf.A4(phi, nx, b0, b1, a, a, s)
                atoms = np.array([A3(G[0], G[1], B[m0]), A3(G[0], G[1], G[1]),
                                  A4(G[1], B[m0 + 1]), A4(B[m0 + 1], G[2]),
                                  A3(G[3], G[2], G[2]), A3(G[3], G[2], B[m0 + 2]),
                                  A3(G[3], G[2], B[m0 + 3])])
                parts = Mx @ atoms
                w = [parts[0], parts[1] + parts[2], parts[3] + parts[4], parts[5], parts[6]]
                nu = 40
                g = synth.geometry(6, 6, 1, a=a, b=a, n_views=1, angles=[phi], s=s, sdd=sdd,
                                   nu=nu, du=dy)
                ks, ws = oracle.entries_2d(g, 0, nx + 3, ny + 3)
                got = dict(zip((ks - nu // 2).tolist(), ws.tolist()))
                for i, m in enumerate(range(m0 - 1, m0 + 4)):
                    assert abs(got.get(m, 0.0) / (a * a) - w[i]) < 1e-10, (phi, nx, ny, m)
                assert set(got) == set(range(m0 - 1, m0 + 4))
                found += 1
    assert found >= 5, found


# ----------------------------------------------------------------------------------------
def test_partition_of_the_fan():
    """P4: summed over a view's elements a pixel's entries give its area inside the fan
    (the full pixel area when all its corners project onto the detector)."""
    g = synth.config("fan2d_64")
    rng = np.random.default_rng(5)
    for _ in range(400):
        v, ix, iy = int(rng.integers(90)), int(rng.integers(64)), int(rng.integers(64))
        phi = g["angles"][v]
        ks, ws = oracle.entries_2d(g, v, ix, iy)
        x0, x1 = _grid(g, ix, 0), _grid(g, ix + 1, 0)
        y0, y1 = _grid(g, iy, 1), _grid(g, iy + 1, 1)
        us = [math.tan(pf.gamma(phi, g["s"], X, Y)) * g["sdd"] for X in (x0, x1) for Y in (y0, y1)]
        if min(us) >= _corner_u(g, 0) and max(us) <= _corner_u(g, g["nu"]):
            assert abs(ws.sum() - 1.0) < 1e-12
        else:
            full = sweep.element_area_sweep_any(phi, g["s"], g["sdd"], _corner_u(g, 0),
                                                _corner_u(g, g["nu"]), x0, x1, y0, y1)
            assert abs(ws.sum() - full) < 1e-12


@pytest.mark.parametrize("phi", [0.0, math.pi / 2, math.pi, 0.3])
def test_column_sum_is_fan_area_in_grid(phi):
    """P4: for an element whose fan enters and leaves the grid box through two opposite
    sides, the entries summed over all pixels equal the fan quadrilateral's area, computed
    from the four analytic crossing points (shoelace)."""
    N, s, sdd = 16, 40.0, 70.0
    g = synth.geometry(N, N, 1, n_views=1, angles=[phi], s=s, sdd=sdd, nu=20, du=1.0)
    x = np.ones((N, N))
    p = oracle.forward_2d(g, x)[0]
    c, sn = math.cos(phi), math.sin(phi)
    for k in range(6, 14):
        u0, u1 = _corner_u(g, k), _corner_u(g, k + 1)
        # the ray through detector coordinate u: S + lam * (-sdd e_s + u e_u), lam in (0, 1]
        pts = []
        for u in (u0, u1):
            d = np.array([-sdd * c - u * sn, -sdd * sn + u * c])
            S = np.array([s * c, s * sn])
            # entry / exit of the box |x|,|y| <= N/2 along the dominant axis
            ax = 0 if abs(d[0]) >= abs(d[1]) else 1
            lams = sorted([(-N / 2 - S[ax]) / d[ax], (N / 2 - S[ax]) / d[ax]])
            P_in, P_out = S + lams[0] * d, S + lams[1] * d
            assert abs(P_in[1 - ax]) <= N / 2 and abs(P_out[1 - ax]) <= N / 2
            pts.append((P_in, P_out))
        quad = np.array([pts[0][0], pts[0][1], pts[1][1], pts[1][0]])
        xq, yq = quad[:, 0], quad[:, 1]
        area = 0.5 * abs(np.dot(xq, np.roll(yq, -1)) - np.dot(yq, np.roll(xq, -1)))
        assert abs(p[k] - area) < 1e-10 * area, (k, p[k], area)


def test_similarity_scaling_and_mirror():
    """P4: scaling every length by t scales W by t^2; mirroring y (phi -> -phi, u -> -u,
    iy -> ny-1-iy, k -> nu-1-k) maps W onto itself."""
    base = dict(a=1.1, b=0.7, s=30.0, sdd=47.0, nu=30, du=0.9)
    ang = np.array([0.2, 1.3, 2.9, -2.2])
    g1 = synth.geometry(10, 12, 1, n_views=4, angles=ang, **base)
    t = 2.5
    g2 = synth.geometry(10, 12, 1, n_views=4, angles=ang,
                        **{k: (v * t if k != "nu" else v) for k, v in base.items()})
    gm = synth.geometry(10, 12, 1, n_views=4, angles=-ang, **base)
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(12, 10))
    p1, p2 = oracle.forward_2d(g1, x), oracle.forward_2d(g2, x)
    assert np.allclose(p2, t * t * p1, rtol=1e-12, atol=1e-12)
    pm = oracle.forward_2d(gm, x[::-1, :].copy())
    assert np.allclose(pm[:, ::-1], p1, rtol=1e-12, atol=1e-12)


def test_oracle_forward_back_adjoint_and_pruning():
    """The oracle's forward and back use the same entries: <Wx, y> = <x, W^T y>; the
    bounding-box pruning loses no entry."""
    g = synth.config("fan2d_64")
    rng = np.random.default_rng(9)
    x = rng.normal(size=(64, 64))
    y = rng.normal(size=(90, 96))
    lhs = float(np.sum(oracle.forward_2d(g, x) * y))
    rhs = float(np.sum(x * oracle.back_2d(g, y)))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    for _ in range(100):
        v, ix, iy = int(rng.integers(90)), int(rng.integers(64)), int(rng.integers(64))
        k1, w1 = oracle.entries_2d(g, v, ix, iy)
        k2, w2 = oracle.entries_2d(g, v, ix, iy, all_elements=True)
        assert k1.tolist() == k2.tolist() and np.allclose(w1, w2, rtol=0, atol=0)


def test_forward_element_matches_full_forward():
    g = synth.config("fan2d_64")
    x = synth.ellipse_phantom(64, 0)
    p = oracle.forward_2d(g, x, views=[3, 40])
    for vi, v in enumerate([3, 40]):
        for k in (10, 48, 70):
            assert abs(oracle.forward_element_2d(g, x, v, k) - p[vi, k]) < 1e-10

"""Pins of the 3D oracle against things other than itself.

* entries against an independent slice-wise integrator (exact sweep areas integrated over
  z by adaptive quadrature);
* Monte Carlo with the detector hit from the paper's ray parametrisation (Eq. (z rotation));
* the paper's 3D closed forms (Section 'The Three-dimensional Case' and its appendix):
  the tetrahedron, Eq. (rel vol 3d) with its C-vector, the phi = 0 form Eq. (vol), the
  top-view triangle Eq. (res vol 3d), and the identities Eq. (f minus g), Eq. (gi gg);
* invariants: partition of the cone, the closed-form volume of an element pyramid through
  the grid box, similarity scaling, mirror symmetry in z, adjointness.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import paper_formulas as pf
from tests import sweep


def _cu(g, k):
    return (k - g["nu"] / 2.0) * g["du"] + g["u_off"]


def _cv(g, l):
    return (l - g["nv"] / 2.0) * g["dv"] + g["v_off"]


def _box(g, ix, iy, iz):
    return ((ix - g["nx"] / 2.0) * g["a"], (ix + 1 - g["nx"] / 2.0) * g["a"],
            (iy - g["ny"] / 2.0) * g["b"], (iy + 1 - g["ny"] / 2.0) * g["b"],
            (iz - g["nz"] / 2.0) * g["c"], (iz + 1 - g["nz"] / 2.0) * g["c"])


SMALL = dict(a=1.2, b=0.9, c=1.1, s=14.0, sdd=23.0, nu=14, nv=12, du=1.3, dv=1.1,
             u_off=0.2, v_off=-0.35)


def test_entries_match_slice_integration():
    """P2 (3D): entries equal the z-integral of exact slice areas."""
    ang = np.array([0.4, 1.1, 2.5, -0.7, -2.0])
    g = synth.geometry(6, 5, 7, n_views=5, angles=ang, **SMALL)
    g["dim"] = 3
    rng = np.random.default_rng(1)
    n = 0
    for _ in range(40):
        v = int(rng.integers(5))
        ix, iy, iz = int(rng.integers(6)), int(rng.integers(5)), int(rng.integers(7))
        kl, ws = oracle.entries_3d(g, v, ix, iy, iz)
        got = {(int(k), int(l)): w for (k, l), w in zip(kl, ws)}
        box = _box(g, ix, iy, iz)
        phi = g["angles"][v]
        ks = sorted({k for k, _ in got} | {min(k for k, _ in got) - 1, max(k for k, _ in got) + 1}) if got else []
        ls = sorted({l for _, l in got} | {min(l for _, l in got) - 1, max(l for _, l in got) + 1}) if got else []
        for k in ks:
            for l in ls:
                if not (0 <= k < g["nu"] and 0 <= l < g["nv"]):
                    continue
                ref = sweep.element_volume_slices(phi, g["s"], g["sdd"], _cu(g, k), _cu(g, k + 1),
                                                  _cv(g, l), _cv(g, l + 1), box)
                assert abs(got.get((k, l), 0.0) - ref) < 1e-9, (v, ix, iy, iz, k, l, got.get((k, l)), ref)
                n += 1
    assert n > 300


def _mc_uv(phi, s, sdd, P):
    """(u, v) of points P (N x 3) from Eq. (z rotation): solve
    P - S = lam (s+d)(cos, sin, 0) + mu_y (sin, -cos, 0) + mu_z (0, 0, -1);
    the ray through P meets the detector at m_y d_y = mu_y / lam, m_z d_z = mu_z / lam."""
    c, sn = math.cos(phi), math.sin(phi)
    M = np.array([[sdd * c, sn, 0.0], [sdd * sn, -c, 0.0], [0.0, 0.0, -1.0]])
    rhs = (P - np.array([s * c, s * sn, 0.0])).T
    lam, muy, muz = np.linalg.solve(M, rhs)
    return muy / lam, muz / lam


def test_monte_carlo_entries():
    ang = np.array([0.0, 0.9, 2.2, 3.6, 5.1])
    g = synth.geometry(5, 4, 6, n_views=5, angles=ang, **SMALL)
    g["dim"] = 3
    rng = np.random.default_rng(4)
    N = 300_000
    for v in range(5):
        for ix, iy, iz in [(0, 0, 0), (2, 1, 3), (4, 3, 5), (1, 2, 2)]:
            x0, x1, y0, y1, z0, z1 = _box(g, ix, iy, iz)
            P = np.stack([rng.uniform(x0, x1, N), rng.uniform(y0, y1, N), rng.uniform(z0, z1, N)], 1)
            u, vv = _mc_uv(g["angles"][v], g["s"], g["sdd"], P)
            k = np.floor((u - g["u_off"]) / g["du"] + g["nu"] / 2.0).astype(int)
            l = np.floor((vv - g["v_off"]) / g["dv"] + g["nv"] / 2.0).astype(int)
            vol = (x1 - x0) * (y1 - y0) * (z1 - z0)
            kl, ws = oracle.entries_3d(g, v, ix, iy, iz)
            got = {(int(a), int(b)): w for (a, b), w in zip(kl, ws)}
            keys = set(got) | set(zip(k.tolist(), l.tolist()))
            for kk, ll in keys:
                if not (0 <= kk < g["nu"] and 0 <= ll < g["nv"]):
                    continue
                p = np.mean((k == kk) & (l == ll))
                sig = vol * math.sqrt(max(p * (1 - p), 1.0 / N) / N)
                assert abs(got.get((kk, ll), 0.0) - vol * p) <= 5 * sig + 1e-12


def test_partition_of_the_cone():
    g = synth.config("cone3d_128")
    rng = np.random.default_rng(6)
    done = 0
    while done < 150:
        v = int(rng.integers(180))
        ix, iy, iz = (int(t) for t in rng.integers(40, 88, size=3))
        kl, ws = oracle.entries_3d(g, v, ix, iy, iz)
        assert abs(ws.sum() - 1.0) < 1e-12
        done += 1


def test_pyramid_volume_through_grid_box():
    """At phi = 0 a central element's pyramid crosses the whole box from x = N/2 to -N/2
    without touching its other faces; its volume in the box is
    (du dv / (3 sdd^2)) ((s + N/2)^3 - (s - N/2)^3)."""
    N, s, sdd = 8, 30.0, 55.0
    g = synth.geometry(N, N, N, n_views=1, angles=[0.0], s=s, sdd=sdd, nu=10, nv=10,
                       du=0.8, dv=0.7)
    g["dim"] = 3
    p = oracle.forward_3d(g, np.ones((N, N, N)))[0]
    ref = g["du"] * g["dv"] / (3 * sdd ** 2) * ((s + N / 2) ** 3 - (s - N / 2) ** 3)
    for k in range(3, 7):
        for l in range(3, 7):
            assert abs(p[l, k] - ref) < 1e-11 * ref, (k, l)


def test_similarity_scaling_and_z_mirror():
    ang = np.array([0.3, 2.0, -1.2])
    g1 = synth.geometry(4, 5, 6, n_views=3, angles=ang, **SMALL)
    t = 1.7
    sc = {k: (v * t if k not in ("nu", "nv") else v) for k, v in SMALL.items()}
    g2 = synth.geometry(4, 5, 6, n_views=3, angles=ang, **sc)
    mir = dict(SMALL, v_off=-SMALL["v_off"])
    g3 = synth.geometry(4, 5, 6, n_views=3, angles=ang, **mir)
    for g in (g1, g2, g3):
        g["dim"] = 3
    x = np.random.default_rng(0).uniform(size=(6, 5, 4))
    p1, p2 = oracle.forward_3d(g1, x), oracle.forward_3d(g2, x)
    assert np.allclose(p2, t ** 3 * p1, rtol=1e-11, atol=1e-12)
    p3 = oracle.forward_3d(g3, x[::-1].copy())
    assert np.allclose(p3[:, ::-1, :], p1, rtol=1e-11, atol=1e-12)


def test_adjoint_and_single_values():
    ang = synth.uniform_angles(6)
    g = synth.geometry(6, 6, 5, n_views=6, angles=ang, **SMALL)
    g["dim"] = 3
    rng = np.random.default_rng(8)
    x = rng.normal(size=(5, 6, 6))
    y = rng.normal(size=(6, 12, 14))
    px = oracle.forward_3d(g, x)
    bx = oracle.back_3d(g, y)
    assert abs(np.sum(px * y) - np.sum(x * bx)) < 1e-10 * abs(np.sum(px * y))
    for (v, k, l) in [(0, 5, 6), (3, 7, 4), (5, 9, 8)]:
        assert abs(oracle.forward_element_3d(g, x, v, k, l) - px[v, l, k]) < 1e-11
    for (ix, iy, iz) in [(0, 0, 0), (3, 2, 4), (5, 5, 1)]:
        assert abs(oracle.back_voxel_3d(g, y, ix, iy, iz) - bx[iz, iy, ix]) < 1e-11


# ----------------------------------------------------------------------------------------
# The paper's 3D closed forms
# ----------------------------------------------------------------------------------------
def _lat(phi, s, sdd, u, keep_below):
    c, sn = math.cos(phi), math.sin(phi)
    pl = np.array([-sdd * sn + u * c, sdd * c + u * sn, 0.0, -u * s])
    return -pl if keep_below else pl


def _above_row(phi, s, sdd, vv):
    """v(P) >= vv  <=>  sdd z - vv t >= 0."""
    c, sn = math.cos(phi), math.sin(phi)
    return np.array([vv * c, vv * sn, sdd, -vv * s])


def test_identities_f_minus_g_and_gi_gg():
    rng = np.random.default_rng(12)
    for _ in range(500):
        phi = rng.uniform(-3, 3)
        bm = rng.uniform(-0.3, 0.3)
        ta = rng.uniform(0.01, 0.3)
        a, b, c, s = rng.uniform(0.5, 2, 3).tolist() + [rng.uniform(20, 40)]
        nx, ny, nz = (int(t) for t in rng.integers(-5, 5, 3))
        g = pf.g_front(phi, bm, ta, nx, nz, a, c, s)
        f = pf.f_rear(phi, bm, ta, nx, nz, a, c, s)
        assert abs((g - f) - math.cos(bm) / math.cos(phi - bm)) < 1e-9 * max(1, abs(g))
        h = pf.h_side(phi, bm, ta, ny, nz, a, b, c, s)
        gg = pf.g_corner(phi, ta, nx, ny, nz, a, b, c, s)
        lhs = (math.cos(phi) * math.cos(phi - bm) / math.cos(bm) * g
               + math.sin(phi) * math.sin(phi - bm) / math.cos(bm) * h)
        assert abs(lhs - gg) < 1e-9 * max(1, abs(gg))


def test_top_view_trapezoid_rel_volume():
    """Eq. (rel vol 3d): relative volume above the row plane v = m_z d_z inside the top-view
    trapezoid between two rays that cross both x-faces, with C from the signs of g, f
    (the plane is kept above the bottom face).  Includes the tetrahedron case C=(1,0,0,0),
    which must also match the printed tetrahedron volume."""
    rng = np.random.default_rng(21)
    a, b, c, s, sdd = 1.0, 1.3, 0.8, 20.0, 32.0
    hits = tetra = 0
    tries = 0
    while hits < 300 and tries < 200000:
        tries += 1
        phi = rng.uniform(-math.pi, math.pi)
        if abs(math.sin(phi)) < 0.05 or abs(math.cos(phi)) < 0.3:
            continue
        nx, ny, nz = int(rng.integers(-4, 4)), int(rng.integers(-4, 4)), int(rng.integers(1, 5))
        x0, x1, y0, y1, z0, z1 = nx * a, (nx + 1) * a, ny * b, (ny + 1) * b, nz * c, (nz + 1) * c
        ys = np.sort(rng.uniform(y0, y1, 2))
        bms = [pf.gamma(phi, s, x0, yy) for yy in ys]
        ok = all(y0 < s * math.sin(phi) - (s * math.cos(phi) - x1) * math.tan(phi - bm) < y1 for bm in bms)
        if not ok:
            continue
        # plane through a random height in the top part of the voxel
        tmid = s - (0.5 * (x0 + x1)) * math.cos(phi) - (0.5 * (y0 + y1)) * math.sin(phi)
        if hits % 2:
            ta = rng.uniform(z0 + 0.55 * c, z1 + 0.3 * c) / tmid
        else:   # planes grazing the top face make the single-vertex (tetrahedron) cases
            ta = rng.uniform(z1 - 0.05 * c, z1 + 0.05 * c) / tmid
        ts = [s - X * math.cos(phi) - Y * math.sin(phi) for X in (x0, x1) for Y in (y0, y1)]
        if ta * min(ts) <= z0:
            continue
        bms.sort()
        u0, u1 = (math.tan(bm) * sdd for bm in bms)
        vol = oracle.clip_volume_3d((x0, x1, y0, y1, z0, z1),
                                    [_lat(phi, s, sdd, u0, False), _lat(phi, s, sdd, u1, True),
                                     _above_row(phi, s, sdd, ta * sdd)])
        gm = pf.g_front(phi, bms[0], ta, nx, nz, a, c, s)
        fm = pf.f_rear(phi, bms[0], ta, nx, nz, a, c, s)
        gm1 = pf.g_front(phi, bms[1], ta, nx, nz, a, c, s)
        fm1 = pf.f_rear(phi, bms[1], ta, nx, nz, a, c, s)
        C = [float(gm > 0), float(fm > 0), float(gm1 > 0), float(fm1 > 0)]
        ref = pf.vol_rel_trapezoid(phi, bms[0], bms[1], ta, C, gm, fm, gm1, fm1, a, b, c)
        assert abs(vol / (a * b * c) - ref) < 1e-9, (vol / (a * b * c), ref, C)
        # a single positive vertex term is the printed tetrahedron volume
        if sum(C) == 1:
            i = C.index(1.0)
            val = (gm, fm, gm1, fm1)[i]
            assert abs(vol - pf.vol_tetra(phi, bms[i // 2], ta, val, a)) < 1e-9
            tetra += 1
        hits += 1
    assert hits >= 300 and tetra >= 3, (hits, tetra)


def test_phi0_rel_volume():
    """Eq. (vol): the phi = 0 limit of Eq. (rel vol 3d) (g, f independent of beta)."""
    rng = np.random.default_rng(22)
    a, b, c, s, sdd = 1.0, 1.0, 1.0, 20.0, 32.0
    phi = 0.0
    hits = 0
    while hits < 100:
        nx, ny, nz = int(rng.integers(-4, 4)), int(rng.integers(-4, 4)), int(rng.integers(1, 5))
        x0, x1, y0, y1, z0, z1 = nx * a, (nx + 1) * a, ny * b, (ny + 1) * b, nz * c, (nz + 1) * c
        ys = np.sort(rng.uniform(y0, y1, 2))
        bms = [pf.gamma(phi, s, x0, yy) for yy in ys]
        if not all(y0 < s * math.sin(phi) - (s * math.cos(phi) - x1) * math.tan(phi - bm) < y1 for bm in bms):
            continue
        tmid = s - 0.5 * (x0 + x1)
        ta = rng.uniform(z0 + 0.55 * c, z1 + 0.3 * c) / tmid
        if ta * (s - x1) <= z0:
            continue
        u0, u1 = (math.tan(bm) * sdd for bm in bms)
        vol = oracle.clip_volume_3d((x0, x1, y0, y1, z0, z1),
                                    [_lat(phi, s, sdd, u0, False), _lat(phi, s, sdd, u1, True),
                                     _above_row(phi, s, sdd, ta * sdd)])
        g = pf.g_front(phi, bms[0], ta, nx, nz, a, c, s)
        f = pf.f_rear(phi, bms[0], ta, nx, nz, a, c, s)
        ref = pf.vol_rel_phi0(bms[0], bms[1], ta, float(g > 0), float(f > 0), g, f, nx, a, b, c, s)
        assert abs(vol / (a * b * c) - ref) < 1e-9, (vol, ref)
        hits += 1


def test_top_view_triangle_rel_volume():
    """Eq. (res vol 3d): relative volume above the row plane inside the top-view triangle
    cut off at V_{n,2} by one ray, with C = (C_y, C_x, C_g) from the signs of g, h, g_g."""
    rng = np.random.default_rng(23)
    a, b, c, s, sdd = 1.0, 1.2, 0.9, 18.0, 30.0
    hits = 0
    tries = 0
    while hits < 300 and tries < 200000:
        tries += 1
        phi = rng.uniform(-math.pi, math.pi)
        if abs(math.sin(phi)) < 0.1 or abs(math.cos(phi)) < 0.1:
            continue
        nx, ny, nz = int(rng.integers(-4, 4)), int(rng.integers(-4, 4)), int(rng.integers(1, 5))
        x0, x1, y0, y1, z0, z1 = nx * a, (nx + 1) * a, ny * b, (ny + 1) * b, nz * c, (nz + 1) * c
        V = {1: (x0, y0), 2: (x1, y0), 3: (x1, y1), 4: (x0, y1)}
        gam = {i: pf.gamma(phi, s, *V[i]) for i in V}
        others = [gam[i] for i in (1, 3, 4)]
        lo, hi = gam[2] < min(others), gam[2] > max(others)
        if not (lo or hi):
            continue
        edge = min(others) if lo else max(others)
        bm = gam[2] + rng.uniform(0.05, 0.95) * (edge - gam[2])
        ts = [s - X * math.cos(phi) - Y * math.sin(phi) for X, Y in V.values()]
        ta = rng.uniform(z0 + 0.55 * c, z1 + 0.3 * c) / (s - x1 * math.cos(phi) - y0 * math.sin(phi))
        if ta * min(ts) <= z0:
            continue
        u = math.tan(bm) * sdd
        vol = oracle.clip_volume_3d((x0, x1, y0, y1, z0, z1),
                                    [_lat(phi, s, sdd, u, keep_below=lo), _above_row(phi, s, sdd, ta * sdd)])
        gm = pf.g_front(phi, bm, ta, nx, nz, a, c, s)
        hm = pf.h_side(phi, bm, ta, ny, nz, a, b, c, s)
        gg = pf.g_corner(phi, ta, nx, ny, nz, a, b, c, s)
        ref = pf.vol_rel_triangle(phi, bm, ta, float(gm > 0), float(hm > 0), float(gg > 0),
                                  gm, hm, gg, a, b, c)
        assert abs(vol / (a * b * c) - ref) < 1e-9, (vol / (a * b * c), ref)
        hits += 1
    assert hits >= 300

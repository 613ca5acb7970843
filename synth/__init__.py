"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no part of the projector arithmetic: it only describes workloads
(grid, detector and orbit sizes) and draws seeded phantoms, angle lists and noise.
Both the oracle and the CUDA path consume what it produces.

Workloads (the paper's datasets are not used; every input is synthetic):

* ``fan2d_64``    2D fan beam, 64x64 unit pixels, 90 views over [0, 2pi), 96 elements of
                  width 1, source-isocentre 200, source-detector 400.
* ``fan2d_512``   2D fan beam, 512x512, 720 views, 768 elements of width 1,
                  source-isocentre 1000, source-detector 1500 (batch of 16 phantoms).
* ``cone3d_128``  3D circular cone beam, 128^3 unit voxels, 180 views, 192x192 detector of
                  unit pixels, source-isocentre 400, source-detector 800.
* ``cone3d_512``  3D cone beam, 512^3, 360 views, 768x768 detector, source-isocentre 1000,
                  source-detector 1500.

Views are phi_v = 2 pi v / N_p, v = 0..N_p-1 (the paper's "equidistant in [0, 2pi)").
Phantoms are a large "body" ellipse (ellipsoid) around the centre plus random inner
ellipses (ellipsoids), evaluated at pixel (voxel) centres: like a scanned object, most of
the field of view is nonzero and the grid's corners are air.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "CONFIGS", "geometry", "uniform_angles", "ellipse_phantom", "ellipsoid_phantom",
    "poisson_sinogram", "serving_requests", "serving_geometry",
]


def uniform_angles(n_views: int) -> np.ndarray:
    """phi_v = 2 pi v / n_views, v = 0..n_views-1 (float64)."""
    return 2.0 * math.pi * np.arange(n_views, dtype=np.float64) / n_views


def geometry(nx, ny, nz, *, a=1.0, b=1.0, c=1.0, n_views, s, sdd, nu, nv=1, du=1.0,
             dv=1.0, u_off=0.0, v_off=0.0, angles=None) -> dict:
    """A workload geometry as a plain dict (lengths in the same unit as the voxel sides)."""
    if angles is None:
        angles = uniform_angles(n_views)
    angles = np.ascontiguousarray(np.asarray(angles, dtype=np.float64))
    assert angles.shape == (n_views,)
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), a=float(a), b=float(b), c=float(c),
                n_views=int(n_views), angles=angles, s=float(s), sdd=float(sdd),
                nu=int(nu), nv=int(nv), du=float(du), dv=float(dv),
                u_off=float(u_off), v_off=float(v_off), dim=3 if nz > 1 or nv > 1 else 2)


def _fan2d_64():
    return geometry(64, 64, 1, n_views=90, s=200.0, sdd=400.0, nu=96)


def _fan2d_512():
    return geometry(512, 512, 1, n_views=720, s=1000.0, sdd=1500.0, nu=768)


def _cone3d_128():
    g = geometry(128, 128, 128, n_views=180, s=400.0, sdd=800.0, nu=192, nv=192)
    g["dim"] = 3
    return g


def _cone3d_512():
    g = geometry(512, 512, 512, n_views=360, s=1000.0, sdd=1500.0, nu=768, nv=768)
    g["dim"] = 3
    return g


CONFIGS = {
    "fan2d_64": _fan2d_64,
    "fan2d_512": _fan2d_512,
    "cone3d_128": _cone3d_128,
    "cone3d_512": _cone3d_512,
}


def config(name: str) -> dict:
    return CONFIGS[name]()


def _body_and_inner(rng, n_inner):
    """Draws (centre offset, semi-axes, value) triples in units of the half-width R: first the
    body (centre within 0.05, semi-axes U[0.75, 0.92], value U[0.1, 0.3]), then the inner
    shapes (centre within 0.7, semi-axes U[0.05, 0.35], value U[0, 1])."""
    out = [("body", 0.05, (0.75, 0.92), (0.1, 0.3))]
    out += [("inner", 0.7, (0.05, 0.35), (0.0, 1.0))] * n_inner
    return out


def ellipse_phantom(n: int, seed: int, n_ellipses: int = 10, ny: int | None = None) -> np.ndarray:
    """A body ellipse and ``n_ellipses`` random ellipses on an n x ny grid of unit pixels
    centred at 0 (R = half the smaller side).

    Body: centre uniform in the disc of radius 0.05 R, semi-axes U[0.75, 0.92] R, value
    U[0.1, 0.3].  Inner ellipses: centre uniform in the disc of radius 0.7 R, semi-axes
    U[0.05, 0.35] R, value U[0, 1].  Orientation U[0, pi).  A pixel takes the sum of the
    values of the ellipses that contain its centre.  Returns float64 [ny][n].
    """
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    xs = (np.arange(n) - n / 2.0 + 0.5)
    ys = (np.arange(ny) - ny / 2.0 + 0.5)
    X, Y = np.meshgrid(xs, ys)
    R = 0.5 * min(n, ny)
    img = np.zeros((ny, n), dtype=np.float64)
    for _, rc, (a0, a1), (v0, v1) in _body_and_inner(rng, n_ellipses):
        r = rc * R * math.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * math.pi)
        cx, cy = r * math.cos(th), r * math.sin(th)
        ax, ay = rng.uniform(a0, a1, size=2) * R
        ang = rng.uniform(0, math.pi)
        val = rng.uniform(v0, v1)
        ca, sa = math.cos(ang), math.sin(ang)
        dx, dy = X - cx, Y - cy
        xr = dx * ca + dy * sa
        yr = -dx * sa + dy * ca
        img[(xr / ax) ** 2 + (yr / ay) ** 2 <= 1.0] += val
    return img


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _ellipsoid_params(n: int, seed: int, n_ellipsoids: int):
    rng = np.random.default_rng(seed)
    R = 0.5 * n
    params = []
    for _, rc, (a0, a1), (v0, v1) in _body_and_inner(rng, n_ellipsoids):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        c = d * rc * R * rng.uniform() ** (1.0 / 3.0)
        ax = rng.uniform(a0, a1, size=3) * R
        Rm = _random_rotation(rng)
        val = rng.uniform(v0, v1)
        params.append((c, ax, Rm, val))
    return params


def ellipsoid_phantom(n: int, seed: int, n_ellipsoids: int = 10, dtype=np.float64,
                      slab: int = 32, workers: int = 1) -> np.ndarray:
    """A body ellipsoid and ``n_ellipsoids`` random ellipsoids on an n^3 grid of unit voxels
    centred at 0 ([nz][ny][nx]; R = n/2).

    Body: centre uniform in the ball of radius 0.05 R, semi-axes U[0.75, 0.92] R, value
    U[0.1, 0.3].  Inner ellipsoids: centre uniform in the ball of radius 0.7 R, semi-axes
    U[0.05, 0.35] R, value U[0, 1].  Uniformly random rotations.  Evaluated slab by slab to
    bound memory (``workers`` threads share the slabs; the result does not depend on it).
    """
    params = _ellipsoid_params(n, seed, n_ellipsoids)
    xs = (np.arange(n) - n / 2.0 + 0.5)
    out = np.zeros((n, n, n), dtype=dtype)
    Y, X = np.meshgrid(xs, xs, indexing="ij")

    def one_slab(z0):
        zs = xs[z0:z0 + slab]
        Z = zs[:, None, None]
        acc = np.zeros((len(zs), n, n), dtype=np.float64)
        for c, ax, Rm, val in params:
            dx, dy, dz = X[None] - c[0], Y[None] - c[1], Z - c[2]
            q = 0.0
            for r in range(3):
                comp = Rm[0, r] * dx + Rm[1, r] * dy + Rm[2, r] * dz
                q = q + (comp / ax[r]) ** 2
            acc[q <= 1.0] += val
        out[z0:z0 + slab] = acc

    if workers > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(one_slab, range(0, n, slab)))
    else:
        for z0 in range(0, n, slab):
            one_slab(z0)
    return out


def ellipsoid_phantom_torch(n: int, seed: int, device, n_ellipsoids: int = 10):
    """The same phantom as ``ellipsoid_phantom`` (same parameter draws), evaluated with torch
    on ``device`` (float32), for large serving requests."""
    import torch
    xs = torch.arange(n, device=device, dtype=torch.float32) - n / 2.0 + 0.5
    Z, Y, X = torch.meshgrid(xs, xs, xs, indexing="ij")
    out = torch.zeros((n, n, n), device=device, dtype=torch.float32)
    for c, ax, Rm, val in _ellipsoid_params(n, seed, n_ellipsoids):
        dx, dy, dz = X - float(c[0]), Y - float(c[1]), Z - float(c[2])
        q = torch.zeros_like(out)
        for r in range(3):
            comp = float(Rm[0, r]) * dx + float(Rm[1, r]) * dy + float(Rm[2, r]) * dz
            q += (comp / float(ax[r])) ** 2
        out += (q <= 1.0).float() * float(val)
    return out


def poisson_sinogram(p: np.ndarray, seed: int, photons: float = 1e5, max_line: float = 3.0):
    """Poisson noise at ``photons`` incident counts.

    The clean line integrals are scaled by kappa so that max(kappa p) = ``max_line``;
    counts ~ Poisson(photons * exp(-kappa p)); the noisy data are
    -ln(max(count, 1) / photons) / kappa.  Returns (noisy p, kappa).
    """
    rng = np.random.default_rng(seed)
    pmax = float(np.max(p))
    kappa = max_line / pmax if pmax > 0 else 1.0
    counts = rng.poisson(photons * np.exp(-kappa * p))
    noisy = -np.log(np.maximum(counts, 1) / photons) / kappa
    return noisy.astype(p.dtype), kappa


SERVING_PROTOCOLS_2D = ((256, 360), (512, 720), (768, 1080), (1024, 1440))
SERVING_PROTOCOLS_3D = ((64, 90), (128, 180), (192, 270), (256, 360))


def serving_geometry(n: int, n_views: int, dim: int) -> dict:
    """The serving mix's geometry for grid side n: s = 1.953 n, source-detector 2.930 n (the
    512-grid ratios), unit voxels and elements, detector 1.5 n (2D) / 1.5 n x 1.5 n (3D)."""
    nd = int(round(1.5 * n))
    nd += nd % 2
    if dim == 2:
        return geometry(n, n, 1, n_views=n_views, s=1.953 * n, sdd=2.930 * n, nu=nd)
    g = geometry(n, n, n, n_views=n_views, s=1.953 * n, sdd=2.930 * n, nu=nd, nv=nd)
    g["dim"] = 3
    return g


def serving_requests(n_requests: int, seed: int, rate_per_s: float):
    """Poisson arrivals of reconstruction requests for the serving mix.

    60% 2D, 40% 3D, each request on one of a scanner's fixed protocols (grid side and views):
    2D N in {256, 512, 768, 1024} with 360 .. 1440 views, 3D N in {64, 128, 192, 256} with
    90 .. 360 views (SERVING_PROTOCOLS_*), chosen uniformly; the geometry of serving_geometry.
    Requests of one protocol share the geometry, as on a scanner.  Each request carries a
    phantom seed.  Returns a list of dicts with arrival times.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        if rng.uniform() < 0.6:
            n, nv = SERVING_PROTOCOLS_2D[int(rng.integers(0, len(SERVING_PROTOCOLS_2D)))]
            g = serving_geometry(n, nv, 2)
        else:
            n, nv = SERVING_PROTOCOLS_3D[int(rng.integers(0, len(SERVING_PROTOCOLS_3D)))]
            g = serving_geometry(n, nv, 3)
        out.append(dict(id=i, arrival=t, geom=g, seed=int(rng.integers(0, 2**31 - 1))))
    return out

"""An independent exact area / volume integrator used to pin the oracle (test-side only).

Area: the region {x in [x0, x1], max_i L_i(x) <= y <= min_j U_j(x)} with linear bounds
L_i, U_j is integrated exactly by sweeping x: the chord length is piecewise linear with
breakpoints where two bounds cross, so the trapezoid rule between sorted breakpoints is
exact.  This shares nothing with polygon clipping.

Volume: integrate the slice area over z with adaptive Gauss-Kronrod quadrature (the slice
area is piecewise quadratic in z).
"""
import itertools
import math
import warnings

import numpy as np
from scipy import integrate


def sweep_area(x0, x1, lows, highs):
    """lows / highs: lists of (A, B) meaning y >= A + B x  /  y <= A + B x."""
    lines = list(lows) + list(highs)
    xs = {x0, x1}
    for (a1, b1), (a2, b2) in itertools.combinations(lines, 2):
        if b1 != b2:
            xc = (a2 - a1) / (b1 - b2)
            if x0 < xc < x1:
                xs.add(xc)
    xs = sorted(xs)

    def chord(x):
        lo = max(a + b * x for a, b in lows)
        hi = min(a + b * x for a, b in highs)
        return max(0.0, hi - lo)

    total = 0.0
    for xa, xb in zip(xs[:-1], xs[1:]):
        total += 0.5 * (xb - xa) * (chord(xa) + chord(xb))
    return total


def ray_line_y(phi, s, sdd, u):
    """The ray through detector coordinate u as y = A + B x (valid when it is not vertical).
    On it  sdd*w - u*t = 0  with w = -x sin + y cos, t = s - x cos - y sin."""
    c, sn = math.cos(phi), math.sin(phi)
    den = sdd * c + u * sn
    return (u * s / den, (sdd * sn - u * c) / den)


def wedge_bounds(phi, s, sdd, u_lo, u_hi, xm):
    """Bounds (lows, highs) in y for u_lo <= u(P) <= u_hi at abscissa near xm.
    u increases with y where x < s cos(phi) (derivative sign of w/t in y)."""
    L0, L1 = ray_line_y(phi, s, sdd, u_lo), ray_line_y(phi, s, sdd, u_hi)
    if xm < s * math.cos(phi):
        return [L0], [L1]
    return [L1], [L0]


def element_area_xsweep(phi, s, sdd, u_lo, u_hi, x0, x1, y0, y1):
    """Area of pixel [x0,x1]x[y0,y1] with u_lo <= u <= u_hi, by the x-sweep.  Requires the
    rays to be non-vertical and s cos(phi) outside [x0, x1]."""
    lows, highs = wedge_bounds(phi, s, sdd, u_lo, u_hi, 0.5 * (x0 + x1))
    return sweep_area(x0, x1, lows + [(y0, 0.0)], highs + [(y1, 0.0)])


def element_area_sweep_any(phi, s, sdd, u_lo, u_hi, x0, x1, y0, y1):
    """Same area; sweeps x when |cos phi| >= |sin phi|, else sweeps y by a transposition
    (x, y, phi) -> (y, x, pi/2 - phi), which maps u to -u."""
    if abs(math.cos(phi)) >= abs(math.sin(phi)):
        return element_area_xsweep(phi, s, sdd, u_lo, u_hi, x0, x1, y0, y1)
    return element_area_xsweep(math.pi / 2 - phi, s, sdd, -u_hi, -u_lo, y0, y1, x0, x1)


def slice_area(phi, s, sdd, u_lo, u_hi, v_lo, v_hi, z, x0, x1, y0, y1):
    """Area at height z of the voxel column [x0,x1]x[y0,y1] inside the element pyramid.
    The row bounds v_lo <= sdd z / t <= v_hi are bounds on the depth t (linear in x, y)."""
    c, sn = math.cos(phi), math.sin(phi)
    lows, highs = wedge_bounds(phi, s, sdd, u_lo, u_hi, 0.5 * (x0 + x1))
    lows = lows + [(y0, 0.0)]
    highs = highs + [(y1, 0.0)]
    # depth band: t in [tmin, tmax] derived from the sign of z and of the row edges
    tmin, tmax = 0.0, math.inf
    for v, is_low in ((v_lo, True), (v_hi, False)):
        # is_low: v(P) >= v_lo  <=>  sdd z - v t >= 0
        # sdd z - v t >= 0 : if v > 0: t <= sdd z / v ; if v < 0: t >= sdd z / v ; v = 0: z >= 0
        sign = 1.0 if is_low else -1.0
        vv, zz = sign * v, sign * sdd * z
        if vv > 0:
            tmax = min(tmax, zz / vv)
        elif vv < 0:
            tmin = max(tmin, zz / vv)
        elif zz < 0:
            return 0.0
    if tmax <= tmin:
        return 0.0
    # t = s - x c - y sn  ->  y = (s - x c - t) / sn  (requires sn != 0)
    for tb, is_min in ((tmin, True), (tmax, False)):
        if not math.isfinite(tb):
            continue
        line = ((s - tb) / sn, -c / sn)
        # t >= tb  <=>  y sn <= s - x c - tb
        upper = (sn > 0) == is_min
        (highs if upper else lows).append(line)
    return sweep_area(x0, x1, lows, highs)


def element_volume_slices(phi, s, sdd, u_lo, u_hi, v_lo, v_hi, box):
    x0, x1, y0, y1, z0, z1 = box
    f = lambda z: slice_area(phi, s, sdd, u_lo, u_hi, v_lo, v_hi, z, x0, x1, y0, y1)
    with warnings.catch_warnings():
        # roundoff warnings at 1e-13 absolute are expected: the tests allow 1e-9
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        val, err = integrate.quad(f, z0, z1, epsabs=1e-13, epsrel=1e-12, limit=200)
    return val

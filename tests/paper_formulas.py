"""The paper's own closed forms, restated for the oracle pins (test-side only).

Each function follows one printed formula; the tests evaluate it on configurations where
the formula applies and compare with the clipping oracle.  Angles follow the paper:
gamma / beta are the top-view angles between the source-origin ray and the ray to a
vertex / detector edge (Notation and Setup), tan(beta) = m d_y / (s + d)
(Eq. (beta_computation)), tan(gamma) from Eq. (gamma_computation) / Eq. (tan beta).
"""
import math


def gamma(phi, s, x, y):
    """Top-view angle of the point (x, y): Eq. (tan beta) / Eq. (gamma_computation)."""
    num = y * math.cos(phi) - x * math.sin(phi)
    den = s - y * math.sin(phi) - x * math.cos(phi)
    return math.atan(num / den)


def beta(m_dy, sdd):
    """Eq. (beta_computation): tan(beta_m) = m d_y / (s + d)."""
    return math.atan(m_dy / sdd)


def A3(phi, g_tri, g_adj, b_m, a, b):
    """Triangle atom, relative to ab (Section 'Triangle').

    A_3(phi, gamma_{n,2}, gamma_{n,1}, beta) = a / (b |sin(2 phi - 2 beta)|) *
        ( sin(phi - gamma_{n,1}) sin(beta - gamma_{n,2}) / sin(gamma_{n,1} - gamma_{n,2}) )^2
    where the triangle's corner is the vertex with angle g_tri and g_adj is the vertex that
    shares the edge of length a with it.  (The printed 'beta_i' is read as beta_m.)
    """
    return a / (b * abs(math.sin(2 * phi - 2 * b_m))) * (
        math.sin(phi - g_adj) * math.sin(b_m - g_tri) / math.sin(g_adj - g_tri)) ** 2


def A4(phi, nx, b_m, b_m1, a, b, s):
    """Trapezoid atom, relative to ab: Eq. (area trapezoid rel)."""
    return (1.0 / b) * abs(s * math.cos(phi) - (nx + 0.5) * a) * abs(
        math.tan(phi - b_m) - math.tan(phi - b_m1))


# ------------------------------------------------------------------------------------
# 3D (Section 'The Three-dimensional Case', Appendix 'The Three-dimensional Case')
# ------------------------------------------------------------------------------------
def tan_alpha(m_dz, sdd):
    """tan(alpha_{m_z}) = m_z d_z / (s + d)."""
    return m_dz / sdd


def g_front(phi, b_m, ta, nx, nz, a, c, s):
    """g_{m_y}: front-face term (x = (n_x+1) a)."""
    return (c / a) * (nz + 1) / ta - math.cos(b_m) / math.cos(phi - b_m) * (
        s * math.cos(phi) - (nx + 1) * a) / a


def f_rear(phi, b_m, ta, nx, nz, a, c, s):
    """f_{m_y}: rear-face term (x = n_x a)."""
    return (c / a) * (nz + 1) / ta - math.cos(b_m) / math.cos(phi - b_m) * (
        s * math.cos(phi) - nx * a) / a


def h_side(phi, b_m, ta, ny, nz, a, b, c, s):
    """h_{m_y}: side-face term (y = n_y b; the printed 'n_y a' is read as n_y b)."""
    return (c / a) * (nz + 1) / ta - math.cos(b_m) / math.sin(phi - b_m) * (
        s * math.sin(phi) - ny * b) / a


def g_corner(phi, ta, nx, ny, nz, a, b, c, s):
    """g_g: the corner term at V_{n,2} = ((n_x+1) a, n_y b)."""
    return (c / a) * (nz + 1) / ta - (s - (nx + 1) * a * math.cos(phi) - ny * b * math.sin(phi)) / a


def vol_tetra(phi, b_m, ta, gval, a):
    """Tetrahedron (one ray meets the front face only): absolute volume."""
    return a ** 3 / 6.0 * abs(ta / math.sin(phi) * math.cos(phi - b_m) / math.cos(b_m) * gval ** 3)


def vol_rel_trapezoid(phi, b_m, b_m1, ta, C, g_m, f_m, g_m1, f_m1, a, b, c):
    """Eq. (rel vol 3d): relative volume above the row plane inside the top-view trapezoid
    between beta_m and beta_{m+1};  C = (C_g,m, C_f,m, C_g,m+1, C_f,m+1)."""
    k_m = math.cos(phi - b_m) / math.cos(b_m)
    k_m1 = math.cos(phi - b_m1) / math.cos(b_m1)
    inner = k_m * (C[0] * g_m ** 3 - C[1] * f_m ** 3) - k_m1 * (C[2] * g_m1 ** 3 - C[3] * f_m1 ** 3)
    return (1.0 / 6.0) * a * a / (b * c) * abs(ta / math.sin(phi) * inner)


def vol_rel_phi0(b_m, b_m1, ta, Cg, Cf, g, f, nx, a, b, c, s):
    """Eq. (vol): the phi = 0 form of Eq. (rel vol 3d)."""
    inner = Cg * g * g * (g + 3 * s / a - 3 * nx - 3) - Cf * f * f * (f + 3 * s / a - 3 * nx)
    return (1.0 / 6.0) * a * a / (b * c) * abs(ta * inner * (math.tan(b_m) - math.tan(b_m1)))


def vol_rel_triangle(phi, b_m, ta, Cy, Cx, Cg, gm, hm, gg, a, b, c):
    """Eq. (res vol 3d): relative volume above the row plane inside the top-view triangle
    cut off at the corner V_{n,2} by the ray beta_m."""
    inner = (Cy * math.cos(phi - b_m) / math.cos(b_m) * gm ** 3
             + Cx * math.tan(phi) * math.sin(phi - b_m) / math.cos(b_m) * hm ** 3
             - Cg / math.cos(phi) * gg ** 3)
    return (1.0 / 6.0) * a * a / (b * c) * abs(ta / math.sin(phi) * inner)

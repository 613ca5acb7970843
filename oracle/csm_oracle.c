/*
 * csm_oracle.c -- plain FP64 CPU oracle for the consistent cone-beam system matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes (the plain definition, not the paper's closed forms):
 *
 *   The source sits at S = (s cos phi, s sin phi, 0) and the flat detector is the plane at
 *   distance d = sdd - s behind the isocentre, perpendicular to the source-isocentre ray
 *   (Section "Notation and Setup", Eq. (z rotation)).  A point P is seen by the detector at
 *
 *       t(P) = s - (P_x cos phi + P_y sin phi)        depth from the source along the axis
 *       u(P) = sdd * ( -P_x sin phi + P_y cos phi ) / t(P)
 *       v(P) = sdd * P_z / t(P)
 *
 *   (Appendix, Eq. (tan beta): tan(gamma) = u / sdd, and Eq. (z expr 1)).  Detector corner k
 *   sits at u_k = (k - nu/2) du + u_off and row corner l at v_l = (l - nv/2) dv + v_off,
 *   so element (k, l) spans [u_k, u_{k+1}] x [v_l, v_{l+1}] (Eq. (2d procedure): element m
 *   lies between the rays beta_m and beta_{m+1}).
 *
 *   The system-matrix entry is the measure of the intersection of the voxel with the cone of
 *   the element (Introduction, Eq. (ip) and the definition of "consistent"):
 *
 *       W[(view,k,l), j] = | voxel_j  intersect  { P : u_k <= u(P) <= u_{k+1},
 *                                                       v_l <= v(P) <= v_{l+1} } |
 *
 *   area in 2D (drop z and v), volume in 3D.  Because t(P) > 0 on the whole grid (the
 *   geometry requires s to exceed the grid's circumradius), each bound is the linear
 *   half-space  sdd*w(P) - u_k*t(P) >= 0  etc., through the source.
 *
 * How: 2D clips the pixel square by the two half-planes (Sutherland-Hodgman) and takes the
 * shoelace area.  3D clips the voxel box, face by face, by the four half-spaces, closes each
 * cut with a cap polygon, and sums pyramid volumes from an interior point.  Candidate
 * elements are those in the bounding box of the projected voxel corners (the pruning can be
 * switched off with all_elements = 1 to show that it loses nothing).  Forward p = W x and
 * back x = W^T p are explicit sums over those entries.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;            /* grid size (nz = 1 for 2D)                   */
    double a, b, c;            /* voxel sides in x, y, z                      */
    int n_views;               /* number of gantry angles                     */
    const double* angles;      /* gantry angles phi [rad], n_views of them    */
    double s;                  /* source - isocentre distance                 */
    double sdd;                /* source - detector distance (s + d)          */
    int nu, nv;                /* detector elements in u (and v; nv = 1 in 2D)*/
    double du, dv;             /* element sizes d_y, d_z                      */
    double u_off, v_off;       /* detector shifts                             */
} orc_geom;

/* ----------------------------------------------------------------------------------------
 * Geometry helpers (Notation and Setup; Appendix Eq. (tan beta), Eq. (z expr 1)).
 * ---------------------------------------------------------------------------------------- */
static double corner_u(const orc_geom* g, int k) { return (k - 0.5 * g->nu) * g->du + g->u_off; }
static double corner_v(const orc_geom* g, int l) { return (l - 0.5 * g->nv) * g->dv + g->v_off; }
static double grid_x(const orc_geom* g, int i) { return (i - 0.5 * g->nx) * g->a; }
static double grid_y(const orc_geom* g, int j) { return (j - 0.5 * g->ny) * g->b; }
static double grid_z(const orc_geom* g, int m) { return (m - 0.5 * g->nz) * g->c; }

/* The linear function  sdd*w(P) - u*t(P)  written as  cx*x + cy*y + c0:
 *   sdd*(-x sin + y cos) - u*(s - x cos - y sin)
 *   = x*(-sdd sin + u cos) + y*(sdd cos + u sin) - u s.
 * It is >= 0 exactly where u(P) >= u (for t(P) > 0). */
static void lateral_plane(const orc_geom* g, double cphi, double sphi, double u, double out[4]) {
    out[0] = -g->sdd * sphi + u * cphi;
    out[1] = g->sdd * cphi + u * sphi;
    out[2] = 0.0;
    out[3] = -u * g->s;
}
/* sdd*z - v*t(P) = x*(v cos) + y*(v sin) + z*sdd - v s;  >= 0 exactly where v(P) >= v. */
static void vertical_plane(const orc_geom* g, double cphi, double sphi, double v, double out[4]) {
    out[0] = v * cphi;
    out[1] = v * sphi;
    out[2] = g->sdd;
    out[3] = -v * g->s;
}

static double proj_u(const orc_geom* g, double cphi, double sphi, double x, double y) {
    double t = g->s - (x * cphi + y * sphi);
    return g->sdd * (-x * sphi + y * cphi) / t;
}
static double proj_v(const orc_geom* g, double cphi, double sphi, double x, double y, double z) {
    double t = g->s - (x * cphi + y * sphi);
    return g->sdd * z / t;
}

/* ----------------------------------------------------------------------------------------
 * 2D: Sutherland-Hodgman clip of a convex polygon by  f(P) = c0 x + c1 y + c3 >= 0.
 * ---------------------------------------------------------------------------------------- */
#define MAXV2 16
typedef struct { int n; double x[MAXV2], y[MAXV2]; } poly2;

static void poly2_clip(poly2* P, const double f[4]) {
    poly2 out; out.n = 0;
    for (int i = 0; i < P->n; ++i) {
        int j = (i + 1) % P->n;
        double xi = P->x[i], yi = P->y[i], xj = P->x[j], yj = P->y[j];
        double fi = f[0] * xi + f[1] * yi + f[3];
        double fj = f[0] * xj + f[1] * yj + f[3];
        if (fi >= 0.0) { out.x[out.n] = xi; out.y[out.n] = yi; out.n++; }
        if ((fi >= 0.0) != (fj >= 0.0)) {
            double tt = fi / (fi - fj);
            out.x[out.n] = xi + tt * (xj - xi);
            out.y[out.n] = yi + tt * (yj - yi);
            out.n++;
        }
    }
    *P = out;
}

static double poly2_area(const poly2* P) {
    double acc = 0.0;
    for (int i = 0; i < P->n; ++i) {
        int j = (i + 1) % P->n;
        acc += P->x[i] * P->y[j] - P->x[j] * P->y[i];
    }
    return 0.5 * fabs(acc);
}

/* Area of the rectangle [x0,x1]x[y0,y1] inside all the given half-planes (n of them). */
double orc_clip_area_2d(double x0, double x1, double y0, double y1, const double* planes, int n) {
    poly2 P; P.n = 4;
    P.x[0] = x0; P.y[0] = y0; P.x[1] = x1; P.y[1] = y0;
    P.x[2] = x1; P.y[2] = y1; P.x[3] = x0; P.y[3] = y1;
    for (int i = 0; i < n && P.n > 0; ++i) poly2_clip(&P, planes + 4 * i);
    return P.n >= 3 ? poly2_area(&P) : 0.0;
}

/* ----------------------------------------------------------------------------------------
 * 3D: convex polyhedron as a list of planar faces; clip by a half-space, close with a cap.
 * ---------------------------------------------------------------------------------------- */
#define MAXV3 24
#define MAXF3 16
typedef struct { int n; double p[MAXV3][3]; } poly3;
typedef struct { int nf; poly3 f[MAXF3]; } polyh;

static void polyh_box(polyh* H, double x0, double x1, double y0, double y1, double z0, double z1) {
    const double X[2] = {x0, x1}, Y[2] = {y0, y1}, Z[2] = {z0, z1};
    /* each face lists its 4 corners in cyclic order */
    static const int faces[6][4][3] = {
        {{0,0,0},{0,1,0},{0,1,1},{0,0,1}}, {{1,0,0},{1,0,1},{1,1,1},{1,1,0}},
        {{0,0,0},{0,0,1},{1,0,1},{1,0,0}}, {{0,1,0},{1,1,0},{1,1,1},{0,1,1}},
        {{0,0,0},{1,0,0},{1,1,0},{0,1,0}}, {{0,0,1},{0,1,1},{1,1,1},{1,0,1}}};
    H->nf = 6;
    for (int f = 0; f < 6; ++f) {
        H->f[f].n = 4;
        for (int v = 0; v < 4; ++v) {
            H->f[f].p[v][0] = X[faces[f][v][0]];
            H->f[f].p[v][1] = Y[faces[f][v][1]];
            H->f[f].p[v][2] = Z[faces[f][v][2]];
        }
    }
}

static double plane_eval(const double pl[4], const double* p) {
    return pl[0] * p[0] + pl[1] * p[1] + pl[2] * p[2] + pl[3];
}

/* Point where the segment p-q meets the plane.  Always interpolate from the
 * lexicographically smaller endpoint so that both faces sharing the edge produce the
 * bit-identical point. */
static void edge_cut(const double pl[4], const double* p, const double* q, double* out) {
    const double* a = p; const double* b = q;
    if (q[0] < p[0] || (q[0] == p[0] && (q[1] < p[1] || (q[1] == p[1] && q[2] < p[2])))) {
        a = q; b = p;
    }
    double fa = plane_eval(pl, a), fb = plane_eval(pl, b);
    double tt = fa / (fa - fb);
    for (int d = 0; d < 3; ++d) out[d] = a[d] + tt * (b[d] - a[d]);
}

static void polyh_clip(polyh* H, const double pl[4]) {
    polyh out; out.nf = 0;
    double cap[MAXV3 * 4][3]; int ncap = 0;
    int face_on_plane = 0;   /* a face lying in the plane already closes the cut */
    for (int f = 0; f < H->nf; ++f) {
        const poly3* F = &H->f[f];
        poly3 G; G.n = 0;
        int on = 1;
        for (int i = 0; i < F->n; ++i) if (plane_eval(pl, F->p[i]) != 0.0) { on = 0; break; }
        if (on) face_on_plane = 1;
        for (int i = 0; i < F->n; ++i) {
            int j = (i + 1) % F->n;
            double fi = plane_eval(pl, F->p[i]), fj = plane_eval(pl, F->p[j]);
            if (fi >= 0.0) {
                memcpy(G.p[G.n++], F->p[i], sizeof(double) * 3);
                if (fi == 0.0 && ncap < MAXV3 * 4) memcpy(cap[ncap++], F->p[i], sizeof(double) * 3);
            }
            if ((fi >= 0.0) != (fj >= 0.0)) {
                double q[3];
                edge_cut(pl, F->p[i], F->p[j], q);
                memcpy(G.p[G.n++], q, sizeof(double) * 3);
                if (ncap < MAXV3 * 4) memcpy(cap[ncap++], q, sizeof(double) * 3);
            }
        }
        if (G.n >= 3 && out.nf < MAXF3) out.f[out.nf++] = G;
    }
    /* cap polygon: unique cut points ordered by angle around their centroid in the plane */
    double uq[MAXV3 * 4][3]; int nu = 0;
    for (int i = 0; i < ncap; ++i) {
        int dup = 0;
        for (int j = 0; j < nu; ++j) {
            double dx = cap[i][0] - uq[j][0], dy = cap[i][1] - uq[j][1], dz = cap[i][2] - uq[j][2];
            if (dx * dx + dy * dy + dz * dz < 1e-26) { dup = 1; break; }
        }
        if (!dup) { memcpy(uq[nu++], cap[i], sizeof(double) * 3); }
    }
    if (!face_on_plane && nu >= 3 && out.nf < MAXF3 && nu <= MAXV3) {
        double cen[3] = {0, 0, 0};
        for (int i = 0; i < nu; ++i) for (int d = 0; d < 3; ++d) cen[d] += uq[i][d] / nu;
        /* in-plane basis e1, e2 orthogonal to the plane normal */
        double n[3] = {pl[0], pl[1], pl[2]};
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int d = 0; d < 3; ++d) n[d] /= nn;
        double r[3] = {1, 0, 0};
        if (fabs(n[0]) > 0.9) { r[0] = 0; r[1] = 1; }
        double e1[3] = {n[1] * r[2] - n[2] * r[1], n[2] * r[0] - n[0] * r[2], n[0] * r[1] - n[1] * r[0]};
        double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int d = 0; d < 3; ++d) e1[d] /= l1;
        double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
        double ang[MAXV3 * 4];
        for (int i = 0; i < nu; ++i) {
            double dx = uq[i][0] - cen[0], dy = uq[i][1] - cen[1], dz = uq[i][2] - cen[2];
            ang[i] = atan2(dx * e2[0] + dy * e2[1] + dz * e2[2], dx * e1[0] + dy * e1[1] + dz * e1[2]);
        }
        /* insertion sort by angle */
        for (int i = 1; i < nu; ++i) {
            double a0 = ang[i]; double p0[3]; memcpy(p0, uq[i], sizeof p0);
            int j = i - 1;
            while (j >= 0 && ang[j] > a0) { ang[j + 1] = ang[j]; memcpy(uq[j + 1], uq[j], sizeof p0); --j; }
            ang[j + 1] = a0; memcpy(uq[j + 1], p0, sizeof p0);
        }
        poly3* C = &out.f[out.nf++];
        C->n = nu;
        for (int i = 0; i < nu; ++i) memcpy(C->p[i], uq[i], sizeof(double) * 3);
    }
    *H = out;
}

/* Volume of a convex polyhedron: sum over faces of (1/3) * area * distance to an interior
 * point (the mean of all face vertices). */
static double polyh_volume(const polyh* H) {
    if (H->nf < 4) return 0.0;
    double c[3] = {0, 0, 0}; int cnt = 0;
    for (int f = 0; f < H->nf; ++f)
        for (int i = 0; i < H->f[f].n; ++i) { for (int d = 0; d < 3; ++d) c[d] += H->f[f].p[i][d]; cnt++; }
    for (int d = 0; d < 3; ++d) c[d] /= cnt;
    double vol = 0.0;
    for (int f = 0; f < H->nf; ++f) {
        const poly3* F = &H->f[f];
        double A[3] = {0, 0, 0};   /* vector area (Newell) */
        for (int i = 0; i < F->n; ++i) {
            const double* p = F->p[i]; const double* q = F->p[(i + 1) % F->n];
            A[0] += p[1] * q[2] - p[2] * q[1];
            A[1] += p[2] * q[0] - p[0] * q[2];
            A[2] += p[0] * q[1] - p[1] * q[0];
        }
        double h = (F->p[0][0] - c[0]) * A[0] + (F->p[0][1] - c[1]) * A[1] + (F->p[0][2] - c[2]) * A[2];
        vol += fabs(h) / 6.0;   /* (1/3) * |A|/2 ... A above is twice the vector area */
    }
    return vol;
}

/* Volume of the box inside all n half-spaces (planes given as 4 doubles each). */
double orc_clip_volume_3d(double x0, double x1, double y0, double y1, double z0, double z1,
                          const double* planes, int n) {
    polyh H; polyh_box(&H, x0, x1, y0, y1, z0, z1);
    for (int i = 0; i < n && H.nf > 0; ++i) polyh_clip(&H, planes + 4 * i);
    return polyh_volume(&H);
}

/* ----------------------------------------------------------------------------------------
 * Entries of W.
 * ---------------------------------------------------------------------------------------- */
/* Index range [k0, k1] of elements whose interval can meet [umin, umax]. */
static void elem_range(double umin, double umax, double c0, double step, int n, int* k0, int* k1) {
    double a0 = floor((umin - c0) / step) - 1.0, a1 = floor((umax - c0) / step) + 1.0;
    if (a0 < 0.0) a0 = 0.0;
    if (a1 > n - 1) a1 = n - 1;
    *k0 = (int)a0; *k1 = (int)a1;
}

/* All nonzero 2D entries of pixel (ix, iy) in view `view`.  Writes element indices and
 * areas; returns the count (<= cap). */
int orc2d_entries(const orc_geom* g, int view, int ix, int iy, int all_elements,
                  int* k_out, double* w_out, int cap) {
    double phi = g->angles[view], cphi = cos(phi), sphi = sin(phi);
    double x0 = grid_x(g, ix), x1 = grid_x(g, ix + 1), y0 = grid_y(g, iy), y1 = grid_y(g, iy + 1);
    int k0 = 0, k1 = g->nu - 1;
    if (!all_elements) {
        double us[4] = {proj_u(g, cphi, sphi, x0, y0), proj_u(g, cphi, sphi, x1, y0),
                        proj_u(g, cphi, sphi, x1, y1), proj_u(g, cphi, sphi, x0, y1)};
        double umin = us[0], umax = us[0];
        for (int i = 1; i < 4; ++i) { umin = fmin(umin, us[i]); umax = fmax(umax, us[i]); }
        elem_range(umin, umax, corner_u(g, 0), g->du, g->nu, &k0, &k1);
        if (umax < corner_u(g, 0) || umin > corner_u(g, g->nu)) return 0;
    }
    int cnt = 0;
    for (int k = k0; k <= k1; ++k) {
        double pl[8];
        lateral_plane(g, cphi, sphi, corner_u(g, k), pl);          /* u(P) >= u_k      */
        lateral_plane(g, cphi, sphi, corner_u(g, k + 1), pl + 4);  /* u(P) <= u_{k+1}  */
        for (int d = 0; d < 4; ++d) pl[4 + d] = -pl[4 + d];
        double w = orc_clip_area_2d(x0, x1, y0, y1, pl, 2);
        if (w > 0.0 && cnt < cap) { k_out[cnt] = k; w_out[cnt] = w; cnt++; }
    }
    return cnt;
}

/* p[view_sel][nu] = W x for the selected views (x is [ny][nx]). */
void orc2d_forward(const orc_geom* g, const double* x, double* p, const int* views, int nsel) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int vi = 0; vi < nsel; ++vi) {
        double* prow = p + (size_t)vi * g->nu;
        for (int k = 0; k < g->nu; ++k) prow[k] = 0.0;
        int ks[64]; double ws[64];
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                double xv = x[(size_t)iy * g->nx + ix];
                int n = orc2d_entries(g, views[vi], ix, iy, 0, ks, ws, 64);
                for (int e = 0; e < n; ++e) prow[ks[e]] += ws[e] * xv;
            }
    }
}

/* x[ny][nx] = W^T p over the selected views (p is [nsel][nu]). */
void orc2d_back(const orc_geom* g, const double* p, double* x, const int* views, int nsel) {
    #pragma omp parallel for schedule(dynamic, 1)
    for (int iy = 0; iy < g->ny; ++iy) {
        int ks[64]; double ws[64];
        for (int ix = 0; ix < g->nx; ++ix) {
            double acc = 0.0;
            for (int vi = 0; vi < nsel; ++vi) {
                int n = orc2d_entries(g, views[vi], ix, iy, 0, ks, ws, 64);
                for (int e = 0; e < n; ++e) acc += ws[e] * p[(size_t)vi * g->nu + ks[e]];
            }
            x[(size_t)iy * g->nx + ix] = acc;
        }
    }
}

/* One detector value p[view][k] = sum_j W x_j, evaluated on its own (for sampled checks). */
double orc2d_forward_element(const orc_geom* g, const double* x, int view, int k) {
    double acc = 0.0;
    int ks[64]; double ws[64];
    for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
            int n = orc2d_entries(g, view, ix, iy, 0, ks, ws, 64);
            for (int e = 0; e < n; ++e) if (ks[e] == k) acc += ws[e] * x[(size_t)iy * g->nx + ix];
        }
    return acc;
}

/* ---------------------------------------------------------------------------------------- */

/* All nonzero 3D entries of voxel (ix,iy,iz) in view `view`: element (k,l) is written as
 * k + nu*l.  Returns the count (<= cap). */
int orc3d_entries(const orc_geom* g, int view, int ix, int iy, int iz, int all_elements,
                  int* kl_out, double* w_out, int cap) {
    double phi = g->angles[view], cphi = cos(phi), sphi = sin(phi);
    double x0 = grid_x(g, ix), x1 = grid_x(g, ix + 1), y0 = grid_y(g, iy), y1 = grid_y(g, iy + 1);
    double z0 = grid_z(g, iz), z1 = grid_z(g, iz + 1);
    int k0 = 0, k1 = g->nu - 1, l0 = 0, l1 = g->nv - 1;
    if (!all_elements) {
        double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
        for (int c = 0; c < 8; ++c) {
            double X = (c & 1) ? x1 : x0, Y = (c & 2) ? y1 : y0, Z = (c & 4) ? z1 : z0;
            double u = proj_u(g, cphi, sphi, X, Y), v = proj_v(g, cphi, sphi, X, Y, Z);
            umin = fmin(umin, u); umax = fmax(umax, u); vmin = fmin(vmin, v); vmax = fmax(vmax, v);
        }
        if (umax < corner_u(g, 0) || umin > corner_u(g, g->nu)) return 0;
        if (vmax < corner_v(g, 0) || vmin > corner_v(g, g->nv)) return 0;
        elem_range(umin, umax, corner_u(g, 0), g->du, g->nu, &k0, &k1);
        elem_range(vmin, vmax, corner_v(g, 0), g->dv, g->nv, &l0, &l1);
    }
    int cnt = 0;
    for (int k = k0; k <= k1; ++k) {
        double pl[16];
        lateral_plane(g, cphi, sphi, corner_u(g, k), pl);
        lateral_plane(g, cphi, sphi, corner_u(g, k + 1), pl + 4);
        for (int d = 0; d < 4; ++d) pl[4 + d] = -pl[4 + d];
        /* clip by the two lateral planes once, then by each row's two planes */
        polyh Hk; polyh_box(&Hk, x0, x1, y0, y1, z0, z1);
        polyh_clip(&Hk, pl);
        if (Hk.nf > 0) polyh_clip(&Hk, pl + 4);
        if (Hk.nf < 4 || polyh_volume(&Hk) <= 0.0) continue;
        for (int l = l0; l <= l1; ++l) {
            vertical_plane(g, cphi, sphi, corner_v(g, l), pl + 8);
            vertical_plane(g, cphi, sphi, corner_v(g, l + 1), pl + 12);
            for (int d = 0; d < 4; ++d) pl[12 + d] = -pl[12 + d];
            polyh H = Hk;
            polyh_clip(&H, pl + 8);
            if (H.nf > 0) polyh_clip(&H, pl + 12);
            double w = polyh_volume(&H);
            if (w > 0.0 && cnt < cap) { kl_out[cnt] = k + g->nu * l; w_out[cnt] = w; cnt++; }
        }
    }
    return cnt;
}

#define CAP3 256

/* p[view_sel][nv][nu] = W x for the selected views (x is [nz][ny][nx]). */
void orc3d_forward(const orc_geom* g, const double* x, double* p, const int* views, int nsel) {
    size_t plane = (size_t)g->nu * g->nv;
    for (size_t i = 0; i < plane * nsel; ++i) p[i] = 0.0;
    for (int vi = 0; vi < nsel; ++vi) {
        double* prow = p + (size_t)vi * plane;
        #pragma omp parallel
        {
            double* loc = (double*)calloc(plane, sizeof(double));
            int kls[CAP3]; double ws[CAP3];
            #pragma omp for schedule(dynamic, 1) collapse(2)
            for (int iz = 0; iz < g->nz; ++iz)
                for (int iy = 0; iy < g->ny; ++iy)
                    for (int ix = 0; ix < g->nx; ++ix) {
                        double xv = x[((size_t)iz * g->ny + iy) * g->nx + ix];
                        if (xv == 0.0) continue;   /* a zero voxel adds nothing */
                        int n = orc3d_entries(g, views[vi], ix, iy, iz, 0, kls, ws, CAP3);
                        for (int e = 0; e < n; ++e) loc[kls[e]] += ws[e] * xv;
                    }
            #pragma omp critical
            for (size_t i = 0; i < plane; ++i) prow[i] += loc[i];
            free(loc);
        }
    }
}

/* x[nz][ny][nx] = W^T p over the selected views (p is [nsel][nv][nu]). */
void orc3d_back(const orc_geom* g, const double* p, double* x, const int* views, int nsel) {
    size_t plane = (size_t)g->nu * g->nv;
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int iz = 0; iz < g->nz; ++iz)
        for (int iy = 0; iy < g->ny; ++iy) {
            int kls[CAP3]; double ws[CAP3];
            for (int ix = 0; ix < g->nx; ++ix) {
                double acc = 0.0;
                for (int vi = 0; vi < nsel; ++vi) {
                    int n = orc3d_entries(g, views[vi], ix, iy, iz, 0, kls, ws, CAP3);
                    for (int e = 0; e < n; ++e) acc += ws[e] * p[(size_t)vi * plane + kls[e]];
                }
                x[((size_t)iz * g->ny + iy) * g->nx + ix] = acc;
            }
        }
}

/* x = W^T p on the z-slab iz0 <= iz < iz1 only (x is [iz1 - iz0][ny][nx], p is
 * [nsel][nv][nu]): the same sums as orc3d_back for those voxels.  Returns the number of
 * nonzero entries applied (for rate accounting). */
long orc3d_back_slab(const orc_geom* g, const double* p, double* x, const int* views, int nsel,
                     int iz0, int iz1) {
    size_t plane = (size_t)g->nu * g->nv;
    long total = 0;
    int nzs = iz1 - iz0;
    #pragma omp parallel for schedule(dynamic, 1) collapse(2) reduction(+:total)
    for (int dz = 0; dz < nzs; ++dz)
        for (int iy = 0; iy < g->ny; ++iy) {
            int kls[CAP3]; double ws[CAP3];
            for (int ix = 0; ix < g->nx; ++ix) {
                double acc = 0.0;
                for (int vi = 0; vi < nsel; ++vi) {
                    int n = orc3d_entries(g, views[vi], ix, iy, iz0 + dz, 0, kls, ws, CAP3);
                    for (int e = 0; e < n; ++e) acc += ws[e] * p[(size_t)vi * plane + kls[e]];
                    total += n;
                }
                x[((size_t)dz * g->ny + iy) * g->nx + ix] = acc;
            }
        }
    return total;
}

/* One back-projected value x_j = sum over the selected views of W^T p (sampled checks). */
double orc3d_back_voxel(const orc_geom* g, const double* p, const int* views, int nsel,
                        int ix, int iy, int iz) {
    size_t plane = (size_t)g->nu * g->nv;
    double acc = 0.0;
    int kls[CAP3]; double ws[CAP3];
    for (int vi = 0; vi < nsel; ++vi) {
        int n = orc3d_entries(g, views[vi], ix, iy, iz, 0, kls, ws, CAP3);
        for (int e = 0; e < n; ++e) acc += ws[e] * p[(size_t)vi * plane + kls[e]];
    }
    return acc;
}

/* One detector value p[view][l][k] = sum_j W x_j.  Voxel columns (ix,iy) whose top view
 * cannot reach element k are skipped, then voxels whose v-range misses row l. */
double orc3d_forward_element(const orc_geom* g, const double* x, int view, int k, int l) {
    double phi = g->angles[view], cphi = cos(phi), sphi = sin(phi);
    double uk0 = corner_u(g, k), uk1 = corner_u(g, k + 1);
    double vl0 = corner_v(g, l), vl1 = corner_v(g, l + 1);
    double total = 0.0;
    #pragma omp parallel for schedule(dynamic, 4) reduction(+:total)
    for (int iy = 0; iy < g->ny; ++iy) {
        int kls[CAP3]; double ws[CAP3];
        for (int ix = 0; ix < g->nx; ++ix) {
            double x0 = grid_x(g, ix), x1 = grid_x(g, ix + 1), y0 = grid_y(g, iy), y1 = grid_y(g, iy + 1);
            double umin = 1e300, umax = -1e300, tmin = 1e300, tmax = -1e300;
            for (int c = 0; c < 4; ++c) {
                double X = (c & 1) ? x1 : x0, Y = (c & 2) ? y1 : y0;
                double u = proj_u(g, cphi, sphi, X, Y);
                double t = g->s - (X * cphi + Y * sphi);
                umin = fmin(umin, u); umax = fmax(umax, u); tmin = fmin(tmin, t); tmax = fmax(tmax, t);
            }
            if (umax < uk0 || umin > uk1) continue;
            for (int iz = 0; iz < g->nz; ++iz) {
                double z0 = grid_z(g, iz), z1 = grid_z(g, iz + 1);
                double va = g->sdd * z0 / tmin, vb = g->sdd * z0 / tmax;
                double vc = g->sdd * z1 / tmin, vd = g->sdd * z1 / tmax;
                double vmin = fmin(fmin(va, vb), fmin(vc, vd)), vmax = fmax(fmax(va, vb), fmax(vc, vd));
                if (vmax < vl0 || vmin > vl1) continue;
                double xv = x[((size_t)iz * g->ny + iy) * g->nx + ix];
                if (xv == 0.0) continue;
                int n = orc3d_entries(g, view, ix, iy, iz, 0, kls, ws, CAP3);
                for (int e = 0; e < n; ++e) if (kls[e] == k + g->nu * l) total += ws[e] * xv;
            }
        }
    }
    return total;
}

/* Explicit sparse W (COO) for small problems.  Row index = (vi*nv + l)*nu + k over the
 * selected views, column index = voxel index.  Returns the number of entries written, or
 * -1 if `cap` was too small. */
long orc3d_coo(const orc_geom* g, const int* views, int nsel, int* rows, int* cols, double* vals, long cap) {
    long cnt = 0;
    int kls[CAP3]; double ws[CAP3];
    for (int vi = 0; vi < nsel; ++vi)
        for (int iz = 0; iz < g->nz; ++iz)
            for (int iy = 0; iy < g->ny; ++iy)
                for (int ix = 0; ix < g->nx; ++ix) {
                    int n = orc3d_entries(g, views[vi], ix, iy, iz, 0, kls, ws, CAP3);
                    for (int e = 0; e < n; ++e) {
                        if (cnt >= cap) return -1;
                        rows[cnt] = vi * g->nu * g->nv + kls[e];
                        cols[cnt] = (iz * g->ny + iy) * g->nx + ix;
                        vals[cnt] = ws[e];
                        cnt++;
                    }
                }
    return cnt;
}

/* Number of nonzero 2D entries over the selected views (for rate accounting). */
long orc2d_count(const orc_geom* g, const int* views, int nsel) {
    long total = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(+:total)
    for (int vi = 0; vi < nsel; ++vi) {
        int ks[64]; double ws[64];
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix)
                total += orc2d_entries(g, views[vi], ix, iy, 0, ks, ws, 64);
    }
    return total;
}

long orc2d_coo(const orc_geom* g, const int* views, int nsel, int* rows, int* cols, double* vals, long cap) {
    long cnt = 0;
    int ks[64]; double ws[64];
    for (int vi = 0; vi < nsel; ++vi)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                int n = orc2d_entries(g, views[vi], ix, iy, 0, ks, ws, 64);
                for (int e = 0; e < n; ++e) {
                    if (cnt >= cap) return -1;
                    rows[cnt] = vi * g->nu + ks[e];
                    cols[cnt] = iy * g->nx + ix;
                    vals[cnt] = ws[e];
                    cnt++;
                }
            }
    return cnt;
}

/* ----------------------------------------------------------------------------------------
 * Line-based comparator matrices (Section "Related work": line-integration methods; Section
 * "Computational complexity": several lines per detector element, averaged).  A ray goes from
 * the source S to the detector point D = S - sdd e_s + u e_u + w e_z of view phi; an
 * element's value is the mean over `lines` rays to u = u_k + (m + 1/2) du / lines (and, in 3D,
 * lines x lines rays with w = v_l + (n + 1/2) dv / lines).
 *   Siddon: the line integral of the piecewise-constant image, i.e. the sum over voxels of the
 *     length of the ray inside each, found as in Siddon's method: every crossing parameter of
 *     the ray with a grid plane, sorted; between consecutive crossings the ray is inside the
 *     voxel that contains the midpoint.
 *   Joseph: the ray sampled at the centre plane of every voxel slice along its major axis,
 *     the image interpolated (linearly in 2D, bilinearly in 3D, zero outside the grid) between
 *     the voxel centres of that slice, each sample weighted by the ray length per slice.
 * 2D when nz == 1 and nv == 1 (z and w ignored).
 * ---------------------------------------------------------------------------------------- */
static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* visit(voxel index, weight) for every voxel the ray meets; ctx passed through */
typedef void (*ray_visit)(void* ctx, size_t vox, double w);

static void ray_siddon(const orc_geom* g, const double S[3], const double d[3], int is3d, ray_visit f, void* ctx) {
    double lo[3] = {grid_x(g, 0), grid_y(g, 0), grid_z(g, 0)};
    double hi[3] = {grid_x(g, g->nx), grid_y(g, g->ny), grid_z(g, g->nz)};
    int n[3] = {g->nx, g->ny, g->nz};
    double h[3] = {g->a, g->b, g->c};
    int dims = is3d ? 3 : 2;
    int cap = g->nx + g->ny + (is3d ? g->nz : 0) + 8;
    double* al = (double*)malloc(sizeof(double) * cap);
    int na = 0;
    al[na++] = 0.0;
    al[na++] = 1.0;
    for (int a = 0; a < dims; ++a) {
        if (d[a] == 0.0) continue;
        for (int i = 0; i <= n[a]; ++i) {
            double t = (lo[a] + i * h[a] - S[a]) / d[a];
            if (t > 0.0 && t < 1.0 && na < cap) al[na++] = t;
        }
    }
    qsort(al, na, sizeof(double), cmp_double);
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + (is3d ? d[2] * d[2] : 0.0));
    for (int m = 0; m + 1 < na; ++m) {
        double t0 = al[m], t1 = al[m + 1];
        if (!(t1 > t0)) continue;
        double tm = 0.5 * (t0 + t1);
        int idx[3] = {0, 0, 0};
        int inside = 1;
        for (int a = 0; a < dims; ++a) {
            double q = S[a] + tm * d[a];
            if (q < lo[a] || q > hi[a]) { inside = 0; break; }
            int i = (int)floor((q - lo[a]) / h[a]);
            if (i < 0 || i >= n[a]) { inside = 0; break; }
            idx[a] = i;
        }
        if (!inside) continue;
        f(ctx, ((size_t)idx[2] * g->ny + idx[1]) * g->nx + idx[0], (t1 - t0) * len);
    }
    free(al);
}

static void ray_joseph(const orc_geom* g, const double S[3], const double d[3], int is3d, ray_visit f, void* ctx) {
    double org[3] = {grid_x(g, 0), grid_y(g, 0), grid_z(g, 0)};
    double h[3] = {g->a, g->b, g->c};
    int n[3] = {g->nx, g->ny, g->nz};
    int m = 0;
    if (fabs(d[1]) > fabs(d[m])) m = 1;
    if (is3d && fabs(d[2]) > fabs(d[m])) m = 2;
    int others[2], no = 0;
    for (int a = 0; a < (is3d ? 3 : 2); ++a) if (a != m) others[no++] = a;
    double len = sqrt(d[0] * d[0] + d[1] * d[1] + (is3d ? d[2] * d[2] : 0.0));
    double wstep = h[m] * len / fabs(d[m]);
    for (int i = 0; i < n[m]; ++i) {
        double cm = org[m] + (i + 0.5) * h[m];
        double t = (cm - S[m]) / d[m];
        if (t < 0.0 || t > 1.0) continue;
        /* position of the sample in voxel-centre units along the other axes */
        double pos[2] = {0.0, 0.0};
        int base[2] = {0, 0};
        for (int o = 0; o < no; ++o) {
            int a = others[o];
            pos[o] = (S[a] + t * d[a] - org[a]) / h[a] - 0.5;
            base[o] = (int)floor(pos[o]);
        }
        int corners = no == 2 ? 4 : 2;
        for (int cidx = 0; cidx < corners; ++cidx) {
            int idx[3] = {0, 0, 0};
            double w = wstep;
            int ok = 1;
            idx[m] = i;
            for (int o = 0; o < no; ++o) {
                int bit = (cidx >> o) & 1;
                int j = base[o] + bit;
                double fr = pos[o] - base[o];
                w *= bit ? fr : 1.0 - fr;
                if (j < 0 || j >= n[others[o]]) ok = 0;
                idx[others[o]] = j;
            }
            if (ok && w != 0.0) f(ctx, ((size_t)idx[2] * g->ny + idx[1]) * g->nx + idx[0], w);
        }
    }
}

typedef struct { const double* x; double acc; } fwd_ctx;
static void fwd_visit(void* c, size_t vox, double w) { fwd_ctx* k = (fwd_ctx*)c; k->acc += w * k->x[vox]; }
typedef struct { double* x; double val; } back_ctx;
static void back_visit(void* c, size_t vox, double w) { back_ctx* k = (back_ctx*)c; k->x[vox] += w * k->val; }

static void element_rays(const orc_geom* g, int model, int lines, int view, int k, int l, ray_visit f, void* ctx) {
    int is3d = !(g->nz == 1 && g->nv == 1);
    double phi = g->angles[view], c = cos(phi), sn = sin(phi);
    int lz = is3d ? lines : 1;
    for (int mz = 0; mz < lz; ++mz) {
        double w = is3d ? corner_v(g, l) + (mz + 0.5) / lz * g->dv : 0.0;
        for (int mu = 0; mu < lines; ++mu) {
            double u = corner_u(g, k) + (mu + 0.5) / lines * g->du;
            double S[3] = {g->s * c, g->s * sn, 0.0};
            double d[3] = {-g->sdd * c - u * sn, -g->sdd * sn + u * c, w};
            if (model == 1) ray_siddon(g, S, d, is3d, f, ctx);
            else ray_joseph(g, S, d, is3d, f, ctx);
        }
    }
}

/* p[vi][nv][nu] = mean over each element's rays of the line integrals of x */
void orc_line_forward(const orc_geom* g, int model, int lines, const double* x, double* p, const int* views, int nsel) {
    int is3d = !(g->nz == 1 && g->nv == 1);
    double norm = 1.0 / (lines * (is3d ? lines : 1));
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int vi = 0; vi < nsel; ++vi)
        for (int l = 0; l < g->nv; ++l)
            for (int k = 0; k < g->nu; ++k) {
                fwd_ctx ctx = {x, 0.0};
                element_rays(g, model, lines, views[vi], k, l, fwd_visit, &ctx);
                p[((size_t)vi * g->nv + l) * g->nu + k] = ctx.acc * norm;
            }
}

/* x = the adjoint of orc_line_forward applied to p (serial: plain sums) */
void orc_line_back(const orc_geom* g, int model, int lines, const double* p, double* x, const int* views, int nsel) {
    int is3d = !(g->nz == 1 && g->nv == 1);
    double norm = 1.0 / (lines * (is3d ? lines : 1));
    size_t nvox = (size_t)g->nx * g->ny * g->nz;
    for (size_t i = 0; i < nvox; ++i) x[i] = 0.0;
    for (int vi = 0; vi < nsel; ++vi)
        for (int l = 0; l < g->nv; ++l)
            for (int k = 0; k < g->nu; ++k) {
                back_ctx ctx = {x, p[((size_t)vi * g->nv + l) * g->nu + k] * norm};
                if (ctx.val != 0.0) element_rays(g, model, lines, views[vi], k, l, back_visit, &ctx);
            }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

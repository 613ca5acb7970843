/* Runs the FP64 oracle on small 2D and 3D geometries under AddressSanitizer and
 * UndefinedBehaviorSanitizer (built by tests/test_oracle_sanitized.py): forward, back,
 * single entries and the COO export, with the adjoint identity <W x, y> = <x, W^T y> as a
 * sanity check.  Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

typedef struct {
    int nx, ny, nz;
    double a, b, c;
    int n_views;
    const double* angles;
    double s;
    double sdd;
    int nu, nv;
    double du, dv;
    double u_off, v_off;
} orc_geom;

void orc2d_forward(const orc_geom* g, const double* x, double* p, const int* views, int nsel);
void orc2d_back(const orc_geom* g, const double* p, double* x, const int* views, int nsel);
void orc3d_forward(const orc_geom* g, const double* x, double* p, const int* views, int nsel);
void orc3d_back(const orc_geom* g, const double* p, double* x, const int* views, int nsel);
long orc3d_coo(const orc_geom* g, const int* views, int nsel, int* rows, int* cols, double* vals, long cap);
long orc2d_coo(const orc_geom* g, const int* views, int nsel, int* rows, int* cols, double* vals, long cap);

static double urand(unsigned* s) { *s = *s * 1664525u + 1013904223u; return (*s >> 8) / 16777216.0; }

static int check(const char* what, const orc_geom* g, int dim) {
    const int nvox = g->nx * g->ny * g->nz, nsino = g->n_views * g->nu * g->nv;
    double* x = malloc(sizeof(double) * nvox);
    double* y = malloc(sizeof(double) * nsino);
    double* p = calloc(nsino, sizeof(double));
    double* b = calloc(nvox, sizeof(double));
    int* views = malloc(sizeof(int) * g->n_views);
    for (int v = 0; v < g->n_views; ++v) views[v] = v;
    unsigned s = 12345u;
    for (int i = 0; i < nvox; ++i) x[i] = urand(&s);
    for (int i = 0; i < nsino; ++i) y[i] = urand(&s);
    if (dim == 2) { orc2d_forward(g, x, p, views, g->n_views); orc2d_back(g, y, b, views, g->n_views); }
    else { orc3d_forward(g, x, p, views, g->n_views); orc3d_back(g, y, b, views, g->n_views); }
    double lhs = 0.0, rhs = 0.0, np = 0.0;
    for (int i = 0; i < nsino; ++i) { lhs += p[i] * y[i]; np += p[i] * p[i]; }
    for (int i = 0; i < nvox; ++i) rhs += x[i] * b[i];
    const long cap = (long)nvox * nsino;
    int* rows = malloc(sizeof(int) * cap);
    int* cols = malloc(sizeof(int) * cap);
    double* vals = malloc(sizeof(double) * cap);
    const long n = dim == 2 ? orc2d_coo(g, views, g->n_views, rows, cols, vals, cap)
                            : orc3d_coo(g, views, g->n_views, rows, cols, vals, cap);
    int ok = isfinite(lhs) && isfinite(rhs) && np > 0.0 && fabs(lhs - rhs) <= 1e-12 * fabs(lhs) && n > 0;
    printf("%s: <Wx,y> = %.15g, <x,W^T y> = %.15g, nnz %ld: %s\n", what, lhs, rhs, n, ok ? "ok" : "FAIL");
    free(x); free(y); free(p); free(b); free(rows); free(cols); free(vals); free(views);
    return ok;
}

int main(void) {
    double ang2[7] = {0.0, 0.3, 1.5707963267948966, 2.2, 3.141592653589793, 4.0, 0.7853981633974483};
    orc_geom g2 = {7, 5, 1, 1.2, 0.9, 1.0, 7, ang2, 14.0, 23.0, 12, 1, 1.1, 1.0, 0.3, 0.0};
    orc_geom g3 = {4, 5, 3, 1.1, 0.9, 1.2, 7, ang2, 14.0, 23.0, 9, 7, 1.2, 1.05, -0.2, 0.35};
    int ok = check("2d", &g2, 2);
    ok &= check("3d", &g3, 3);
    return ok ? 0 : 1;
}

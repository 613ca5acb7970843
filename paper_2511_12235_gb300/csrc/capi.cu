// capi.cu -- the C ABI (include/csm.h): geometry validation and device tables, dispatch of
// forward / back to the 2D and 3D kernels, status reporting.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <new>

#include "csm_internal.cuh"

namespace csm {

static thread_local char g_cuda_err[256] = {0};

void set_cuda_error(cudaError_t e) {
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

csm_status check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return CSM_ECUDA;
    }
    return CSM_OK;
}

Geo make_geo(const csm_geom_s* g) {
    Geo o;
    o.nx = g->nx; o.ny = g->ny; o.nz = g->nz; o.nu = g->nu; o.nv = g->nv; o.n_views = g->n_views;
    o.a_d = g->a; o.b_d = g->b; o.c_d = g->c; o.s_d = g->s; o.sdd_d = g->sdd;
    o.du_d = g->du; o.dv_d = g->dv;
    o.u0_d = (-0.5 * g->nu) * g->du + g->u_off;
    o.v0_d = (-0.5 * g->nv) * g->dv + g->v_off;
    o.x0_d = -0.5 * g->nx * g->a; o.y0_d = -0.5 * g->ny * g->b; o.z0_d = -0.5 * g->nz * g->c;
    o.a = (float)o.a_d; o.b = (float)o.b_d; o.c = (float)o.c_d; o.s = (float)o.s_d;
    o.sdd = (float)o.sdd_d; o.du = (float)o.du_d; o.dv = (float)o.dv_d; o.u0 = (float)o.u0_d;
    o.v0 = (float)o.v0_d; o.x0 = (float)o.x0_d; o.y0 = (float)o.y0_d; o.z0 = (float)o.z0_d;
    o.idu_d = 1.0 / o.du_d; o.idv_d = 1.0 / o.dv_d; o.ic_d = 1.0 / o.c_d;
    o.idu = (float)o.idu_d; o.idv = (float)o.idv_d; o.ic = (float)o.ic_d;
    o.qmax_d = std::max(fabs(o.v0_d), fabs(o.v0_d + g->nv * o.dv_d)) / o.sdd_d;
    o.dq_d = o.dv_d / o.sdd_d;
    o.qmax = (float)o.qmax_d; o.dq = (float)o.dq_d;
    o.axis_sigma = g->t.axis_sigma; o.cs_f = g->t.cs_f; o.cs_d = g->t.cs_d;
    o.line_fx = g->t.line_fx; o.line_d = g->t.line_d; o.inv_f = g->t.inv_f; o.inv_d = g->t.inv_d;
    o.wrange = g->t.wrange; o.rowq_f = g->t.rowq_f; o.rowq_d = g->t.rowq_d;
    o.rowq4 = g->t.rowq4;
    o.colt_fx = g->t.colt_fx;
    o.colt_d = g->t.colt_d;
    const size_t nel = (size_t)g->n_views * g->nv * g->nu;
    o.ew_f = g->w_block ? (const float*)g->w_block : nullptr;
    o.ew_d = g->w_block ? (const double*)((const char*)g->w_block + ((nel * sizeof(float) + 255) & ~(size_t)255)) : nullptr;
    return o;
}

// ---------------------------------------------------------------------------------------
// Host construction of the per-view tables, FP64.
//
// The ray through detector corner u is { P : sdd w(P) - u t(P) = 0 } with
// w = -x sin + y cos and t = s - x cos - y sin (Appendix Eq. (tan beta): tan beta = u/sdd;
// Eq. (y expression) / Eq. (x expression) write the same ray as y(x) or x(y)).
//   walking x:  y(x) = (u s + x (sdd sin - u cos)) / (sdd cos + u sin)
//   walking y:  x(y) = (u s - y (sdd cos + u sin)) / (u cos - sdd sin)
// A view walks the axis along which the source lies outside the grid's extent (then u is
// monotone along every cross line, so the corner lines are ordered by k), preferring the
// axis closer to the central ray (the paper's rotation of the frame by pi/2, Section
// "The Two-dimensional Case").
// ---------------------------------------------------------------------------------------
static const double kFar = 1073741824.0;  // 2^30 cells: "entirely outside the grid"

static csm_status build_tables(csm_geom_s* g) {
    const int V = g->n_views, nu = g->nu, nv = g->nv;
    const double D = g->sdd, s = g->s;
    const double hx = 0.5 * g->nx * g->a, hy = 0.5 * g->ny * g->b;
    const double x0 = -hx, y0 = -hy;
    std::vector<int> axis_sigma(2 * V);
    std::vector<float> cs_f(2 * V);
    std::vector<double> cs_d(2 * V);
    std::vector<long long> line_fx(2 * (size_t)V * (nu + 1));
    std::vector<double> line_d(2 * (size_t)V * (nu + 1));
    std::vector<float> inv_f((size_t)V * (nu + 1));
    std::vector<double> inv_d((size_t)V * (nu + 1));
    std::vector<int> wrange(2 * (size_t)V * nu);
    std::vector<float> rowq_f(nv + 1);
    std::vector<double> rowq_d(nv + 1);

    for (int v = 0; v < V; ++v) {
        const double c = cos(g->angles[v]), sn = sin(g->angles[v]);
        cs_f[2 * v] = (float)c; cs_f[2 * v + 1] = (float)sn;
        cs_d[2 * v] = c; cs_d[2 * v + 1] = sn;
        const double m0 = s * fabs(c) - hx, m1 = s * fabs(sn) - hy;
        int axis;
        if (fabs(c) >= fabs(sn)) axis = m0 > 0 ? 0 : 1;
        else axis = m1 > 0 ? 1 : 0;
        const double margin = axis == 0 ? m0 : m1;
        if (!(margin > 0)) return CSM_EGEOM;
        // u increases with y along x = const iff s cos - x > 0 (axis 0);
        // u increases with x along y = const iff y - s sin > 0 (axis 1).
        const int sigma = axis == 0 ? (c > 0 ? 1 : -1) : (sn < 0 ? 1 : -1);
        axis_sigma[2 * v] = axis; axis_sigma[2 * v + 1] = sigma;
        const int nw = axis == 0 ? g->nx : g->ny;
        const int nc = axis == 0 ? g->ny : g->nx;
        const double hw = axis == 0 ? g->a : g->b, hc = axis == 0 ? g->b : g->a;
        // grid's u-range (for rays that never cross the walked extent)
        double umin = 1e300, umax = -1e300;
        for (int cc = 0; cc < 4; ++cc) {
            double X = (cc & 1) ? hx : -hx, Y = (cc & 2) ? hy : -hy;
            double t = s - X * c - Y * sn;
            double u = D * (-X * sn + Y * c) / t;
            umin = std::min(umin, u); umax = std::max(umax, u);
        }
        std::vector<double> P0(nu + 1), DL(nu + 1);
        for (int k = 0; k <= nu; ++k) {
            const double u = (k - 0.5 * nu) * g->du + g->u_off;
            double den, p0, dl;
            if (axis == 0) {
                den = D * c + u * sn;
                p0 = ((u * s + x0 * (D * sn - u * c)) / den - y0) / hc;
                dl = (D * sn - u * c) / den * hw / hc;
            } else {
                den = u * c - D * sn;
                p0 = ((u * s - y0 * (D * c + u * sn)) / den - x0) / hc;
                dl = -(D * c + u * sn) / den * hw / hc;
            }
            const double pend = p0 + nw * dl;
            bool far_lo = false, far_hi = false;
            if (!(fabs(den) > 1e-9 * (D + fabs(u))) || !std::isfinite(p0) || !std::isfinite(dl)) {
                // the ray never crosses the walked extent: all pixels lie on one side
                bool all_below_u = u >= umax;   // every pixel has u(P) < u_k
                bool below_line = (sigma > 0) ? all_below_u : !all_below_u;
                far_hi = below_line; far_lo = !below_line;
            } else if (p0 < -4 && pend < -4) {
                far_lo = true;
            } else if (p0 > nc + 4 && pend > nc + 4) {
                far_hi = true;
            }
            if (far_lo) { p0 = -kFar; dl = 0; }
            if (far_hi) { p0 = kFar; dl = 0; }
            if (fabs(p0) > kFar || fabs(p0 + nw * dl) > kFar) return CSM_EGEOM;
            P0[k] = p0; DL[k] = dl;
            const size_t e = (size_t)v * (nu + 1) + k;
            line_d[2 * e] = p0; line_d[2 * e + 1] = dl;
            line_fx[2 * e] = llround(p0 * 4294967296.0);
            line_fx[2 * e + 1] = llround(dl * 4294967296.0);
            const double ad = fabs(dl);
            inv_d[e] = ad > 0 ? 0.5 / ad : 0.0;
            inv_f[e] = ad > 0 ? (float)(0.5 / ad) : 0.0f;
            if (ad > 0 && !std::isfinite(inv_f[e])) inv_f[e] = 3.0e38f;
        }
        // walk range of each element's strip: {upper line >= 0} and {lower line <= nc}
        for (int k = 0; k < nu; ++k) {
            const int ku = sigma > 0 ? k + 1 : k, kl = sigma > 0 ? k : k + 1;
            double lo = 0.0, hi = (double)nw;
            auto clip_ge = [&](double p0, double dl, double val) {  // p0 + w dl >= val
                if (dl > 0) lo = std::max(lo, (val - p0) / dl);
                else if (dl < 0) hi = std::min(hi, (val - p0) / dl);
                else if (p0 < val) hi = -1.0;
            };
            auto clip_le = [&](double p0, double dl, double val) {  // p0 + w dl <= val
                if (dl > 0) hi = std::min(hi, (val - p0) / dl);
                else if (dl < 0) lo = std::max(lo, (val - p0) / dl);
                else if (p0 > val) hi = -1.0;
            };
            clip_ge(P0[ku], DL[ku], 0.0);
            clip_le(P0[kl], DL[kl], (double)nc);
            int w0 = 0, w1 = 0;
            if (hi >= lo) {
                w0 = std::max(0, (int)floor(lo) - 1);
                w1 = std::min(nw, (int)ceil(hi) + 1);
                if (w1 < w0) w1 = w0;
            }
            wrange[2 * ((size_t)v * nu + k)] = w0;
            wrange[2 * ((size_t)v * nu + k) + 1] = w1;
        }
    }
    for (int l = 0; l <= nv; ++l) {
        double vv = (l - 0.5 * nv) * g->dv + g->v_off;
        rowq_d[l] = vv / D;
        rowq_f[l] = (float)(vv / D);
    }
    // depth of column centres per view, t_c / c = T0 + ix Tx + iy Ty (32.32 fixed point and
    // double), so that the kernels form it without FP64 arithmetic
    const size_t nct = g->dim == 3 ? 3 * (size_t)V : 3;
    std::vector<long long> colt_fx(nct, 0);
    std::vector<double> colt_d(nct, 0.0);
    if (g->dim == 3) {
        for (int v = 0; v < V; ++v) {
            const double c = cos(g->angles[v]), sn = sin(g->angles[v]);
            const double T0 = (s - (x0 + 0.5 * g->a) * c - (y0 + 0.5 * g->b) * sn) / g->c;
            const double Tx = -g->a * c / g->c, Ty = -g->b * sn / g->c;
            if (fabs(T0) + fabs(Tx) * g->nx + fabs(Ty) * g->ny > kFar) return CSM_EGEOM;
            colt_d[3 * v] = T0; colt_d[3 * v + 1] = Tx; colt_d[3 * v + 2] = Ty;
            colt_fx[3 * v] = llround(T0 * 4294967296.0);
            colt_fx[3 * v + 1] = llround(Tx * 4294967296.0);
            colt_fx[3 * v + 2] = llround(Ty * 4294967296.0);
        }
    }
    // row corners as float pairs (q = hi + lo) with 1/|q|, for the FP32 height of a row plane
    std::vector<float> rowq4(4 * (size_t)(nv + 1), 0.0f);
    for (int l = 0; l <= nv; ++l) {
        const double q = rowq_d[l];
        const float hi = (float)q;
        rowq4[4 * l] = hi;
        rowq4[4 * l + 1] = (float)(q - (double)hi);
        rowq4[4 * l + 2] = q != 0.0 ? (float)(1.0 / fabs(q)) : 0.0f;
    }

    // one device block for everything
    auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
    size_t off = 0;
    size_t o_as = off; off += al(axis_sigma.size() * sizeof(int));
    size_t o_csf = off; off += al(cs_f.size() * sizeof(float));
    size_t o_csd = off; off += al(cs_d.size() * sizeof(double));
    size_t o_lfx = off; off += al(line_fx.size() * sizeof(long long));
    size_t o_ld = off; off += al(line_d.size() * sizeof(double));
    size_t o_if = off; off += al(inv_f.size() * sizeof(float));
    size_t o_id = off; off += al(inv_d.size() * sizeof(double));
    size_t o_wr = off; off += al(wrange.size() * sizeof(int));
    size_t o_rf = off; off += al(rowq_f.size() * sizeof(float));
    size_t o_rd = off; off += al(rowq_d.size() * sizeof(double));
    size_t o_q4 = off; off += al(rowq4.size() * sizeof(float));
    size_t o_cfx = off; off += al(colt_fx.size() * sizeof(long long));
    size_t o_cd = off; off += al(colt_d.size() * sizeof(double));
    size_t o_cnt = off; off += al(sizeof(unsigned long long));
    std::vector<char> host(off, 0);
    memcpy(&host[o_as], axis_sigma.data(), axis_sigma.size() * sizeof(int));
    memcpy(&host[o_csf], cs_f.data(), cs_f.size() * sizeof(float));
    memcpy(&host[o_csd], cs_d.data(), cs_d.size() * sizeof(double));
    memcpy(&host[o_lfx], line_fx.data(), line_fx.size() * sizeof(long long));
    memcpy(&host[o_ld], line_d.data(), line_d.size() * sizeof(double));
    memcpy(&host[o_if], inv_f.data(), inv_f.size() * sizeof(float));
    memcpy(&host[o_id], inv_d.data(), inv_d.size() * sizeof(double));
    memcpy(&host[o_wr], wrange.data(), wrange.size() * sizeof(int));
    memcpy(&host[o_rf], rowq_f.data(), rowq_f.size() * sizeof(float));
    memcpy(&host[o_rd], rowq_d.data(), rowq_d.size() * sizeof(double));
    memcpy(&host[o_q4], rowq4.data(), rowq4.size() * sizeof(float));
    memcpy(&host[o_cfx], colt_fx.data(), colt_fx.size() * sizeof(long long));
    memcpy(&host[o_cd], colt_d.data(), colt_d.size() * sizeof(double));
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, off);
    if (e != cudaSuccess) { set_cuda_error(e); return e == cudaErrorMemoryAllocation ? CSM_ENOMEM : CSM_ECUDA; }
    e = cudaMemcpy(d, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_cuda_error(e); cudaFree(d); return CSM_ECUDA; }
    char* b = (char*)d;
    g->d_block = d; g->d_bytes = off;
    g->t.axis_sigma = (int*)(b + o_as);
    g->t.cs_f = (float*)(b + o_csf);
    g->t.cs_d = (double*)(b + o_csd);
    g->t.line_fx = (long long*)(b + o_lfx);
    g->t.line_d = (double*)(b + o_ld);
    g->t.inv_f = (float*)(b + o_if);
    g->t.inv_d = (double*)(b + o_id);
    g->t.wrange = (int*)(b + o_wr);
    g->t.rowq_f = (float*)(b + o_rf);
    g->t.rowq_d = (double*)(b + o_rd);
    g->t.rowq4 = (float4*)(b + o_q4);
    g->t.colt_fx = (long long*)(b + o_cfx);
    g->t.colt_d = (double*)(b + o_cd);
    g->t.counter = (unsigned long long*)(b + o_cnt);
    return CSM_OK;
}

static csm_status finish_create(csm_geom_s* g, const double* angles, csm_geom_t* out) {
    g->angles.resize(g->n_views);
    for (int v = 0; v < g->n_views; ++v) {
        g->angles[v] = angles ? angles[v] : 2.0 * M_PI * v / g->n_views;
        if (!std::isfinite(g->angles[v])) return CSM_EINVAL;
    }
    // the cone must lie between source and detector: s beyond the grid's circumradius
    double hz = g->dim == 3 ? 0.5 * g->nz * g->c : 0.0;
    double r = sqrt(pow(0.5 * g->nx * g->a, 2) + pow(0.5 * g->ny * g->b, 2));
    if (!(g->s > r) || !(g->sdd > g->s)) return CSM_EGEOM;
    if (g->dim == 3) {
        // detector rows one voxel can reach in one view: its v-extent at the nearest depth
        double tmin = g->s - r, diag = sqrt(g->a * g->a + g->b * g->b);
        double vext = g->sdd * (g->c / tmin + hz * diag / (tmin * tmin));
        if (vext / g->dv + 3.0 > (double)kMaxRowCorners) return CSM_EUNSUPPORTED;
        // corner lines that can cross one cell: its u-extent over du, plus one
        double tanb = std::max(fabs((-0.5 * g->nu) * g->du + g->u_off), fabs((0.5 * g->nu) * g->du + g->u_off)) / g->sdd;
        double uext = g->sdd * diag * (1.0 + tanb) / tmin;
        if (floor(uext / g->du) + 1.0 > (double)kMaxG) return CSM_EUNSUPPORTED;
        // the kernels index one view's projections with 32-bit integers
        if ((double)g->nv * g->nu >= 2147483647.0) return CSM_EUNSUPPORTED;
    }
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    csm_status st = build_tables(g);
    if (st != CSM_OK) return st;
    *out = g;
    return CSM_OK;
}

static bool pos(double v) { return std::isfinite(v) && v > 0; }

// The geometry's tables live on the device it was created on: a call made with another
// device current would hand the kernels pointers into another GPU's memory.
static csm_status check_device(const csm_geom_s* g) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    return dev == g->device ? CSM_OK : CSM_EINVAL;
}

}  // namespace csm

using namespace csm;

extern "C" {

csm_status csm_geom_create_2d(const csm_geom2d_desc* d, csm_geom_t* out) {
    if (!d || !out) return CSM_EINVAL;
    *out = nullptr;
    if (d->nx <= 0 || d->ny <= 0 || d->n_views <= 0 || d->nu <= 0) return CSM_EINVAL;
    if (!pos(d->a) || !pos(d->b) || !pos(d->s) || !pos(d->sdd) || !pos(d->du) || !std::isfinite(d->u_off))
        return CSM_EINVAL;
    csm_geom_s* g = new (std::nothrow) csm_geom_s();
    if (!g) return CSM_ENOMEM;
    g->dim = 2; g->nx = d->nx; g->ny = d->ny; g->nz = 1; g->a = d->a; g->b = d->b; g->c = 1.0;
    g->n_views = d->n_views; g->s = d->s; g->sdd = d->sdd; g->nu = d->nu; g->nv = 1;
    g->du = d->du; g->dv = 1.0; g->u_off = d->u_off; g->v_off = 0.0;
    csm_status st = finish_create(g, d->angles, out);
    if (st != CSM_OK) { delete g; *out = nullptr; }
    return st;
}

csm_status csm_geom_create_3d(const csm_geom3d_desc* d, csm_geom_t* out) {
    if (!d || !out) return CSM_EINVAL;
    *out = nullptr;
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || d->n_views <= 0 || d->nu <= 0 || d->nv <= 0)
        return CSM_EINVAL;
    if (!pos(d->a) || !pos(d->b) || !pos(d->c) || !pos(d->s) || !pos(d->sdd) || !pos(d->du) ||
        !pos(d->dv) || !std::isfinite(d->u_off) || !std::isfinite(d->v_off))
        return CSM_EINVAL;
    csm_geom_s* g = new (std::nothrow) csm_geom_s();
    if (!g) return CSM_ENOMEM;
    g->dim = 3; g->nx = d->nx; g->ny = d->ny; g->nz = d->nz; g->a = d->a; g->b = d->b; g->c = d->c;
    g->n_views = d->n_views; g->s = d->s; g->sdd = d->sdd; g->nu = d->nu; g->nv = d->nv;
    g->du = d->du; g->dv = d->dv; g->u_off = d->u_off; g->v_off = d->v_off;
    csm_status st = finish_create(g, d->angles, out);
    if (st != CSM_OK) { delete g; *out = nullptr; }
    return st;
}

void csm_geom_free(csm_geom_t g) {
    if (!g) return;
    if (g->d_block || g->w_block) {
        // release the table on the device that holds it, then restore the caller's device
        int prev = -1;
        const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
        if (have_prev && prev != g->device) cudaSetDevice(g->device);
        if (g->d_block) cudaFree(g->d_block);
        if (g->w_block) cudaFree(g->w_block);
        if (have_prev && prev != g->device) cudaSetDevice(prev);
    }
    delete g;
}

csm_status csm_geom_set_element_weights(csm_geom_t g, const double* weights) {
    if (!g) return CSM_EINVAL;
    csm_status dv = check_device(g);
    if (dv != CSM_OK) return dv;
    const size_t nel = (size_t)g->n_views * g->nv * g->nu;
    if (!weights) {
        if (g->w_block) {
            cudaError_t e = cudaFree(g->w_block);
            g->w_block = nullptr;
            if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
        }
        return CSM_OK;
    }
    for (size_t i = 0; i < nel; ++i)
        if (!std::isfinite(weights[i])) return CSM_EINVAL;
    const size_t of = (nel * sizeof(float) + 255) & ~(size_t)255;
    std::vector<char> host(of + nel * sizeof(double));
    float* wf = (float*)host.data();
    for (size_t i = 0; i < nel; ++i) wf[i] = (float)weights[i];
    memcpy(host.data() + of, weights, nel * sizeof(double));
    if (!g->w_block) {
        cudaError_t e = cudaMalloc(&g->w_block, host.size());
        if (e != cudaSuccess) {
            g->w_block = nullptr;
            set_cuda_error(e);
            return e == cudaErrorMemoryAllocation ? CSM_ENOMEM : CSM_ECUDA;
        }
    }
    cudaError_t e = cudaMemcpy(g->w_block, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    return CSM_OK;
}

static bool valid_dtype(csm_dtype t) { return t == CSM_F32 || t == CSM_F64 || t == CSM_BF16 || t == CSM_F16; }

csm_status csm_workspace_bytes(csm_geom_t g, int op, int64_t batch, csm_dtype compute, size_t* bytes) {
    if (!g || !bytes || batch < 0 || op < 0 || op > 3 || !valid_dtype(compute)) return CSM_EINVAL;
    bool dbl = compute == CSM_F64;
    *bytes = g->dim == 2 ? workspace_2d(g, op, batch, dbl) : workspace_3d(g, op, batch, dbl);
    return CSM_OK;
}

csm_status csm_forward(csm_geom_t g, const void* x, void* p, int64_t batch, csm_dtype xdt, csm_dtype pdt,
                       int flags, void* ws, size_t ws_bytes, void* stream) {
    if (!g || batch < 0 || !valid_dtype(xdt) || !valid_dtype(pdt)) return CSM_EINVAL;
    if (batch == 0) return CSM_OK;
    if (!x || !p) return CSM_EINVAL;
    if (flags & ~(CSM_ACCUMULATE | CSM_RELATIVE_WEIGHTS | CSM_VOXEL_DRIVEN)) return CSM_EINVAL;
    csm_status dv = check_device(g);
    if (dv != CSM_OK) return dv;
    cudaStream_t st = (cudaStream_t)stream;
    return g->dim == 2 ? forward_2d(g, x, p, batch, xdt, pdt, flags, ws, ws_bytes, st)
                       : forward_3d(g, x, p, batch, xdt, pdt, flags, ws, ws_bytes, st);
}

csm_status csm_back(csm_geom_t g, const void* p, void* x, int64_t batch, csm_dtype pdt, csm_dtype xdt,
                    int flags, void* ws, size_t ws_bytes, void* stream) {
    if (!g || batch < 0 || !valid_dtype(xdt) || !valid_dtype(pdt)) return CSM_EINVAL;
    if (batch == 0) return CSM_OK;
    if (!x || !p) return CSM_EINVAL;
    if (flags & ~(CSM_ACCUMULATE | CSM_RELATIVE_WEIGHTS)) return CSM_EINVAL;
    csm_status dv = check_device(g);
    if (dv != CSM_OK) return dv;
    cudaStream_t st = (cudaStream_t)stream;
    return g->dim == 2 ? back_2d(g, p, x, batch, pdt, xdt, flags, ws, ws_bytes, st)
                       : back_3d(g, p, x, batch, pdt, xdt, flags, ws, ws_bytes, st);
}

csm_status csm_nnz(csm_geom_t g, int64_t* nnz, void* stream) {
    if (!g || !nnz) return CSM_EINVAL;
    if (g->nnz >= 0) { *nnz = g->nnz; return CSM_OK; }
    csm_status dv = check_device(g);
    if (dv != CSM_OK) return dv;
    int64_t n = 0;
    csm_status st = g->dim == 2 ? nnz_2d(g, &n, (cudaStream_t)stream) : nnz_3d(g, &n, (cudaStream_t)stream);
    if (st == CSM_OK) { g->nnz = n; *nnz = n; }
    return st;
}

csm_status csm_sync_status(void* stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    return CSM_OK;
}

const char* csm_status_string(csm_status s) {
    switch (s) {
        case CSM_OK: return "ok";
        case CSM_EINVAL: return "invalid argument";
        case CSM_EGEOM: return "unsupported geometry (the source must lie outside the grid's circumcircle, sdd > s)";
        case CSM_ENOMEM: return "out of device memory";
        case CSM_ECUDA: return "CUDA error";
        case CSM_EUNSUPPORTED: return "not supported";
        case CSM_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* csm_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"

extern "C" csm_status csm_launch_count(uint64_t* count) {
    if (!count) return CSM_EINVAL;
    *count = (uint64_t)g_launches.load(std::memory_order_relaxed);
    return CSM_OK;
}

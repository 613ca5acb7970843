// proj3d.cu -- 3D circular cone-beam projectors: p = W x (ray-driven gather over row
// bundles) and x = W^T p (voxel-driven gather), every entry W_ij evaluated on the fly.
//
// Entry (Section "The Three-dimensional Case"): the volume of voxel j inside the pyramid of
// element (k, l), i.e. between the lateral planes of corners k, k+1 (the 2D rays, seen from
// the top) and the row planes {v(P) = v_l}, {v(P) = v_{l+1}}, where v(P) = sdd z / t(P) so
// that row plane l is z = q_l t(P), q_l = v_l / sdd (Appendix Eq. (z expr 1)).
//
// Composition.  For a top-view atom R (the part of the voxel's top-view cell below one corner
// line: the triangle / trapezoid / pentagon of the 2D case) and a row corner l,
//     Phi_l(R) = integral over R of  clamp(q_l t - z0, 0, c)  dA
// is the volume of the voxel above R and below row plane l (the paper's Vol_rel with its
// C-vector: the clamp's two kinks are where the plane meets the voxel's bottom and top
// faces).  The element's volume is the double difference
//     W_{k,l} = [Phi_{l+1} - Phi_l](below line k+1) - [Phi_{l+1} - Phi_l](below line k),
// the m_z subtraction Vol_res = Vol_rel(m_z - 1) - Vol_rel(m_z) and the top-view sums of the
// 2D procedure.  Because it uses both clamp kinks, any number of rows per voxel is handled
// (the paper restricts its experiments to three).
//
// Each Phi is two integrals of relu(g + q t') over the polygon R (t' = depth relative to the
// cell centre).  They are evaluated exactly: 0 when the linear function is <= 0 on R,
// g A + q M1 when it is >= 0 on R, and otherwise by the divergence theorem as a sum over
// R's edges,  -(1/q) sum_e w_e E3(l_P, l_Q),  where w_e is the outward edge normal (times
// length) projected on the source direction and E3 the exact mean of relu^2 / 2 along the
// edge.  These are the paper's cubic terms C g^3 (Eq. (rel vol 3d), Eq. (res vol 3d)) written
// per edge instead of per vertex, which removes the 1/sin(phi), 1/cos(phi) factors of the
// printed forms (their singular views, Eq. (vol)) from the arithmetic.
#include <algorithm>

#include "csm_internal.cuh"

namespace csm {

static int chunk3(int64_t batch) {
    if (batch >= 4) return 4;
    if (batch >= 2) return 2;
    return 1;
}
static size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }
constexpr int RB = 8;   // detector rows per forward thread

size_t workspace_3d(const csm_geom_s* g, int op, int64_t batch, bool dbl) {
    if (batch <= 0) return 0;
    const size_t es = dbl ? 8 : 4;
    const size_t nb = chunk3(batch);
    if (op == 0) return 2 * al256((size_t)g->nx * g->ny * g->nz * nb * es);
    return al256((size_t)g->n_views * g->nv * g->nu * nb * es);
}

template <int NB> struct Vec3 { static constexpr int W = NB; };

template <typename T>
__device__ __forceinline__ T load_any3(const void* base, size_t i, int dt) {
    switch (dt) {
        case CSM_F64: return (T)((const double*)base)[i];
        case CSM_BF16: return (T)__bfloat162float(((const __nv_bfloat16*)base)[i]);
        case CSM_F16: return (T)__half2float(((const __half*)base)[i]);
        default: return (T)((const float*)base)[i];
    }
}

template <typename T>
__device__ __forceinline__ void store_any3(void* base, size_t i, int dt, T v, bool acc) {
    switch (dt) {
        case CSM_F64: { double* q = (double*)base + i; *q = acc ? *q + (double)v : (double)v; break; }
        case CSM_BF16: {
            __nv_bfloat16* q = (__nv_bfloat16*)base + i;
            float cur = acc ? __bfloat162float(*q) : 0.0f;
            *q = __float2bfloat16_rn(cur + (float)v);
            break;
        }
        case CSM_F16: {
            __half* q = (__half*)base + i;
            float cur = acc ? __half2float(*q) : 0.0f;
            *q = __float2half_rn(cur + (float)v);
            break;
        }
        default: { float* q = (float*)base + i; *q = acc ? *q + (float)v : (float)v; break; }
    }
}

template <typename T> struct G3;
template <> struct G3<float> {
    static __device__ __forceinline__ float s(const Geo& g) { return g.s; }
    static __device__ __forceinline__ float sdd(const Geo& g) { return g.sdd; }
    static __device__ __forceinline__ float a(const Geo& g) { return g.a; }
    static __device__ __forceinline__ float b(const Geo& g) { return g.b; }
    static __device__ __forceinline__ float c(const Geo& g) { return g.c; }
    static __device__ __forceinline__ float x0(const Geo& g) { return g.x0; }
    static __device__ __forceinline__ float y0(const Geo& g) { return g.y0; }
    static __device__ __forceinline__ float z0(const Geo& g) { return g.z0; }
    static __device__ __forceinline__ float u0(const Geo& g) { return g.u0; }
    static __device__ __forceinline__ float v0(const Geo& g) { return g.v0; }
    static __device__ __forceinline__ float du(const Geo& g) { return g.du; }
    static __device__ __forceinline__ float dv(const Geo& g) { return g.dv; }
    static __device__ __forceinline__ float cs(const Geo& g, int v, int i) { return g.cs_f[2 * v + i]; }
    static __device__ __forceinline__ float q(const Geo& g, int l) { return g.rowq_f[l]; }
    static __device__ __forceinline__ float div(float x, float y) { return __fdividef(x, y); }
    static constexpr float eps = 1e-3f;
};
template <> struct G3<double> {
    static __device__ __forceinline__ double s(const Geo& g) { return g.s_d; }
    static __device__ __forceinline__ double sdd(const Geo& g) { return g.sdd_d; }
    static __device__ __forceinline__ double a(const Geo& g) { return g.a_d; }
    static __device__ __forceinline__ double b(const Geo& g) { return g.b_d; }
    static __device__ __forceinline__ double c(const Geo& g) { return g.c_d; }
    static __device__ __forceinline__ double x0(const Geo& g) { return g.x0_d; }
    static __device__ __forceinline__ double y0(const Geo& g) { return g.y0_d; }
    static __device__ __forceinline__ double z0(const Geo& g) { return g.z0_d; }
    static __device__ __forceinline__ double u0(const Geo& g) { return g.u0_d; }
    static __device__ __forceinline__ double v0(const Geo& g) { return g.v0_d; }
    static __device__ __forceinline__ double du(const Geo& g) { return g.du_d; }
    static __device__ __forceinline__ double dv(const Geo& g) { return g.dv_d; }
    static __device__ __forceinline__ double cs(const Geo& g, int v, int i) { return g.cs_d[2 * v + i]; }
    static __device__ __forceinline__ double q(const Geo& g, int l) { return g.rowq_d[l]; }
    static __device__ __forceinline__ double div(double x, double y) { return x / y; }
    static constexpr double eps = 1e-9;
};

// Row-plane height above the grid's bottom face at the centre of column (ix, iy), in units
// of c; the local height above voxel iz's bottom face is (G - iz) c.
struct RowF {
    long long G;
    __device__ __forceinline__ void at(const Geo& g, int v, int l, int ix, int iy) {
        const long long* e = g.rowp_fx + 3 * ((size_t)v * (g.nv + 1) + l);
        G = e[0] + (long long)ix * e[1] + (long long)iy * e[2];
    }
    __device__ __forceinline__ float rel(int iz) const {   // G - iz in float, exact integer part
        int hi = (int)(G >> 32);
        unsigned lo = (unsigned)(G & 0xffffffffull);
        return (float)(hi - iz) + (float)lo * 2.3283064365386963e-10f;
    }
};
struct RowD {
    double G;
    __device__ __forceinline__ void at(const Geo& g, int v, int l, int ix, int iy) {
        const double* e = g.rowp_d + 3 * ((size_t)v * (g.nv + 1) + l);
        G = e[0] + (double)ix * e[1] + (double)iy * e[2];
    }
    __device__ __forceinline__ double rel(int iz) const { return G - (double)iz; }
};
template <typename T> struct RowOf;
template <> struct RowOf<float> { using type = RowF; };
template <> struct RowOf<double> { using type = RowD; };

// ---------------------------------------------------------------------------------------
// Top-view atom: the part of a cell below one corner line, as a 6-vertex polygon
//   (0,0) (1,0) (1,h1) (xi_hi,h(xi_hi)) (xi_lo,h(xi_lo)) (0,h0)      (cell units, CCW)
// with h = clamp(line, 0, 1) and xi_hi / xi_lo the points where the line crosses the cross
// faces (coinciding vertices give zero-length edges).  Stored per vertex: depth t' relative
// to the cell centre; per edge: w_e = e_s . (outward normal x length); and the area A, the
// first moment M1 = integral of t' dA, and the depth range.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Atom {
    T t[6], w[6];
    T tmin, tmax, A, M1;
    bool empty;
};

template <typename T>
__device__ __forceinline__ T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

template <typename T>
__device__ __forceinline__ void make_atom(Atom<T>& P, T lam0, T lam1, T hw, T hc, int axis, T cs, T sn) {
    if (lam0 <= T(0) && lam1 <= T(0)) {
        P.empty = true;
        P.A = T(0); P.M1 = T(0); P.tmin = T(0); P.tmax = T(0);
        return;
    }
    P.empty = false;
    const T dl = lam1 - lam0;
    T xa = T(1), xb = T(1);
    if (dl != T(0)) {
        const T r = G3<T>::div(T(1), dl);
        xa = clamp01(-lam0 * r);
        xb = clamp01((T(1) - lam0) * r);
    }
    const T xhi = xa > xb ? xa : xb, xlo = xa > xb ? xb : xa;
    const T XI[6] = {T(0), T(1), T(1), xhi, xlo, T(0)};
    const T ET[6] = {T(0), T(0), clamp01(lam1), clamp01(lam0 + dl * xhi), clamp01(lam0 + dl * xlo), clamp01(lam0)};
    T DX[6], DY[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const T dw = (XI[i] - T(0.5)) * hw, dc = (ET[i] - T(0.5)) * hc;
        DX[i] = axis == 0 ? dw : dc;
        DY[i] = axis == 0 ? dc : dw;
        P.t[i] = -(DX[i] * cs + DY[i] * sn);
    }
    const T orient = axis == 0 ? T(1) : T(-1);
    T a2 = T(0), m = T(0);
    P.tmin = P.t[0];
    P.tmax = P.t[0];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int j = (i + 1) % 6;
        P.w[i] = orient * (cs * (DY[j] - DY[i]) - sn * (DX[j] - DX[i]));
        a2 += XI[i] * ET[j] - XI[j] * ET[i];
        m -= P.w[i] * (P.t[i] * P.t[i] + P.t[i] * P.t[j] + P.t[j] * P.t[j]);
        P.tmin = P.t[i] < P.tmin ? P.t[i] : P.tmin;
        P.tmax = P.t[i] > P.tmax ? P.t[i] : P.tmax;
    }
    P.A = T(0.5) * a2 * hw * hc;
    P.M1 = m * T(1.0 / 6.0);
}

// mean of relu(x)^2 / 2 for x linear from p to q along a segment
template <typename T>
__device__ __forceinline__ T e3(T p, T q) {
    const T mx = p > q ? p : q, mn = p > q ? q : p;
    if (mn >= T(0)) return (p * p + p * q + q * q) * T(1.0 / 6.0);
    if (mx <= T(0)) return T(0);
    return G3<T>::div(mx * mx * mx, T(6) * (mx - mn));
}

// integral over the atom of relu(g + q t')
template <typename T>
__device__ __forceinline__ T relu_int(const Atom<T>& P, T g, T q) {
    if (P.empty) return T(0);
    const T lo = g + q * (q > T(0) ? P.tmin : P.tmax);
    const T hi = g + q * (q > T(0) ? P.tmax : P.tmin);
    if (hi <= T(0)) return T(0);
    if (lo >= T(0)) return g * P.A + q * P.M1;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int j = (i + 1) % 6;
        acc += P.w[i] * e3(g + q * P.t[i], g + q * P.t[j]);
    }
    return -G3<T>::div(acc, q);
}

// Phi = integral over the atom of clamp(g + q t', 0, c): the voxel volume above the atom and
// below the row plane whose height above the voxel's bottom face at the cell centre is g.
template <typename T>
__device__ __forceinline__ T phi_row(const Atom<T>& P, T g, T q, T c) {
    if (P.empty) return T(0);
    return relu_int(P, g, q) - relu_int(P, g - c, q);
}

// Elements / rows a voxel (column corners X0..Y1, heights z0..z1) can reach in view v.
template <typename T>
__device__ __forceinline__ bool voxel_footprint(const Geo& g, int v, T X0, T X1, T Y0, T Y1, T z0, T z1, int& k0,
                                                int& k1, int& l0, int& l1) {
    const T c = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
    const T s = G3<T>::s(g), D = G3<T>::sdd(g);
    T umin = T(1e30), umax = T(-1e30), tmin = T(1e30), tmax = T(-1e30);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const T X = (q & 1) ? X1 : X0, Y = (q & 2) ? Y1 : Y0;
        const T t = s - X * c - Y * sn;
        const T u = G3<T>::div(D * (Y * c - X * sn), t);
        umin = u < umin ? u : umin;
        umax = u > umax ? u : umax;
        tmin = t < tmin ? t : tmin;
        tmax = t > tmax ? t : tmax;
    }
    const T vlo = D * (z0 < T(0) ? G3<T>::div(z0, tmin) : G3<T>::div(z0, tmax));
    const T vhi = D * (z1 > T(0) ? G3<T>::div(z1, tmin) : G3<T>::div(z1, tmax));
    const T idu = T(1) / G3<T>::du(g), idv = T(1) / G3<T>::dv(g);
    T f0 = floor((umin - G3<T>::u0(g)) * idu - G3<T>::eps), f1 = floor((umax - G3<T>::u0(g)) * idu + G3<T>::eps);
    T h0 = floor((vlo - G3<T>::v0(g)) * idv - G3<T>::eps), h1 = floor((vhi - G3<T>::v0(g)) * idv + G3<T>::eps);
    if (f1 < T(0) || f0 > T(g.nu - 1) || h1 < T(0) || h0 > T(g.nv - 1)) return false;
    k0 = f0 < T(0) ? 0 : (int)f0;
    k1 = f1 > T(g.nu - 1) ? g.nu - 1 : (int)f1;
    l0 = h0 < T(0) ? 0 : (int)h0;
    l1 = h1 > T(g.nv - 1) ? g.nv - 1 : (int)h1;
    if (l1 - l0 + 2 > kMaxRowCorners) l1 = l0 + kMaxRowCorners - 2;   // excluded by the geometry check
    return k0 <= k1 && l0 <= l1;
}

// ---------------------------------------------------------------------------------------
// Layouts.  Forward reads x as xs0[ix][q][iz][iy][VW] (walk x) / xs1[iy][q][iz][ix][VW]
// (walk y): lanes handle neighbouring elements, i.e. neighbouring cross cells.  Back reads
// p as ps[v][q][l][k][VW].
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
__global__ void prep_vol_3d(const void* __restrict__ x, int xdt, int B, int b_off, int nx, int ny, int nz,
                            T* __restrict__ xs0, T* __restrict__ xs1) {
    const size_t n = (size_t)nx * ny * nz;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((size_t)nx * ny));
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const int b = b_off + bb;
        const T val = b < B ? load_any3<T>(x, (size_t)b * n + i, xdt) : T(0);
        xs0[((((size_t)ix) * nz + iz) * ny + iy) * NB + bb] = val;
        xs1[((((size_t)iy) * nz + iz) * nx + ix) * NB + bb] = val;
    }
}

template <typename T, int NB>
__global__ void prep_sino_3d(const void* __restrict__ p, int pdt, int B, int b_off, size_t n, T* __restrict__ ps) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const int b = b_off + bb;
        ps[i * NB + bb] = b < B ? load_any3<T>(p, (size_t)b * n + i, pdt) : T(0);
    }
}

template <typename T, int NB>
__device__ __forceinline__ void fma_vec(T (&acc)[NB], T wt, const T* __restrict__ src) {
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] += wt * __ldg(src + i);
}

// ---------------------------------------------------------------------------------------
// Back projection: one thread per voxel loops over all views; per view it builds the
// top-view atoms of the corner lines of its footprint one after the other, evaluates Phi at
// the row corners of its footprint, and forms the element volumes as double differences.
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(128) back3d_vox(Geo g, const T* __restrict__ ps, void* __restrict__ x, int xdt,
                                                  int B, int b_off, T scale, int accumulate) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 4 + threadIdx.y, iz = blockIdx.z;
    if (ix >= g.nx || iy >= g.ny) return;
    using L = typename LineOf<T>::type;
    using R = typename RowOf<T>::type;
    const T a = G3<T>::a(g), b = G3<T>::b(g), c = G3<T>::c(g);
    const T X0 = G3<T>::x0(g) + ix * a, X1 = X0 + a, Y0 = G3<T>::y0(g) + iy * b, Y1 = Y0 + b;
    const T Z0 = G3<T>::z0(g) + iz * c, Z1 = Z0 + c;
    T acc[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] = T(0);
    for (int v = 0; v < g.n_views; ++v) {
        int k0, k1, l0, l1;
        if (!voxel_footprint<T>(g, v, X0, X1, Y0, Y1, Z0, Z1, k0, k1, l0, l1)) continue;
        const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
        const int w = axis == 0 ? ix : iy, cc = axis == 0 ? iy : ix;
        const T hw = axis == 0 ? a : b, hc = axis == 0 ? b : a;
        const T cs = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
        const int nrc = l1 - l0 + 2;
        T gr[kMaxRowCorners], qr[kMaxRowCorners], prev[kMaxRowCorners], cur[kMaxRowCorners];
#pragma unroll
        for (int r = 0; r < kMaxRowCorners; ++r) {
            if (r < nrc) {
                R row;
                row.at(g, v, l0 + r, ix, iy);
                gr[r] = row.rel(iz) * c;
                qr[r] = G3<T>::q(g, l0 + r);
            } else {
                gr[r] = T(0);
                qr[r] = T(0);
            }
        }
        Atom<T> P;
        {
            L line;
            line.load(g, v, k0, w);
            T y0, y1;
            line.offsets(cc, y0, y1);
            make_atom<T>(P, y0, y1, hw, hc, axis, cs, sn);
#pragma unroll
            for (int r = 0; r < kMaxRowCorners; ++r) prev[r] = r < nrc ? phi_row<T>(P, gr[r], qr[r], c) : T(0);
        }
        const T* pv = ps + (size_t)v * g.nv * g.nu * NB;
        for (int k = k0; k <= k1; ++k) {
            L line;
            line.load(g, v, k + 1, w);
            T y0, y1;
            line.offsets(cc, y0, y1);
            make_atom<T>(P, y0, y1, hw, hc, axis, cs, sn);
#pragma unroll
            for (int r = 0; r < kMaxRowCorners; ++r) cur[r] = r < nrc ? phi_row<T>(P, gr[r], qr[r], c) : T(0);
#pragma unroll
            for (int r = 0; r < kMaxRowCorners - 1; ++r) {
                if (r < nrc - 1) {
                    T wt = (cur[r + 1] - cur[r]) - (prev[r + 1] - prev[r]);
                    wt = sigma > 0 ? wt : -wt;
                    if (wt != T(0)) fma_vec<T, NB>(acc, wt, pv + ((size_t)(l0 + r) * g.nu + k) * NB);
                }
            }
#pragma unroll
            for (int r = 0; r < kMaxRowCorners; ++r) prev[r] = cur[r];
        }
    }
    const size_t vox = ((size_t)iz * g.ny + iy) * g.nx + ix;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int bidx = b_off + i;
        if (bidx < B) store_any3<T>(x, (size_t)bidx * nvox + vox, xdt, acc[i] * scale, accumulate != 0);
    }
}

// ---------------------------------------------------------------------------------------
// Forward projection, ray-driven: one thread per (view, element column k, bundle of RB
// detector rows).  The thread walks the top-view strip of column k cell by cell (as in 2D);
// in each cell it builds the two atoms of its corner lines once, then visits the voxels of
// the column that its rows reach and accumulates W * x for each of its rows.
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(64) fwd3d_ray(Geo g, const T* __restrict__ xs0, const T* __restrict__ xs1,
                                                void* __restrict__ p, int pdt, int B, int b_off, T scale,
                                                int accumulate) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    const int lb = blockIdx.z * RB;
    if (k >= g.nu) return;
    const int nrow = min(RB, g.nv - lb);
    using L = typename LineOf<T>::type;
    using R = typename RowOf<T>::type;
    const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
    const int nc = axis == 0 ? g.ny : g.nx;
    const T* __restrict__ xs = axis == 0 ? xs0 : xs1;
    const T a = G3<T>::a(g), b = G3<T>::b(g), c = G3<T>::c(g);
    const T hw = axis == 0 ? a : b, hc = axis == 0 ? b : a;
    const T cs = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
    // largest change of a row plane's height across a cell, in units of c
    const T tr = T(0.5) * (fabs(a * cs) + fabs(b * sn));
    T qr[RB + 1];
    T qmax = T(0);
#pragma unroll
    for (int r = 0; r <= RB; ++r) {
        qr[r] = r <= nrow ? G3<T>::q(g, lb + r) : T(0);
        qmax = fabs(qr[r]) > qmax ? fabs(qr[r]) : qmax;
    }
    const T margin = qmax * tr / c + T(1e-3);
    const int w0 = g.wrange[2 * ((size_t)v * g.nu + k)], w1 = g.wrange[2 * ((size_t)v * g.nu + k) + 1];
    L la, lb_;
    la.load(g, v, k, w0);
    lb_.load(g, v, k + 1, w0);
    T acc[RB][NB];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int i = 0; i < NB; ++i) acc[r][i] = T(0);
    for (int w = w0; w < w1; ++w) {
        int clo = min(la.cell_lo(), lb_.cell_lo());
        int chi = max(la.cell_hi(), lb_.cell_hi());
        clo = max(clo, 0);
        chi = min(chi, nc - 1);
        for (int cc = clo; cc <= chi; ++cc) {
            T a0, a1, b0, b1;
            la.offsets(cc, a0, a1);
            lb_.offsets(cc, b0, b1);
            Atom<T> Pa, Pb;
            make_atom<T>(Pa, a0, a1, hw, hc, axis, cs, sn);
            make_atom<T>(Pb, b0, b1, hw, hc, axis, cs, sn);
            if (Pa.empty && Pb.empty) continue;
            const int ix = axis == 0 ? w : cc, iy = axis == 0 ? cc : w;
            // row-plane heights at this column relative to voxel zb, float
            R r0, rn;
            r0.at(g, v, lb, ix, iy);
            rn.at(g, v, lb + nrow, ix, iy);
            const T zlo = floor(r0.rel(0) - margin), zhi = floor(rn.rel(0) + margin);
            if (zhi < T(0) || zlo > T(g.nz - 1)) continue;
            const int izlo = zlo < T(0) ? 0 : (int)zlo;
            const int izhi = zhi > T(g.nz - 1) ? g.nz - 1 : (int)zhi;
            if (izlo > izhi) continue;
            T gz[RB + 1];
#pragma unroll
            for (int r = 0; r <= RB; ++r) {
                if (r <= nrow) {
                    R row;
                    row.at(g, v, lb + r, ix, iy);
                    gz[r] = row.rel(izlo);
                } else {
                    gz[r] = T(0);
                }
            }
            const T* xcol = xs + ((size_t)w * g.nz) * nc * NB + (size_t)cc * NB;
            for (int iz = izlo; iz <= izhi; ++iz) {
                const T dz = T(iz - izlo);
                T fa[RB + 1], fb[RB + 1];
#pragma unroll
                for (int r = 0; r <= RB; ++r) {
                    fa[r] = T(0);
                    fb[r] = T(0);
                    if (r <= nrow) {
                        const T h = gz[r] - dz;   // plane height above the voxel's bottom, units of c
                        if (h + margin <= T(0)) {
                            // plane below the voxel everywhere in the cell: nothing below it
                        } else if (h - margin >= T(1)) {
                            fa[r] = c * Pa.A;   // whole voxel column part below the plane
                            fb[r] = c * Pb.A;
                        } else {
                            fa[r] = phi_row<T>(Pa, h * c, qr[r], c);
                            fb[r] = phi_row<T>(Pb, h * c, qr[r], c);
                        }
                    }
                }
                T xv[NB];
#pragma unroll
                for (int i = 0; i < NB; ++i) xv[i] = __ldg(xcol + (size_t)iz * nc * NB + i);
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (r < nrow) {
                        T wt = (fb[r + 1] - fb[r]) - (fa[r + 1] - fa[r]);
                        wt = sigma > 0 ? wt : -wt;
#pragma unroll
                        for (int i = 0; i < NB; ++i) acc[r][i] += wt * xv[i];
                    }
                }
            }
        }
        la.step();
        lb_.step();
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        if (r < nrow) {
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int bidx = b_off + i;
                if (bidx < B)
                    store_any3<T>(p, (((size_t)bidx * g.n_views + v) * g.nv + lb + r) * g.nu + k, pdt,
                                  acc[r][i] * scale, accumulate != 0);
            }
        }
    }
}

// Number of (voxel, view, element) whose volume exceeds 1e-6 of the voxel's.
__global__ void __launch_bounds__(128) nnz3d_kernel(Geo g, unsigned long long* counter) {
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 4 + threadIdx.y, iz = blockIdx.z;
    unsigned long long cnt = 0;
    if (ix < g.nx && iy < g.ny) {
        const float a = g.a, b = g.b, c = g.c;
        const float X0 = g.x0 + ix * a, X1 = X0 + a, Y0 = g.y0 + iy * b, Y1 = Y0 + b;
        const float Z0 = g.z0 + iz * c, Z1 = Z0 + c;
        const float thr = 1e-6f * a * b * c;   // above 1e-6 of the voxel's volume
        for (int v = 0; v < g.n_views; ++v) {
            int k0, k1, l0, l1;
            if (!voxel_footprint<float>(g, v, X0, X1, Y0, Y1, Z0, Z1, k0, k1, l0, l1)) continue;
            const int axis = g.axis_sigma[2 * v];
            const int w = axis == 0 ? ix : iy, cc = axis == 0 ? iy : ix;
            const float hw = axis == 0 ? a : b, hc = axis == 0 ? b : a;
            const float cs = g.cs_f[2 * v], sn = g.cs_f[2 * v + 1];
            const int nrc = l1 - l0 + 2;
            float gr[kMaxRowCorners], qr[kMaxRowCorners], prev[kMaxRowCorners], cur[kMaxRowCorners];
#pragma unroll
            for (int r = 0; r < kMaxRowCorners; ++r) {
                RowF row;
                row.at(g, v, l0 + (r < nrc ? r : 0), ix, iy);
                gr[r] = row.rel(iz) * c;
                qr[r] = g.rowq_f[l0 + (r < nrc ? r : 0)];
            }
            Atom<float> P;
            LineF line;
            float y0, y1;
            line.load(g, v, k0, w);
            line.offsets(cc, y0, y1);
            make_atom<float>(P, y0, y1, hw, hc, axis, cs, sn);
#pragma unroll
            for (int r = 0; r < kMaxRowCorners; ++r) prev[r] = r < nrc ? phi_row<float>(P, gr[r], qr[r], c) : 0.0f;
            for (int k = k0; k <= k1; ++k) {
                line.load(g, v, k + 1, w);
                line.offsets(cc, y0, y1);
                make_atom<float>(P, y0, y1, hw, hc, axis, cs, sn);
#pragma unroll
                for (int r = 0; r < kMaxRowCorners; ++r) cur[r] = r < nrc ? phi_row<float>(P, gr[r], qr[r], c) : 0.0f;
#pragma unroll
                for (int r = 0; r < kMaxRowCorners - 1; ++r)
                    if (r < nrc - 1) cnt += fabsf((cur[r + 1] - cur[r]) - (prev[r + 1] - prev[r])) > thr;
#pragma unroll
                for (int r = 0; r < kMaxRowCorners; ++r) prev[r] = cur[r];
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (threadIdx.x == 0 && cnt) atomicAdd(counter, cnt);
}

// ---------------------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
static csm_status run_fwd3(const csm_geom_s* gh, const void* x, void* p, int64_t batch, csm_dtype xdt,
                           csm_dtype pdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    const size_t nvox = (size_t)gh->nx * gh->ny * gh->nz;
    const size_t half = al256(nvox * NB * sizeof(T));
    T* xs0 = (T*)ws;
    T* xs1 = (T*)((char*)ws + half);
    // the atoms' integrals are volumes in world units already
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1.0 / (gh->a * gh->b * gh->c)) : T(1);
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        prep_vol_3d<T, NB><<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(x, (int)xdt, (int)batch, (int)b0,
                                                                          gh->nx, gh->ny, gh->nz, xs0, xs1);
        dim3 fb(64), fg((gh->nu + 63) / 64, gh->n_views, (gh->nv + RB - 1) / RB);
        fwd3d_ray<T, NB><<<fg, fb, 0, st>>>(g, xs0, xs1, p, (int)pdt, (int)batch, (int)b0, scale,
                                           (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status e = check_launch();
        if (e != CSM_OK) return e;
    }
    return CSM_OK;
}

template <typename T, int NB>
static csm_status run_back3(const csm_geom_s* gh, const void* p, void* x, int64_t batch, csm_dtype pdt,
                            csm_dtype xdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    T* ps = (T*)ws;
    // the atoms' integrals are volumes in world units already
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1.0 / (gh->a * gh->b * gh->c)) : T(1);
    const size_t n = (size_t)gh->n_views * gh->nv * gh->nu;
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        prep_sino_3d<T, NB><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, (int)pdt, (int)batch, (int)b0, n, ps);
        dim3 bb(32, 4), bg((gh->nx + 31) / 32, (gh->ny + 3) / 4, gh->nz);
        back3d_vox<T, NB><<<bg, bb, 0, st>>>(g, ps, x, (int)xdt, (int)batch, (int)b0, scale,
                                            (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status e = check_launch();
        if (e != CSM_OK) return e;
    }
    return CSM_OK;
}

csm_status forward_3d(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt, csm_dtype pdt,
                      int flags, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    if (flags & CSM_VOXEL_DRIVEN) return CSM_EUNSUPPORTED;
    if (!ws || ws_bytes < workspace_3d(g, 0, batch, dbl)) return CSM_EINVAL;
    if (g->nz > 65535 || g->n_views > 65535) return CSM_EUNSUPPORTED;
    switch (chunk3(batch)) {
        case 4: return dbl ? run_fwd3<double, 4>(g, x, p, batch, xdt, pdt, flags, ws, st)
                           : run_fwd3<float, 4>(g, x, p, batch, xdt, pdt, flags, ws, st);
        case 2: return dbl ? run_fwd3<double, 2>(g, x, p, batch, xdt, pdt, flags, ws, st)
                           : run_fwd3<float, 2>(g, x, p, batch, xdt, pdt, flags, ws, st);
        default: return dbl ? run_fwd3<double, 1>(g, x, p, batch, xdt, pdt, flags, ws, st)
                            : run_fwd3<float, 1>(g, x, p, batch, xdt, pdt, flags, ws, st);
    }
}

csm_status back_3d(const csm_geom_s* g, const void* p, void* x, int64_t batch, csm_dtype pdt, csm_dtype xdt,
                   int flags, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    if (!ws || ws_bytes < workspace_3d(g, 1, batch, dbl)) return CSM_EINVAL;
    if (g->nz > 65535) return CSM_EUNSUPPORTED;
    switch (chunk3(batch)) {
        case 4: return dbl ? run_back3<double, 4>(g, p, x, batch, pdt, xdt, flags, ws, st)
                           : run_back3<float, 4>(g, p, x, batch, pdt, xdt, flags, ws, st);
        case 2: return dbl ? run_back3<double, 2>(g, p, x, batch, pdt, xdt, flags, ws, st)
                           : run_back3<float, 2>(g, p, x, batch, pdt, xdt, flags, ws, st);
        default: return dbl ? run_back3<double, 1>(g, p, x, batch, pdt, xdt, flags, ws, st)
                            : run_back3<float, 1>(g, p, x, batch, pdt, xdt, flags, ws, st);
    }
}

csm_status nnz_3d(const csm_geom_s* gh, int64_t* out, cudaStream_t st) {
    const Geo g = make_geo(gh);
    cudaError_t e = cudaMemsetAsync(gh->t.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    dim3 bb(32, 4), bg((gh->nx + 31) / 32, (gh->ny + 3) / 4, gh->nz);
    nnz3d_kernel<<<bg, bb, 0, st>>>(g, gh->t.counter);
    csm_status s = check_launch();
    if (s != CSM_OK) return s;
    unsigned long long h = 0;
    e = cudaMemcpyAsync(&h, gh->t.counter, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    *out = (int64_t)h;
    return CSM_OK;
}

}  // namespace csm

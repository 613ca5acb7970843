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

size_t workspace_3d(const csm_geom_s* g, int op, int64_t batch, bool dbl) {
    if (batch <= 0) return 0;
    const size_t es = dbl ? 8 : 4;
    const size_t nb = chunk3(batch);
    const size_t vol = al256((size_t)g->nx * g->ny * g->nz * nb * es);
    const size_t sino = al256((size_t)g->n_views * g->nv * g->nu * nb * es);
    if (op == 0) return 2 * vol;   // the volume in both walk layouts
    return sino;
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
// Edge form of a top-view atom for repeated evaluation.  Per edge: the depths t' of its two
// ends, w_e = e_s . (outward normal x length) and 1 / |t'_a - t'_b|; zero-length edges are
// dropped.  The tail moment
//     M_s(T) = integral over the atom of relu(s t' - T) dA   (s = +1 or -1)
// is  -(s/6) sum_e w_e E_e  with E_e = a^2 + a b + b^2 (both ends beyond T) or
// a^3 / |t'_a - t'_b| (one end beyond T), a >= b the parts of the ends beyond T: the same
// edge sum as above with the per-edge division precomputed.
// ---------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

template <typename T>
struct AtomE {
    T ta[6], tb[6], w[6], inv[6];
    T A, M1, tmin, tmax;
    int ne;
};

template <typename T>
__device__ __forceinline__ void make_atom_e(AtomE<T>& P, T lam0, T lam1, T hw, T hc, int axis, T cs, T sn) {
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
    T DX[6], DY[6], TP[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const T dw = (XI[i] - T(0.5)) * hw, dc = (ET[i] - T(0.5)) * hc;
        DX[i] = axis == 0 ? dw : dc;
        DY[i] = axis == 0 ? dc : dw;
        TP[i] = -(DX[i] * cs + DY[i] * sn);
    }
    const T orient = axis == 0 ? T(1) : T(-1);
    T a2 = T(0), m = T(0), tmin = TP[0], tmax = TP[0];
    int ne = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int j = (i + 1) % 6;
        a2 += XI[i] * ET[j] - XI[j] * ET[i];
        tmin = TP[i] < tmin ? TP[i] : tmin;
        tmax = TP[i] > tmax ? TP[i] : tmax;
        if (XI[i] == XI[j] && ET[i] == ET[j]) continue;
        const T w = orient * (cs * (DY[j] - DY[i]) - sn * (DX[j] - DX[i]));
        const T d = fabs(TP[i] - TP[j]);
        m -= w * (TP[i] * TP[i] + TP[i] * TP[j] + TP[j] * TP[j]);
        P.ta[ne] = TP[i];
        P.tb[ne] = TP[j];
        P.w[ne] = w;
        P.inv[ne] = d > T(0) ? G3<T>::div(T(1), d) : T(0);
        ++ne;
    }
    P.ne = ne;
    P.A = T(0.5) * a2 * hw * hc;
    P.M1 = m * T(1.0 / 6.0);
    P.tmin = tmin;
    P.tmax = tmax;
}

template <typename T>
__device__ __forceinline__ T tail_moment(const AtomE<T>& P, T Tq, T s) {
    T acc = T(0);
    for (int e = 0; e < P.ne; ++e) {
        const T pa = s * P.ta[e] - Tq, pb = s * P.tb[e] - Tq;
        const T mx = pa > pb ? pa : pb, mn = pa > pb ? pb : pa;
        const T a = mx > T(0) ? mx : T(0), b = mn > T(0) ? mn : T(0);
        const T E = b > T(0) ? (a * a + a * b + b * b) : a * a * a * P.inv[e];
        acc += P.w[e] * E;
    }
    return -s * acc * T(1.0 / 6.0);
}

// Phi = integral over the atom of clamp(g + q t', 0, c); iq = 1 / |q|.  In the flipped frame
// s t' the clamp's kinks sit at T0 = -g/|q| (bottom face) and T1 = (c - g)/|q| (top face);
// only a kink inside the atom's depth range needs the edge sum, and normally only one is
// inside, so one tail evaluation serves both terms (a second one only for voxels thinner
// than the plane's rise across the atom).
template <typename T>
__device__ __forceinline__ T phi_e(const AtomE<T>& P, T g, T q, T iq, T c) {
    if (q == T(0)) return (g < T(0) ? T(0) : (g > c ? c : g)) * P.A;
    const T s = q > T(0) ? T(1) : T(-1), qa = fabs(q);
    const T T0 = -g * iq, T1 = (c - g) * iq;
    const T lo = s > T(0) ? P.tmin : -P.tmax, hi = s > T(0) ? P.tmax : -P.tmin;
    const T lin0 = g * P.A + qa * s * P.M1;        // q |q| M(T0) when T0 <= lo
    const T lin1 = lin0 - c * P.A;                 // q |q| M(T1) when T1 <= lo
    const bool in0 = T0 > lo && T0 < hi, in1 = T1 > lo && T1 < hi;
    if (!in0 && !in1) return T1 <= lo ? c * P.A : (T0 >= hi ? T(0) : lin0);
    const T tl = qa * tail_moment(P, in0 ? T0 : T1, s);
    const T P0 = in0 ? tl : (T0 <= lo ? lin0 : T(0));
    T P1 = in1 ? tl : (T1 >= hi ? T(0) : lin1);
    if (in0 && in1) P1 = qa * tail_moment(P, T1, s);
    return P0 - P1;
}

// ---------------------------------------------------------------------------------------
// Column-view machinery shared by the voxel-driven 3D kernels.  For one voxel column (cell)
// and one view: the corner lines of the footprint are classified as below the cell (the
// atom "cell below the line" is empty), above it (the atom is the whole cell) or crossing
// it; only crossing lines get their own atom.  Element column k then has the weight
//     W(k, l) = sigma [S(line k+1, l) - S(line k, l)],  S(line, l) = Phi(line, l+1) - Phi(line, l)
// with S = 0 for empty and S = S_full for whole-cell lines, so only the element columns next
// to a crossing line carry weight.
// ---------------------------------------------------------------------------------------
template <typename T>
struct ColumnView {
    int ok, axis, sigma, k_first, ng;   // elements k_first .. k_first + ng (ng + 1 columns)
    T tmin_w, tmax_w;                   // world depth range of the column
    T margin;                           // largest |t'| in the cell
};

// Classification of the corner lines of one column's footprint (identical in every lane of
// a warp that handles the column): elements k_first .. k_first + ng carry weight, the
// crossing lines are k_first + 1 .. k_first + ng.
template <typename T>
__device__ __forceinline__ void column_view(const Geo& g, int v, int ix, int iy, ColumnView<T>& cv) {
    using L = typename LineOf<T>::type;
    const T a = G3<T>::a(g), b = G3<T>::b(g);
    const T X0 = G3<T>::x0(g) + ix * a, X1 = X0 + a, Y0 = G3<T>::y0(g) + iy * b, Y1 = Y0 + b;
    const T cs = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
    const T s = G3<T>::s(g), D = G3<T>::sdd(g);
    T umin = T(1e30), umax = T(-1e30), tmin = T(1e30), tmax = T(-1e30);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const T X = (q & 1) ? X1 : X0, Y = (q & 2) ? Y1 : Y0;
        const T t = s - X * cs - Y * sn;
        const T u = G3<T>::div(D * (Y * cs - X * sn), t);
        umin = u < umin ? u : umin;
        umax = u > umax ? u : umax;
        tmin = t < tmin ? t : tmin;
        tmax = t > tmax ? t : tmax;
    }
    cv.tmin_w = tmin;
    cv.tmax_w = tmax;
    cv.margin = T(0.5) * (fabs(a * cs) + fabs(b * sn));
    const T idu = T(1) / G3<T>::du(g);
    T f0 = floor((umin - G3<T>::u0(g)) * idu - G3<T>::eps), f1 = floor((umax - G3<T>::u0(g)) * idu + G3<T>::eps);
    cv.ok = 0;
    if (f1 < T(0) || f0 > T(g.nu - 1)) return;
    const int k0 = f0 < T(0) ? 0 : (int)f0, k1 = f1 > T(g.nu - 1) ? g.nu - 1 : (int)f1;
    const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
    cv.axis = axis;
    cv.sigma = sigma;
    const int w = axis == 0 ? ix : iy, cc = axis == 0 ? iy : ix;
    // lines k0 .. k1+1 in order; "before" type: empty for sigma > 0, whole cell for sigma < 0
    int ga = -1, gb = -1;
    for (int k = k0; k <= k1 + 1; ++k) {
        L line;
        line.load(g, v, k, w);
        T y0, y1;
        line.offsets(cc, y0, y1);
        const bool empty = y0 <= T(0) && y1 <= T(0), full = y0 >= T(1) && y1 >= T(1);
        const bool before = sigma > 0 ? empty : full, after = sigma > 0 ? full : empty;
        if (ga < 0 && !before) ga = k;
        if (!after) gb = k;
    }
    if (ga < 0) ga = k1 + 2;              // every line of the footprint is of the "before" type
    if (gb < 0) gb = k0 - 1;              // every line is of the "after" type
    if (gb < ga - 1) gb = ga - 1;
    int ng = gb - ga + 1;
    ng = ng > kMaxG ? kMaxG : ng;          // excluded by the geometry check
    cv.ng = ng;
    cv.k_first = ga - 1;
    cv.ok = 1;
}

// Atom of crossing line i (0 <= i < cv.ng) of the column.
template <typename T>
__device__ __forceinline__ void crossing_atom(const Geo& g, int v, int ix, int iy, const ColumnView<T>& cv, int i,
                                              AtomE<T>& P) {
    using L = typename LineOf<T>::type;
    const int axis = cv.axis;
    const int w = axis == 0 ? ix : iy, cc = axis == 0 ? iy : ix;
    const T a = G3<T>::a(g), b = G3<T>::b(g);
    L line;
    line.load(g, v, cv.k_first + 1 + i, w);
    T y0, y1;
    line.offsets(cc, y0, y1);
    make_atom_e<T>(P, y0, y1, axis == 0 ? a : b, axis == 0 ? b : a, axis, G3<T>::cs(g, v, 0), G3<T>::cs(g, v, 1));
}

template <typename T>
__device__ __forceinline__ void full_atom(const Geo& g, int v, AtomE<T>& P) {
    const int axis = g.axis_sigma[2 * v];
    const T a = G3<T>::a(g), b = G3<T>::b(g);
    make_atom_e<T>(P, T(2), T(2), axis == 0 ? a : b, axis == 0 ? b : a, axis, G3<T>::cs(g, v, 0), G3<T>::cs(g, v, 1));
}

// Rows of voxel [z0w, z1w] (world) seen from a column with depth range [tmin, tmax].
template <typename T>
__device__ __forceinline__ bool voxel_rows(const Geo& g, T z0w, T z1w, T tmin, T tmax, int& l0, int& l1) {
    const T D = G3<T>::sdd(g);
    const T vlo = D * (z0w < T(0) ? G3<T>::div(z0w, tmin) : G3<T>::div(z0w, tmax));
    const T vhi = D * (z1w > T(0) ? G3<T>::div(z1w, tmin) : G3<T>::div(z1w, tmax));
    const T idv = T(1) / G3<T>::dv(g);
    T h0 = floor((vlo - G3<T>::v0(g)) * idv - G3<T>::eps), h1 = floor((vhi - G3<T>::v0(g)) * idv + G3<T>::eps);
    if (h1 < T(0) || h0 > T(g.nv - 1)) return false;
    l0 = h0 < T(0) ? 0 : (int)h0;
    l1 = h1 > T(g.nv - 1) ? g.nv - 1 : (int)h1;
    return l0 <= l1;
}

// Visits every nonzero W(k, l) of voxel iz in the column (ix, iy) for view v:
// emit(k, l, W).  atoms: the column-view's crossing-line atoms; full: the whole-cell atom;
// scratch: this lane's 2 (kMaxG + 1) slots, 32 elements apart (one per lane of the warp), for
// Phi per atom on two consecutive row corner planes.
template <typename T, typename Emit>
__device__ __forceinline__ void voxel_entries(const Geo& g, int v, int ix, int iy, int iz, const ColumnView<T>& cv,
                                              const AtomE<T>* atoms, const AtomE<T>& full, T* scratch, Emit&& emit) {
    using R = typename RowOf<T>::type;
    const T c = G3<T>::c(g);
    const T z0w = G3<T>::z0(g) + iz * c;
    int l0, l1;
    if (!voxel_rows<T>(g, z0w, z0w + c, cv.tmin_w, cv.tmax_w, l0, l1)) return;
    const int ng = cv.ng, na = ng + 1;
    // PHI(b, j): Phi of atom j (0: the whole cell, j > 0: crossing line j - 1) on the row
    // corner plane held in buffer b; buffers alternate between the corners r - 1 and r
#define PHI(b, j) scratch[((b) * (kMaxG + 1) + (j)) * 32]
#pragma unroll 1
    for (int r = l0; r <= l1 + 1; ++r) {
        const int cur = r & 1, prv = cur ^ 1;
        R row;
        row.at(g, v, r, ix, iy);
        const T h = row.rel(iz);                 // plane height above the voxel bottom, units of c
        const T q = G3<T>::q(g, r);
        const T m = fabs(q) * cv.margin / c;     // height change across the cell, units of c
        const int cls = h + m <= T(0) ? 0 : (h - m >= T(1) ? 2 : 1);   // below / above / crossing
        const T gw = h * c, iq = q != T(0) ? G3<T>::div(T(1), fabs(q)) : T(0);
#pragma unroll 1
        for (int j = 0; j < na; ++j) {
            const AtomE<T>& P = j == 0 ? full : atoms[j - 1];
            PHI(cur, j) = cls == 0 ? T(0) : (cls == 2 ? c * P.A : phi_e<T>(P, gw, q, iq, c));
        }
        if (r == l0) continue;
        // W(k, l) = sigma [S(k+1) - S(k)] with S = 0 (empty lines), S_full (whole-cell lines)
        // or the crossing lines' S, over the element columns k_first .. k_first + ng
        const int l = r - 1;
        const T sf = PHI(cur, 0) - PHI(prv, 0);
        T prevS = cv.sigma > 0 ? T(0) : sf;
#pragma unroll 1
        for (int j = 0; j <= ng; ++j) {
            const T S = j < ng ? PHI(cur, j + 1) - PHI(prv, j + 1) : (cv.sigma > 0 ? sf : T(0));
            const int k = cv.k_first + j;
            const T wt = cv.sigma > 0 ? S - prevS : prevS - S;
            if (k >= 0 && k < g.nu && wt != T(0)) emit(k, l, wt);
            prevS = S;
        }
    }
#undef PHI
}

// ---------------------------------------------------------------------------------------
// Back projection: one warp per voxel column and window of 32 voxels in z (one voxel per
// lane).  All lanes of a warp share the column's view geometry: per view the lanes classify
// the footprint's corner lines identically, lanes 0 .. ng-1 build the crossing lines' atoms
// in parallel (warp-private shared memory) and the last lane the whole-cell atom; then each
// lane forms its voxel's entries and accumulates W p.
// ---------------------------------------------------------------------------------------
constexpr int BW = 4;   // warps (columns) per block

template <typename T, int NB>
__global__ void __launch_bounds__(32 * BW) back3d_vox(Geo g, const T* __restrict__ ps, void* __restrict__ x, int xdt,
                                                      int B, int b_off, T scale, int accumulate) {
    __shared__ AtomE<T> atoms_s[BW][kMaxG + 1];
    __shared__ T scratch_s[BW][2 * (kMaxG + 1) * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = blockIdx.x * BW + wid;
    if (col >= g.nx * g.ny) return;                       // whole warp leaves together
    const int ix = col % g.nx, iy = col / g.nx;
    const int iz = blockIdx.y * 32 + lane;
    AtomE<T>* atoms = atoms_s[wid];
    AtomE<T>& full = atoms_s[wid][kMaxG];
    T* scratch = scratch_s[wid] + lane;
    T acc[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] = T(0);
    for (int v = 0; v < g.n_views; ++v) {
        ColumnView<T> cv;
        column_view<T>(g, v, ix, iy, cv);
        if (!cv.ok) continue;                              // warp-uniform
        __syncwarp();
        if (lane < cv.ng) crossing_atom<T>(g, v, ix, iy, cv, lane, atoms[lane]);
        if (lane == 31) full_atom<T>(g, v, full);
        __syncwarp();
        if (iz < g.nz) {
            const T* pv = ps + (size_t)v * g.nv * g.nu * NB;
            voxel_entries<T>(g, v, ix, iy, iz, cv, atoms, full, scratch, [&](int k, int l, T wt) {
                fma_vec<T, NB>(acc, wt, pv + ((size_t)l * g.nu + k) * NB);
            });
        }
    }
    if (iz >= g.nz) return;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    const size_t vox = ((size_t)iz * g.ny + iy) * g.nx + ix;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int bidx = b_off + i;
        if (bidx < B) store_any3<T>(x, (size_t)bidx * nvox + vox, xdt, acc[i] * scale, accumulate != 0);
    }
}

// ---------------------------------------------------------------------------------------
// Forward projection, ray-driven with row windows: one warp per (view, detector column k,
// window of RW consecutive rows).  The warp walks the top-view strip of column k cell by
// cell (as in 2D); per cell two lanes build the atoms of the strip's corner lines, then the
// lanes take the voxels of the column that the window's rows reach (one voxel per lane,
// 32 at a time), form their entries for column k and add W x into per-row sums in shared
// memory, which the warp writes to p at the end (each element written by exactly one warp).
// ---------------------------------------------------------------------------------------
constexpr int FW = 4;       // warps per block
constexpr int RWMAX = 96;   // rows per warp (upper bound of the window)

template <typename T, int NB>
__global__ void __launch_bounds__(32 * FW) fwd3d_rw(Geo g, int rw, const T* __restrict__ xs0, const T* __restrict__ xs1,
                                                    void* __restrict__ p, int pdt, int B, int b_off, T scale,
                                                    int accumulate) {
    __shared__ AtomE<T> atoms_s[FW][2];
    __shared__ T rows_s[FW][RWMAX * NB];
    using L = typename LineOf<T>::type;
    using R = typename RowOf<T>::type;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = blockIdx.x * FW + wid;
    const int v = blockIdx.y;
    const int L0 = blockIdx.z * rw;
    if (k >= g.nu || L0 >= g.nv) return;                  // whole warp leaves together
    const int nrow = min(rw, g.nv - L0);
    T* rows = rows_s[wid];
    for (int i = lane; i < nrow * NB; i += 32) rows[i] = T(0);
    const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
    const int nc = axis == 0 ? g.ny : g.nx;
    const T* __restrict__ xs = axis == 0 ? xs0 : xs1;
    const T a = G3<T>::a(g), b = G3<T>::b(g), c = G3<T>::c(g);
    const T hw = axis == 0 ? a : b, hc = axis == 0 ? b : a;
    const T cs = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
    const T margin = T(0.5) * (fabs(a * cs) + fabs(b * sn));
    const T q_lo = G3<T>::q(g, L0), q_hi = G3<T>::q(g, L0 + nrow);
    const T mz = (fabs(q_lo) > fabs(q_hi) ? fabs(q_lo) : fabs(q_hi)) * margin / c + T(1e-3);
    const int w0 = g.wrange[2 * ((size_t)v * g.nu + k)], w1 = g.wrange[2 * ((size_t)v * g.nu + k) + 1];
    L la, lb;
    la.load(g, v, k, w0);
    lb.load(g, v, k + 1, w0);
    AtomE<T>& Pa = atoms_s[wid][0];
    AtomE<T>& Pb = atoms_s[wid][1];
    __syncwarp();
    for (int w = w0; w < w1; ++w) {
        int clo = min(la.cell_lo(), lb.cell_lo());
        int chi = max(la.cell_hi(), lb.cell_hi());
        clo = max(clo, 0);
        chi = min(chi, nc - 1);
        for (int cc = clo; cc <= chi; ++cc) {
            T a0, a1, b0, b1;
            la.offsets(cc, a0, a1);
            lb.offsets(cc, b0, b1);
            const bool ea = a0 <= T(0) && a1 <= T(0), eb = b0 <= T(0) && b1 <= T(0);
            const bool fa = a0 >= T(1) && a1 >= T(1), fb = b0 >= T(1) && b1 >= T(1);
            if ((ea && eb) || (fa && fb)) continue;        // the strip misses this cell (warp-uniform)
            const int ix = axis == 0 ? w : cc, iy = axis == 0 ? cc : w;
            R rl, rh;
            rl.at(g, v, L0, ix, iy);
            rh.at(g, v, L0 + nrow, ix, iy);
            const T zlo = floor(rl.rel(0) - mz), zhi = floor(rh.rel(0) + mz);
            if (zhi < T(0) || zlo > T(g.nz - 1)) continue;
            const int izlo = zlo < T(0) ? 0 : (int)zlo;
            const int izhi = zhi > T(g.nz - 1) ? g.nz - 1 : (int)zhi;
            __syncwarp();
            if (lane == 0 && !ea) make_atom_e<T>(Pa, a0, a1, hw, hc, axis, cs, sn);
            if (lane == 1 && !eb) make_atom_e<T>(Pb, b0, b1, hw, hc, axis, cs, sn);
            __syncwarp();
            const T* xcol = xs + ((size_t)w * g.nz) * nc * NB + (size_t)cc * NB;
            for (int zb = izlo; zb <= izhi; zb += 32) {
                const int iz = zb + lane;
                if (iz > izhi) continue;
                T xv[NB];
                bool any = false;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    xv[i] = __ldg(xcol + (size_t)iz * nc * NB + i);
                    any |= xv[i] != T(0);
                }
                if (!any) continue;
                int l0, l1;
                // rows of this voxel at this cell, clipped to the window
                {
                    const T z0w = G3<T>::z0(g) + iz * c;
                    const T s = G3<T>::s(g);
                    T tmin = T(1e30), tmax = T(-1e30);
                    const T X0 = G3<T>::x0(g) + ix * a, Y0 = G3<T>::y0(g) + iy * b;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const T t = s - (X0 + ((qq & 1) ? a : T(0))) * cs - (Y0 + ((qq & 2) ? b : T(0))) * sn;
                        tmin = t < tmin ? t : tmin;
                        tmax = t > tmax ? t : tmax;
                    }
                    if (!voxel_rows<T>(g, z0w, z0w + c, tmin, tmax, l0, l1)) continue;
                }
                if (l1 < L0 || l0 >= L0 + nrow) continue;
                // Phi of both lines at corners l0 .. l1+1; entries of rows in the window
                T pa = T(0), pb = T(0);
                for (int r = l0; r <= l1 + 1; ++r) {
                    R row;
                    row.at(g, v, r, ix, iy);
                    const T h = row.rel(iz);
                    const T q = G3<T>::q(g, r);
                    const T m = fabs(q) * margin / c;
                    T ca, cb;
                    if (h + m <= T(0)) {
                        ca = T(0);
                        cb = T(0);
                    } else if (h - m >= T(1)) {
                        ca = ea ? T(0) : c * Pa.A;
                        cb = eb ? T(0) : c * Pb.A;
                    } else {
                        const T gw = h * c, iq = q != T(0) ? G3<T>::div(T(1), fabs(q)) : T(0);
                        ca = ea ? T(0) : phi_e<T>(Pa, gw, q, iq, c);
                        cb = eb ? T(0) : phi_e<T>(Pb, gw, q, iq, c);
                    }
                    if (r > l0) {
                        const int l = r - 1;
                        if (l >= L0 && l < L0 + nrow) {
                            T wt = (cb - pb) - (ca - pa);
                            wt = sigma > 0 ? wt : -wt;
                            if (wt != T(0)) {
#pragma unroll
                                for (int i = 0; i < NB; ++i) atomicAdd(&rows[(l - L0) * NB + i], wt * xv[i]);
                            }
                        }
                    }
                    pa = ca;
                    pb = cb;
                }
            }
        }
        la.step();
        lb.step();
    }
    __syncwarp();
    for (int j = lane; j < nrow; j += 32) {
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int bidx = b_off + i;
            if (bidx < B)
                store_any3<T>(p, (((size_t)bidx * g.n_views + v) * g.nv + L0 + j) * g.nu + k, pdt,
                              rows[j * NB + i] * scale, accumulate != 0);
        }
    }
}

// Number of (voxel, view, element) whose volume exceeds 1e-6 of the voxel's (column-warps as
// in the back projection).
__global__ void __launch_bounds__(32 * BW) nnz3d_kernel(Geo g, unsigned long long* counter) {
    __shared__ AtomE<float> atoms_s[BW][kMaxG + 1];
    __shared__ float scratch_s[BW][2 * (kMaxG + 1) * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = blockIdx.x * BW + wid;
    if (col >= g.nx * g.ny) return;
    const int ix = col % g.nx, iy = col / g.nx;
    const int iz = blockIdx.y * 32 + lane;
    AtomE<float>* atoms = atoms_s[wid];
    AtomE<float>& full = atoms_s[wid][kMaxG];
    float* scratch = scratch_s[wid] + lane;
    const float thr = 1e-6f * g.a * g.b * g.c;
    unsigned long long cnt = 0;
    for (int v = 0; v < g.n_views; ++v) {
        ColumnView<float> cv;
        column_view<float>(g, v, ix, iy, cv);
        if (!cv.ok) continue;
        __syncwarp();
        if (lane < cv.ng) crossing_atom<float>(g, v, ix, iy, cv, lane, atoms[lane]);
        if (lane == 31) full_atom<float>(g, v, full);
        __syncwarp();
        if (iz < g.nz)
            voxel_entries<float>(g, v, ix, iy, iz, cv, atoms, full, scratch,
                                 [&](int, int, float wt) { cnt += fabsf(wt) > thr; });
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(counter, cnt);
}

// ---------------------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------------------
// Rows per forward warp: the voxels those rows reach in one cell (at the largest depth) fit
// in two passes of 32 lanes.
static int rows_per_warp(const csm_geom_s* g) {
    const double r = sqrt(pow(0.5 * g->nx * g->a, 2) + pow(0.5 * g->ny * g->b, 2));
    const double tmax = g->s + r;
    int rw = (int)floor(60.0 * g->sdd * g->c / (tmax * g->dv));
    return std::max(8, std::min(RWMAX, rw));
}

template <typename T, int NB>
static csm_status run_fwd3(const csm_geom_s* gh, const void* x, void* p, int64_t batch, csm_dtype xdt,
                           csm_dtype pdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    const size_t nvox = (size_t)gh->nx * gh->ny * gh->nz;
    const size_t half = al256(nvox * NB * sizeof(T));
    // the atoms' integrals are volumes in world units already
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1.0 / (gh->a * gh->b * gh->c)) : T(1);
    T* xs0 = (T*)ws;
    T* xs1 = (T*)((char*)ws + half);
    const int rw = rows_per_warp(gh);
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        prep_vol_3d<T, NB><<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(x, (int)xdt, (int)batch, (int)b0,
                                                                          gh->nx, gh->ny, gh->nz, xs0, xs1);
        dim3 fb(32 * FW), fg((gh->nu + FW - 1) / FW, gh->n_views, (gh->nv + rw - 1) / rw);
        fwd3d_rw<T, NB><<<fg, fb, 0, st>>>(g, rw, xs0, xs1, p, (int)pdt, (int)batch, (int)b0, scale,
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
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1.0 / (gh->a * gh->b * gh->c)) : T(1);
    const size_t n = (size_t)gh->n_views * gh->nv * gh->nu;
    const size_t ncol = (size_t)gh->nx * gh->ny;
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        prep_sino_3d<T, NB><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, (int)pdt, (int)batch, (int)b0, n, ps);
        dim3 bb(32 * BW), bg((unsigned)((ncol + BW - 1) / BW), (gh->nz + 31) / 32);
        back3d_vox<T, NB><<<bg, bb, 0, st>>>(g, ps, x, (int)xdt, (int)batch, (int)b0, scale,
                                            (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status r = check_launch();
        if (r != CSM_OK) return r;
    }
    return CSM_OK;
}

csm_status forward_3d(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt, csm_dtype pdt,
                      int flags, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    if (flags & CSM_VOXEL_DRIVEN) return CSM_EUNSUPPORTED;
    if (!ws || ws_bytes < workspace_3d(g, 0, batch, dbl)) return CSM_EINVAL;
    if (g->n_views > 65535 || (g->nv + 7) / 8 > 65535) return CSM_EUNSUPPORTED;
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
    if ((g->nz + 31) / 32 > 65535) return CSM_EUNSUPPORTED;
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
    const size_t ncol = (size_t)gh->nx * gh->ny;
    dim3 bb(32 * BW), bg((unsigned)((ncol + BW - 1) / BW), (gh->nz + 31) / 32);
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

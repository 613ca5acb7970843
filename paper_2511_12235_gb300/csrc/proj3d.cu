// proj3d.cu -- 3D circular cone-beam projectors: p = W x (ray-driven gather, a warp per
// group of detector columns) and x = W^T p (voxel-driven gather, a warp per voxel column),
// every entry W_ij evaluated on the fly.
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
// cell centre), i.e. the tail moment M(T) = integral over R of relu(t' - T) dA at the two
// kinks.  M is a cubic in T between consecutive vertex depths of R; each atom gets a table of
// those pieces (see "Tail-moment table" below), from the divergence-theorem edge sum that is
// the paper's cubic terms C g^3 (Eq. (rel vol 3d), Eq. (res vol 3d)) written per edge.
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
    // back: the differenced sinogram, 4 values per (view, corner 0..nu, plane slot 0..nv+1)
    const size_t sino = al256((size_t)g->n_views * (g->nu + 1) * (g->nv + 2) * 4 * nb * es);
    // the volume in both walk layouts and each column's range of nonzero voxels
    if (op == 0) return 2 * vol + al256((size_t)g->nx * g->ny * sizeof(int2));
    if (op == 2) {                 // voxel-driven forward: one item's layouts and its sinogram sums
        const size_t vol1 = al256((size_t)g->nx * g->ny * g->nz * es);
        return 2 * vol1 + al256((size_t)g->n_views * g->nv * g->nu * es);
    }
    if (op == 3) return sino + vol;   // back into BF16 / F16 x: and the chunk's sums in FP32 (FP64)
    return sino;
}

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
    static __device__ __forceinline__ float idu(const Geo& g) { return g.idu; }
    static __device__ __forceinline__ float idv(const Geo& g) { return g.idv; }
    static __device__ __forceinline__ float ic(const Geo& g) { return g.ic; }
    static __device__ __forceinline__ float cs(const Geo& g, int v, int i) { return g.cs_f[2 * v + i]; }
    static __device__ __forceinline__ float q(const Geo& g, int l) { return g.rowq_f[l]; }
    static __device__ __forceinline__ float qmax(const Geo& g) { return g.qmax; }
    static __device__ __forceinline__ float dq(const Geo& g) { return g.dq; }
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
    static __device__ __forceinline__ double idu(const Geo& g) { return g.idu_d; }
    static __device__ __forceinline__ double idv(const Geo& g) { return g.idv_d; }
    static __device__ __forceinline__ double ic(const Geo& g) { return g.ic_d; }
    static __device__ __forceinline__ double cs(const Geo& g, int v, int i) { return g.cs_d[2 * v + i]; }
    static __device__ __forceinline__ double q(const Geo& g, int l) { return g.rowq_d[l]; }
    static __device__ __forceinline__ double qmax(const Geo& g) { return g.qmax_d; }
    static __device__ __forceinline__ double dq(const Geo& g) { return g.dq_d; }
    static __device__ __forceinline__ double div(double x, double y) { return x / y; }
    static constexpr double eps = 1e-9;
};

// Depth of the centre of column (ix, iy) in view v over c, t_c / c = T0 + ix Tx + iy Ty
// (per-view table).  FP32: summed in 32.32 fixed point (exact) and returned as the pair
// integer part + fraction, both exact in float; FP64: in double.
__device__ __forceinline__ void column_depth(const Geo& g, int v, int ix, int iy, float& hi, float& lo) {
    const long long* e = g.colt_fx + 3 * v;
    const long long t = e[0] + (long long)ix * e[1] + (long long)iy * e[2];
    hi = (float)(int)(t >> 32);
    lo = (float)(unsigned)(t & 0xffffffffll) * 2.3283064365386963e-10f;
}
__device__ __forceinline__ void column_depth(const Geo& g, int v, int ix, int iy, double& hi, double& lo) {
    const double* e = g.colt_d + 3 * v;
    hi = e[0] + (double)ix * e[1] + (double)iy * e[2];
    lo = 0.0;
}

// Height of row corner plane l above the bottom face of voxel iz at the column centre, in
// units of c:  h = q_l t_c / c - (iz - nz / 2)  (the plane is z = q_l t, the voxel's bottom
// z0 + iz c).  FP32: the product of the float pairs q = qh + ql and t_c / c = dh + dl with
// its rounding error recovered by an FMA, so h carries an absolute error of a few 1e-7
// whatever the magnitudes of q t_c / c and iz.  Also returns q and 1/|q| (0 for q = 0).
__device__ __forceinline__ float plane_height(const Geo& g, int l, int iz, float dh, float dl, float& q, float& iq) {
    const float4 r = __ldg(g.rowq4 + l);
    const float p = r.x * dh;
    const float e = fmaf(r.x, dh, -p);
    const float izp = (float)iz - 0.5f * (float)g.nz;
    q = r.x;
    iq = r.z;
    return (p - izp) + (e + fmaf(r.x, dl, r.y * dh));
}
__device__ __forceinline__ double plane_height(const Geo& g, int l, int iz, double dh, double, double& q, double& iq) {
    q = g.rowq_d[l];
    iq = q != 0.0 ? 1.0 / fabs(q) : 0.0;
    return q * dh - ((double)iz - 0.5 * (double)g.nz);
}

// ---------------------------------------------------------------------------------------
// Layouts.  The forward deals the voxels of one column to the lanes of a warp, so it reads x
// with z innermost: xs0[ix][iy][iz][NB] (walk x) / xs1[iy][ix][iz][NB] (walk y).  The back
// projection deals neighbouring voxels of a column to neighbouring lanes, whose rows of the
// detector are neighbours too, so it reads p with the rows innermost: ps[v][k][l][NB].
// Both copies are made by 32 x 32 tiled transposes through shared memory (coalesced reads
// and writes).
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(256) prep_vol_3d(const void* __restrict__ x, int xdt, int B, int b_off, int nx,
                                                   int ny, int nz, T* __restrict__ xs0, T* __restrict__ xs1) {
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, z0 = blockIdx.y * 32, iy = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t n = (size_t)nx * ny * nz;
    for (int bb = 0; bb < NB; ++bb) {
        const int b = b_off + bb;
        for (int j = ty; j < 32; j += 8) {
            const int ix = x0 + tx, iz = z0 + j;
            T val = T(0);
            if (ix < nx && iz < nz && b < B) val = load_any3<T>(x, (size_t)b * n + ((size_t)iz * ny + iy) * nx + ix, xdt);
            tile[j][tx] = val;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int ix = x0 + j, iz = z0 + tx;
            if (ix < nx && iz < nz) {
                const T val = tile[tx][j];
                xs0[(((size_t)ix * ny + iy) * nz + iz) * NB + bb] = val;
                xs1[(((size_t)iy * nx + ix) * nz + iz) * NB + bb] = val;
            }
        }
        __syncthreads();
    }
}

// First and last voxel of each column (ix, iy) that holds a nonzero value of the chunk's items
// (lo > hi when there is none), from the z-innermost copy: one warp per column, the lanes
// reading 32 neighbouring voxels at a time.  The forward skips columns without one and limits
// the planes of the others to their range.
template <typename T, int NB>
__global__ void __launch_bounds__(256) col_range_3d(const T* __restrict__ xs0, int ncol, int nz,
                                                    int2* __restrict__ rng) {
    const int lane = threadIdx.x & 31;
    const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (col >= ncol) return;                               // whole warp leaves together
    const T* __restrict__ xc = xs0 + (size_t)col * nz * NB;
    int lo = 0x7fffffff, hi = -1;
    for (int zb = 0; zb < nz; zb += 32) {
        const int iz = zb + lane;
        bool nzv = false;
        if (iz < nz) {
#pragma unroll
            for (int i = 0; i < NB; ++i) nzv |= xc[(size_t)iz * NB + i] != T(0);
        }
        const unsigned m = __ballot_sync(0xffffffffu, nzv);
        if (m) {
            if (lo == 0x7fffffff) lo = zb + __ffs(m) - 1;
            hi = zb + 31 - __clz(m);
        }
    }
    if (lane == 0) rng[col] = make_int2(lo, hi);
}

// The back projection reads, per view, corner / element column i = 0 .. nu and plane slot
// r = 0 .. nv + 1 (p = 0 outside the detector), the four values
//     .x  DD(i, r) = Dc(i, r - 1) - Dc(i, r)      Dc(i, l) = p(i - 1, l) - p(i, l)
//     .y  Dc(i, r - 1)
//     .z  Dy(i, r) = p(i, r - 1) - p(i, r)
//     .w  p(i, r - 1)
// stored as q[v][i][r][component][NB] (the sums by parts of the voxel_back_fast form).  Each
// block differences a 32 x 32 tile of p held in shared memory with a one-element halo.
template <typename T, int NB>
__global__ void __launch_bounds__(256) prep_diff_3d(Geo g, const void* __restrict__ p, int pdt, int B, int b_off,
                                                    int nu, int nv, T* __restrict__ q) {
    __shared__ T tile[34][34];   // p(i0 - 1 + a, r0 - 1 + b) at tile[b][a], a, b in [0, 33]
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32, v = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const size_t plane = (size_t)nu * nv;
    const size_t nvw = plane * gridDim.z;
    const size_t slots = (size_t)(nu + 1) * (nv + 2);
    for (int bb = 0; bb < NB; ++bb) {
        const int b = b_off + bb;
        for (int e = ty * 32 + tx; e < 34 * 34; e += 256) {
            const int ta = e % 34, tb = e / 34;
            const int k = i0 - 1 + ta, l = r0 - 1 + tb;
            T val = T(0);
            if (k >= 0 && k < nu && l >= 0 && l < nv && b < B)
                val = elem_weight<T>(g, (size_t)v * plane + (size_t)l * nu + k) *
                      load_any3<T>(p, (size_t)b * nvw + (size_t)v * plane + (size_t)l * nu + k, pdt);
            tile[tb][ta] = val;
        }
        __syncthreads();
        // thread (tx, ty): plane slot r = r0 + tx (coalesced writes along r), corners i0 + ty + 8 j
        const int r = r0 + tx;
        for (int j = ty; j < 32; j += 8) {
            const int i = i0 + j;
            if (i <= nu && r <= nv + 1) {
                // tile coordinates of p(i - 1, r - 1): (a, b) = (j, tx)
                const T pm1 = tile[tx][j], p0m1 = tile[tx][j + 1];     // p(i-1, r-1), p(i, r-1)
                const T pm0 = tile[tx + 1][j], p00 = tile[tx + 1][j + 1];  // p(i-1, r),   p(i, r)
                const T dcm = pm1 - p0m1, dc0 = pm0 - p00;
                T* dst = q + (((size_t)v * slots + (size_t)i * (nv + 2) + r) * 4) * NB + bb;
                dst[0] = dcm - dc0;
                dst[NB] = dcm;
                dst[2 * NB] = p0m1 - p00;
                dst[3 * NB] = p0m1;
            }
        }
        __syncthreads();
    }
}

template <typename T, int NB>
__device__ __forceinline__ void fma_vec(T (&acc)[NB], T wt, const T* __restrict__ src) {
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] += wt * __ldg(src + i);
}

// ---------------------------------------------------------------------------------------
// Tail-moment table of a top-view atom.  The tail moment
//     M(T) = integral over the atom of relu(t' - T) dA
// (t' = depth relative to the cell centre) is a cubic in T between consecutive vertex depths
// of the atom: by the divergence theorem it is  -(1/6) sum_e w_e E_e(T)  over the atom's
// edges, w_e = e_s . (outward normal x length) projected on the source direction and
// E_e = a^2 + a b + b^2 (both ends beyond T) or a^3 / |t'_a - t'_b| (one end beyond T),
// a >= b the parts of the ends beyond T.  These are the paper's cubic terms C g^3
// (Eq. (rel vol 3d), Eq. (res vol 3d)) written per edge instead of per vertex, which removes
// the 1/sin(phi), 1/cos(phi) factors of the printed forms (their singular views, Eq. (vol))
// from the arithmetic.  The table holds the six vertex depths sorted, tau_0 <= .. <= tau_5,
// and per piece the Taylor coefficients of M at the piece's base:
//     piece 0      T <  tau_0                linear  M(tau_0) - A (T - tau_0)
//     piece p      tau_{p-1} <= T < tau_p    cubic, base tau_{p-1}   (p = 1 .. 5)
//     piece 6      T >= tau_5                zero
// so that M costs six comparisons and three FMAs, the same for every lane.
// ---------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

template <typename T>
struct __align__(16) AtomP {
    T cf[7][4];   // per piece: M and its first three derivatives / n! at the piece's base
    T tau[6];     // sorted vertex depths
    T A;          // area
    T M1;         // first moment of the depth t' over the atom (integral of t' dA)
};

template <typename T> struct Cf4;
template <> struct Cf4<float> {
    float x, y, z, w;
    __device__ __forceinline__ void load(const float* p) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        x = v.x; y = v.y; z = v.z; w = v.w;
    }
};
template <> struct Cf4<double> {
    double x, y, z, w;
    __device__ __forceinline__ void load(const double* p) {
        const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
        x = v0.x; y = v0.y; z = v1.x; w = v1.y;
    }
};

// Piece p (1 <= p <= 5) of the table of the atom "cell below the line with offsets lam0, lam1
// at the walk boundaries" (units of hc; lam >= 1 on both ends: the whole cell); the call with
// p == 1 also writes tau, A and pieces 0 and 6.  Every lane that builds a piece of the same
// atom computes the same vertices and the same sorted depths.
template <typename T>
__device__ __forceinline__ void build_piece(AtomP<T>& P, int p, T lam0, T lam1, T hw, T hc, int axis, T cs, T sn) {
    const T dl = lam1 - lam0;
    T xa = T(1), xb = T(1);
    if (dl != T(0)) {
        const T r = G3<T>::div(T(1), dl);
        xa = clamp01(-lam0 * r);
        xb = clamp01((T(1) - lam0) * r);
    }
    const T xhi = xa > xb ? xa : xb, xlo = xa > xb ? xb : xa;
    // vertices in cell units (walk coordinate XI, cross coordinate ET), counter-clockwise
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
    T ts[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) ts[i] = TP[i];
    // sorting network for six keys
#define CSM_CX(i, j) { const T lo_ = ts[i] < ts[j] ? ts[i] : ts[j], hi_ = ts[i] < ts[j] ? ts[j] : ts[i]; ts[i] = lo_; ts[j] = hi_; }
    CSM_CX(0, 5) CSM_CX(1, 3) CSM_CX(2, 4) CSM_CX(1, 2) CSM_CX(3, 4) CSM_CX(0, 3)
    CSM_CX(2, 5) CSM_CX(0, 1) CSM_CX(2, 3) CSM_CX(4, 5) CSM_CX(1, 2) CSM_CX(3, 4)
#undef CSM_CX
    T base = ts[0], top = ts[1];
#pragma unroll
    for (int i = 1; i < 5; ++i)
        if (p == i + 1) { base = ts[i]; top = ts[i + 1]; }
    const T mid = T(0.5) * (base + top);
    const T orient = axis == 0 ? T(1) : T(-1);
    T c0 = T(0), c1 = T(0), c2 = T(0), c3 = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int j = (i + 1) % 6;
        const T w = orient * (cs * (DY[j] - DY[i]) - sn * (DX[j] - DX[i]));
        const T hi = TP[i] > TP[j] ? TP[i] : TP[j], lo = TP[i] > TP[j] ? TP[j] : TP[i];
        const T a = hi - base, b = lo - base;
        if (mid < lo) {                 // both ends beyond T on the whole piece
            c0 += w * (a * a + a * b + b * b);
            c1 -= w * T(3) * (a + b);
            c2 += w * T(3);
        } else if (mid < hi) {          // one end beyond
            const T inv = G3<T>::div(T(1), hi - lo);
            c0 += w * a * a * a * inv;
            c1 -= w * T(3) * a * a * inv;
            c2 += w * T(3) * a * inv;
            c3 -= w * inv;
        }
    }
    const T k = T(-1.0 / 6.0);
    T* row = P.cf[p];
    row[0] = k * c0; row[1] = k * c1; row[2] = k * c2; row[3] = k * c3;
    if (p == 1) {
        P.cf[0][0] = k * c0; P.cf[0][1] = k * c1; P.cf[0][2] = T(0); P.cf[0][3] = T(0);
        P.cf[6][0] = T(0); P.cf[6][1] = T(0); P.cf[6][2] = T(0); P.cf[6][3] = T(0);
        // area and first moment of t' by a fan of triangles from the cell centre (where t' = 0):
        // each edge's triangle has signed area cr/2 and mean t' (TP_i + TP_j)/3
        T a2 = T(0), m6 = T(0);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const int j = (i + 1) % 6;
            const T cr = (XI[i] - T(0.5)) * (ET[j] - T(0.5)) - (XI[j] - T(0.5)) * (ET[i] - T(0.5));
            a2 += cr;
            m6 += cr * (TP[i] + TP[j]);
            P.tau[i] = ts[i];
        }
        P.A = T(0.5) * a2 * hw * hc;
        P.M1 = m6 * hw * hc * T(1.0 / 6.0);
    }
}

// M(x) from the table; tau: the table's sorted depths, already in registers.
template <typename T>
__device__ __forceinline__ T eval_m(const AtomP<T>& P, const T (&tau)[6], T x) {
    int idx = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) idx += x >= tau[i] ? 1 : 0;
    const T base = P.tau[idx > 0 ? idx - 1 : 0];
    Cf4<T> c;
    c.load(P.cf[idx]);
    const T d = x - base;
    return ((c.w * d + c.z) * d + c.y) * d + c.x;
}

// Phi = integral over the atom of clamp(g + q t', 0, c) dA, iq = 1 / |q| (0 for q = 0).
// The clamp is relu(g + q t') - relu(g + q t' - c), whose kinks are the plane's crossings of
// the voxel's bottom and top faces; for q > 0 the two relu integrals are |q| M(-g/|q|) and
// |q| M((c - g)/|q|), for q < 0 the mirror relu(-y) = relu(y) - y gives
// |q| [M(g/|q|) - M((g - c)/|q|)] + c A.
template <typename T>
__device__ __forceinline__ T phi_p(const AtomP<T>& P, T g, T q, T iq, T c) {
    const T qa = fabs(q), sg = q < T(0) ? T(-1) : T(1);
    const T x0 = -g * iq * sg, x1 = (c - g) * iq * sg;
    T tau[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) tau[i] = P.tau[i];
    const T r = qa * (eval_m<T>(P, tau, x0) - eval_m<T>(P, tau, x1)) + (q < T(0) ? c * P.A : T(0));
    return q == T(0) ? (g < T(0) ? T(0) : (g > c ? c : g)) * P.A : r;
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
    int kin;                            // all of them on the detector
    T tmin_w, tmax_w;                   // world depth range of the column
    T margin_c;                         // largest |t'| in the cell, in units of the voxel height c
    T dh, dl;                           // centre depth / c as a pair (column_depth)
    int fast;                           // planes meet voxel faces one at a time (see face_kink)
};

// Classification of the corner lines of one column's footprint, computed cooperatively by
// the 32 lanes of a warp (the result is identical in every lane): the four cell corners are
// projected by lane groups of four, the lines k0 .. k1+1 of the footprint are classified one
// per lane, and ballots give the first and last line that is not of the "before" / "after"
// type.  Elements k_first .. k_first + ng carry weight, the crossing lines are
// k_first + 1 .. k_first + ng.  With [klo, khi] only those lines are classified (lines below
// the footprint count as "before", lines above it as "after"): the entries of the elements
// klo .. khi-1 are then exact, the others must not be used.  cv.ok = 0 when the cell gives
// those elements no weight.
template <typename T>
__device__ __forceinline__ void column_view(const Geo& g, int v, int ix, int iy, int lane, ColumnView<T>& cv,
                                            int klo = 0, int khi = 0x7fffffff) {
    using L = typename LineOf<T>::type;
    const T a = G3<T>::a(g), b = G3<T>::b(g);
    const T X0 = G3<T>::x0(g) + ix * a, Y0 = G3<T>::y0(g) + iy * b;
    const T cs = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
    const T s = G3<T>::s(g), D = G3<T>::sdd(g);
    const int qd = lane & 3;
    const T X = X0 + ((qd & 1) ? a : T(0)), Y = Y0 + ((qd & 2) ? b : T(0));
    const T t = s - X * cs - Y * sn;
    const T u = G3<T>::div(D * (Y * cs - X * sn), t);
    T umin = u, umax = u, tmin = t, tmax = t;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        const T u2 = __shfl_xor_sync(0xffffffffu, umin, o), u3 = __shfl_xor_sync(0xffffffffu, umax, o);
        const T t2 = __shfl_xor_sync(0xffffffffu, tmin, o), t3 = __shfl_xor_sync(0xffffffffu, tmax, o);
        umin = u2 < umin ? u2 : umin;
        umax = u3 > umax ? u3 : umax;
        tmin = t2 < tmin ? t2 : tmin;
        tmax = t3 > tmax ? t3 : tmax;
    }
    cv.tmin_w = tmin;
    cv.tmax_w = tmax;
    column_depth(g, v, ix, iy, cv.dh, cv.dl);
    cv.margin_c = T(0.5) * (fabs(a * cs) + fabs(b * sn)) * G3<T>::ic(g);
    {
        // A row plane dips below / rises above a horizontal voxel face inside the cell only
        // within m = |q| margin_c (units of c) of it.  When 2 m is below the smallest spacing
        // of neighbouring planes at this column (dq t_min / c) and m < 1/2, at most one plane
        // does so at each face and no plane does so at both faces of one voxel.
        const T m = G3<T>::qmax(g) * cv.margin_c;
        const T pitch = G3<T>::dq(g) * tmin * G3<T>::ic(g);
        cv.fast = (T(2) * m + T(0.02) < pitch) && (m < T(0.45));
    }
    const T idu = G3<T>::idu(g);
    T f0 = floor((umin - G3<T>::u0(g)) * idu - G3<T>::eps), f1 = floor((umax - G3<T>::u0(g)) * idu + G3<T>::eps);
    cv.ok = 0;
    if (f1 < T(0) || f0 > T(g.nu - 1)) return;
    const int k0 = f0 < T(0) ? 0 : (int)f0, k1 = f1 > T(g.nu - 1) ? g.nu - 1 : (int)f1;
    const int la = k0 > klo ? k0 : klo, lb = k1 + 1 < khi ? k1 + 1 : khi;   // lines classified
    if (la > lb) return;
    const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
    cv.axis = axis;
    cv.sigma = sigma;
    const int w = axis == 0 ? ix : iy, cc = axis == 0 ? iy : ix;
    // line la + lane; "before" type: empty for sigma > 0, whole cell for sigma < 0
    bool not_before = false, not_after = false;
    if (lane <= lb - la) {
        L line;
        line.load(g, v, la + lane, w);
        T y0, y1;
        line.offsets(cc, y0, y1);
        const bool empty = y0 <= T(0) && y1 <= T(0), full = y0 >= T(1) && y1 >= T(1);
        not_before = !(sigma > 0 ? empty : full);
        not_after = !(sigma > 0 ? full : empty);
    }
    const unsigned mb = __ballot_sync(0xffffffffu, not_before), ma = __ballot_sync(0xffffffffu, not_after);
    const int ga = mb ? la + __ffs(mb) - 1 : lb + 1;     // every line is of the "before" type
    int gb = ma ? la + 31 - __clz(ma) : la - 1;          // every line is of the "after" type
    if (gb < ga - 1) gb = ga - 1;
    int ng = gb - ga + 1;
    ng = ng > kMaxG ? kMaxG : ng;          // excluded by the geometry check
    cv.ng = ng;
    cv.k_first = ga - 1;
    cv.kin = cv.k_first >= 0 && cv.k_first + ng < g.nu;
    cv.ok = 1;
}

// Voxels of the grid that the detector's rows can reach from a column with world depth range
// [tmin, tmax] (conservative by one voxel on each side; the exact row range of each voxel is
// decided by voxel_rows).
template <typename T>
__device__ __forceinline__ void cone_z_range(const Geo& g, T tmin, T tmax, int& izlo, int& izhi) {
    const T D = G3<T>::sdd(g), vb = G3<T>::v0(g), vt = vb + T(g.nv) * G3<T>::dv(g);
    const T zmin = G3<T>::div(vb * (vb < T(0) ? tmax : tmin), D);
    const T zmax = G3<T>::div(vt * (vt > T(0) ? tmax : tmin), D);
    const T ic = G3<T>::ic(g);
    T lo = floor((zmin - G3<T>::z0(g)) * ic) - T(1), hi = floor((zmax - G3<T>::z0(g)) * ic) + T(1);
    lo = lo < T(0) ? T(0) : lo;
    hi = hi > T(g.nz - 1) ? T(g.nz - 1) : hi;
    izlo = (int)lo;
    izhi = hi < lo ? izlo - 1 : (int)hi;
}

// Piece p of the table of atom i of the column: crossing line i for 0 <= i < cv.ng, the whole
// cell for i = cv.ng (a line above the cell).  One code path for both, so that the lanes
// building them do not diverge.
template <typename T>
__device__ __forceinline__ void column_piece(const Geo& g, int v, int ix, int iy, const ColumnView<T>& cv, int i,
                                             int p, AtomP<T>& P) {
    using L = typename LineOf<T>::type;
    const int axis = cv.axis;
    const int w = axis == 0 ? ix : iy, cc = axis == 0 ? iy : ix;
    const T a = G3<T>::a(g), b = G3<T>::b(g);
    T y0 = T(2), y1 = T(2);
    if (i < cv.ng) {
        L line;
        line.load(g, v, cv.k_first + 1 + i, w);
        line.offsets(cc, y0, y1);
    }
    build_piece<T>(P, p, y0, y1, axis == 0 ? a : b, axis == 0 ? b : a, axis, G3<T>::cs(g, v, 0), G3<T>::cs(g, v, 1));
}

// Builds the tables of the column's ng + 1 atoms, one (atom, piece) per lane.
template <typename T>
__device__ __forceinline__ void column_atoms(const Geo& g, int v, int ix, int iy, const ColumnView<T>& cv, int lane,
                                             AtomP<T>* atoms) {
    for (int it = lane; it < (cv.ng + 1) * 5; it += 32) {
        const int i = it / 5, p = it - 5 * i + 1;
        column_piece<T>(g, v, ix, iy, cv, i, p, atoms[i == cv.ng ? kMaxG : i]);
    }
}

// Rows of voxel [z0w, z1w] (world) seen from a column with depth range [tmin, tmax].
template <typename T>
__device__ __forceinline__ bool voxel_rows(const Geo& g, T z0w, T z1w, T tmin, T tmax, int& l0, int& l1) {
    const T D = G3<T>::sdd(g);
    const T vlo = D * (z0w < T(0) ? G3<T>::div(z0w, tmin) : G3<T>::div(z0w, tmax));
    const T vhi = D * (z1w > T(0) ? G3<T>::div(z1w, tmin) : G3<T>::div(z1w, tmax));
    const T idv = G3<T>::idv(g);
    T h0 = floor((vlo - G3<T>::v0(g)) * idv - G3<T>::eps), h1 = floor((vhi - G3<T>::v0(g)) * idv + G3<T>::eps);
    if (h1 < T(0) || h0 > T(g.nv - 1)) return false;
    l0 = h0 < T(0) ? 0 : (int)h0;
    l1 = h1 > T(g.nv - 1) ? g.nv - 1 : (int)h1;
    return l0 <= l1;
}

// Visits every nonzero W(k, l) of voxel iz in the column (ix, iy) for view v through a sink:
// sink.add(k, l, W) for each entry.  atoms: the column-view's crossing-line atoms; full: the
// whole-cell atom.
template <typename T, typename Sink>
__device__ __forceinline__ void voxel_entries(const Geo& g, int v, int ix, int iy, int iz, const ColumnView<T>& cv,
                                              const AtomP<T>* atoms, const AtomP<T>& full, Sink& sink) {
    const T c = G3<T>::c(g);
    const T z0w = G3<T>::z0(g) + iz * c;
    int l0, l1;
    if (!voxel_rows<T>(g, z0w, z0w + c, cv.tmin_w, cv.tmax_w, l0, l1)) return;
    const int ng = cv.ng, na = ng + 1;
    // pc[j] / pp[j]: Phi of atom j (0: the whole cell, j > 0: crossing line j - 1) on the row
    // corner planes r and r - 1 (registers: the loops over atoms are unrolled, their bounds
    // are the same in every lane of the warp)
    T pc[kMaxG + 1], pp[kMaxG + 1];
#pragma unroll
    for (int j = 0; j <= kMaxG; ++j) pp[j] = T(0);
#pragma unroll 1
    for (int r = l0; r <= l1 + 1; ++r) {
        T q, iq;
        const T h = plane_height(g, r, iz, cv.dh, cv.dl, q, iq);   // above the voxel bottom, units of c
        const T m = fabs(q) * cv.margin_c;       // height change across the cell, units of c
        const int cls = h + m <= T(0) ? 0 : (h - m >= T(1) ? 2 : 1);   // below / above / crossing
        const T gw = h * c;
#pragma unroll
        for (int j = 0; j <= kMaxG; ++j) {
            if (j < na) {
                const AtomP<T>& P = j == 0 ? full : atoms[j - 1];
                pc[j] = cls == 0 ? T(0) : (cls == 2 ? c * P.A : phi_p<T>(P, gw, q, iq, c));
            } else {
                pc[j] = T(0);
            }
        }
        if (r > l0) {
            // W(k, l) = sigma [S(k+1) - S(k)] with S = 0 (empty lines), S_full (whole-cell
            // lines) or the crossing lines' S, over the element columns k_first .. k_first + ng
            const int l = r - 1;
            const T sf = pc[0] - pp[0];
            T prevS = cv.sigma > 0 ? T(0) : sf;
#pragma unroll
            for (int j = 0; j <= kMaxG; ++j) {
                if (j <= ng) {
                    const T S = j < ng ? pc[j < kMaxG ? j + 1 : kMaxG] - pp[j < kMaxG ? j + 1 : kMaxG] : (cv.sigma > 0 ? sf : T(0));
                    const int k = cv.k_first + j;
                    const T wt = cv.sigma > 0 ? S - prevS : prevS - S;
                    if ((cv.kin || (k >= 0 && k < g.nu)) && wt != T(0)) sink.add(k, l, wt);
                    prevS = S;
                }
            }
        }
#pragma unroll
        for (int j = 0; j <= kMaxG; ++j) pp[j] = pc[j];
    }
}

// ---------------------------------------------------------------------------------------
// Faces and kinks (the fast form of Phi).  With y = g + q t' the plane's height above the
// voxel's bottom face,  clamp(y, 0, c) = y + relu(-y) - relu(y - c).  A plane whose height
// range over the cell (h +- m in units of c, m = |q| margin_c) lies inside (0, 1) therefore has
// the linear Phi = g A + q M1 (A the atom's area, M1 its first moment of t'), a plane below
// the voxel Phi = 0 and one above Phi = c A.  Only a plane within m of a face needs the tail
// moments, and its correction is one number per (face, atom): the volume on the minority side
// of the plane next to the face,
//     K_f = integral over the atom of relu(s (g_f + q t')),   s = -sign(g_f)   (g_f: the
// plane's height above face f at the cell centre),
// which enters the voxel above the face with + and the voxel below it with -:
//     Phi(plane, voxel iz) = base(h) + K_iz - K_{iz+1},
//     base(h) = 0 (h < 0), g A + q M1 (0 <= h < 1), c A (h >= 1),  h at the cell centre.
// With relu(q (t' - x)), x = -g / q, one table evaluation gives K: |q| M(x) or |q| H(x) with
// the head moment H(x) = integral of relu(x - t') = x A - M1 + M(x).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T kink_tail(const AtomP<T>& P, T gw, T q, T iq, bool below) {
    T tau[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) tau[i] = P.tau[i];
    const T x = -gw * (q < T(0) ? -iq : iq);
    const bool use_m = below == (q > T(0));
    const T mv = eval_m<T>(P, tau, x);
    return fabs(q) * (use_m ? mv : mv + (x * P.A - P.M1));
}

// The plane (if any) that meets the bottom face of voxel iz inside the cell: returns its index
// rb (or -1) with its height hb above the face (units of c), q and 1/|q|; ra receives the first
// plane whose height at the cell centre is at or above the face (0 .. nv + 1), ha and qa its
// height above the face and q when ra <= nv.  Requires cv.fast.
template <typename T>
__device__ __forceinline__ int face_plane(const Geo& g, int iz, const ColumnView<T>& cv, int& ra, T& ha, T& qa,
                                          T& hb, T& qb, T& iqb) {
    // nearest planes: q t_c / c = iz - nz/2 at the face, planes q_r = (v0 + r dv) / sdd
    const T fz = T(iz) - T(0.5) * T(g.nz);
    const T qf = G3<T>::div(fz, cv.dh + cv.dl);
    const T rf = (qf * G3<T>::sdd(g) - G3<T>::v0(g)) * G3<T>::idv(g);
    const T rfl = floor(rf);
    // the two planes around the face (plane heights increase with r)
    const int r0 = rfl < T(-1) ? -1 : (rfl > T(g.nv) ? g.nv : (int)rfl);
    int rb = -1;
    hb = T(0);
    qb = T(0);
    iqb = T(0);
    ra = r0 + 1;
    ha = T(0);
    qa = T(0);
    bool found = false;
#pragma unroll
    for (int c2 = 0; c2 < 2; ++c2) {
        const int r = r0 + c2;
        if (r >= 0 && r <= g.nv) {
            T q, iq;
            const T h = plane_height(g, r, iz, cv.dh, cv.dl, q, iq);
            if (!found && h >= T(0)) { ra = r; ha = h; qa = q; found = true; }
            if (fabs(h) < fabs(q) * cv.margin_c) { rb = r; hb = h; qb = q; iqb = iq; }
        }
    }
    return rb;
}

// face_plane, and the plane's K for the whole-cell atom (slot 0) and each crossing line's atom
// (slots 1 .. ng), written to kslot.
template <typename T>
__device__ __forceinline__ int face_kink(const Geo& g, int iz, const ColumnView<T>& cv, const AtomP<T>* atoms,
                                         const AtomP<T>& full, T* kslot, int& ra, T& ha, T& qa) {
    T hb, qb, iqb;
    const int rb = face_plane<T>(g, iz, cv, ra, ha, qa, hb, qb, iqb);
    const int na = cv.ng + 1;
    const T gw = hb * G3<T>::c(g);
#pragma unroll
    for (int j = 0; j <= kMaxG; ++j) {
        if (j < na) {
            T kv = T(0);
            if (rb >= 0) kv = kink_tail<T>(j == 0 ? full : atoms[j - 1], gw, qb, iqb, hb < T(0));
            kslot[j] = kv;
        }
    }
    return rb;
}

// Where the columns of one (voxel column, view) sit in the differenced sinogram: the first
// crossing line k1, the boundary column bcol of the whole-cell lines (valid when bok) and the
// sign sb it carries after telescoping.
struct BackCols {
    int k1, bcol;
    bool bok;
    float sb;
};
template <typename T>
__device__ __forceinline__ BackCols back_cols(const Geo& g, const ColumnView<T>& cv) {
    BackCols bc;
    bc.bcol = cv.sigma > 0 ? cv.k_first + cv.ng : cv.k_first;
    bc.bok = bc.bcol >= 0 && bc.bcol < g.nu;
    bc.sb = cv.sigma > 0 ? 1.0f : -1.0f;
    bc.k1 = cv.k_first + 1;
    return bc;
}

// The back projection's term of one face f (the bottom face of voxel iz): with the plane rb that
// meets it inside the cell and the K of each atom, F_f = sum over atoms of K times the atom's
// column of the differenced sinogram at plane rb.  It enters voxel iz with + and voxel iz - 1
// with - (Phi = base + K_iz - K_{iz+1}), so each face's term is formed once, by the lane of
// the voxel above it.  Returns rb; ra, ha, qa as face_plane.
template <typename T, int NB>
__device__ __forceinline__ int face_back(const Geo& g, int iz, const ColumnView<T>& cv, const AtomP<T>* atoms,
                                         const AtomP<T>& full, const T* __restrict__ qv, const BackCols& bc, int& ra,
                                         T& ha, T& qa, T (&ff)[NB]) {
    T hb, qb, iqb;
    const int rb = face_plane<T>(g, iz, cv, ra, ha, qa, hb, qb, iqb);
#pragma unroll
    for (int n = 0; n < NB; ++n) ff[n] = T(0);
    if (rb >= 0) {
        const int ns = g.nv + 2;
        const T gw = hb * G3<T>::c(g);
        const bool below = hb < T(0);
#pragma unroll
        for (int j = 0; j < kMaxG; ++j)
            if (j < cv.ng)
                fma_vec<T, NB>(ff, kink_tail<T>(atoms[j], gw, qb, iqb, below),
                               qv + (((size_t)(bc.k1 + j) * ns + rb) * 4 + 0) * NB);
        if (bc.bok)
            fma_vec<T, NB>(ff, T(bc.sb) * kink_tail<T>(full, gw, qb, iqb, below),
                           qv + (((size_t)bc.bcol * ns + rb) * 4 + 2) * NB);
    }
    return rb;
}

// Back projection of one voxel for one view in the fast form, by sums by parts over the
// detector's columns and rows.  With Phi_i(r) the volume of the voxel below row plane r and
// below corner line i (lines left of the footprint: empty or the whole cell, right of it:
// the other), the voxel's value  sum_{k,l} W(k, l) p(k, l)  equals
//     sigma sum_i sum_r Phi_i(r) DD(i, r)      (p = 0 outside the detector),
// Phi_i(r) = 0 for planes below the voxel and c A_i for planes above it, and the lines of
// the whole-cell type telescope into the footprint's boundary column b.  What remains per
// line: the planes whose centre lies in the voxel (ra .. rtop - 1) with the linear Phi, the
// first plane above (c A_i Dc(i, rtop - 1)), and the two face corrections K.  q: this view's
// differenced projections (prep_diff_3d).
template <typename T, int NB>
__device__ __forceinline__ void voxel_back_fast(const Geo& g, int iz, const ColumnView<T>& cv, const AtomP<T>* atoms,
                                                const AtomP<T>& full, const T* __restrict__ qv, const BackCols& bc,
                                                int ra, T ha, T qa, int rtop, const T (&corr)[NB], T (&sum)[NB]) {
    const int ng = cv.ng;
    const int ns = g.nv + 2;
    const T c = G3<T>::c(g);
    const int bcol = bc.bcol, k1 = bc.k1;
    const bool bok = bc.bok;
    const T sb = T(bc.sb);
    auto at = [&](int i, int r, int comp) { return qv + (((size_t)i * ns + r) * 4 + comp) * NB; };
    T acc[NB];
#pragma unroll
    for (int n = 0; n < NB; ++n) acc[n] = corr[n];   // the two faces' terms
    const int rlo = ra < 0 ? 0 : ra, rhi = rtop > g.nv + 1 ? g.nv + 1 : rtop;
    T q = qa, hr = ha;                  // the first plane's height came with ra
    for (int r = rlo; r < rhi; ++r) {   // planes with their centre inside the voxel (r <= nv)
        T iq;
        if (r != rlo) hr = plane_height(g, r, iz, cv.dh, cv.dl, q, iq);
        const T gw = hr * c;
#pragma unroll
        for (int j = 0; j < kMaxG; ++j) {
            if (j < ng) {
                const AtomP<T>& P = atoms[j];
                fma_vec<T, NB>(acc, gw * P.A + q * P.M1, at(k1 + j, r, 0));
            }
        }
        if (bok) fma_vec<T, NB>(acc, sb * gw * full.A, at(bcol, r, 2));
    }
    // the first plane above the voxel: the telescoped sum of every plane above it
#pragma unroll
    for (int j = 0; j < kMaxG; ++j)
        if (j < ng) fma_vec<T, NB>(acc, c * atoms[j].A, at(k1 + j, rhi, 1));
    if (bok) fma_vec<T, NB>(acc, sb * c * full.A, at(bcol, rhi, 3));
    const T sg = cv.sigma > 0 ? T(1) : T(-1);
#pragma unroll
    for (int n = 0; n < NB; ++n) sum[n] = sg * acc[n];
}

// voxel_entries with the fast form of Phi: rb / kb the plane meeting the voxel's bottom face and
// its K per atom, rt / kt the same for the top face (from the voxel above).
template <typename T, typename Sink>
__device__ __forceinline__ void voxel_entries_fast(const Geo& g, int ix, int iy, int iz, const ColumnView<T>& cv,
                                                   const AtomP<T>* atoms, const AtomP<T>& full, int rb,
                                                   const T* kb, int rt, const T* kt, Sink& sink) {
    const T c = G3<T>::c(g);
    const T z0w = G3<T>::z0(g) + iz * c;
    int l0, l1;
    if (!voxel_rows<T>(g, z0w, z0w + c, cv.tmin_w, cv.tmax_w, l0, l1)) return;
    const int ng = cv.ng, na = ng + 1;
    T pc[kMaxG + 1], pp[kMaxG + 1];
#pragma unroll
    for (int j = 0; j <= kMaxG; ++j) pp[j] = T(0);
#pragma unroll 1
    for (int r = l0; r <= l1 + 1; ++r) {
        T q, iq;
        const T h = plane_height(g, r, iz, cv.dh, cv.dl, q, iq);   // above the voxel bottom, units of c
        const T gw = h * c;
        const int cls = h < T(0) ? 0 : (h >= T(1) ? 2 : 1);
        const bool on_b = r == rb, on_t = r == rt;
#pragma unroll
        for (int j = 0; j <= kMaxG; ++j) {
            if (j < na) {
                const AtomP<T>& P = j == 0 ? full : atoms[j - 1];
                T v = cls == 0 ? T(0) : (cls == 2 ? c * P.A : gw * P.A + q * P.M1);
                if (on_b) v += kb[j];
                if (on_t) v -= kt[j];
                pc[j] = v;
            } else {
                pc[j] = T(0);
            }
        }
        if (r > l0) {
            const int l = r - 1;
            const T sf = pc[0] - pp[0];
            T prevS = cv.sigma > 0 ? T(0) : sf;
#pragma unroll
            for (int j = 0; j <= kMaxG; ++j) {
                if (j <= ng) {
                    const T S = j < ng ? pc[j < kMaxG ? j + 1 : kMaxG] - pp[j < kMaxG ? j + 1 : kMaxG] : (cv.sigma > 0 ? sf : T(0));
                    const int k = cv.k_first + j;
                    const T wt = cv.sigma > 0 ? S - prevS : prevS - S;
                    if ((cv.kin || (k >= 0 && k < g.nu)) && wt != T(0)) sink.add(k, l, wt);
                    prevS = S;
                }
            }
        }
#pragma unroll
        for (int j = 0; j <= kMaxG; ++j) pp[j] = pc[j];
    }
}

// Per-warp shared slots of the face corrections: one row of kKs values per lane.
constexpr int kKs = kMaxG + 3;   // 9: rows of neighbouring lanes fall in different banks

// Sink of the back projection: W p gathered from this view's projections.
template <typename T, int NB>
struct GatherSink {
    const T* pv;        // this view's differenced projections (prep_diff_3d); p(k, l) is the .w
    int nv;             // value at slot (k, l + 1)
    T sum[NB];
    __device__ __forceinline__ void add(int k, int l, T wt) {
        fma_vec<T, NB>(sum, wt, pv + ((size_t)(k * (nv + 2) + l + 1) * 4 + 3) * NB);
    }
};

// ---------------------------------------------------------------------------------------
// Back projection: one warp per voxel column and window of ZW voxels in z (ZW = 64, 128 or
// 256, the largest that still gives the grid enough warps).  All lanes of a
// warp share the column's view geometry: per view the warp classifies the footprint's corner
// lines, lanes 0 .. ng build the column's atoms in parallel (warp-private shared memory),
// then the voxels of the window that the view's cone reaches are dealt to the lanes in
// order (32 at a time), each lane forming its voxel's entries and adding W p to the voxel's
// sum in shared memory.  The sums are written once at the end.
// ---------------------------------------------------------------------------------------
constexpr int BW = 4;     // warps (columns) per block
constexpr int ZWN = 64;   // voxels of a column per warp in the nnz count

template <typename T, int NB, int ZW>
__global__ void __launch_bounds__(32 * BW, sizeof(T) == 8 ? 3 : 8) back3d_vox(Geo g, const T* __restrict__ ps, void* __restrict__ x, int xdt,
                                                      int B, int b_off, T scale, int accumulate, int v_begin, int v_end) {
    __shared__ AtomP<T> atoms_s[BW][kMaxG + 1];
    __shared__ T acc_s[BW][NB * ZW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = blockIdx.x * BW + wid;
    if (col >= g.nx * g.ny) return;                       // whole warp leaves together
    const int ix = col % g.nx, iy = col / g.nx;
    const int zb = blockIdx.y * ZW, ze = min(zb + ZW, g.nz);
    AtomP<T>* atoms = atoms_s[wid];
    T* acc = acc_s[wid];                                  // acc[b * ZW + (iz - zb)]
    for (int i = lane; i < NB * ZW; i += 32) acc[i] = T(0);
    for (int v = v_begin; v < v_end; ++v) {
        ColumnView<T> cv;
        column_view<T>(g, v, ix, iy, lane, cv);
        if (!cv.ok) continue;                              // warp-uniform
        int z0, z1;
        cone_z_range<T>(g, cv.tmin_w, cv.tmax_w, z0, z1);
        z0 = max(z0, zb);
        z1 = min(z1, ze - 1);
        if (z0 > z1) continue;
        __syncwarp();
        column_atoms<T>(g, v, ix, iy, cv, lane, atoms);
        __syncwarp();
        GatherSink<T, NB> sink;
        sink.pv = ps + (size_t)v * (g.nu + 1) * (g.nv + 2) * 4 * NB;
        sink.nv = g.nv;
        if (cv.fast) {
            const BackCols bc = back_cols<T>(g, cv);
            // 31 voxels per pass; lane 31 forms the term of the face above the last of them
            for (int zc = z0; zc <= z1; zc += 31) {
                const int iz = zc + lane;
                int ra = 0;
                T ha = T(0), qa = T(0), ff[NB];
#pragma unroll
                for (int i = 0; i < NB; ++i) ff[i] = T(0);
                if (iz <= z1 + 1) face_back<T, NB>(g, iz, cv, atoms, atoms[kMaxG], sink.pv, bc, ra, ha, qa, ff);
                const int rtop = __shfl_down_sync(0xffffffffu, ra, 1);
                T corr[NB];
#pragma unroll
                for (int i = 0; i < NB; ++i) corr[i] = ff[i] - __shfl_down_sync(0xffffffffu, ff[i], 1);
                if (lane < 31 && iz <= z1) {
                    T vs[NB];
                    voxel_back_fast<T, NB>(g, iz, cv, atoms, atoms[kMaxG], sink.pv, bc, ra, ha, qa, rtop, corr, vs);
#pragma unroll
                    for (int i = 0; i < NB; ++i) acc[i * ZW + iz - zb] += vs[i];
                }
            }
        } else {
            for (int iz = z0 + lane; iz <= z1; iz += 32) {
#pragma unroll
                for (int i = 0; i < NB; ++i) sink.sum[i] = T(0);
                voxel_entries<T>(g, v, ix, iy, iz, cv, atoms, atoms[kMaxG], sink);
#pragma unroll
                for (int i = 0; i < NB; ++i) acc[i * ZW + iz - zb] += sink.sum[i];
            }
        }
    }
    __syncwarp();
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    for (int iz = zb + lane; iz < ze; iz += 32) {
        const size_t vox = ((size_t)iz * g.ny + iy) * g.nx + ix;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int bidx = b_off + i;
            if (bidx < B) store_any3<T>(x, (size_t)bidx * nvox + vox, xdt, acc[i * ZW + iz - zb] * scale, accumulate != 0);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Forward projection, ray-driven over element groups: one warp per (view, group of KW
// neighbouring detector columns kg .. kg+KW-1, window of rw consecutive rows; KW = 8 when
// that still gives 16384 warps, else 4).  The warp
// walks the union of the group's top-view strips cell by cell (as in 2D); per cell it
// classifies the group's KW + 1 corner lines (column_view restricted to them), builds the
// tables of the crossing ones (one (line, piece) per lane; the whole-cell table is built once
// per warp), then the lanes take the voxels of the column that the window's rows reach (one
// voxel per lane, 32 at a time), form their entries with the back projection's voxel_entries
// and add W x into per-(column, row) sums in shared memory, which the warp writes to p at the
// end (each element written by exactly one warp).  A line's table serves the two columns it
// bounds, so the group shares them; cells whose voxels in reach are all zero are skipped
// before any table is built.  The window is as tall as a shared-memory budget allows (384
// rows for one FP32 batch item).
// ---------------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------------
// One cell of the forward projection in the fast form, the lanes taking row planes.  With
// C_a(r) = sum_iz x(iz) Phi_a(r, iz) for atom a (whole cell or below a crossing line) and
// plane r, an element column k of the footprint receives on row l
//     p(k, l) += sigma [T(line k + 1, l) - T(line k, l)],   T_a(l) = C_a(l + 1) - C_a(l),
// with T = 0 or T of the whole cell for the lines outside the footprint (as in voxel_entries).
// Plane r has its centre in voxel i_r (height h in [0, 1) above its bottom): every voxel
// below it has Phi = c A, voxel i_r the linear Phi, and a face the plane meets inside the cell
// moves K from one side to the other, so
//     C_a(r) = c A_a X(i_r) + C'_a(r),  C'_a(r) = (g A_a + q M1_a) x(i_r) + K_a (x above - x below)
// (X: the sum of x below a voxel) and T_a(l) = c A_a [x(i_l) + .. + x(i_{l+1} - 1)] + C'_a(l+1)
// - C'_a(l).  Each lane computes C' of its plane, takes its neighbour's (plane l + 1) by a
// shuffle, and adds its row's sums: rows are owned by lanes (no atomics, fixed order).  Rows
// whose two planes both lie below or both above the grid get T = 0 and are skipped.
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
__device__ __forceinline__ void cell_forward_fast(const Geo& g, const ColumnView<T>& cv, const AtomP<T>* atoms,
                                                  const AtomP<T>& full, const T* __restrict__ xcol, int lane, int kg,
                                                  int nk, int L0, int nrow, int rw, T* rows, int zlo, int zhi) {
    const T c = G3<T>::c(g);
    const int ng = cv.ng, na = ng + 1;
    // planes that can reach the nonzero voxels zlo .. zhi: around the heights zlo - 1 and zhi + 2
    // (m < 1/2); rows between two planes both below or both above them add exactly nothing
    const T tc = cv.dh + cv.dl;
    const T ra_f = (G3<T>::div(T(zlo - 1) - T(0.5) * T(g.nz), tc) * G3<T>::sdd(g) - G3<T>::v0(g)) * G3<T>::idv(g);
    const T rb_f = (G3<T>::div(T(zhi + 2) - T(0.5) * T(g.nz), tc) * G3<T>::sdd(g) - G3<T>::v0(g)) * G3<T>::idv(g);
    const int plast = L0 + nrow;                      // planes L0 .. L0 + nrow bound the window's rows
    int r_first = L0, r_last = plast;
    {
        const T lo = floor(ra_f) - T(1), hi = floor(rb_f) + T(2);
        if (lo > T(r_first)) r_first = lo > T(plast) ? plast : (int)lo;
        if (hi < T(r_last)) r_last = hi < T(r_first) ? r_first : (int)hi;
    }
    auto xat = [&](int iz, int n) { return (iz >= 0 && iz < g.nz) ? __ldg(xcol + (size_t)iz * NB + n) : T(0); };
#pragma unroll 1
    for (int rc = r_first; rc < r_last; rc += 31) {
        const int r = rc + lane;
        T cp[kMaxG + 1][NB];
#pragma unroll
        for (int j = 0; j <= kMaxG; ++j)
#pragma unroll
            for (int n = 0; n < NB; ++n) cp[j][n] = T(0);
        int izr = 0;
        if (r <= r_last) {
            T q, iq;
            // the voxel holding the plane's centre: a rough height above the grid's bottom (off by
            // at most one voxel near a face), then the exact height relative to that voxel
            izr = (int)floor(G3<T>::q(g, r) * (cv.dh + cv.dl) + T(0.5) * T(g.nz));
            T h = plane_height(g, r, izr, cv.dh, cv.dl, q, iq);       // the same, relative to voxel izr
            if (h < T(0)) { izr -= 1; h += T(1); }
            else if (h >= T(1)) { izr += 1; h -= T(1); }
            const T m = fabs(q) * cv.margin_c;
            T x0[NB], dx[NB];
            const bool kb = h < m, kt = h > T(1) - m;
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                x0[n] = xat(izr, n);
                dx[n] = kb ? x0[n] - xat(izr - 1, n) : (kt ? xat(izr + 1, n) - x0[n] : T(0));
            }
            const T gw = h * c;
            const T gk = kb ? gw : gw - c;      // height above the face the plane meets
#pragma unroll
            for (int j = 0; j <= kMaxG; ++j) {
                if (j < na) {
                    const AtomP<T>& P = j == 0 ? full : atoms[j - 1];
                    const T L = gw * P.A + q * P.M1;
                    T K = T(0);
                    if (kb || kt) K = kink_tail<T>(P, gk, q, iq, kt);
#pragma unroll
                    for (int n = 0; n < NB; ++n) cp[j][n] = L * x0[n] + K * dx[n];
                }
            }
        }
        const int izn = __shfl_down_sync(0xffffffffu, izr, 1);
        // in place: cp becomes T' = C'(l + 1) - C'(l)
        T (&tv)[kMaxG + 1][NB] = cp;
#pragma unroll
        for (int j = 0; j <= kMaxG; ++j) {
            if (j < na) {
#pragma unroll
                for (int n = 0; n < NB; ++n) tv[j][n] = __shfl_down_sync(0xffffffffu, cp[j][n], 1) - cp[j][n];
            }
        }
        const int l = r;
        if (lane < 31 && l < r_last) {
            // voxels from i_l up to i_{l+1} - 1 lie between the two planes
            T sx[NB];
#pragma unroll
            for (int n = 0; n < NB; ++n) sx[n] = T(0);
            const int za = izr < 0 ? 0 : izr, zb = izn > g.nz ? g.nz : izn;
            for (int iz = za; iz < zb; ++iz) {
#pragma unroll
                for (int n = 0; n < NB; ++n) sx[n] += __ldg(xcol + (size_t)iz * NB + n);
            }
            T* row = rows + (size_t)(l - L0) * NB;
            T sf[NB], prev[NB];
#pragma unroll
            for (int n = 0; n < NB; ++n) {
                sf[n] = tv[0][n] + c * full.A * sx[n];
                prev[n] = cv.sigma > 0 ? T(0) : sf[n];
            }
#pragma unroll
            for (int j = 0; j <= kMaxG; ++j) {
                if (j <= ng) {
                    const int k = cv.k_first + j;
                    const bool inside = k >= kg && k < kg + nk;
                    const T cA = j < ng ? c * atoms[j < kMaxG ? j : kMaxG - 1].A : T(0);
#pragma unroll
                    for (int n = 0; n < NB; ++n) {
                        const T S = j < ng ? tv[j < kMaxG ? j + 1 : kMaxG][n] + cA * sx[n] : (cv.sigma > 0 ? sf[n] : T(0));
                        const T wt = cv.sigma > 0 ? S - prev[n] : prev[n] - S;
                        if (inside) row[(size_t)(k - kg) * rw * NB + n] += wt;
                        prev[n] = S;
                    }
                }
            }
        }
    }
}

constexpr int FW = 4;                // warps per block

// Sink of the forward projection: W x added to the (column, row) sums of the warp's group.
template <typename T, int NB>
struct RowSink {
    T* rows;
    int rw, kg, nk, L0, nrow;
    T xv[NB];
    __device__ __forceinline__ void add(int k, int l, T wt) {
        const int kk = k - kg, ll = l - L0;
        if (kk >= 0 && kk < nk && ll >= 0 && ll < nrow) {
#pragma unroll
            for (int i = 0; i < NB; ++i) atomicAdd(&rows[(kk * rw + ll) * NB + i], wt * xv[i]);
        }
    }
};
constexpr int FWD_SMEM = 32 * 1024;  // shared-memory budget of one block's row sums (256 rows at KW = 8)

template <typename T, int NB, int KW>
__global__ void __launch_bounds__(32 * FW, sizeof(T) == 8 ? 3 : 6) fwd3d_grp(Geo g, int rw, const T* __restrict__ xs0,
                                                     const T* __restrict__ xs1, const int2* __restrict__ rng,
                                                     void* __restrict__ p, int pdt, int B, int b_off, T scale,
                                                     int accumulate) {
    __shared__ AtomP<T> atoms_s[FW][kMaxG + 1];
    extern __shared__ __align__(16) unsigned char fwd_dyn[];   // [FW][KW][rw][NB] sums
    using L = typename LineOf<T>::type;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int kg = (blockIdx.x * FW + wid) * KW;
    const int v = blockIdx.y;
    const int L0 = blockIdx.z * rw;
    if (kg >= g.nu || L0 >= g.nv) return;                 // whole warp leaves together
    const int nk = min(KW, g.nu - kg), nrow = min(rw, g.nv - L0);
    T* rows = reinterpret_cast<T*>(fwd_dyn) + (size_t)wid * KW * rw * NB;   // [(k - kg) * rw + row][NB]
    for (int i = lane; i < KW * rw * NB; i += 32) rows[i] = T(0);
    AtomP<T>* atoms = atoms_s[wid];
    const int axis = g.axis_sigma[2 * v];
    const int nc = axis == 0 ? g.ny : g.nx;
    const T* __restrict__ xs = axis == 0 ? xs0 : xs1;
    const T a = G3<T>::a(g), b = G3<T>::b(g), c = G3<T>::c(g);
    const T hw = axis == 0 ? a : b, hc = axis == 0 ? b : a;
    const T cs = G3<T>::cs(g, v, 0), sn = G3<T>::cs(g, v, 1);
    const T margin_c = T(0.5) * (fabs(a * cs) + fabs(b * sn)) * G3<T>::ic(g);   // units of c
    const T q_lo = G3<T>::q(g, L0), q_hi = G3<T>::q(g, L0 + nrow);
    const T mz = (fabs(q_lo) > fabs(q_hi) ? fabs(q_lo) : fabs(q_hi)) * margin_c + T(1e-3);
    // walk range: the union of the group's elements' ranges
    int w0 = 0x7fffffff, w1 = -1;
    if (lane < nk) {
        w0 = g.wrange[2 * ((size_t)v * g.nu + kg + lane)];
        w1 = g.wrange[2 * ((size_t)v * g.nu + kg + lane) + 1];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        w0 = min(w0, __shfl_xor_sync(0xffffffffu, w0, o));
        w1 = max(w1, __shfl_xor_sync(0xffffffffu, w1, o));
    }
    L la, lb;
    la.load(g, v, kg, w0);
    lb.load(g, v, kg + nk, w0);
    // the whole-cell table is the same in every cell of the view: built once
    if (lane < 5) build_piece<T>(atoms[kMaxG], lane + 1, T(2), T(2), hw, hc, axis, cs, sn);
    __syncwarp();
    for (int w = w0; w < w1; ++w) {
        int clo = min(la.cell_lo(), lb.cell_lo());
        int chi = max(la.cell_hi(), lb.cell_hi());
        clo = max(clo, 0);
        chi = min(chi, nc - 1);
        for (int cc = clo; cc <= chi; ++cc) {
            const int ix = axis == 0 ? w : cc, iy = axis == 0 ? cc : w;
            const int2 cr = rng[(size_t)ix * g.ny + iy];   // the column's nonzero voxels
            if (cr.x > cr.y) continue;                     // none: the cell adds nothing
            // voxels of the column that the window's rows reach (from the column's centre depth)
            T dh, dl, qq, iqq;
            column_depth(g, v, ix, iy, dh, dl);
            const T zlo = floor(plane_height(g, L0, 0, dh, dl, qq, iqq) - mz);
            const T zhi = floor(plane_height(g, L0 + nrow, 0, dh, dl, qq, iqq) + mz);
            if (zhi < T(0) || zlo > T(g.nz - 1)) continue;
            const int izlo = zlo < T(0) ? 0 : (int)zlo;
            const int izhi = zhi > T(g.nz - 1) ? g.nz - 1 : (int)zhi;
            // the nonzero voxels in reach: cells with none add nothing and are skipped before any
            // set-up; planes below or above all of them add nothing either
            const int znz_lo = max(cr.x, izlo), znz_hi = min(cr.y, izhi);
            if (znz_lo > znz_hi) continue;
            ColumnView<T> cv;
            column_view<T>(g, v, ix, iy, lane, cv, kg, kg + nk);
            if (!cv.ok) continue;                          // warp-uniform
            const T* xcol = xs + ((size_t)w * nc + cc) * g.nz * NB;
            __syncwarp();
            for (int it = lane; it < cv.ng * 5; it += 32) {
                const int i = it / 5;
                column_piece<T>(g, v, ix, iy, cv, i, it - 5 * i + 1, atoms[i]);
            }
            __syncwarp();
            if (cv.fast) {
                cell_forward_fast<T, NB>(g, cv, atoms, atoms[kMaxG], xcol, lane, kg, nk, L0, nrow, rw, rows, znz_lo,
                                         znz_hi);
                __syncwarp();
                continue;
            }
            for (int zb = izlo; zb <= izhi; zb += 32) {
                const int iz = zb + lane;
                if (iz > izhi) continue;
                T xv[NB];
                bool any = false;
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    xv[i] = __ldg(xcol + (size_t)iz * NB + i);
                    any |= xv[i] != T(0);
                }
                if (!any) continue;
                RowSink<T, NB> sink{rows, rw, kg, nk, L0, nrow};
#pragma unroll
                for (int i = 0; i < NB; ++i) sink.xv[i] = xv[i];
                voxel_entries<T>(g, v, ix, iy, iz, cv, atoms, atoms[kMaxG], sink);
            }
        }
        la.step();
        lb.step();
    }
    __syncwarp();
    for (int idx = lane; idx < nk * nrow; idx += 32) {
        const int j = idx / nk, kk = idx - j * nk;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int bidx = b_off + i;
            if (bidx < B)
                store_any3<T>(p, (((size_t)bidx * g.n_views + v) * g.nv + L0 + j) * g.nu + kg + kk, pdt,
                              rows[(kk * rw + j) * NB + i] * scale *
                                  elem_weight<T>(g, ((size_t)v * g.nv + L0 + j) * g.nu + kg + kk),
                              accumulate != 0);
        }
    }
}

// Number of (voxel, view, element) whose volume exceeds 1e-6 of the voxel's (column-warps as
// in the back projection).
struct CountSink {
    float thr;
    unsigned long long n;
    __device__ __forceinline__ void add(int, int, float wt) { n += fabsf(wt) > thr; }
};

__global__ void __launch_bounds__(32 * BW) nnz3d_kernel(Geo g, unsigned long long* counter) {
    __shared__ AtomP<float> atoms_s[BW][kMaxG + 1];
    __shared__ float ks_s[BW][32 * kKs];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = blockIdx.x * BW + wid;
    if (col >= g.nx * g.ny) return;
    const int ix = col % g.nx, iy = col / g.nx;
    const int zb = blockIdx.y * ZWN, ze = min(zb + ZWN, g.nz);
    AtomP<float>* atoms = atoms_s[wid];
    float* ks = ks_s[wid];
    const float thr = 1e-6f * g.a * g.b * g.c;
    unsigned long long cnt = 0;
    for (int v = 0; v < g.n_views; ++v) {
        ColumnView<float> cv;
        column_view<float>(g, v, ix, iy, lane, cv);
        if (!cv.ok) continue;
        int z0, z1;
        cone_z_range<float>(g, cv.tmin_w, cv.tmax_w, z0, z1);
        z0 = max(z0, zb);
        z1 = min(z1, ze - 1);
        if (z0 > z1) continue;
        __syncwarp();
        column_atoms<float>(g, v, ix, iy, cv, lane, atoms);
        __syncwarp();
        CountSink sink{thr, 0ull};
        if (cv.fast) {
            for (int zc = z0; zc <= z1; zc += 31) {
                const int iz = zc + lane;
                int ra = 0;
                float ha_, qa_;   // unused here
                const int rb = iz <= z1 + 1 ? face_kink<float>(g, iz, cv, atoms, atoms[kMaxG], ks + lane * kKs, ra, ha_, qa_) : -1;
                __syncwarp();
                const int rt = __shfl_down_sync(0xffffffffu, rb, 1);
                if (lane < 31 && iz <= z1)
                    voxel_entries_fast<float>(g, ix, iy, iz, cv, atoms, atoms[kMaxG], rb, ks + lane * kKs, rt,
                                              ks + (lane + 1) * kKs, sink);
                __syncwarp();
            }
        } else {
            for (int iz = z0 + lane; iz <= z1; iz += 32)
                voxel_entries<float>(g, v, ix, iy, iz, cv, atoms, atoms[kMaxG], sink);
        }
        cnt += sink.n;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(counter, cnt);
}

// ---------------------------------------------------------------------------------------
// Forward projection, voxel-driven (the scatter form of the paper's Algorithm 1): warps over
// voxel columns as in the back projection; each warp adds its voxels' entries W x into
// shared-memory partial sums of the detector rows its chunk of voxels reaches (one per
// footprint column and row), then adds every nonzero partial to the sinogram sums in global
// memory with one atomic.  Entries beyond the partials' row range go to global memory
// directly.  The order of the FP additions is not fixed.
// ---------------------------------------------------------------------------------------
constexpr int kPR = 128;   // partial rows per footprint column

template <typename T>
struct PartialSink {
    T* part;            // [kMaxG + 1][kPR]
    T* pacc;            // this view's sums, [nv][nu]
    int lbase, kfirst, nu;
    T xv;
    __device__ __forceinline__ void add(int k, int l, T wt) {
        const int j = k - kfirst, r = l - lbase;
        if (j >= 0 && j <= kMaxG && r >= 0 && r < kPR) atomicAdd(part + j * kPR + r, wt * xv);
        else atomicAdd(pacc + (size_t)l * nu + k, wt * xv);
    }
};

template <typename T, int ZW>
__global__ void __launch_bounds__(32 * BW) fwd3d_vox(Geo g, const T* __restrict__ xs0, T* __restrict__ pacc) {
    __shared__ AtomP<T> atoms_s[BW][kMaxG + 1];
    __shared__ T ks_s[BW][32 * kKs];
    __shared__ T part_s[BW][(kMaxG + 1) * kPR];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = blockIdx.x * BW + wid;
    if (col >= g.nx * g.ny) return;
    const int ix = col % g.nx, iy = col / g.nx;
    const int zb = blockIdx.y * ZW, ze = min(zb + ZW, g.nz);
    AtomP<T>* atoms = atoms_s[wid];
    T* ks = ks_s[wid];
    T* part = part_s[wid];
    for (int i = lane; i < (kMaxG + 1) * kPR; i += 32) part[i] = T(0);
    const T* xcol = xs0 + ((size_t)ix * g.ny + iy) * g.nz;
    const T c = G3<T>::c(g);
    for (int v = 0; v < g.n_views; ++v) {
        ColumnView<T> cv;
        column_view<T>(g, v, ix, iy, lane, cv);
        if (!cv.ok) continue;
        int z0, z1;
        cone_z_range<T>(g, cv.tmin_w, cv.tmax_w, z0, z1);
        z0 = max(z0, zb);
        z1 = min(z1, ze - 1);
        if (z0 > z1) continue;
        // skip columns whose voxels in reach are all zero
        bool nzv = false;
        for (int zc = z0; zc <= z1 && !__any_sync(0xffffffffu, nzv); zc += 32)
            if (zc + lane <= z1) nzv = __ldg(xcol + zc + lane) != T(0);
        if (!__any_sync(0xffffffffu, nzv)) continue;
        __syncwarp();
        column_atoms<T>(g, v, ix, iy, cv, lane, atoms);
        __syncwarp();
        PartialSink<T> sink;
        sink.part = part;
        sink.pacc = pacc + (size_t)v * g.nv * g.nu;
        sink.kfirst = cv.k_first;
        sink.nu = g.nu;
        const int step = cv.fast ? 31 : 32;
        for (int zc = z0; zc <= z1; zc += step) {
            const int iz = zc + lane;
            const bool mine = lane < step && iz <= z1;
            const T xv = mine ? __ldg(xcol + iz) : T(0);
            // rows the chunk reaches start at the lowest voxel's first row
            int l0 = g.nv, l1 = -1;
            if (mine && xv != T(0)) {
                const T z0w = G3<T>::z0(g) + iz * c;
                if (!voxel_rows<T>(g, z0w, z0w + c, cv.tmin_w, cv.tmax_w, l0, l1)) { l0 = g.nv; l1 = -1; }
            }
            const int lbase = __reduce_min_sync(0xffffffffu, (unsigned)(l0 + 1)) - 1;
            const int ltop = (int)__reduce_max_sync(0xffffffffu, (unsigned)(l1 + 1)) - 1;
            sink.lbase = lbase;
            sink.xv = xv;
            if (cv.fast) {
                int ra = 0;
                T ha_, qa_;   // unused here
                const bool need = mine && xv != T(0);
                const bool below = __shfl_up_sync(0xffffffffu, need, 1);
                const int rb = ((need || (lane > 0 && below)) && iz <= z1 + 1)
                                   ? face_kink<T>(g, iz, cv, atoms, atoms[kMaxG], ks + lane * kKs, ra, ha_, qa_) : -1;
                __syncwarp();
                const int rt = __shfl_down_sync(0xffffffffu, rb, 1);
                if (need)
                    voxel_entries_fast<T>(g, ix, iy, iz, cv, atoms, atoms[kMaxG], rb, ks + lane * kKs, rt,
                                          ks + (lane + 1) * kKs, sink);
            } else if (mine && xv != T(0)) {
                voxel_entries<T>(g, v, ix, iy, iz, cv, atoms, atoms[kMaxG], sink);
            }
            __syncwarp();
            // flush the partials of the rows reached (elements on the detector only)
            if (ltop >= lbase) {
                const int span = min(ltop - lbase + 1, kPR);
                for (int j = 0; j <= cv.ng; ++j) {
                    const int k = cv.k_first + j;
                    for (int r = lane; r < span; r += 32) {
                        const T val = part[j * kPR + r];
                        if (val != T(0)) {
                            if (k >= 0 && k < g.nu) atomicAdd(sink.pacc + (size_t)(lbase + r) * g.nu + k, val);
                            part[j * kPR + r] = T(0);
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
}

// p = scale * w * sums (+ p with CSM_ACCUMULATE), in p's storage type.
template <typename T>
__global__ void finish_scatter_3d(Geo g, const T* __restrict__ pacc, void* __restrict__ p, int pdt, int b, T scale,
                                  int accumulate) {
    const size_t n = (size_t)g.n_views * g.nv * g.nu;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        store_any3<T>(p, (size_t)b * n + i, pdt, pacc[i] * scale * elem_weight<T>(g, i), accumulate != 0);
}

template <typename T>
static csm_status run_fwd3_vox(const csm_geom_s* gh, const void* x, void* p, int64_t batch, csm_dtype xdt,
                               csm_dtype pdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    const size_t nvox = (size_t)gh->nx * gh->ny * gh->nz;
    const size_t vol1 = al256(nvox * sizeof(T));
    T* xs0 = (T*)ws;
    T* xs1 = (T*)((char*)ws + vol1);
    T* pacc = (T*)((char*)ws + 2 * vol1);
    const size_t nsino = (size_t)gh->n_views * gh->nv * gh->nu;
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1.0 / (gh->a * gh->b * gh->c)) : T(1);
    const size_t ncol = (size_t)gh->nx * gh->ny;
    constexpr int ZW = 64;
    for (int64_t b = 0; b < batch; ++b) {
        dim3 tb(32, 8), tg((gh->nx + 31) / 32, (gh->nz + 31) / 32, gh->ny);
        note_launch(), prep_vol_3d<T, 1><<<tg, tb, 0, st>>>(x, (int)xdt, (int)batch, (int)b, gh->nx, gh->ny, gh->nz, xs0, xs1);
        cudaError_t e = cudaMemsetAsync(pacc, 0, nsino * sizeof(T), st);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
        dim3 bb(32 * BW), bg((unsigned)((ncol + BW - 1) / BW), (gh->nz + ZW - 1) / ZW);
        note_launch(), fwd3d_vox<T, ZW><<<bg, bb, 0, st>>>(g, xs0, pacc);
        note_launch(), finish_scatter_3d<T><<<1216, 256, 0, st>>>(g, pacc, p, (int)pdt, (int)b, scale, (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status s = check_launch();
        if (s != CSM_OK) return s;
    }
    return CSM_OK;
}

// ---------------------------------------------------------------------------------------
// Sparse export: the same per-voxel entries (column-warps, 64-voxel windows as the count),
// written as rows of W^T (voxels; per-voxel counts and write positions kept in shared memory,
// so the entries of a row come in view, row, column order) or of W (elements; atomics).
// ---------------------------------------------------------------------------------------
template <typename T>
struct ExportSink {
    const Geo* g;
    ExportArgs a;
    T thr, scale;
    long long vox;     // this voxel's index (column of W)
    int base;          // row index of this view's first element
    int nu;
    int n;             // entries so far (mode 0) / write position (mode 1)
    __device__ __forceinline__ void add(int k, int l, T wt) {
        if (!(fabs(wt) > thr)) return;
        const long long row_e = (long long)base + (long long)l * nu + k;
        const T v = wt * scale * elem_weight<T>(*g, (size_t)row_e);
        switch (a.mode) {
            case 0: ++n; break;
            case 1: {
                const long long slot = a.row_ptr[vox] + n++;
                a.col[slot] = (int)row_e;
                if (a.dbl) ((double*)a.val)[slot] = (double)v;
                else ((float*)a.val)[slot] = (float)v;
                break;
            }
            case 2: atomicAdd(a.counts + row_e, 1ull); break;
            default: {
                const long long slot = a.row_ptr[row_e] + atomicAdd(a.cursor + row_e, 1);
                a.col[slot] = (int)vox;
                if (a.dbl) ((double*)a.val)[slot] = (double)v;
                else ((float*)a.val)[slot] = (float)v;
                break;
            }
        }
    }
};

template <typename T>
__global__ void __launch_bounds__(32 * BW) export3d_kernel(Geo g, ExportArgs ea) {
    __shared__ AtomP<T> atoms_s[BW][kMaxG + 1];
    __shared__ T ks_s[BW][32 * kKs];
    __shared__ int pos_s[BW][ZWN];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int col = blockIdx.x * BW + wid;
    if (col >= g.nx * g.ny) return;
    const int ix = col % g.nx, iy = col / g.nx;
    const int zb = blockIdx.y * ZWN, ze = min(zb + ZWN, g.nz);
    AtomP<T>* atoms = atoms_s[wid];
    T* ks = ks_s[wid];
    int* pos = pos_s[wid];
    for (int i = lane; i < ZWN; i += 32) pos[i] = 0;
    ExportSink<T> sink;
    sink.g = &g;
    sink.a = ea;
    sink.thr = (T)ea.thr;
    sink.scale = (T)ea.scale;
    sink.nu = g.nu;
    for (int v = 0; v < g.n_views; ++v) {
        ColumnView<T> cv;
        column_view<T>(g, v, ix, iy, lane, cv);
        if (!cv.ok) continue;
        int z0, z1;
        cone_z_range<T>(g, cv.tmin_w, cv.tmax_w, z0, z1);
        z0 = max(z0, zb);
        z1 = min(z1, ze - 1);
        if (z0 > z1) continue;
        __syncwarp();
        column_atoms<T>(g, v, ix, iy, cv, lane, atoms);
        __syncwarp();
        sink.base = v * g.nv * g.nu;
        if (cv.fast) {
            for (int zc = z0; zc <= z1; zc += 31) {
                const int iz = zc + lane;
                int ra = 0;
                T ha_, qa_;   // unused here
                const int rb = iz <= z1 + 1 ? face_kink<T>(g, iz, cv, atoms, atoms[kMaxG], ks + lane * kKs, ra, ha_, qa_) : -1;
                __syncwarp();
                const int rt = __shfl_down_sync(0xffffffffu, rb, 1);
                if (lane < 31 && iz <= z1) {
                    sink.vox = ((long long)iz * g.ny + iy) * g.nx + ix;
                    sink.n = pos[iz - zb];
                    voxel_entries_fast<T>(g, ix, iy, iz, cv, atoms, atoms[kMaxG], rb, ks + lane * kKs, rt,
                                          ks + (lane + 1) * kKs, sink);
                    pos[iz - zb] = sink.n;
                }
                __syncwarp();
            }
        } else {
            for (int iz = z0 + lane; iz <= z1; iz += 32) {
                sink.vox = ((long long)iz * g.ny + iy) * g.nx + ix;
                sink.n = pos[iz - zb];
                voxel_entries<T>(g, v, ix, iy, iz, cv, atoms, atoms[kMaxG], sink);
                pos[iz - zb] = sink.n;
            }
        }
    }
    __syncwarp();
    if (ea.mode == 0)
        for (int iz = zb + lane; iz < ze; iz += 32)
            ea.counts[((long long)iz * g.ny + iy) * g.nx + ix] = (unsigned long long)pos[iz - zb];
}

csm_status export_3d(const csm_geom_s* gh, const ExportArgs& a, cudaStream_t st) {
    const Geo g = make_geo(gh);
    const size_t ncol = (size_t)gh->nx * gh->ny;
    dim3 bb(32 * BW), bg((unsigned)((ncol + BW - 1) / BW), (gh->nz + ZWN - 1) / ZWN);
    if (a.dbl) note_launch(), export3d_kernel<double><<<bg, bb, 0, st>>>(g, a);
    else note_launch(), export3d_kernel<float><<<bg, bb, 0, st>>>(g, a);
    return check_launch();
}

// ---------------------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------------------
// Rows per forward warp: all of them when the block's row sums fit the shared-memory budget,
// else the largest window that does (at least 32 rows).
static int rows_per_warp(const csm_geom_s* g, int kw, int nb, size_t elem) {
    const int cap = (int)(FWD_SMEM / ((size_t)FW * kw * nb * elem));
    return std::max(32, std::min(g->nv, cap));
}

template <typename T, int NB, int KW>
static csm_status launch_fwd3(const Geo& g, const csm_geom_s* gh, const T* xs0, const T* xs1, const int2* rng, void* p,
                              int64_t batch, csm_dtype pdt, int64_t b0, T scale, int flags, cudaStream_t st) {
    const int rw = rows_per_warp(gh, KW, NB, sizeof(T));
    const size_t dyn = (size_t)FW * KW * rw * NB * sizeof(T);
    if (dyn > 16 * 1024) {      // with the static tables above the default 48 KiB per block
        cudaError_t e = cudaFuncSetAttribute(fwd3d_grp<T, NB, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    }
    dim3 fb(32 * FW), fg((gh->nu + FW * KW - 1) / (FW * KW), gh->n_views, (gh->nv + rw - 1) / rw);
    note_launch(), fwd3d_grp<T, NB, KW><<<fg, fb, dyn, st>>>(g, rw, xs0, xs1, rng, p, (int)pdt, (int)batch, (int)b0, scale,
                                              (flags & CSM_ACCUMULATE) ? 1 : 0);
    return check_launch();
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
    int2* rng = (int2*)((char*)ws + 2 * half);
    const int ncol = gh->nx * gh->ny;
    const bool wide = (size_t)((gh->nu + 7) / 8) * gh->n_views >= 16384;
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        dim3 tb(32, 8), tg((gh->nx + 31) / 32, (gh->nz + 31) / 32, gh->ny);
        note_launch(), prep_vol_3d<T, NB><<<tg, tb, 0, st>>>(x, (int)xdt, (int)batch, (int)b0, gh->nx, gh->ny, gh->nz, xs0, xs1);
        note_launch(), col_range_3d<T, NB><<<(unsigned)((ncol + 7) / 8), 256, 0, st>>>(xs0, ncol, gh->nz, rng);
        csm_status e = wide ? launch_fwd3<T, NB, 8>(g, gh, xs0, xs1, rng, p, batch, pdt, b0, scale, flags, st)
                            : launch_fwd3<T, NB, 4>(g, gh, xs0, xs1, rng, p, batch, pdt, b0, scale, flags, st);
        if (e != CSM_OK) return e;
    }
    return CSM_OK;
}

// Window height of the back projection: the largest of 512 / 256 / 128 / 64 voxels (at most
// 512 voxel sums per warp in shared memory: NB x ZW <= 512; 128 in FP64) that is not much
// taller than the grid and still leaves one warp per SM lane group (152 SMs x 32 warps).  A
// taller window shares a column's per-view set-up (corner classification, atom tables) among
// more voxels.
static int back_window(const csm_geom_s* g, bool dbl, int nb) {
    const size_t ncol = (size_t)g->nx * g->ny;
    const int top = dbl ? 128 : 512 / nb;
    for (int zw = top; zw > 64; zw >>= 1)
        if (g->nz > zw / 2 && ncol * (size_t)((g->nz + zw - 1) / zw) >= 152 * 32) return zw;
    return 64;
}

// Views per back-projection launch: every resident warp works on the same few views, so their
// slices of the differenced sinogram stay in L2 (about 64 MiB of them, one batch item's worth,
// so that the grouping and the summation order do not depend on the batch) instead of every
// warp reading its own view from DRAM.  Each group adds its sums to x (read-modify-write, one
// warp per voxel, a fixed order).  Sums for x in another type (BF16, F16) go through an FP32
// / FP64 copy when the workspace holds one (op 3), else one launch covers all views.
static int back_view_group(const csm_geom_s* g, size_t elem, csm_dtype xdt, bool dbl) {
    const bool exact_x = dbl ? xdt == CSM_F64 : xdt == CSM_F32;
    const size_t slice = (size_t)(g->nu + 1) * (g->nv + 2) * 4 * elem;
    if (!exact_x) return g->n_views;
    const size_t v = ((size_t)64 << 20) / (slice > 0 ? slice : 1);
    return (int)std::max<size_t>(1, std::min<size_t>(v, (size_t)g->n_views));
}

template <typename T, int NB, int ZW>
static csm_status launch_back3(const Geo& g, const csm_geom_s* gh, const T* ps, void* x, int64_t batch,
                               csm_dtype xdt, int64_t b0, T scale, int flags, cudaStream_t st) {
    const size_t ncol = (size_t)gh->nx * gh->ny;
    dim3 bb(32 * BW), bg((unsigned)((ncol + BW - 1) / BW), (gh->nz + ZW - 1) / ZW);
    const int vg = back_view_group(gh, sizeof(T), xdt, sizeof(T) == 8);
    for (int v0 = 0; v0 < gh->n_views; v0 += vg) {
        const int acc = (v0 > 0 || (flags & CSM_ACCUMULATE)) ? 1 : 0;
        note_launch(), back3d_vox<T, NB, ZW><<<bg, bb, 0, st>>>(g, ps, x, (int)xdt, (int)batch, (int)b0, scale, acc, v0,
                                                std::min(v0 + vg, gh->n_views));
        csm_status s = check_launch();
        if (s != CSM_OK) return s;
    }
    return CSM_OK;
}

// x (any storage type) from the FP32 / FP64 sums of a chunk of batch items, rounded once.
template <typename T>
__global__ void __launch_bounds__(256) sums_to_x_3d(const T* __restrict__ xacc, size_t n, void* __restrict__ x,
                                                    int xdt, size_t off, int accumulate) {
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256)
        store_any3<T>(x, off + i, xdt, xacc[i], accumulate != 0);
}

// xacc: when not null, the chunk's sums are formed in this FP32 / FP64 copy (the view groups
// adding into it) and then written to x in its storage type; else they go to x directly.
template <typename T, int NB>
static csm_status run_back3(const csm_geom_s* gh, const void* p, void* x, int64_t batch, csm_dtype pdt,
                            csm_dtype xdt, int flags, void* ws, T* xacc, cudaStream_t st) {
    const Geo g = make_geo(gh);
    T* ps = (T*)ws;
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1.0 / (gh->a * gh->b * gh->c)) : T(1);
    const int zw = back_window(gh, sizeof(T) == 8, NB);
    constexpr int kTop = sizeof(T) == 8 ? 128 : 512 / NB;   // largest window instantiated
    const csm_dtype tdt = sizeof(T) == 8 ? CSM_F64 : CSM_F32;
    const size_t nvox = (size_t)gh->nx * gh->ny * gh->nz;
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        dim3 tb(32, 8), tg((gh->nu + 1 + 31) / 32, (gh->nv + 2 + 31) / 32, gh->n_views);
        note_launch(), prep_diff_3d<T, NB><<<tg, tb, 0, st>>>(g, p, (int)pdt, (int)batch, (int)b0, gh->nu, gh->nv, ps);
        // target of the projector launches: x itself, or the chunk's sums (items 0 .. nbc - 1)
        const int64_t nbc = std::min<int64_t>(NB, batch - b0);
        void* xt = xacc ? (void*)xacc : x;
        const csm_dtype xtdt = xacc ? tdt : xdt;
        const int64_t bt = xacc ? nbc : batch, b0t = xacc ? 0 : b0;
        const int ft = xacc ? (flags & ~CSM_ACCUMULATE) : flags;
        csm_status r;
        if (zw >= kTop) r = launch_back3<T, NB, kTop>(g, gh, ps, xt, bt, xtdt, b0t, scale, ft, st);
        else if (zw >= 256) r = launch_back3<T, NB, (kTop >= 256 ? 256 : 64)>(g, gh, ps, xt, bt, xtdt, b0t, scale, ft, st);
        else if (zw == 128) r = launch_back3<T, NB, 128>(g, gh, ps, xt, bt, xtdt, b0t, scale, ft, st);
        else r = launch_back3<T, NB, 64>(g, gh, ps, xt, bt, xtdt, b0t, scale, ft, st);
        if (r != CSM_OK) return r;
        if (xacc) {
            note_launch(), sums_to_x_3d<T><<<1216, 256, 0, st>>>(xacc, (size_t)nbc * nvox, x, (int)xdt, (size_t)b0 * nvox,
                                                                 (flags & CSM_ACCUMULATE) ? 1 : 0);
            r = check_launch();
            if (r != CSM_OK) return r;
        }
    }
    return CSM_OK;
}

csm_status forward_3d(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt, csm_dtype pdt,
                      int flags, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    if (g->n_views > 65535 || (g->nv + 31) / 32 > 65535 || g->ny > 65535 || (g->nz + 31) / 32 > 65535)
        return CSM_EUNSUPPORTED;
    if (flags & CSM_VOXEL_DRIVEN) {
        if (!ws || ws_bytes < workspace_3d(g, 2, batch, dbl)) return CSM_EINVAL;
        return dbl ? run_fwd3_vox<double>(g, x, p, batch, xdt, pdt, flags, ws, st)
                   : run_fwd3_vox<float>(g, x, p, batch, xdt, pdt, flags, ws, st);
    }
    if (!ws || ws_bytes < workspace_3d(g, 0, batch, dbl)) return CSM_EINVAL;
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
    if ((g->nz + 63) / 64 > 65535 || g->n_views > 65535 || (g->nv + 31) / 32 > 65535) return CSM_EUNSUPPORTED;
    // x in another type than the arithmetic (BF16, F16, FP32 under FP64): with the larger
    // workspace (op 3) the sums are formed in an FP32 / FP64 copy, so that the back projection
    // runs in view groups and x is still rounded once; else one launch over all views
    const bool exact_x = dbl ? xdt == CSM_F64 : xdt == CSM_F32;
    const size_t sino = workspace_3d(g, 1, batch, dbl);
    void* xacc = (!exact_x && ws_bytes >= workspace_3d(g, 3, batch, dbl)) ? (char*)ws + sino : nullptr;
    switch (chunk3(batch)) {
        case 4: return dbl ? run_back3<double, 4>(g, p, x, batch, pdt, xdt, flags, ws, (double*)xacc, st)
                           : run_back3<float, 4>(g, p, x, batch, pdt, xdt, flags, ws, (float*)xacc, st);
        case 2: return dbl ? run_back3<double, 2>(g, p, x, batch, pdt, xdt, flags, ws, (double*)xacc, st)
                           : run_back3<float, 2>(g, p, x, batch, pdt, xdt, flags, ws, (float*)xacc, st);
        default: return dbl ? run_back3<double, 1>(g, p, x, batch, pdt, xdt, flags, ws, (double*)xacc, st)
                            : run_back3<float, 1>(g, p, x, batch, pdt, xdt, flags, ws, (float*)xacc, st);
    }
}

csm_status nnz_3d(const csm_geom_s* gh, int64_t* out, cudaStream_t st) {
    const Geo g = make_geo(gh);
    cudaError_t e = cudaMemsetAsync(gh->t.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    const size_t ncol = (size_t)gh->nx * gh->ny;
    dim3 bb(32 * BW), bg((unsigned)((ncol + BW - 1) / BW), (gh->nz + ZWN - 1) / ZWN);
    note_launch(), nnz3d_kernel<<<bg, bb, 0, st>>>(g, gh->t.counter);
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

// lines.cu -- line-based comparator projectors: the system matrices the paper compares the
// consistent one with (Section "Related work": line-integration methods; Section
// "Computational complexity": several lines per detector element, averaged).
//
//   Siddon:  W_ij = length of the ray inside voxel j (exact ray-box intersection lengths,
//            traversed voxel by voxel).
//   Joseph:  the ray is sampled at the centre plane of every voxel slice along its major axis;
//            the volume is interpolated (linearly in 2D, bilinearly in 3D) between the voxel
//            centres of that slice; each sample is weighted by the ray length per slice.
//
// A detector element's value is the mean of the line integrals along `lines` rays from the
// source to evenly spaced points of the element (lines x lines points in 3D): ray m hits
// u = u_k + (m + 1/2) du / lines.  The back projection is the exact adjoint: the same rays,
// the same weights, added to the volume with atomics (in no fixed order).
#include "csm_internal.cuh"

namespace csm {

template <typename T> struct LT;
template <> struct LT<float> {
    static __device__ __forceinline__ float cs(const Geo& g, int v, int i) { return g.cs_f[2 * v + i]; }
};
template <> struct LT<double> {
    static __device__ __forceinline__ double cs(const Geo& g, int v, int i) { return g.cs_d[2 * v + i]; }
};

template <typename T>
__device__ __forceinline__ T ld_any(const void* base, size_t i, int dt) {
    switch (dt) {
        case CSM_F64: return (T)((const double*)base)[i];
        case CSM_BF16: return (T)__bfloat162float(((const __nv_bfloat16*)base)[i]);
        case CSM_F16: return (T)__half2float(((const __half*)base)[i]);
        default: return (T)((const float*)base)[i];
    }
}

template <typename T>
__device__ __forceinline__ void st_any(void* base, size_t i, int dt, T v, bool acc) {
    switch (dt) {
        case CSM_F64: { double* q = (double*)base + i; *q = acc ? *q + (double)v : (double)v; break; }
        case CSM_BF16: {
            __nv_bfloat16* q = (__nv_bfloat16*)base + i;
            *q = __float2bfloat16_rn((acc ? __bfloat162float(*q) : 0.0f) + (float)v);
            break;
        }
        case CSM_F16: {
            __half* q = (__half*)base + i;
            *q = __float2half_rn((acc ? __half2float(*q) : 0.0f) + (float)v);
            break;
        }
        default: { float* q = (float*)base + i; *q = acc ? *q + (float)v : (float)v; break; }
    }
}

// One ray of view v to detector point (u, w): source S, direction d = D - S (parameter
// alpha in [0, 1] from S to D).
template <typename T>
struct Ray {
    T sx, sy, sz, dx, dy, dz;
    __device__ __forceinline__ void make(const Geo& g, int v, T u, T w) {
        const T c = LT<T>::cs(g, v, 0), s = LT<T>::cs(g, v, 1);
        const T S = (T)g.s_d, D = (T)g.sdd_d;
        sx = S * c; sy = S * s; sz = T(0);
        dx = -D * c - u * s;
        dy = -D * s + u * c;
        dz = w;
    }
};

// Visitor interface: f(cell index along x, y, z, weight) for each voxel the ray meets.
// Siddon: voxels traversed in order with their intersection lengths (3D; 2D with nz = 1,
// c the unit height and dz = 0).
template <typename T, typename F>
__device__ __forceinline__ void siddon(const Geo& g, const Ray<T>& r, F&& f) {
    const T x0 = (T)g.x0_d, y0 = (T)g.y0_d, z0 = (T)g.z0_d;
    const T a = (T)g.a_d, b = (T)g.b_d, c = (T)g.c_d;
    const T x1 = x0 + g.nx * a, y1 = y0 + g.ny * b, z1 = z0 + g.nz * c;
    T amin = T(0), amax = T(1);
    // slab intersections
    auto slab = [&](T s0, T d, T lo, T hi) {
        if (d != T(0)) {
            T t0 = (lo - s0) / d, t1 = (hi - s0) / d;
            if (t0 > t1) { const T t = t0; t0 = t1; t1 = t; }
            amin = t0 > amin ? t0 : amin;
            amax = t1 < amax ? t1 : amax;
        } else if (s0 < lo || s0 > hi) {
            amax = T(-1);
        }
    };
    slab(r.sx, r.dx, x0, x1);
    slab(r.sy, r.dy, y0, y1);
    slab(r.sz, r.dz, z0, z1);
    if (!(amax > amin)) return;
    const T len = sqrt(r.dx * r.dx + r.dy * r.dy + r.dz * r.dz);
    // the voxel at the entry point (middle of the first step, robust at faces)
    const T am = amin;
    int ix = (int)floor((r.sx + am * r.dx - x0) / a), iy = (int)floor((r.sy + am * r.dy - y0) / b);
    int iz = (int)floor((r.sz + am * r.dz - z0) / c);
    // nudge into the grid when the entry point lies on its boundary
    ix = ix < 0 ? 0 : (ix >= g.nx ? g.nx - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= g.ny ? g.ny - 1 : iy);
    iz = iz < 0 ? 0 : (iz >= g.nz ? g.nz - 1 : iz);
    const int stx = r.dx > T(0) ? 1 : -1, sty = r.dy > T(0) ? 1 : -1, stz = r.dz > T(0) ? 1 : -1;
    const T big = T(1e30);
    T tdx = r.dx != T(0) ? a / fabs(r.dx) : big, tdy = r.dy != T(0) ? b / fabs(r.dy) : big;
    T tdz = r.dz != T(0) ? c / fabs(r.dz) : big;
    T tmx = r.dx != T(0) ? (x0 + (ix + (stx > 0 ? 1 : 0)) * a - r.sx) / r.dx : big;
    T tmy = r.dy != T(0) ? (y0 + (iy + (sty > 0 ? 1 : 0)) * b - r.sy) / r.dy : big;
    T tmz = r.dz != T(0) ? (z0 + (iz + (stz > 0 ? 1 : 0)) * c - r.sz) / r.dz : big;
    T acur = amin;
    for (int guard = 0; guard < g.nx + g.ny + g.nz + 3; ++guard) {
        T an = tmx < tmy ? tmx : tmy;
        an = tmz < an ? tmz : an;
        const T aend = an < amax ? an : amax;
        if (aend > acur) f(ix, iy, iz, (aend - acur) * len);
        acur = aend;
        if (acur >= amax) break;
        if (an == tmx) { ix += stx; tmx += tdx; }
        else if (an == tmy) { iy += sty; tmy += tdy; }
        else { iz += stz; tmz += tdz; }
        if (ix < 0 || ix >= g.nx || iy < 0 || iy >= g.ny || iz < 0 || iz >= g.nz) break;
    }
}

// Joseph: slices along the ray's major axis; the other coordinates are interpolated between
// voxel centres (bilinear in 3D; in 2D the z part is one slice with weight 1).
template <typename T, typename F>
__device__ __forceinline__ void joseph(const Geo& g, const Ray<T>& r, F&& f) {
    const T ax = fabs(r.dx), ay = fabs(r.dy), az = fabs(r.dz);
    const int m = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    const T org[3] = {(T)g.x0_d, (T)g.y0_d, (T)g.z0_d};
    const T h[3] = {(T)g.a_d, (T)g.b_d, (T)g.c_d};
    const int n[3] = {g.nx, g.ny, g.nz};
    const T s[3] = {r.sx, r.sy, r.sz}, d[3] = {r.dx, r.dy, r.dz};
    const int p = m == 0 ? 1 : 0, q = m == 2 ? 1 : 2;    // the two other axes
    const T len = sqrt(r.dx * r.dx + r.dy * r.dy + r.dz * r.dz);
    const T wstep = h[m] * len / fabs(d[m]);               // ray length per slice
    for (int i = 0; i < n[m]; ++i) {
        const T xm = org[m] + (i + T(0.5)) * h[m];
        const T al = (xm - s[m]) / d[m];
        if (al < T(0) || al > T(1)) continue;
        const T tp = (s[p] + al * d[p] - org[p]) / h[p] - T(0.5);
        const T tq = (s[q] + al * d[q] - org[q]) / h[q] - T(0.5);
        const T fp = floor(tp), fq = floor(tq);
        const int jp = (int)fp, jq = (int)fq;
        const T wp = tp - fp, wq = tq - fq;
#pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
#pragma unroll
            for (int cq = 0; cq < 2; ++cq) {
                const int kp = jp + cp, kq = jq + cq;
                if (kp < 0 || kp >= n[p] || kq < 0 || kq >= n[q]) continue;
                const T w = (cp ? wp : T(1) - wp) * (cq ? wq : T(1) - wq);
                if (w == T(0)) continue;
                int idx[3];
                idx[m] = i; idx[p] = kp; idx[q] = kq;
                f(idx[0], idx[1], idx[2], wstep * w);
            }
        }
    }
}

// In 2D (nz = 1, z0 = -c/2) the rays have dz = 0 and z = 0: Joseph's third axis has one
// voxel centre at z = 0, interpolation weight 1.

template <typename T>
__global__ void __launch_bounds__(128) line_fwd(Geo g, int model, int lines, const void* __restrict__ x, int xdt,
                                                void* __restrict__ p, int pdt, int b, int accumulate) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y, v = blockIdx.z;
    if (k >= g.nu) return;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    const void* xb = (const char*)x + 0;
    const size_t xoff = (size_t)b * nvox;
    const int lz = g.nz > 1 || g.nv > 1 ? lines : 1;     // rows of sub-rays (3D)
    T acc = T(0);
    for (int mz = 0; mz < lz; ++mz) {
        const T w = g.nv > 1 || g.nz > 1 ? (T)(g.v0_d + (l + (mz + 0.5) / lz) * g.dv_d) : T(0);
        for (int mu = 0; mu < lines; ++mu) {
            const T u = (T)(g.u0_d + (k + (mu + 0.5) / lines) * g.du_d);
            Ray<T> r;
            r.make(g, v, u, w);
            auto vis = [&](int ix, int iy, int iz, T wt) {
                acc += wt * ld_any<T>(xb, xoff + ((size_t)iz * g.ny + iy) * g.nx + ix, xdt);
            };
            if (model == CSM_LINE_SIDDON) siddon<T>(g, r, vis);
            else joseph<T>(g, r, vis);
        }
    }
    acc /= (T)(lines * lz);
    st_any<T>(p, (((size_t)b * g.n_views + v) * g.nv + l) * g.nu + k, pdt, acc, accumulate != 0);
}

template <typename T>
__global__ void __launch_bounds__(128) line_back(Geo g, int model, int lines, const void* __restrict__ p, int pdt,
                                                 T* __restrict__ x, int b) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int l = blockIdx.y, v = blockIdx.z;
    if (k >= g.nu) return;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    const int lz = g.nz > 1 || g.nv > 1 ? lines : 1;
    const T pv = ld_any<T>(p, (((size_t)b * g.n_views + v) * g.nv + l) * g.nu + k, pdt) / (T)(lines * lz);
    if (pv == T(0)) return;
    T* xb = x + (size_t)b * nvox;
    for (int mz = 0; mz < lz; ++mz) {
        const T w = g.nv > 1 || g.nz > 1 ? (T)(g.v0_d + (l + (mz + 0.5) / lz) * g.dv_d) : T(0);
        for (int mu = 0; mu < lines; ++mu) {
            const T u = (T)(g.u0_d + (k + (mu + 0.5) / lines) * g.du_d);
            Ray<T> r;
            r.make(g, v, u, w);
            auto vis = [&](int ix, int iy, int iz, T wt) {
                atomicAdd(xb + ((size_t)iz * g.ny + iy) * g.nx + ix, wt * pv);
            };
            if (model == CSM_LINE_SIDDON) siddon<T>(g, r, vis);
            else joseph<T>(g, r, vis);
        }
    }
}

}  // namespace csm

using namespace csm;

extern "C" {

static csm_status line_args(csm_geom_t g, int model, int lines, int64_t batch, csm_dtype a, csm_dtype b) {
    if (!g || batch < 0 || lines < 1 || lines > 64) return CSM_EINVAL;
    if (model != CSM_LINE_SIDDON && model != CSM_LINE_JOSEPH) return CSM_EINVAL;
    auto ok = [](csm_dtype t) { return t == CSM_F32 || t == CSM_F64 || t == CSM_BF16 || t == CSM_F16; };
    if (!ok(a) || !ok(b)) return CSM_EINVAL;
    if (g->n_views > 65535 || g->nv > 65535) return CSM_EUNSUPPORTED;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    return dev == g->device ? CSM_OK : CSM_EINVAL;
}

csm_status csm_forward_line(csm_geom_t g, int model, int lines, const void* x, void* p, int64_t batch, csm_dtype xdt,
                            csm_dtype pdt, int flags, void* stream) {
    csm_status s = line_args(g, model, lines, batch, xdt, pdt);
    if (s != CSM_OK) return s;
    if (flags & ~CSM_ACCUMULATE) return CSM_EINVAL;
    if (batch == 0) return CSM_OK;
    if (!x || !p) return CSM_EINVAL;
    const Geo geo = make_geo(g);
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    dim3 blk(128), grd((g->nu + 127) / 128, g->nv, g->n_views);
    for (int64_t b = 0; b < batch; ++b) {
        if (dbl) note_launch(), line_fwd<double><<<grd, blk, 0, (cudaStream_t)stream>>>(geo, model, lines, x, (int)xdt, p, (int)pdt,
                                                                        (int)b, flags & CSM_ACCUMULATE);
        else note_launch(), line_fwd<float><<<grd, blk, 0, (cudaStream_t)stream>>>(geo, model, lines, x, (int)xdt, p, (int)pdt,
                                                                      (int)b, flags & CSM_ACCUMULATE);
        s = check_launch();
        if (s != CSM_OK) return s;
    }
    return CSM_OK;
}

csm_status csm_back_line(csm_geom_t g, int model, int lines, const void* p, void* x, int64_t batch, csm_dtype pdt,
                         csm_dtype xdt, int flags, void* stream) {
    csm_status s = line_args(g, model, lines, batch, pdt, xdt);
    if (s != CSM_OK) return s;
    if (flags & ~CSM_ACCUMULATE) return CSM_EINVAL;
    if (xdt != CSM_F32 && xdt != CSM_F64) return CSM_EUNSUPPORTED;   // added to with atomics
    if (batch == 0) return CSM_OK;
    if (!x || !p) return CSM_EINVAL;
    const Geo geo = make_geo(g);
    const size_t nvox = (size_t)g->nx * g->ny * g->nz;
    if (!(flags & CSM_ACCUMULATE)) {
        cudaError_t e = cudaMemsetAsync(x, 0, nvox * batch * (xdt == CSM_F64 ? 8 : 4), (cudaStream_t)stream);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    }
    dim3 blk(128), grd((g->nu + 127) / 128, g->nv, g->n_views);
    for (int64_t b = 0; b < batch; ++b) {
        if (xdt == CSM_F64) note_launch(), line_back<double><<<grd, blk, 0, (cudaStream_t)stream>>>(geo, model, lines, p, (int)pdt,
                                                                                   (double*)x, (int)b);
        else note_launch(), line_back<float><<<grd, blk, 0, (cudaStream_t)stream>>>(geo, model, lines, p, (int)pdt, (float*)x, (int)b);
        s = check_launch();
        if (s != CSM_OK) return s;
    }
    return CSM_OK;
}

}  // extern "C"

// csm_internal.cuh -- geometry handle, kernel parameter blocks and the shared device math
// of the projectors.  Included by every translation unit of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/csm.h"

namespace csm {

// ---------------------------------------------------------------------------------------
// Geometry handle (host).  The device block holds, per view:
//   axis_sigma[v] = {axis, sigma}: axis 0 walks the grid along x (pixel columns) and writes
//       every corner ray as a line y(x); axis 1 walks along y with lines x(y).  sigma = +1
//       when the line of corner k+1 lies above (larger cross coordinate) the line of k.
//   cs[v]       = {cos phi, sin phi}
//   line_fx     = per corner k: the line's cross coordinate in cell units at walk boundary
//                 w = 0 and its step per cell, both 32.32 fixed point (int64)
//   line_d      = the same two numbers in double
//   inv2        = 1 / (2 |step|) per corner (float and double)
//   wrange      = per element k: the walk cells [w0, w1) where its strip meets the grid
//   rows (3D)   = per row corner l: q_l = v_l / sdd (float and double), and q_l as a float
//                 pair hi + lo with 1/|q_l| (float4), from which the kernels form the height
//                 of the plane { v(P) = v_l } = { z = q_l t(P) } at a column centre
//   columns (3D) = per view the depth of column centres over c, T0 + ix Tx + iy Ty
//                 (32.32 fixed point and double)
// ---------------------------------------------------------------------------------------
struct DeviceTables {
    int* axis_sigma = nullptr;     // [V][2]
    float* cs_f = nullptr;         // [V][2]
    double* cs_d = nullptr;        // [V][2]
    long long* line_fx = nullptr;  // [V][nu+1][2]
    double* line_d = nullptr;      // [V][nu+1][2]
    float* inv_f = nullptr;        // [V][nu+1]
    double* inv_d = nullptr;       // [V][nu+1]
    int* wrange = nullptr;         // [V][nu][2]
    float* rowq_f = nullptr;       // [nv+1]
    double* rowq_d = nullptr;      // [nv+1]
    float4* rowq4 = nullptr;       // [nv+1] {q hi, q lo, 1/|q|, 0}
    long long* colt_fx = nullptr;  // [V][3] column-centre depth / c = T0 + ix Tx + iy Ty, 32.32 (3D)
    double* colt_d = nullptr;      // [V][3]
    unsigned long long* counter = nullptr;  // scratch word for csm_nnz
};

}  // namespace csm

struct csm_geom_s {
    int dim = 2;
    int nx = 0, ny = 0, nz = 1;
    double a = 1, b = 1, c = 1;
    int n_views = 0;
    std::vector<double> angles;
    double s = 0, sdd = 0;
    int nu = 0, nv = 1;
    double du = 1, dv = 1, u_off = 0, v_off = 0;
    int device = 0;
    void* w_block = nullptr;       // per-element sensitivity weights (float then double), or none
    void* d_block = nullptr;
    size_t d_bytes = 0;
    csm::DeviceTables t;
    int64_t nnz = -1;
};

namespace csm {

// Parameters passed by value to the kernels.
struct Geo {
    int nx, ny, nz, nu, nv, n_views;
    // grid and detector in float and double
    float a, b, c, s, sdd, du, dv, u0, v0, x0, y0, z0;
    double a_d, b_d, c_d, s_d, sdd_d, du_d, dv_d, u0_d, v0_d, x0_d, y0_d, z0_d;
    // reciprocals 1/du, 1/dv, 1/c (rounded from FP64), so that no kernel divides by them
    float idu, idv, ic;
    double idu_d, idv_d, ic_d;
    // row planes: largest |q_l| = |v_l| / sdd over the detector's row corners, and the step
    // dq = dv / sdd between neighbouring corners (3D)
    float qmax, dq;
    double qmax_d, dq_d;
    const int* axis_sigma;
    const float* cs_f;
    const double* cs_d;
    const long long* line_fx;
    const double* line_d;
    const float* inv_f;
    const double* inv_d;
    const int* wrange;
    const float* rowq_f;
    const double* rowq_d;
    const float4* rowq4;
    const long long* colt_fx;
    const double* colt_d;
    // per-element sensitivity weights w[v][l][k] (NULL: all 1), float and double copies
    const float* ew_f;
    const double* ew_d;
};

Geo make_geo(const csm_geom_s* g);

// Sensitivity weight of element i = (v nv + l) nu + k (1 without weights).
template <typename T> __device__ __forceinline__ T elem_weight(const Geo& g, size_t i);
template <> __device__ __forceinline__ float elem_weight<float>(const Geo& g, size_t i) {
    return g.ew_f ? g.ew_f[i] : 1.0f;
}
template <> __device__ __forceinline__ double elem_weight<double>(const Geo& g, size_t i) {
    return g.ew_d ? g.ew_d[i] : 1.0;
}

// Most detector row corners (rows + 1) that one voxel's footprint can span in one view; the
// 3D kernels keep one value per corner in registers.  Geometries beyond it are refused.
constexpr int kMaxRowCorners = 8;
// Most corner lines that cross one voxel column's cell in one view; the voxel-driven 3D
// kernels keep one top-view atom per crossing line in shared memory.  Checked on the host.
constexpr int kMaxG = 6;

// thread-local record of the last CUDA error text
void set_cuda_error(cudaError_t e);
csm_status check_launch();
// counts one kernel launch issued from the host (every launch site of the library calls it
// just before its <<< >>>; csm_launch_count reads the total)
void note_launch();

// ---------------------------------------------------------------------------------------
// Element conversions for storage types.
// ---------------------------------------------------------------------------------------
template <typename S> __device__ __forceinline__ float to_f(S v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<double>(double v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

template <typename T, typename S> __device__ __forceinline__ T load_as(const S* p) { return (T)to_f<S>(*p); }
template <> __device__ __forceinline__ double load_as<double, double>(const double* p) { return *p; }
template <> __device__ __forceinline__ float load_as<float, float>(const float* p) { return *p; }

template <typename S> __device__ __forceinline__ S from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_f<double>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

template <typename S, typename T> __device__ __forceinline__ void store_as(S* p, T v, bool acc) {
    float cur = acc ? to_f<S>(*p) : 0.0f;
    *p = from_f<S>(cur + (float)v);
}
template <> __device__ __forceinline__ void store_as<double, double>(double* p, double v, bool acc) {
    *p = acc ? *p + v : v;
}
template <> __device__ __forceinline__ void store_as<float, float>(float* p, float v, bool acc) {
    *p = acc ? *p + v : v;
}

// ---------------------------------------------------------------------------------------
// The 2D atom: the fraction of a unit cell lying below a straight line.
//
// Walking the grid along one axis, every corner ray is a straight line across a cell.  Its
// cross coordinates at the two walk-faces of the cell, measured in cell units from the
// cell's lower cross-face, are p and q.  The part of the cell below the line is
//   - a trapezoid when the line crosses both walk-faces inside the cell (the paper's A_4
//     between two such rays, Eq. (area trapezoid rel): height x mid-line),
//   - a corner triangle, or the cell minus one, when the line leaves through a cross-face
//     (the paper's A_3, Section "Triangle"),
// i.e. clamp(line, 0, 1) integrated over the cell.  With relu(y) - relu(y - 1) = clamp and
// the exact mean of relu over a linear segment,
//      mean_{tau in [0,1]} relu(p + (q - p) tau) = (p + q)/2            if p, q >= 0
//                                              = 0                       if p, q <= 0
//                                              = max(p,q)^2 / (2|q - p|) otherwise,
// where 1 / (2|q - p|) is a per-line constant (the line's step per cell), so the atom needs
// no division.  An element's weight is the difference of the atoms of its two corner rays
// (the cumulative form of the sums and differences of Eq. (2d procedure)).
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T relu_mean(T p, T q, T inv2) {
    T mx = p > q ? p : q;
    T mn = p > q ? q : p;
    if (mn >= T(0)) return T(0.5) * (p + q);
    if (mx <= T(0)) return T(0);
    return mx * mx * inv2;
}

// Branch-free form of the same atom (selects instead of branches): lanes of a warp that sit
// in different cases issue the same instructions.  Exactly 1 when the line lies above the
// cell and exactly 0 when it lies below.
template <typename T>
__device__ __forceinline__ T relu_mean_sel(T p, T q, T inv2) {
    const T mx = p > q ? p : q, mn = p > q ? q : p;
    const T r = mx > T(0) ? mx : T(0);
    return mn >= T(0) ? T(0.5) * (p + q) : r * r * inv2;
}

template <typename T>
__device__ __forceinline__ T cell_atom(T p, T q, T inv2) {
    const T mn = p > q ? q : p;
    const T v = relu_mean_sel(p, q, inv2) - relu_mean_sel(p - T(1), q - T(1), inv2);
    return mn >= T(1) ? T(1) : v;
}

template <typename T>
__device__ __forceinline__ T cell_below(T p, T q, T inv2) {
    T mx = p > q ? p : q;
    T mn = p > q ? q : p;
    if (mn >= T(1)) return T(1);
    if (mx <= T(0)) return T(0);
    if (mn >= T(0) && mx <= T(1)) return T(0.5) * (p + q);
    return relu_mean(p, q, inv2) - relu_mean(p - T(1), q - T(1), inv2);
}

// Cross coordinate of a corner line relative to cell c, at walk boundaries w and w+1.
// Float path: 32.32 fixed point, exact stepping, so the local offset carries no error from
// the magnitude of the absolute position.  Double path: double arithmetic.
struct LineF {
    long long p, d;   // position at walk boundary w, step per cell
    __device__ __forceinline__ void load(const Geo& g, int v, int k, int w) {
        const long long* e = g.line_fx + 2 * ((size_t)v * (g.nu + 1) + k);
        d = e[1];
        p = e[0] + (long long)w * d;
    }
    __device__ __forceinline__ void step() { p += d; }
    __device__ __forceinline__ int cell_lo() const {   // floor of min(position at w, w+1)
        long long q = p + d;
        return (int)((p < q ? p : q) >> 32);
    }
    __device__ __forceinline__ int cell_hi() const {
        long long q = p + d;
        return (int)((p > q ? p : q) >> 32);
    }
    static __device__ __forceinline__ float local(long long P, int c) {
        int hi = (int)(P >> 32);
        unsigned lo = (unsigned)(P & 0xffffffffull);
        return (float)(hi - c) + (float)lo * 2.3283064365386963e-10f;
    }
    __device__ __forceinline__ void offsets(int c, float& ya, float& yb) const {
        ya = local(p, c);
        yb = local(p + d, c);
    }
    // offsets at the walk faces w, w + 1, w + 2 (two neighbouring columns)
    __device__ __forceinline__ void offsets3(int c, float& ya, float& yb, float& yc) const {
        ya = local(p, c);
        yb = local(p + d, c);
        yc = local(p + 2 * d, c);
    }
};

struct LineD {
    double p, d;
    __device__ __forceinline__ void load(const Geo& g, int v, int k, int w) {
        const double* e = g.line_d + 2 * ((size_t)v * (g.nu + 1) + k);
        d = e[1];
        p = e[0] + (double)w * d;
    }
    __device__ __forceinline__ void step() { p += d; }
    __device__ __forceinline__ int cell_lo() const { return (int)floor(fmin(p, p + d)); }
    __device__ __forceinline__ int cell_hi() const { return (int)floor(fmax(p, p + d)); }
    __device__ __forceinline__ void offsets(int c, double& ya, double& yb) const {
        ya = p - (double)c;
        yb = (p + d) - (double)c;
    }
    __device__ __forceinline__ void offsets3(int c, double& ya, double& yb, double& yc) const {
        ya = p - (double)c;
        yb = (p + d) - (double)c;
        yc = (p + 2.0 * d) - (double)c;
    }
};

template <typename T> struct LineOf;
template <> struct LineOf<float> { using type = LineF; };
template <> struct LineOf<double> { using type = LineD; };

template <typename T> __device__ __forceinline__ T inv_of(const Geo& g, int v, int k);
template <> __device__ __forceinline__ float inv_of<float>(const Geo& g, int v, int k) {
    return g.inv_f[(size_t)v * (g.nu + 1) + k];
}
template <> __device__ __forceinline__ double inv_of<double>(const Geo& g, int v, int k) {
    return g.inv_d[(size_t)v * (g.nu + 1) + k];
}

// Launch entry points implemented per dimension.
csm_status forward_2d(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt,
                      csm_dtype pdt, int flags, void* ws, size_t ws_bytes, cudaStream_t st);
csm_status back_2d(const csm_geom_s* g, const void* p, void* x, int64_t batch, csm_dtype pdt,
                   csm_dtype xdt, int flags, void* ws, size_t ws_bytes, cudaStream_t st);
size_t workspace_2d(const csm_geom_s* g, int op, int64_t batch, bool dbl);
csm_status nnz_2d(const csm_geom_s* g, int64_t* out, cudaStream_t st);

// Sparse export (sparse.cu drives these passes over every entry with |w| > thr, scaled by
// `scale`).  Rows of W^T are voxels, rows of W detector elements (v nv + l) nu + k.
//   mode 0: rows of W^T, counts[voxel] = number of entries     (no atomics)
//   mode 1: rows of W^T, fill from row_ptr in (view, row, column) order (sorted columns)
//   mode 2: rows of W,   counts[element] += 1                   (atomics)
//   mode 3: rows of W,   fill at row_ptr[element] + cursor[element]++ (atomics; rows sorted later)
struct ExportArgs {
    int mode;
    double thr, scale;
    unsigned long long* counts;
    const long long* row_ptr;
    int* cursor;
    int* col;
    void* val;
    int dbl;   // values (and arithmetic) in FP64
};
csm_status export_2d(const csm_geom_s* g, const ExportArgs& a, cudaStream_t st);
csm_status export_3d(const csm_geom_s* g, const ExportArgs& a, cudaStream_t st);

csm_status forward_3d(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt,
                      csm_dtype pdt, int flags, void* ws, size_t ws_bytes, cudaStream_t st);
csm_status back_3d(const csm_geom_s* g, const void* p, void* x, int64_t batch, csm_dtype pdt,
                   csm_dtype xdt, int flags, void* ws, size_t ws_bytes, cudaStream_t st);
size_t workspace_3d(const csm_geom_s* g, int op, int64_t batch, bool dbl);
csm_status nnz_3d(const csm_geom_s* g, int64_t* out, cudaStream_t st);

}  // namespace csm

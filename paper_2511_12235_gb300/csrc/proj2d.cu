// proj2d.cu -- 2D fan-beam projectors: p = W x (ray-driven gather) and x = W^T p
// (voxel-driven gather), with every entry W_ij evaluated on the fly.
//
// Entry of W (Introduction, Eq. (ip)): the area of pixel j inside the fan of element k,
// i.e. between the rays to detector corners k and k+1.  Each view walks the grid along one
// axis (the paper's frame rotation by pi/2 so that the rays cross the walked cells from
// one walk-face to the other, Section "The Two-dimensional Case"); inside a cell every corner
// ray is a straight line, the area below it is a trapezoid or a corner triangle (the
// paper's A_4 and A_3 atoms), and the element's area is the difference of the two corner
// rays' atoms (the sums / differences of Eq. (2d procedure) in cumulative form).
#include <algorithm>

#include "csm_internal.cuh"

namespace csm {

static int chunk_for(int64_t batch) {
    if (batch >= 16) return 16;
    if (batch >= 8) return 8;
    if (batch >= 4) return 4;
    if (batch >= 2) return 2;
    return 1;
}

static size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

size_t workspace_2d(const csm_geom_s* g, int op, int64_t batch, bool dbl) {
    if (batch <= 0) return 0;
    const size_t es = dbl ? 8 : 4;
    const size_t nb = chunk_for(batch);
    if (op == 0) return 2 * al256((size_t)g->nx * g->ny * nb * es);
    if (op == 2) return al256((size_t)g->n_views * g->nu * es);   // voxel-driven forward: sums of one item
    return al256((size_t)g->n_views * g->nu * nb * es);
}

// ---------------------------------------------------------------------------------------
// Layout kernels: gather a chunk of NB batch items into pixel-major, batch-interleaved
// copies (one per walk axis) so that the projector reads NB contiguous values per cell.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T load_any(const void* base, size_t i, int dt) {
    switch (dt) {
        case CSM_F64: return (T)((const double*)base)[i];
        case CSM_BF16: return (T)__bfloat162float(((const __nv_bfloat16*)base)[i]);
        case CSM_F16: return (T)__half2float(((const __half*)base)[i]);
        default: return (T)((const float*)base)[i];
    }
}

template <typename T>
__device__ __forceinline__ void store_any(void* base, size_t i, int dt, T v, bool acc) {
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

// Batch items are grouped in vectors of VW = min(NB, 4); a chunk of NB items is stored as
// Q = NB / VW planes so that the lanes of a warp, which visit neighbouring cells, read
// neighbouring 16-byte vectors:
//   walk x:  xs0[((ix * Q + q) * ny + iy) * VW + r]      (b = q * VW + r)
//   walk y:  xs1[((iy * Q + q) * nx + ix) * VW + r]
template <int NB> struct Vec { static constexpr int W = NB < 4 ? NB : 4; static constexpr int Q = NB / W; };

template <typename T, int NB>
__global__ void __launch_bounds__(256) prep_image_2d(const void* __restrict__ x, int xdt, int B, int b_off,
                                                     int nx, int ny, T* __restrict__ xs0, T* __restrict__ xs1) {
    constexpr int VW = Vec<NB>::W, Q = Vec<NB>::Q;
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int bb = 0; bb < NB; ++bb) {
        const int b = b_off + bb, q = bb / VW, r = bb % VW;
        for (int j = ty; j < 32; j += 8) {
            int ix = bx + tx, iy = by + j;
            T val = T(0);
            if (ix < nx && iy < ny && b < B) val = load_any<T>(x, ((size_t)b * ny + iy) * nx + ix, xdt);
            tile[j][tx] = val;
            if (ix < nx && iy < ny) xs1[(((size_t)iy * Q + q) * nx + ix) * VW + r] = val;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            int ix = bx + j, iy = by + tx;
            if (ix < nx && iy < ny) xs0[(((size_t)ix * Q + q) * ny + iy) * VW + r] = tile[tx][j];
        }
        __syncthreads();
    }
}

// p[b][v][k] -> ps[((v * Q + q) * nu + k) * VW + r]
// (the element's sensitivity weight applied: the back projection of diag(w) p)
template <typename T, int NB>
__global__ void prep_sino_2d(Geo g, const void* __restrict__ p, int pdt, int B, int b_off, int V, int nu,
                             T* __restrict__ ps) {
    constexpr int VW = Vec<NB>::W, Q = Vec<NB>::Q;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * nu) return;
    const size_t v = i / nu, k = i % nu;
    const T w = elem_weight<T>(g, i);
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
        const int b = b_off + bb;
        ps[((v * Q + bb / VW) * nu + k) * VW + bb % VW] = b < B ? w * load_any<T>(p, (size_t)b * V * nu + i, pdt) : T(0);
    }
}

// acc[b] += wt * value[b] for the NB items of one cell; `base` points at the cell's first
// vector and consecutive planes are `plane` elements apart.
template <typename T, int NB> struct Cell;   // the NB values of one cell, in registers
template <int NB> struct Cell<float, NB> {
    static constexpr int Q = Vec<NB>::Q;
    float4 v[Q];
    __device__ __forceinline__ void load(const float* __restrict__ base, size_t plane) {
        if constexpr (Vec<NB>::W == 4) {
#pragma unroll
            for (int q = 0; q < Q; ++q) v[q] = __ldg(reinterpret_cast<const float4*>(base + q * plane));
        } else {
#pragma unroll
            for (int r = 0; r < NB; ++r) (&v[0].x)[r] = __ldg(base + r);
        }
    }
    // pairs of items with the packed FP32x2 FMA (one instruction per two items, the same
    // IEEE fused multiply-add per item as the scalar form)
    __device__ __forceinline__ void fma(float (&acc)[NB], float wt) const {
        if constexpr (NB % 2 == 0) {
            const float2 w2 = make_float2(wt, wt);
#pragma unroll
            for (int i = 0; i < NB; i += 2) {
                const float2 a = __ffma2_rn(make_float2((&v[0].x)[i], (&v[0].x)[i + 1]), w2,
                                            make_float2(acc[i], acc[i + 1]));
                acc[i] = a.x;
                acc[i + 1] = a.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < NB; ++i) acc[i] += wt * (&v[0].x)[i];
        }
    }
};
template <int NB> struct Cell<double, NB> {
    static constexpr int Q = Vec<NB>::Q, W = Vec<NB>::W;
    double v[NB];
    __device__ __forceinline__ void load(const double* __restrict__ base, size_t plane) {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int r = 0; r < W; ++r) v[q * W + r] = __ldg(base + q * plane + r);
    }
    __device__ __forceinline__ void fma(double (&acc)[NB], double wt) const {
#pragma unroll
        for (int i = 0; i < NB; ++i) acc[i] += wt * v[i];
    }
};

// ---------------------------------------------------------------------------------------
// Forward, ray-driven: one thread per (view, pair of neighbouring elements k, k+1) (E = 2;
// one element per thread, E = 1, when pairs would leave too few threads).  The thread walks
// the cells of its fan strip (between corner lines k and k+E) along the view's walk axis; in
// each walked column it visits the cells between the outer lines, loads each cell's NB batch
// values once and accumulates  W * x  for its elements (their weights are differences of
// neighbouring lines' cell atoms).  A block holds 16 threads of each of 4 neighbouring views:
// their strips cover nearly the same cells, so a cell fetched into L1 for one view serves
// the others.
// ---------------------------------------------------------------------------------------
template <typename T, int NB, int E>
__global__ void __launch_bounds__(64) fwd2d_ray(Geo g, const T* __restrict__ xs0, const T* __restrict__ xs1,
                                                 void* __restrict__ p, int pdt, int B, int b_off, T scale,
                                                 int accumulate) {
    const int k = (blockIdx.x * 16 + (threadIdx.x & 15)) * E;
    const int v = blockIdx.y * 4 + (threadIdx.x >> 4);
    if (k >= g.nu || v >= g.n_views) return;
    const bool two = E == 2 && k + 1 < g.nu;
    const int kc = two ? k + 2 : k + 1;            // outer line of the pair
    const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
    const int nc = axis == 0 ? g.ny : g.nx;
    const T* __restrict__ xs = axis == 0 ? xs0 : xs1;
    const int* wr = g.wrange + 2 * ((size_t)v * g.nu + k);
    const int w0 = two ? min(wr[0], wr[2]) : wr[0], w1 = two ? max(wr[1], wr[3]) : wr[1];
    using L = typename LineOf<T>::type;
    L la, lb, lc;
    la.load(g, v, k, w0);
    lb.load(g, v, k + 1, w0);
    lc.load(g, v, kc, w0);
    const T ia = inv_of<T>(g, v, k), ib = inv_of<T>(g, v, k + 1), ic = inv_of<T>(g, v, kc);
    T acc[NB], acc2[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) acc[i] = acc2[i] = T(0);
    for (int w = w0; w < w1; ++w) {
        int clo = min(la.cell_lo(), lc.cell_lo());
        int chi = max(la.cell_hi(), lc.cell_hi());
        const int c0 = max(clo, 0);
        chi = min(chi, nc - 1);
        if (c0 <= chi) {
            // the lines' cross offsets at the two walk faces, relative to cell c0, converted
            // once per column; per cell only an integer shift remains
            T a0, a1, b0, b1, e0, e1;
            la.offsets(c0, a0, a1);
            lb.offsets(c0, b0, b1);
            lc.offsets(c0, e0, e1);
            const T* xw = xs + ((size_t)w * Vec<NB>::Q * nc) * Vec<NB>::W;
            for (int c = c0; c <= chi; ++c) {
                // the cell's values first: their latency overlaps the weight arithmetic
                Cell<T, NB> cell;
                cell.load(xw + (size_t)c * Vec<NB>::W, (size_t)nc * Vec<NB>::W);
                const T fa = cell_atom(a0, a1, ia), fb = cell_atom(b0, b1, ib);
                const T wt = sigma > 0 ? fb - fa : fa - fb;
                cell.fma(acc, wt);
                if constexpr (E == 2) {
                    const T fc = cell_atom(e0, e1, ic);
                    const T wt2 = sigma > 0 ? fc - fb : fb - fc;
                    cell.fma(acc2, wt2);
                }
                a0 -= T(1);
                a1 -= T(1);
                b0 -= T(1);
                b1 -= T(1);
                e0 -= T(1);
                e1 -= T(1);
            }
        }
        la.step();
        lb.step();
        lc.step();
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = b_off + i;
        if (b < B) {
            store_any<T>(p, ((size_t)b * g.n_views + v) * g.nu + k, pdt,
                         acc[i] * scale * elem_weight<T>(g, (size_t)v * g.nu + k), accumulate != 0);
            if (two) store_any<T>(p, ((size_t)b * g.n_views + v) * g.nu + k + 1, pdt,
                                  acc2[i] * scale * elem_weight<T>(g, (size_t)v * g.nu + k + 1), accumulate != 0);
        }
    }
}

template <typename T> __device__ __forceinline__ T cs_of(const Geo& g, int v, int i);
template <> __device__ __forceinline__ float cs_of<float>(const Geo& g, int v, int i) { return g.cs_f[2 * v + i]; }
template <> __device__ __forceinline__ double cs_of<double>(const Geo& g, int v, int i) { return g.cs_d[2 * v + i]; }

template <typename T> struct GeoT;
template <> struct GeoT<float> {
    static __device__ __forceinline__ float s(const Geo& g) { return g.s; }
    static __device__ __forceinline__ float sdd(const Geo& g) { return g.sdd; }
    static __device__ __forceinline__ float u0(const Geo& g) { return g.u0; }
    static __device__ __forceinline__ float du(const Geo& g) { return g.du; }
    static __device__ __forceinline__ float idu(const Geo& g) { return g.idu; }
    static __device__ __forceinline__ float x0(const Geo& g) { return g.x0; }
    static __device__ __forceinline__ float y0(const Geo& g) { return g.y0; }
    static __device__ __forceinline__ float a(const Geo& g) { return g.a; }
    static __device__ __forceinline__ float b(const Geo& g) { return g.b; }
};
template <> struct GeoT<double> {
    static __device__ __forceinline__ double s(const Geo& g) { return g.s_d; }
    static __device__ __forceinline__ double sdd(const Geo& g) { return g.sdd_d; }
    static __device__ __forceinline__ double u0(const Geo& g) { return g.u0_d; }
    static __device__ __forceinline__ double du(const Geo& g) { return g.du_d; }
    static __device__ __forceinline__ double idu(const Geo& g) { return g.idu_d; }
    static __device__ __forceinline__ double x0(const Geo& g) { return g.x0_d; }
    static __device__ __forceinline__ double y0(const Geo& g) { return g.y0_d; }
    static __device__ __forceinline__ double a(const Geo& g) { return g.a_d; }
    static __device__ __forceinline__ double b(const Geo& g) { return g.b_d; }
};

// Elements [k0, k1] whose interval can meet the pixel's projection: the detector
// coordinates of its corners (Appendix Eq. (tan beta): u = sdd tan gamma).  The range is
// widened by a margin far above the rounding error of u (1e-3 element in FP32), so an
// element is never missed; an element included by the margin gets an exact zero weight.
template <typename T> __device__ __forceinline__ T quick_div(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float quick_div<float>(float a, float b) { return __fdividef(a, b); }
template <typename T> struct RangeEps;
template <> struct RangeEps<float> { static constexpr float v = 1e-3f; };
template <> struct RangeEps<double> { static constexpr double v = 1e-9; };

template <typename T>
__device__ __forceinline__ bool pixel_elements(const Geo& g, int v, T X0, T X1, T Y0, T Y1, int& k0, int& k1) {
    const T c = cs_of<T>(g, v, 0), sn = cs_of<T>(g, v, 1);
    const T s = GeoT<T>::s(g), D = GeoT<T>::sdd(g);
    T umin = T(1e30), umax = T(-1e30);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const T X = (q & 1) ? X1 : X0, Y = (q & 2) ? Y1 : Y0;
        const T t = s - X * c - Y * sn;
        const T u = quick_div<T>(D * (Y * c - X * sn), t);
        umin = u < umin ? u : umin;
        umax = u > umax ? u : umax;
    }
    const T inv_du = GeoT<T>::idu(g);
    T f0 = floor((umin - GeoT<T>::u0(g)) * inv_du - RangeEps<T>::v);
    T f1 = floor((umax - GeoT<T>::u0(g)) * inv_du + RangeEps<T>::v);
    f0 = f0 < T(-2) ? T(-2) : (f0 > T(g.nu + 2) ? T(g.nu + 2) : f0);
    f1 = f1 < T(-2) ? T(-2) : (f1 > T(g.nu + 2) ? T(g.nu + 2) : f1);
    k0 = max((int)f0, 0);
    k1 = min((int)f1, g.nu - 1);
    return k0 <= k1;
}

// ---------------------------------------------------------------------------------------
// Back projection, gather form, two pixels per thread.  A block holds a 16 x 8 pixel tile and
// BG view groups (views v = g, g + BG, ...).  Each thread takes two pixels that are
// neighbours along the view's walk axis: for the views walked along x (axis 0) the pairs
// (ix, ix + 1), for the views walked along y the pairs (iy, iy + 1), so every thread runs two
// phases with two different pairs.  The two pixels of a pair lie in neighbouring columns of
// the same cell row, so they share
//   - the element range (the projection of the 2 x 1 rectangle's four corners),
//   - the corner lines: one line load gives the offsets at the walk faces w, w + 1, w + 2,
//   - each element's NB sinogram values (one load serves both pixels' entries),
// while each keeps its own cell atoms and sums.  An element outside one pixel's footprint
// gets an exact zero weight there (both corner lines' atoms are 0 or both are 1).  The
// phases' and groups' sums meet in shared memory and are added in a fixed order
// (deterministic, no atomics).  The same cell atoms as the forward kernel give the same
// entries up to the FP32 rounding of the offsets.
// ---------------------------------------------------------------------------------------
constexpr int BTX = 16, BTY = 8, BG = 4;        // pixel tile 16 x 8, 4 view groups
constexpr int kBackPix = BTX * BTY;              // pixels per tile
constexpr int kBackThreads = kBackPix / 2 * BG;  // one pair per thread and group: 256

template <typename T, int NB>
__device__ __forceinline__ void back_pair_phase(const Geo& g, const T* __restrict__ ps, int phase, int grp, int w,
                                                int c, T RX0, T RX1, T RY0, T RY1, T (&acc1)[NB],
                                                T (&acc2)[NB]) {
    constexpr int VW = Vec<NB>::W, Q = Vec<NB>::Q;
    using L = typename LineOf<T>::type;
    const size_t plane = (size_t)g.nu * VW;
    for (int v = grp; v < g.n_views; v += BG) {
        if (g.axis_sigma[2 * v] != phase) continue;
        int k0, k1;
        if (!pixel_elements<T>(g, v, RX0, RX1, RY0, RY1, k0, k1)) continue;
        const int sigma = g.axis_sigma[2 * v + 1];
        L l;
        l.load(g, v, k0, w);
        T y0, y1, y2;
        l.offsets3(c, y0, y1, y2);
        T inv = inv_of<T>(g, v, k0);
        T prev1 = cell_atom(y0, y1, inv), prev2 = cell_atom(y1, y2, inv);
        const T* pv = ps + (size_t)v * Q * plane;
        for (int k = k0; k <= k1; ++k) {
            Cell<T, NB> cell;
            cell.load(pv + (size_t)k * VW, plane);   // issued before the weight arithmetic
            l.load(g, v, k + 1, w);
            l.offsets3(c, y0, y1, y2);
            inv = inv_of<T>(g, v, k + 1);
            const T cur1 = cell_atom(y0, y1, inv), cur2 = cell_atom(y1, y2, inv);
            const T wt1 = sigma > 0 ? cur1 - prev1 : prev1 - cur1;
            const T wt2 = sigma > 0 ? cur2 - prev2 : prev2 - cur2;
            prev1 = cur1;
            prev2 = cur2;
            cell.fma(acc1, wt1);
            cell.fma(acc2, wt2);
        }
    }
}

// shared memory: BG x NB x kBackPix sums (pixel innermost: conflict-free in both directions)
template <typename T, int NB> constexpr size_t back2d_smem() { return (size_t)BG * NB * kBackPix * sizeof(T); }

template <typename T, int NB>
__global__ void __launch_bounds__(kBackThreads) back2d_vox(Geo g, const T* __restrict__ ps, void* __restrict__ x,
                                                         int xdt, int B, int b_off, T scale, int accumulate) {
    extern __shared__ __align__(16) unsigned char back_smem[];
    T* part = reinterpret_cast<T*>(back_smem);   // [BG][NB][kBackPix]
    const int tid = threadIdx.x;
    const int grp = tid / (kBackPix / 2), t = tid % (kBackPix / 2);
    const int bx = blockIdx.x * BTX, by = blockIdx.y * BTY;
    T* mine = part + (size_t)grp * NB * kBackPix;
    const T A = GeoT<T>::a(g), Bh = GeoT<T>::b(g), XO = GeoT<T>::x0(g), YO = GeoT<T>::y0(g);
    T acc1[NB], acc2[NB];

    // phase 0: views walked along x, pairs (ix, ix + 1)
    {
        const int px = 2 * (t % (BTX / 2)), py = t / (BTX / 2);
        const int ix = bx + px, iy = by + py;
#pragma unroll
        for (int i = 0; i < NB; ++i) acc1[i] = acc2[i] = T(0);
        if (ix < g.nx && iy < g.ny) {
            const T X0 = XO + ix * A, Y0 = YO + iy * Bh;
            back_pair_phase<T, NB>(g, ps, 0, grp, ix, iy, X0, X0 + 2 * A, Y0, Y0 + Bh, acc1, acc2);
        }
        const int p0 = py * BTX + px;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            mine[i * kBackPix + p0] = acc1[i];
            mine[i * kBackPix + p0 + 1] = acc2[i];
        }
    }
    // phase 1: views walked along y, pairs (iy, iy + 1)
    const int qx = t % BTX, qy = 2 * (t / BTX);
    {
        const int ix = bx + qx, iy = by + qy;
#pragma unroll
        for (int i = 0; i < NB; ++i) acc1[i] = acc2[i] = T(0);
        if (ix < g.nx && iy < g.ny) {
            const T X0 = XO + ix * A, Y0 = YO + iy * Bh;
            back_pair_phase<T, NB>(g, ps, 1, grp, iy, ix, X0, X0 + A, Y0, Y0 + 2 * Bh, acc1, acc2);
        }
    }
    __syncthreads();   // every phase-0 sum is in shared memory
    {
        const int p0 = qy * BTX + qx;
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            mine[i * kBackPix + p0] += acc1[i];
            mine[i * kBackPix + p0 + BTX] += acc2[i];
        }
    }
    __syncthreads();
    for (int e = tid; e < NB * kBackPix; e += kBackThreads) {
        const int i = e / kBackPix, pix = e % kBackPix;
        const int ix = bx + pix % BTX, iy = by + pix / BTX, b = b_off + i;
        if (ix >= g.nx || iy >= g.ny || b >= B) continue;
        T s = part[e];
#pragma unroll
        for (int gg = 1; gg < BG; ++gg) s += part[(size_t)gg * NB * kBackPix + e];
        store_any<T>(x, ((size_t)b * g.ny + iy) * g.nx + ix, xdt, s * scale, accumulate != 0);
    }
}

// ---------------------------------------------------------------------------------------
// Forward projection, voxel-driven (the scatter form of the paper's Algorithm 1): a block of
// 16 x 16 pixels takes a set of views; per view its pixels add their entries W x into
// shared-memory partial sums of the elements the block reaches (found by a block-wide
// min / max of the pixels' element ranges), then every nonzero partial is added to the
// sinogram sums in global memory with one atomic.  The order of the FP additions is not
// fixed.
// ---------------------------------------------------------------------------------------
constexpr int kPE = 256;      // partial elements per block and view
constexpr int kVPB = 8;       // views per block

template <typename T>
__global__ void __launch_bounds__(256) fwd2d_vox(Geo g, const void* __restrict__ x, int xdt, int b,
                                                 T* __restrict__ pacc) {
    __shared__ T part[kPE];
    __shared__ int kr[2];
    const int ix = blockIdx.x * 16 + threadIdx.x, iy = blockIdx.y * 16 + threadIdx.y;
    const int tid = threadIdx.y * 16 + threadIdx.x;
    const bool inside = ix < g.nx && iy < g.ny;
    const T xv = inside ? load_any<T>(x, ((size_t)b * g.ny + iy) * g.nx + ix, xdt) : T(0);
    const T X0 = GeoT<T>::x0(g) + ix * GeoT<T>::a(g), X1 = X0 + GeoT<T>::a(g);
    const T Y0 = GeoT<T>::y0(g) + iy * GeoT<T>::b(g), Y1 = Y0 + GeoT<T>::b(g);
    using L = typename LineOf<T>::type;
    for (int i = tid; i < kPE; i += 256) part[i] = T(0);
    const int v_end = min((int)(blockIdx.z + 1) * kVPB, g.n_views);
    for (int v = blockIdx.z * kVPB; v < v_end; ++v) {
        int k0 = 0, k1 = -1;
        const bool has = inside && xv != T(0) && pixel_elements<T>(g, v, X0, X1, Y0, Y1, k0, k1);
        if (tid == 0) { kr[0] = 0x7fffffff; kr[1] = -1; }
        __syncthreads();
        if (has) { atomicMin(kr, k0); atomicMax(kr + 1, k1); }
        __syncthreads();
        const int kb = kr[0], ke = kr[1];
        if (ke >= kb) {                                   // block-uniform
            if (has) {
                const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
                const int w = axis == 0 ? ix : iy, c = axis == 0 ? iy : ix;
                L l;
                l.load(g, v, k0, w);
                T y0, y1;
                l.offsets(c, y0, y1);
                T prev = cell_atom(y0, y1, inv_of<T>(g, v, k0));
                for (int k = k0; k <= k1; ++k) {
                    l.load(g, v, k + 1, w);
                    l.offsets(c, y0, y1);
                    const T cur = cell_atom(y0, y1, inv_of<T>(g, v, k + 1));
                    const T wt = sigma > 0 ? cur - prev : prev - cur;
                    prev = cur;
                    if (wt != T(0)) {
                        if (k - kb < kPE) atomicAdd(part + (k - kb), wt * xv);
                        else atomicAdd(pacc + (size_t)v * g.nu + k, wt * xv);
                    }
                }
            }
            __syncthreads();
            const int span = min(ke - kb + 1, kPE);
            for (int i = tid; i < span; i += 256) {
                const T val = part[i];
                if (val != T(0)) {
                    atomicAdd(pacc + (size_t)v * g.nu + kb + i, val);
                    part[i] = T(0);
                }
            }
        }
        __syncthreads();
    }
}

// p = scale * w * sums (+ p with CSM_ACCUMULATE), in p's storage type.
template <typename T>
__global__ void finish_scatter_2d(Geo g, const T* __restrict__ pacc, void* __restrict__ p, int pdt, int b, T scale,
                                  int accumulate) {
    const size_t n = (size_t)g.n_views * g.nu;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        store_any<T>(p, (size_t)b * n + i, pdt, pacc[i] * scale * elem_weight<T>(g, i), accumulate != 0);
}

template <typename T>
static csm_status run_forward_vox(const csm_geom_s* gh, const void* x, void* p, int64_t batch, csm_dtype xdt,
                                  csm_dtype pdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    T* pacc = (T*)ws;
    const size_t n = (size_t)gh->n_views * gh->nu;
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1) : T(gh->a * gh->b);
    dim3 bb(16, 16), bg((gh->nx + 15) / 16, (gh->ny + 15) / 16, (gh->n_views + kVPB - 1) / kVPB);
    for (int64_t b = 0; b < batch; ++b) {
        cudaError_t e = cudaMemsetAsync(pacc, 0, n * sizeof(T), st);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
        note_launch(), fwd2d_vox<T><<<bg, bb, 0, st>>>(g, x, (int)xdt, (int)b, pacc);
        note_launch(), finish_scatter_2d<T><<<1216, 256, 0, st>>>(g, pacc, p, (int)pdt, (int)b, scale, (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status s = check_launch();
        if (s != CSM_OK) return s;
    }
    return CSM_OK;
}

// Number of (pixel, view, element) whose area exceeds 1e-6 of the pixel's.
__global__ void __launch_bounds__(256) nnz2d_kernel(Geo g, unsigned long long* counter) {
    const int ix = blockIdx.x * 16 + threadIdx.x, iy = blockIdx.y * 16 + threadIdx.y;
    unsigned long long cnt = 0;
    if (ix < g.nx && iy < g.ny) {
        const float X0 = g.x0 + ix * g.a, X1 = X0 + g.a, Y0 = g.y0 + iy * g.b, Y1 = Y0 + g.b;
        for (int v = 0; v < g.n_views; ++v) {
            int k0, k1;
            if (!pixel_elements<float>(g, v, X0, X1, Y0, Y1, k0, k1)) continue;
            const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
            const int w = axis == 0 ? ix : iy, c = axis == 0 ? iy : ix;
            LineF l;
            l.load(g, v, k0, w);
            float y0, y1;
            l.offsets(c, y0, y1);
            float prev = cell_below(y0, y1, inv_of<float>(g, v, k0));
            for (int k = k0; k <= k1; ++k) {
                l.load(g, v, k + 1, w);
                l.offsets(c, y0, y1);
                const float cur = cell_below(y0, y1, inv_of<float>(g, v, k + 1));
                const float wt = sigma > 0 ? cur - prev : prev - cur;
                prev = cur;
                cnt += wt > 1e-6f;   // above 1e-6 of the pixel area (FP32 resolves it)
            }
        }
    }
    // warp reduce then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x + 16 * threadIdx.y) % 32 == 0 && cnt) atomicAdd(counter, cnt);
}

// Sparse export: thread per pixel, its entries in view then element order (the back
// projection's cell atoms), written as rows of W^T (pixels) or of W (elements) as described by
// ExportArgs in csm_internal.cuh.
template <typename T>
__global__ void __launch_bounds__(256) export2d_kernel(Geo g, ExportArgs ea) {
    const int ix = blockIdx.x * 16 + threadIdx.x, iy = blockIdx.y * 16 + threadIdx.y;
    if (ix >= g.nx || iy >= g.ny) return;
    const long long pix = (long long)iy * g.nx + ix;
    const T thr = (T)ea.thr, scale = (T)ea.scale;
    const T X0 = GeoT<T>::x0(g) + ix * GeoT<T>::a(g), X1 = X0 + GeoT<T>::a(g);
    const T Y0 = GeoT<T>::y0(g) + iy * GeoT<T>::b(g), Y1 = Y0 + GeoT<T>::b(g);
    using L = typename LineOf<T>::type;
    long long n = 0;
    for (int v = 0; v < g.n_views; ++v) {
        int k0, k1;
        if (!pixel_elements<T>(g, v, X0, X1, Y0, Y1, k0, k1)) continue;
        const int axis = g.axis_sigma[2 * v], sigma = g.axis_sigma[2 * v + 1];
        const int w = axis == 0 ? ix : iy, c = axis == 0 ? iy : ix;
        L l;
        l.load(g, v, k0, w);
        T y0, y1;
        l.offsets(c, y0, y1);
        T prev = cell_atom(y0, y1, inv_of<T>(g, v, k0));
        for (int k = k0; k <= k1; ++k) {
            l.load(g, v, k + 1, w);
            l.offsets(c, y0, y1);
            const T cur = cell_atom(y0, y1, inv_of<T>(g, v, k + 1));
            const T wt = sigma > 0 ? cur - prev : prev - cur;
            prev = cur;
            if (!(fabs(wt) > thr)) continue;
            const long long row_e = (long long)v * g.nu + k;
            const T ew = elem_weight<T>(g, (size_t)row_e);
            switch (ea.mode) {
                case 0: ++n; break;
                case 1: {
                    const long long slot = ea.row_ptr[pix] + n++;
                    ea.col[slot] = (int)row_e;
                    if (ea.dbl) ((double*)ea.val)[slot] = (double)(wt * scale * ew);
                    else ((float*)ea.val)[slot] = (float)(wt * scale * ew);
                    break;
                }
                case 2: atomicAdd(ea.counts + row_e, 1ull); break;
                default: {
                    const long long slot = ea.row_ptr[row_e] + atomicAdd(ea.cursor + row_e, 1);
                    ea.col[slot] = (int)pix;
                    if (ea.dbl) ((double*)ea.val)[slot] = (double)(wt * scale * ew);
                    else ((float*)ea.val)[slot] = (float)(wt * scale * ew);
                    break;
                }
            }
        }
    }
    if (ea.mode == 0) ea.counts[pix] = (unsigned long long)n;
}

csm_status export_2d(const csm_geom_s* gh, const ExportArgs& a, cudaStream_t st) {
    const Geo g = make_geo(gh);
    dim3 bb(16, 16), bg((gh->nx + 15) / 16, (gh->ny + 15) / 16);
    if (a.dbl) note_launch(), export2d_kernel<double><<<bg, bb, 0, st>>>(g, a);
    else note_launch(), export2d_kernel<float><<<bg, bb, 0, st>>>(g, a);
    return check_launch();
}

// ---------------------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
static csm_status run_forward(const csm_geom_s* gh, const void* x, void* p, int64_t batch, csm_dtype xdt,
                              csm_dtype pdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    const size_t half = al256((size_t)gh->nx * gh->ny * NB * sizeof(T));
    T* xs0 = (T*)ws;
    T* xs1 = (T*)((char*)ws + half);
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1) : T(gh->a * gh->b);
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        dim3 pb(32, 8), pg((gh->nx + 31) / 32, (gh->ny + 31) / 32);
        note_launch(), prep_image_2d<T, NB><<<pg, pb, 0, st>>>(x, (int)xdt, (int)batch, (int)b0, gh->nx, gh->ny, xs0, xs1);
        // pairs of elements per thread when that still leaves 64 Ki threads
        const bool pair = (size_t)(gh->nu / 2) * gh->n_views >= 65536;
        dim3 fb(64), fg(pair ? (gh->nu + 31) / 32 : (gh->nu + 15) / 16, (gh->n_views + 3) / 4);
        if (pair)
            note_launch(), fwd2d_ray<T, NB, 2><<<fg, fb, 0, st>>>(g, xs0, xs1, p, (int)pdt, (int)batch, (int)b0, scale,
                                                  (flags & CSM_ACCUMULATE) ? 1 : 0);
        else
            note_launch(), fwd2d_ray<T, NB, 1><<<fg, fb, 0, st>>>(g, xs0, xs1, p, (int)pdt, (int)batch, (int)b0, scale,
                                                  (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status e = check_launch();
        if (e != CSM_OK) return e;
    }
    return CSM_OK;
}

template <typename T, int NB>
static csm_status run_back(const csm_geom_s* gh, const void* p, void* x, int64_t batch, csm_dtype pdt,
                           csm_dtype xdt, int flags, void* ws, cudaStream_t st) {
    const Geo g = make_geo(gh);
    T* ps = (T*)ws;
    const T scale = (flags & CSM_RELATIVE_WEIGHTS) ? T(1) : T(gh->a * gh->b);
    const size_t n = (size_t)gh->n_views * gh->nu;
    constexpr size_t smem = back2d_smem<T, NB>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(back2d_vox<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    }
    for (int64_t b0 = 0; b0 < batch; b0 += NB) {
        note_launch(), prep_sino_2d<T, NB><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, p, (int)pdt, (int)batch, (int)b0,
                                                                         gh->n_views, gh->nu, ps);
        dim3 bb(kBackThreads), bg((gh->nx + BTX - 1) / BTX, (gh->ny + BTY - 1) / BTY);
        note_launch(), back2d_vox<T, NB><<<bg, bb, smem, st>>>(g, ps, x, (int)xdt, (int)batch, (int)b0, scale,
                                               (flags & CSM_ACCUMULATE) ? 1 : 0);
        csm_status e = check_launch();
        if (e != CSM_OK) return e;
    }
    return CSM_OK;
}

template <typename T>
static csm_status fwd_nb(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt, csm_dtype pdt,
                         int flags, void* ws, cudaStream_t st) {
    switch (chunk_for(batch)) {
        case 16: return run_forward<T, 16>(g, x, p, batch, xdt, pdt, flags, ws, st);
        case 8: return run_forward<T, 8>(g, x, p, batch, xdt, pdt, flags, ws, st);
        case 4: return run_forward<T, 4>(g, x, p, batch, xdt, pdt, flags, ws, st);
        case 2: return run_forward<T, 2>(g, x, p, batch, xdt, pdt, flags, ws, st);
        default: return run_forward<T, 1>(g, x, p, batch, xdt, pdt, flags, ws, st);
    }
}

template <typename T>
static csm_status back_nb(const csm_geom_s* g, const void* p, void* x, int64_t batch, csm_dtype pdt, csm_dtype xdt,
                          int flags, void* ws, cudaStream_t st) {
    switch (chunk_for(batch)) {
        case 16: return run_back<T, 16>(g, p, x, batch, pdt, xdt, flags, ws, st);
        case 8: return run_back<T, 8>(g, p, x, batch, pdt, xdt, flags, ws, st);
        case 4: return run_back<T, 4>(g, p, x, batch, pdt, xdt, flags, ws, st);
        case 2: return run_back<T, 2>(g, p, x, batch, pdt, xdt, flags, ws, st);
        default: return run_back<T, 1>(g, p, x, batch, pdt, xdt, flags, ws, st);
    }
}

csm_status forward_2d(const csm_geom_s* g, const void* x, void* p, int64_t batch, csm_dtype xdt, csm_dtype pdt,
                      int flags, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    if (flags & CSM_VOXEL_DRIVEN) {
        if (!ws || ws_bytes < workspace_2d(g, 2, batch, dbl)) return CSM_EINVAL;
        if ((g->n_views + kVPB - 1) / kVPB > 65535) return CSM_EUNSUPPORTED;
        return dbl ? run_forward_vox<double>(g, x, p, batch, xdt, pdt, flags, ws, st)
                   : run_forward_vox<float>(g, x, p, batch, xdt, pdt, flags, ws, st);
    }
    if (!ws || ws_bytes < workspace_2d(g, 0, batch, dbl)) return CSM_EINVAL;
    if ((g->n_views + 3) / 4 > 65535) return CSM_EUNSUPPORTED;
    return dbl ? fwd_nb<double>(g, x, p, batch, xdt, pdt, flags, ws, st)
               : fwd_nb<float>(g, x, p, batch, xdt, pdt, flags, ws, st);
}

csm_status back_2d(const csm_geom_s* g, const void* p, void* x, int64_t batch, csm_dtype pdt, csm_dtype xdt,
                   int flags, void* ws, size_t ws_bytes, cudaStream_t st) {
    const bool dbl = xdt == CSM_F64 || pdt == CSM_F64;
    if (!ws || ws_bytes < workspace_2d(g, 1, batch, dbl)) return CSM_EINVAL;
    return dbl ? back_nb<double>(g, p, x, batch, pdt, xdt, flags, ws, st)
               : back_nb<float>(g, p, x, batch, pdt, xdt, flags, ws, st);
}

csm_status nnz_2d(const csm_geom_s* gh, int64_t* out, cudaStream_t st) {
    const Geo g = make_geo(gh);
    cudaError_t e = cudaMemsetAsync(gh->t.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    dim3 bb(16, 16), bg((gh->nx + 15) / 16, (gh->ny + 15) / 16);
    note_launch(), nnz2d_kernel<<<bg, bb, 0, st>>>(g, gh->t.counter);
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

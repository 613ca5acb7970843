// sparse.cu -- the system matrix W as an explicit sparse matrix (CSR), computed on the device
// from the same closed-form entries as the projectors, and the CSR kernels that row-action
// methods (SART) need: sparse matrix-vector products and row normalisation.
#include "csm_internal.cuh"

namespace csm {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;                              // per thread
constexpr int kScanBlock = kScanThreads * kScanItems;      // elements per block

static size_t al32(size_t n) { return (n + 31) & ~(size_t)31; }

// In-place exclusive prefix sums of d[0 .. n) per block of kScanBlock; block totals to sums.
__global__ void __launch_bounds__(kScanThreads) scan_block(long long* __restrict__ d, size_t n,
                                                          long long* __restrict__ sums) {
    __shared__ long long part[kScanThreads];
    const size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? d[base + i] : 0;
        const long long t = v[i];
        v[i] = run;
        run += t;
    }
    part[threadIdx.x] = run;
    __syncthreads();
    // exclusive scan of the thread totals (Hillis-Steele on kScanThreads values)
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const long long add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    const long long off = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) d[base + i] = v[i] + off;
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = part[kScanThreads - 1];
}

__global__ void scan_add(long long* __restrict__ d, size_t n, const long long* __restrict__ offs) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] += offs[i / kScanBlock];
}

static size_t scan_tmp_elems(size_t n) {
    size_t t = 0;
    while (n > 1) {
        n = (n + kScanBlock - 1) / kScanBlock;
        t += al32(n);
    }
    return t + 32;
}

static csm_status scan_exclusive(long long* d, size_t n, long long* tmp, cudaStream_t st) {
    const size_t nb = (n + kScanBlock - 1) / kScanBlock;
    note_launch(), scan_block<<<(unsigned)nb, kScanThreads, 0, st>>>(d, n, tmp);
    csm_status s = check_launch();
    if (s != CSM_OK || nb <= 1) return s;
    s = scan_exclusive(tmp, nb, tmp + al32(nb), st);
    if (s != CSM_OK) return s;
    note_launch(), scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, n, tmp);
    return check_launch();
}

// Rows of W come out of the fill pass in no particular order: sort each row by column.
template <typename T>
__global__ void sort_rows(size_t n_rows, const long long* __restrict__ row_ptr, int* __restrict__ col,
                          T* __restrict__ val) {
    const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const long long a = row_ptr[r], b = row_ptr[r + 1];
    for (long long i = a + 1; i < b; ++i) {
        const int c = col[i];
        const T v = val[i];
        long long j = i - 1;
        while (j >= a && col[j] > c) {
            col[j + 1] = col[j];
            val[j + 1] = val[j];
            --j;
        }
        col[j + 1] = c;
        val[j + 1] = v;
    }
}

// y[r] = alpha sum_j val[j] x[col[j]] + beta y[r], a warp per row, fixed summation order.
template <typename T>
__global__ void __launch_bounds__(256) csr_spmv_kernel(size_t n_rows, const long long* __restrict__ row_ptr,
                                                       const int* __restrict__ col, const T* __restrict__ val,
                                                       T alpha, const T* __restrict__ x, T beta, T* __restrict__ y) {
    const size_t r = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n_rows) return;
    const long long a = row_ptr[r], b = row_ptr[r + 1];
    T s = T(0);
    for (long long j = a + lane; j < b; j += 32) s += val[j] * __ldg(x + col[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[r] = alpha * s + (beta != T(0) ? beta * y[r] : T(0));
}

// Divides every row by its sum (rows summing to 0 are left as they are); row sums to `sums`.
template <typename T>
__global__ void __launch_bounds__(256) csr_normalize_kernel(size_t n_rows, const long long* __restrict__ row_ptr,
                                                            T* __restrict__ val, T* __restrict__ sums) {
    const size_t r = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n_rows) return;
    const long long a = row_ptr[r], b = row_ptr[r + 1];
    T s = T(0);
    for (long long j = a + lane; j < b; j += 32) s += val[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (s != T(0)) {
        const T inv = T(1) / s;
        for (long long j = a + lane; j < b; j += 32) val[j] *= inv;
    }
    if (sums && lane == 0) sums[r] = s;
}

static bool export_shape(const csm_geom_s* g, int flags, size_t* n_rows, size_t* n_cols) {
    const size_t nvox = (size_t)g->nx * g->ny * g->nz;
    const size_t nel = (size_t)g->n_views * g->nv * g->nu;
    *n_rows = (flags & CSM_EXPORT_TRANSPOSE) ? nvox : nel;
    *n_cols = (flags & CSM_EXPORT_TRANSPOSE) ? nel : nvox;
    return *n_rows < 2147483647ull && *n_cols < 2147483647ull;
}

static size_t export_ws(size_t n_rows, int flags) {
    size_t b = (al32(scan_tmp_elems(n_rows + 1)) * sizeof(long long) + 255) & ~(size_t)255;
    if (!(flags & CSM_EXPORT_TRANSPOSE)) b += ((n_rows * sizeof(int)) + 255) & ~(size_t)255;
    return b;
}

}  // namespace csm

using namespace csm;

extern "C" {

csm_status csm_export_workspace_bytes(csm_geom_t g, int flags, size_t* bytes) {
    if (!g || !bytes || (flags & ~(CSM_EXPORT_TRANSPOSE | CSM_RELATIVE_WEIGHTS))) return CSM_EINVAL;
    size_t nr, nc;
    if (!export_shape(g, flags, &nr, &nc)) return CSM_EUNSUPPORTED;
    *bytes = export_ws(nr, flags);
    return CSM_OK;
}

csm_status csm_export_csr(csm_geom_t g, int flags, csm_dtype val_dt, int64_t* row_ptr, int32_t* col_idx, void* val,
                          int64_t capacity, int64_t* nnz, void* workspace, size_t workspace_bytes, void* stream) {
    if (!g || !row_ptr || !nnz || (flags & ~(CSM_EXPORT_TRANSPOSE | CSM_RELATIVE_WEIGHTS))) return CSM_EINVAL;
    if (val_dt != CSM_F32 && val_dt != CSM_F64) return CSM_EINVAL;
    size_t nr, nc;
    if (!export_shape(g, flags, &nr, &nc)) return CSM_EUNSUPPORTED;
    if (!workspace || workspace_bytes < export_ws(nr, flags)) return CSM_EINVAL;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    if (dev != g->device) return CSM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const bool tr = (flags & CSM_EXPORT_TRANSPOSE) != 0;
    const bool dbl = val_dt == CSM_F64;
    const double meas = g->dim == 3 ? g->a * g->b * g->c : g->a * g->b;
    long long* tmp = (long long*)workspace;
    int* cursor = (int*)((char*)workspace + ((al32(scan_tmp_elems(nr + 1)) * sizeof(long long) + 255) & ~(size_t)255));
    ExportArgs a;
    // entries below the resolution of the arithmetic are not stored: 1e-6 (FP32) or 1e-12
    // (FP64) of the voxel measure; the 2D kernels work with fractions of the pixel
    a.thr = (dbl ? 1e-12 : 1e-6) * (g->dim == 3 ? meas : 1.0);
    a.scale = g->dim == 3 ? ((flags & CSM_RELATIVE_WEIGHTS) ? 1.0 / meas : 1.0)
                          : ((flags & CSM_RELATIVE_WEIGHTS) ? 1.0 : meas);
    a.counts = (unsigned long long*)row_ptr;
    a.row_ptr = (const long long*)row_ptr;
    a.cursor = cursor;
    a.col = col_idx;
    a.val = val;
    a.dbl = dbl ? 1 : 0;
    // count
    e = cudaMemsetAsync(row_ptr, 0, (nr + 1) * sizeof(int64_t), st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    a.mode = tr ? 0 : 2;
    csm_status s = g->dim == 3 ? export_3d(g, a, st) : export_2d(g, a, st);
    if (s != CSM_OK) return s;
    s = scan_exclusive((long long*)row_ptr, nr + 1, tmp, st);
    if (s != CSM_OK) return s;
    long long total = 0;
    e = cudaMemcpyAsync(&total, row_ptr + nr, sizeof total, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    *nnz = total;
    if (!col_idx || !val) return CSM_OK;
    if (capacity < total) return CSM_EINVAL;
    // fill
    if (!tr) {
        e = cudaMemsetAsync(cursor, 0, nr * sizeof(int), st);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    }
    a.mode = tr ? 1 : 3;
    s = g->dim == 3 ? export_3d(g, a, st) : export_2d(g, a, st);
    if (s != CSM_OK) return s;
    if (!tr) {
        const unsigned blocks = (unsigned)((nr + 127) / 128);
        if (dbl) note_launch(), sort_rows<double><<<blocks, 128, 0, st>>>(nr, (const long long*)row_ptr, col_idx, (double*)val);
        else note_launch(), sort_rows<float><<<blocks, 128, 0, st>>>(nr, (const long long*)row_ptr, col_idx, (float*)val);
        s = check_launch();
        if (s != CSM_OK) return s;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    return CSM_OK;
}

csm_status csm_csr_spmv(int64_t n_rows, const int64_t* row_ptr, const int32_t* col_idx, const void* val,
                        csm_dtype dt, double alpha, const void* x, double beta, void* y, void* stream) {
    if (n_rows < 0 || (n_rows > 0 && (!row_ptr || !col_idx || !val || !x || !y))) return CSM_EINVAL;
    if (dt != CSM_F32 && dt != CSM_F64) return CSM_EINVAL;
    if (n_rows == 0) return CSM_OK;
    const size_t threads = (size_t)n_rows * 32;
    if ((threads + 255) / 256 > 2147483647ull) return CSM_EUNSUPPORTED;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (dt == CSM_F64)
        note_launch(), csr_spmv_kernel<double><<<blocks, 256, 0, st>>>((size_t)n_rows, (const long long*)row_ptr, col_idx,
                                                         (const double*)val, alpha, (const double*)x, beta, (double*)y);
    else
        note_launch(), csr_spmv_kernel<float><<<blocks, 256, 0, st>>>((size_t)n_rows, (const long long*)row_ptr, col_idx,
                                                        (const float*)val, (float)alpha, (const float*)x, (float)beta,
                                                        (float*)y);
    return check_launch();
}

csm_status csm_csr_normalize_rows(int64_t n_rows, const int64_t* row_ptr, void* val, csm_dtype dt, void* row_sums,
                                  void* stream) {
    if (n_rows < 0 || (n_rows > 0 && (!row_ptr || !val))) return CSM_EINVAL;
    if (dt != CSM_F32 && dt != CSM_F64) return CSM_EINVAL;
    if (n_rows == 0) return CSM_OK;
    const size_t threads = (size_t)n_rows * 32;
    if ((threads + 255) / 256 > 2147483647ull) return CSM_EUNSUPPORTED;
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    cudaStream_t st = (cudaStream_t)stream;
    if (dt == CSM_F64)
        note_launch(), csr_normalize_kernel<double><<<blocks, 256, 0, st>>>((size_t)n_rows, (const long long*)row_ptr, (double*)val,
                                                              (double*)row_sums);
    else
        note_launch(), csr_normalize_kernel<float><<<blocks, 256, 0, st>>>((size_t)n_rows, (const long long*)row_ptr, (float*)val,
                                                             (float*)row_sums);
    return check_launch();
}

}  // extern "C"

// vecops.cu -- batched vector kernels for the reconstruction solvers (CG least squares,
// Nesterov's accelerated gradient on the Tikhonov objective, power iteration for ||W||;
// Section "Numerical Experiments", Eq. (exp_tikh)).  Scalars that the iterations derive from
// inner products stay in device memory, so a whole iteration can be captured in a CUDA graph.
#include <mutex>

#include "csm_internal.cuh"

namespace csm {

constexpr int kDotBlocks = 256;    // partial sums per batch item (first stage)
constexpr int kDotThreads = 256;

template <typename T>
__device__ __forceinline__ double ld(const void* p, size_t i, int dt) {
    switch (dt) {
        case CSM_F64: return ((const double*)p)[i];
        case CSM_BF16: return (double)__bfloat162float(((const __nv_bfloat16*)p)[i]);
        case CSM_F16: return (double)__half2float(((const __half*)p)[i]);
        default: return (double)((const float*)p)[i];
    }
}

// Stage 1: block (j, b) sums a[b, i] * b[b, i] over a grid-stride range of i in FP64.
__global__ void __launch_bounds__(kDotThreads) dot_partial(const void* __restrict__ a, const void* __restrict__ b,
                                                           int dt, int64_t n, double* __restrict__ part) {
    const int bb = blockIdx.y;
    const size_t off = (size_t)bb * n;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)kDotBlocks * kDotThreads)
        s += ld<double>(a, off + i, dt) * ld<double>(b, off + i, dt);
    __shared__ double red[kDotThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)bb * kDotBlocks + blockIdx.x] = red[0];
}

// Stage 2: one block per batch item adds its partials in a fixed order.
__global__ void __launch_bounds__(kDotThreads) dot_final(const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double red[kDotThreads];
    double s = 0.0;
    for (int j = threadIdx.x; j < kDotBlocks; j += kDotThreads) s += part[(size_t)blockIdx.x * kDotBlocks + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

__device__ __forceinline__ double coeff(double c, const double* num, const double* den, int b, bool den_sqrt) {
    double v = c;
    if (num) v *= num[b];
    if (den) {
        double d = den_sqrt ? sqrt(den[b]) : den[b];
        v = d != 0.0 ? v / d : 0.0;
    }
    return v;
}

// y[b, i] = A_b x[b, i] + B_b y[b, i]
__global__ void axpby_kernel(int64_t n, int64_t batch, int dt, double ac, const double* __restrict__ an,
                             const double* __restrict__ ad, const void* __restrict__ x, double bc,
                             const double* __restrict__ bn, const double* __restrict__ bd, void* __restrict__ y,
                             int den_sqrt) {
    const int b = blockIdx.y;
    const double A = coeff(ac, an, ad, b, den_sqrt & 1), B = coeff(bc, bn, bd, b, den_sqrt & 2);
    const size_t off = (size_t)b * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        switch (dt) {
            case CSM_F64: {
                double* q = (double*)y + off + i;
                const double xv = x ? ((const double*)x)[off + i] : 0.0;
                *q = A * xv + (B != 0.0 ? B * *q : 0.0);
                break;
            }
            case CSM_F32: {
                float* q = (float*)y + off + i;
                const float xv = x ? ((const float*)x)[off + i] : 0.0f;
                *q = (float)A * xv + (B != 0.0 ? (float)B * *q : 0.0f);
                break;
            }
            case CSM_BF16: {
                __nv_bfloat16* q = (__nv_bfloat16*)y + off + i;
                const float xv = x ? __bfloat162float(((const __nv_bfloat16*)x)[off + i]) : 0.0f;
                *q = __float2bfloat16_rn((float)A * xv + (B != 0.0 ? (float)B * __bfloat162float(*q) : 0.0f));
                break;
            }
            default: {
                __half* q = (__half*)y + off + i;
                const float xv = x ? __half2float(((const __half*)x)[off + i]) : 0.0f;
                *q = __float2half_rn((float)A * xv + (B != 0.0 ? (float)B * __half2float(*q) : 0.0f));
                break;
            }
        }
    }
}

// out[i] = num[i] / den[i], 0 where den[i] == 0
__global__ void ediv_kernel(int64_t n, int dt, const void* __restrict__ num, const void* __restrict__ den,
                            void* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (dt == CSM_F64) {
            const double d = ((const double*)den)[i];
            ((double*)out)[i] = d != 0.0 ? ((const double*)num)[i] / d : 0.0;
        } else {
            const float d = ((const float*)den)[i];
            ((float*)out)[i] = d != 0.0f ? ((const float*)num)[i] / d : 0.0f;
        }
    }
}

// Per-slot FISTA momentum for batches whose items are at different iterations: item b takes
// theta = table[k[b]] (0 beyond the table), writes 1 + theta and theta, and counts k[b] up.
__global__ void fista_coeffs_kernel(int64_t batch, const double* __restrict__ table, int n_table, int* __restrict__ k,
                                    double* __restrict__ one_plus, double* __restrict__ theta) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const int kk = k[b];
    const double th = (kk >= 0 && kk < n_table) ? table[kk] : 0.0;
    one_plus[b] = 1.0 + th;
    theta[b] = th;
    k[b] = kk + 1;
}

size_t dot_workspace_bytes(int64_t batch) { return (size_t)batch * kDotBlocks * sizeof(double); }

csm_status dot_launch(const void* a, const void* b, int64_t n, int64_t batch, csm_dtype dt, double* out,
                      double* part, cudaStream_t st) {
    dim3 g1(kDotBlocks, (unsigned)batch);
    note_launch(), dot_partial<<<g1, kDotThreads, 0, st>>>(a, b, (int)dt, n, part);
    note_launch(), dot_final<<<(unsigned)batch, kDotThreads, 0, st>>>(part, out);
    return check_launch();
}

// ---------------------------------------------------------------------------------------
// Allocation-free inner products.  Some callers cannot allocate device memory for the
// partial sums: code that has handed all device memory to a pool allocator, plug-ins that
// are given no allocator, and latency-critical loops where cudaMalloc / cudaFree, which may
// synchronise the device, are not acceptable.  For them the first-stage partials live in a
// fixed array in the library's own device memory, sized for kDotNoAllocMaxBatch items
// (128 KiB); every GPU that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------------------
constexpr int kDotNoAllocMaxBatch = 64;
static __device__ __align__(256) double g_dot_scratch[kDotNoAllocMaxBatch * kDotBlocks];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
struct ScratchSlot {
    unsigned long long ctx_id;   // CUDA context the address belongs to (0: none yet)
    double* addr;
};
static ScratchSlot g_scratch[kMaxDevices] = {};

// Identifier of the current CUDA context (unique within the process; 0 when no context is
// current yet), through the driver entry points that the runtime hands out, so the library
// needs no link to libcuda.  Called with g_scratch_mu held.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
static CtxGetCurrentFn g_ctx_get_current = nullptr;
static CtxGetIdFn g_ctx_get_id = nullptr;
static csm_status current_context_id(unsigned long long* id) {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) return CSM_ECUDA;
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    void* ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0) return CSM_ECUDA;
    *id = 0;
    if (ctx && g_ctx_get_id(ctx, id) != 0) return CSM_ECUDA;
    return CSM_OK;
}

// Device address of g_dot_scratch in the current device's context.  In host code the
// array's name denotes a host-side stand-in, so the address is looked up with the device
// current: the first time the device is used, and again whenever its context has changed
// (after cudaDeviceReset the old address would point into released memory); it is cached
// per device together with the context's identifier.
static csm_status dot_scratch_address(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    if (dev < 0 || dev >= kMaxDevices) return CSM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long ctx = 0;
    csm_status s = current_context_id(&ctx);
    if (s != CSM_OK) return s;
    ScratchSlot& slot = g_scratch[dev];
    if (!slot.addr || ctx == 0 || slot.ctx_id != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_scratch);   // makes the device's context current
        if (e != cudaSuccess || !p) {
            set_cuda_error(e);
            return CSM_ECUDA;
        }
        s = current_context_id(&ctx);
        if (s != CSM_OK) return s;
        slot.addr = (double*)p;
        slot.ctx_id = ctx;
    }
    *out = slot.addr;
    return CSM_OK;
}

}  // namespace csm

using namespace csm;

extern "C" {

csm_status csm_dot_workspace_bytes(int64_t batch, size_t* bytes) {
    if (batch <= 0 || batch > 65535 || !bytes) return CSM_EINVAL;
    *bytes = dot_workspace_bytes(batch);
    return CSM_OK;
}

csm_status csm_dot(const void* a, const void* b, int64_t n, int64_t batch, csm_dtype dt, double* out,
                   void* workspace, size_t workspace_bytes, void* stream) {
    if (!a || !b || !out || n < 0 || batch <= 0 || batch > 65535) return CSM_EINVAL;
    if (dt != CSM_F32 && dt != CSM_F64 && dt != CSM_BF16 && dt != CSM_F16) return CSM_EINVAL;
    if (!workspace || workspace_bytes < dot_workspace_bytes(batch)) return CSM_EINVAL;
    return dot_launch(a, b, n, batch, dt, out, (double*)workspace, (cudaStream_t)stream);
}

csm_status csm_axpby(int64_t n, int64_t batch, csm_dtype dt, double a_c, const double* a_num, const double* a_den,
                     const void* x, double b_c, const double* b_num, const double* b_den, void* y, int flags,
                     void* stream) {
    if (!y || n < 0 || batch <= 0 || batch > 65535) return CSM_EINVAL;
    if (dt != CSM_F32 && dt != CSM_F64 && dt != CSM_BF16 && dt != CSM_F16) return CSM_EINVAL;
    if (n == 0) return CSM_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;   // 8 blocks of 256 per SM on 152 SMs, grid-stride beyond
    dim3 grid((unsigned)blocks, (unsigned)batch);
    note_launch(), axpby_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(n, batch, (int)dt, a_c, a_num, a_den, x, b_c, b_num, b_den,
                                                        y, flags);
    return check_launch();
}

csm_status csm_fista_coeffs(int64_t batch, const double* theta_table, int n_table, int32_t* k, double* one_plus_theta,
                            double* theta, void* stream) {
    if (batch < 0 || n_table < 0 || (batch > 0 && (!k || !one_plus_theta || !theta || (n_table > 0 && !theta_table))))
        return CSM_EINVAL;
    if (batch == 0) return CSM_OK;
    note_launch(), fista_coeffs_kernel<<<(unsigned)((batch + 127) / 128), 128, 0, (cudaStream_t)stream>>>(batch, theta_table, n_table,
                                                                                          k, one_plus_theta, theta);
    return check_launch();
}

csm_status csm_ediv(int64_t n, csm_dtype dt, const void* num, const void* den, void* out, void* stream) {
    if (n < 0 || (n > 0 && (!num || !den || !out))) return CSM_EINVAL;
    if (dt != CSM_F32 && dt != CSM_F64) return CSM_EINVAL;
    if (n == 0) return CSM_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    note_launch(), ediv_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, (int)dt, num, den, out);
    return check_launch();
}

csm_status csm_dot_noalloc(const void* a, const void* c, int64_t n, int64_t batch, csm_dtype dt, double* out,
                           void* stream) {
    if (!a || !c || !out || n < 0 || batch <= 0) return CSM_EINVAL;
    if (batch > kDotNoAllocMaxBatch) return CSM_EINVAL;   // beyond the fixed scratch array
    if (dt != CSM_F32 && dt != CSM_F64 && dt != CSM_BF16 && dt != CSM_F16) return CSM_EINVAL;
    double* part = nullptr;
    csm_status s = dot_scratch_address(&part);
    if (s != CSM_OK) return s;
    // every partial slot the second stage reads is written by the first: nothing to clear
    return dot_launch(a, c, n, batch, dt, out, part, (cudaStream_t)stream);
}

}  // extern "C"

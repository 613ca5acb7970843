// peak.cu -- FP32 / FP64 fused multiply-add throughput of the current GPU, measured by a
// kernel of independent FMA chains.  The projectors are bound by the issue rate of plain
// arithmetic (no tensor cores: the entries are geometry, not a dense contraction), so their
// roofline is the FMA rate measured here on the same device and at the same clocks.
#include "csm_internal.cuh"

namespace csm {

constexpr int kPeakChains = 8;     // independent accumulators per thread (hide FMA latency)
constexpr int kPeakThreads = 256;
__device__ double g_peak_sink;   // written only by a result the chains cannot reach

// Every thread runs kPeakChains independent chains a <- a * m + c for `iters` rounds (2 flops
// per FMA).  m and c come from the host, so the compiler cannot fold the chains; the result
// is written only when it equals a value the chains cannot reach, so the work stays live.
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chains(int64_t iters, T m, T c) {
    T a[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) a[i] = fma(a[i], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += a[i];
    if (s == T(-12345.678)) g_peak_sink = (double)s;
}

}  // namespace csm

using namespace csm;

extern "C" csm_status csm_fma_rate(csm_dtype dt, int64_t iters, int blocks_per_sm, int launches, double* flops,
                                   double* seconds, void* stream) {
    if (!flops || !seconds || iters <= 0 || blocks_per_sm <= 0 || launches <= 0) return CSM_EINVAL;
    if (dt != CSM_F32 && dt != CSM_F64) return CSM_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        if (e0) cudaEventDestroy(e0);
        return CSM_ECUDA;
    }
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    e = cudaEventRecord(e0, st);
    for (int l = 0; l < launches && e == cudaSuccess; ++l) {
        if (dt == CSM_F32)
            note_launch(), fma_chains<float><<<grid, kPeakThreads, 0, st>>>(iters, 1.0000001f, -1e-7f);
        else
            note_launch(), fma_chains<double><<<grid, kPeakThreads, 0, st>>>(iters, 1.0000000001, -1e-10);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) { set_cuda_error(e); return CSM_ECUDA; }
    *flops = 2.0 * 16.0 * kPeakChains * (double)iters * (double)grid * kPeakThreads * (double)launches;
    *seconds = 1e-3 * (double)ms;
    return CSM_OK;
}

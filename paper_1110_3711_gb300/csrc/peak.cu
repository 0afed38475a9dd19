// Measurement helper (not part of the method): the rate of independent fused
// multiply-adds, the arithmetic roofline that bounds PI (float32 in the split
// form, float64 in the FP64 form).  Every thread runs 8 independent FMA chains
// (more than the FMA latency in cycles divided by the issue interval), 2048
// threads per SM; the chains converge to c / (1 - b) > 0, so the guarded store
// of their sum never happens but keeps them live.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaChains = 8;
constexpr int kFmaUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kFmaThreads) k_fma_rate(int iters, T b, T c, T *out)
{
    T a[kFmaChains];
#pragma unroll
    for (int u = 0; u < kFmaChains; ++u) a[u] = (T)(threadIdx.x + u) * (T)1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < kFmaUnroll; ++r) {
#pragma unroll
            for (int u = 0; u < kFmaChains; ++u) a[u] = fma(a[u], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int u = 0; u < kFmaChains; ++u) s += a[u];
    if (s == (T)-1) out[0] = s;
}

template <typename T>
int fma_rate(void *scratch, cudaStream_t st, int iters, double *flops)
{
    int dev = 0, sms = 0;
    if (check_cuda(cudaGetDevice(&dev))) return SPH_ERR_CUDA;
    if (check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
        return SPH_ERR_CUDA;
    const int blocks = sms * (2048 / kFmaThreads);
    cudaEvent_t e0, e1;
    if (check_cuda(cudaEventCreate(&e0))) return SPH_ERR_CUDA;
    if (check_cuda(cudaEventCreate(&e1))) {
        cudaEventDestroy(e0);
        return SPH_ERR_CUDA;
    }
    int rc = SPH_OK;
    T *out = (T *)scratch;
    k_fma_rate<T><<<blocks, kFmaThreads, 0, st>>>(iters / 4 + 1, (T)0.999, (T)1e-4, out);
    cudaEventRecord(e0, st);
    k_fma_rate<T><<<blocks, kFmaThreads, 0, st>>>(iters, (T)0.999, (T)1e-4, out);
    cudaEventRecord(e1, st);
    rc = check_cuda(cudaGetLastError());
    if (!rc) rc = check_cuda(cudaEventSynchronize(e1));
    float ms = 0.0f;
    if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double fmas = (double)blocks * kFmaThreads * (double)iters * kFmaUnroll * kFmaChains;
    *flops = ms > 0.0f ? 2.0 * fmas / (1e-3 * (double)ms) : 0.0;
    return SPH_OK;
}

}  // namespace

}  // namespace sph

extern "C" int sph_fma_rate(int precision, void *scratch, void *stream, double *flops)
{
    if (!scratch || !flops) return SPH_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // about 10 ms per timed launch at the nominal rates (float32 about 40e12
    // FMA/s, float64 about 0.6e12 FMA/s on 152 SMs)
    if (precision == SPH_FP32_SPLIT) return sph::fma_rate<float>(scratch, st, 8192, flops);
    if (precision == SPH_FP64) return sph::fma_rate<double>(scratch, st, 128, flops);
    return SPH_ERR_INVALID_ARG;
}

// Measured FMA issue rates of the device (a diagnostic for the FP64 and FP32
// arithmetic rooflines; no counterpart in the paper).  Each thread runs eight
// independent FMA chains so that the pipe, not the FMA latency, limits the
// rate; the grid fills every SM several times over.
#include <cuda_runtime.h>

#include "tl.h"
#include "tl_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(const T *in, T *out, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = in[c] + (T)threadIdx.x;
    for (int i = 0; i < kIters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345e-30) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

template <typename T>
int time_chains(int sms, cudaStream_t st, double *rate)
{
    T *buf = nullptr;
    if (cudaMalloc(&buf, 4096 * sizeof(T)) != cudaSuccess) return tl::set_error(TL_ENOMEM, "probe buffer", "");
    cudaMemsetAsync(buf, 0, 4096 * sizeof(T), st);
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chains<T><<<blocks, 256, 0, st>>>(buf, buf + 2048, (T)0.999, (T)1e-3);  // warm-up
    cudaEventRecord(e0, st);
    fma_chains<T><<<blocks, 256, 0, st>>>(buf, buf + 2048, (T)0.999, (T)1e-3);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) return tl::set_error(TL_ECUDA, "probe: ", cudaGetErrorString(e));
    *rate = (double)blocks * 256.0 * kChains * kIters / (ms * 1e-3);
    return TL_OK;
}

}  // namespace

extern "C" int tl_probe_fma_rates(double *fp64_fma_per_s, double *fp32_fma_per_s, void *cuda_stream)
{
    tl::set_error(TL_OK, "", "");
    if (!fp64_fma_per_s || !fp32_fma_per_s) return tl::set_error(TL_EINVAL, "NULL argument", "");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return tl::set_error(TL_ECUDA, "device query: ", cudaGetErrorString(e));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc = time_chains<double>(sms, st, fp64_fma_per_s);
    if (rc) return rc;
    return time_chains<float>(sms, st, fp32_fma_per_s);
}

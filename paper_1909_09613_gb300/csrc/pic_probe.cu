// Arithmetic-peak probe for the roofline denominators (not part of the PIC path): every thread
// runs a long chain of independent FMAs on registers; the rate over all SMs is the measured
// FMA peak of the device in the precision asked for.
#include "pic.h"

#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T *out, int iters, T a, T b)
{
    T r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = r[i] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += r[i];
    if (s == (T)12345.678) out[0] = s;  // keeps the chain live
}

template <typename T>
int run_probe(double *tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PIC_ECUDA;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return PIC_ENOMEM;
    const int blocks = sms * 8, threads = 256;
    const int iters = sizeof(T) == 8 ? 2048 : 32768;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma<T><<<blocks, threads>>>(out, iters / 8, (T)0.999999, (T)1e-7);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        k_fma<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return PIC_ECUDA;
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return PIC_OK;
}

}  // namespace

extern "C" int pic_probe_fma_peak(int kind, double *tflops)
{
    if (!tflops) return PIC_EINVAL;
    if (kind == 0) return run_probe<double>(tflops);
    if (kind == 1) return run_probe<float>(tflops);
    return PIC_EINVAL;
}

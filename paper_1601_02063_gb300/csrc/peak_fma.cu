// FMA-chain microbenchmark of the FP32 and FP64 vector pipes.  The measured rate is the
// denominator of the integrator's compute roofline (the device reports no FP64/FP32 peak).
// Each thread runs 8 independent dependency chains so that FMA latency is hidden.
#include <cuda_runtime.h>

#include "odx_internal.h"

namespace odx {

template <typename T>
__global__ void __launch_bounds__(256) fma_chain_kernel(T *out, int iters, T b, T c)
{
    T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = x0 * b + c;
            x1 = x1 * b + c;
            x2 = x2 * b + c;
            x3 = x3 * b + c;
            x4 = x4 * b + c;
            x5 = x5 * b + c;
            x6 = x6 * b + c;
            x7 = x7 * b + c;
        }
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true
}

cudaError_t run_fma_peak(int32_t precision, int32_t num_sms, double *flops)
{
    const int threads = 256, blocks = num_sms * 8;
    const int iters = (precision == ODX_FP64) ? 64 : 4096;
    void *out = nullptr;
    cudaError_t err = cudaMalloc(&out, (size_t)threads * blocks * sizeof(double));
    if (err != cudaSuccess) return err;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        if (precision == ODX_FP64)
            fma_chain_kernel<double><<<blocks, threads>>>((double *)out, iters, 0.999999, 1e-7);
        else
            fma_chain_kernel<float><<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
    }
    err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double fl = 2.0 * 8.0 * 16.0 * (double)iters * threads * blocks;
    *flops = fl / (best * 1e-3);
    return err;
}

}  // namespace odx

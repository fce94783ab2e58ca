// peak.cu -- FMA-chain throughput probe for the FP32 / FP64 pipe roofline denominators.
//
// Every thread runs 8 independent dependent-FMA chains (enough to hide the pipe
// latency), the grid fills every SM several times over, and the result is folded into
// one store so the compiler keeps the arithmetic.  2 flops per FMA.
#include <cuda_runtime.h>

#include "css_internal.h"

namespace {

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;

template <class T>
__global__ void k_fma(T a, T b, T* out) {
    T x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int it = 0; it < ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s == (T)-1.2345) out[0] = s;   // practically never true; keeps the chains live
}

}  // namespace

namespace cssi {

cudaError_t measure_fma_peak(int precision, int sm_count, cudaStream_t st, double* flops) {
    const int threads = 256, blocks = sm_count * 16;
    void* out = nullptr;
    cudaError_t e = cudaMalloc(&out, 16);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        if (precision == CSS_FP64) k_fma<double><<<blocks, threads, 0, st>>>(0.999999, 1e-7, (double*)out);
        else k_fma<float><<<blocks, threads, 0, st>>>(0.999999f, 1e-7f, (float*)out);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    *flops = 2.0 * CHAINS * (double)ITERS * threads * (double)blocks / (best * 1e-3);
    return cudaGetLastError();
}

}  // namespace cssi

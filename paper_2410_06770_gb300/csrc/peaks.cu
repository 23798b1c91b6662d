// peaks.cu -- microbenchmarks of the arithmetic pipes and HBM the xGETT
// kernels run on, so roofline fractions can use measured denominators:
// FP64 FMA (DFMA), FP64 tensor MMA (mma.sync f64, DMMA) in three shapes,
// FP32 FMA, and an HBM copy.  Each kernel keeps enough independent chains in
// flight to saturate its pipe; the result is the best of several timed runs.
#include <cuda_runtime.h>

#include <algorithm>

#include "gett_bench.h"

namespace {

constexpr int CHAINS = 8;

template <class T>
__global__ void fma_peak_kernel(T *out, int iters, T x, T y)
{
    T acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = acc[c] * x + y;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c];
    if (s == (T)-1.2345) out[threadIdx.x] = s;  // keep the chains alive
}

// mma.sync f64, shape selected by SHAPE: 0 = m8n8k4, 1 = m16n8k4, 2 = m16n8k8
template <int SHAPE>
__global__ void dmma_peak_kernel(double *out, int iters)
{
    double a[4], b[2], c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 1.0 + 1e-9 * (threadIdx.x + i);
    b[0] = 0.5;
    b[1] = 0.25;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[j][i] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if constexpr (SHAPE == 0) {
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                             : "+d"(c[j][0]), "+d"(c[j][1])
                             : "d"(a[0]), "d"(b[0]));
            } else if constexpr (SHAPE == 1) {
                asm volatile(
                    "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                    "{%0,%1,%2,%3};"
                    : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                    : "d"(a[0]), "d"(a[1]), "d"(b[0]));
            } else {
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                    "{%8,%9}, {%0,%1,%2,%3};"
                    : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                    : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
            }
        }
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) s += c[j][i];
    if (s == -1.2345) out[threadIdx.x] = s;
}

__global__ void copy_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <class F>
float best_ms(F launch, int reps)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();  // warm-up
    launch();
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

extern "C" int gett_measure_peaks(gett_peaks *out, size_t copy_bytes)
{
    if (!out) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double *scratch = nullptr;
    if (cudaMalloc(&scratch, 4096 * sizeof(double)) != cudaSuccess) return -6;
    const int threads = 256, blocks = sms * 8;
    const int iters = 4096;
    {
        float ms = best_ms([&] { fma_peak_kernel<double><<<blocks, threads>>>(scratch, iters, 0.999, 1e-3); }, 5);
        out->dfma_tflops = 2.0 * CHAINS * iters * (double)threads * blocks / (ms * 1e-3) / 1e12;
    }
    {
        float ms = best_ms([&] {
            fma_peak_kernel<float><<<blocks, threads>>>((float *)scratch, iters * 4, 0.999f, 1e-3f);
        }, 5);
        out->ffma_tflops = 2.0 * CHAINS * iters * 4.0 * threads * blocks / (ms * 1e-3) / 1e12;
    }
    const int dit = 1024;
    const double warps = (double)blocks * threads / 32;
    {
        float ms = best_ms([&] { dmma_peak_kernel<0><<<blocks, threads>>>(scratch, dit); }, 5);
        out->dmma_m8n8k4_tflops = 4.0 * dit * warps * (2.0 * 8 * 8 * 4) / (ms * 1e-3) / 1e12;
    }
    {
        float ms = best_ms([&] { dmma_peak_kernel<1><<<blocks, threads>>>(scratch, dit); }, 5);
        out->dmma_m16n8k4_tflops = 4.0 * dit * warps * (2.0 * 16 * 8 * 4) / (ms * 1e-3) / 1e12;
    }
    {
        float ms = best_ms([&] { dmma_peak_kernel<2><<<blocks, threads>>>(scratch, dit); }, 5);
        out->dmma_m16n8k8_tflops = 4.0 * dit * warps * (2.0 * 16 * 8 * 8) / (ms * 1e-3) / 1e12;
    }
    cudaFree(scratch);
    out->copy_gbs = 0;
    if (copy_bytes >= (1 << 20)) {
        void *a = nullptr, *b = nullptr;
        if (cudaMalloc(&a, copy_bytes) == cudaSuccess && cudaMalloc(&b, copy_bytes) == cudaSuccess) {
            cudaMemset(a, 0, copy_bytes);
            size_t n = copy_bytes / sizeof(float4);
            float ms = best_ms([&] {
                copy_kernel<<<sms * 16, 512>>>((const float4 *)a, (float4 *)b, n);
            }, 10);
            out->copy_gbs = 2.0 * n * sizeof(float4) / (ms * 1e-3) / 1e9;
        }
        if (a) cudaFree(a);
        if (b) cudaFree(b);
    }
    out->sms = sms;
    cudaError_t e = cudaDeviceSynchronize();
    return e == cudaSuccess ? 0 : -4;
}

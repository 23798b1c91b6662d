// peaks.cu -- microbenchmarks of the arithmetic pipes and HBM the xGETT
// kernels run on, so roofline fractions can use measured denominators:
// FP64 FMA (DFMA), FP64 tensor MMA (mma.sync f64, DMMA) in three shapes,
// FP32 FMA, INT8 tensor MMA (mma.sync s8, the only INT8 tensor instruction
// sm_103a offers), the 5th-generation tensor core (tcgen05.mma) with bf16
// and with e4m3 operands, and an HBM copy.  Each kernel keeps enough
// independent work in flight to saturate its pipe; the result is the best of
// several timed runs.  These numbers decide which slice type the split
// precision form uses.
#include <cuda_runtime.h>

#include <algorithm>

#include "gett_bench.h"
#include "tc_common.cuh"

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

// FP64 pipes side by side: even warps run the DMMA (m8n8k4) chains, odd warps
// the DFMA chains, to see whether the two FP64 paths add up on this GPU.
__global__ void fp64_mixed_kernel(double *out, int dmma_iters, int fma_iters)
{
    const int warp = threadIdx.x >> 5;
    double s = 0;
    if ((warp & 1) == 0) {
        double a = 1.0 + 1e-9 * threadIdx.x, b = 0.5, c[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j][0] = c[j][1] = 0.0;
        for (int it = 0; it < dmma_iters; ++it) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                             : "+d"(c[j][0]), "+d"(c[j][1])
                             : "d"(a), "d"(b));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) s += c[j][0] + c[j][1];
    } else {
        double acc[CHAINS];
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) acc[c] = (double)(threadIdx.x + c);
        for (int i = 0; i < fma_iters; ++i) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) acc[c] = acc[c] * 0.999 + 1e-3;
        }
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) s += acc[c];
    }
    if (s == -1.2345) out[threadIdx.x] = s;
}

// mma.sync s8 -> s32, m16n8k32: four independent accumulators a warp
__global__ void imma_peak_kernel(int *out, int iters)
{
    uint32_t a[4], b[2];
    int c[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = 0x01010101u * (uint32_t)(threadIdx.x + i);
    b[0] = 0x01020304u;
    b[1] = 0x04030201u;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[j][i] = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(c[j][0]), "+r"(c[j][1]), "+r"(c[j][2]), "+r"(c[j][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) s += c[j][i];
    if (s == 12345) out[threadIdx.x] = s;
}

// tcgen05.mma issue rate: one CTA per SM, one thread issues `iters` x 4
// MMAs of 128 x 256 (x 16 bf16 or x 32 e4m3 along K) from two zeroed
// 128-byte-swizzled shared tiles into one TMEM accumulator, commits and waits
// (bounded) for completion.  KIND 0: kind::f16 with bf16 operands; KIND 1:
// kind::f8f6f4 with e4m3 operands.  Both read 32 bytes of every operand row
// per instruction.
constexpr int TCP_M = 128, TCP_N = 256;
constexpr int TCP_A_BYTES = TCP_M * 128, TCP_B_BYTES = TCP_N * 128;
constexpr int TCP_SMEM = TCP_A_BYTES + TCP_B_BYTES + 1024;

template <int KIND>
__global__ void __launch_bounds__(128, 1) tc_peak_kernel(int iters, int *err)
{
    extern __shared__ uint8_t tcp_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tcp_raw) + 1023) & ~uintptr_t(1023));
    for (int i = threadIdx.x; i < (TCP_A_BYTES + TCP_B_BYTES) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(base)[i] = make_uint4(0, 0, 0, 0);
    // the tensor core reads shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        gett::tc::mbar_init(&bar, 1);
        gett::tc::fence_barrier_init();
    }
    if (threadIdx.x < 32) gett::tc::tmem_alloc(&slot, TCP_N);
    __syncthreads();
    gett::tc::tc_fence_after();
    const uint32_t tmem = slot;
    if (threadIdx.x == 0) {
        const uint64_t ad = gett::tc::smem_desc_sw128(gett::tc::smem_u32(base));
        const uint64_t bd = gett::tc::smem_desc_sw128(gett::tc::smem_u32(base + TCP_A_BYTES));
        constexpr uint32_t idesc = KIND == 0 ? gett::tc::idesc_bf16_f32(TCP_M, TCP_N)
                                             : ((1u << 4) | ((uint32_t)(TCP_N >> 3) << 17) |
                                                ((uint32_t)(TCP_M >> 4) << 24));  // D f32, A, B e4m3 (0)
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t acc = (it > 0 || j > 0) ? 1u : 0u;
                if constexpr (KIND == 0) {
                    gett::tc::umma_bf16(tmem, ad + (uint64_t)(j * 2), bd + (uint64_t)(j * 2), idesc, acc);
                } else {
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad + (uint64_t)(j * 2)), "l"(bd + (uint64_t)(j * 2)), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
        }
        gett::tc::umma_commit(&bar);
        if (!gett::tc::mbar_wait(&bar, 0, err, gett::tc::ERR_WAIT_ACC_FULL)) gett::tc::mbar_drain(&bar, 0);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        gett::tc::tc_fence_after();
        gett::tc::tmem_dealloc(tmem, TCP_N);
    }
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
    {
        // the two FP64 paths together: half the warps each; the DMMA half's
        // flops are scaled by the measured rate ratio so that, if the paths
        // are independent, both halves take the same time.  A warp's DFMA
        // work is 32 * 2 * CHAINS * fit flops, its DMMA work 4 * dmi * 512
        const double ratio = out->dfma_tflops > 0 ? out->dmma_m8n8k4_tflops / out->dfma_tflops : 1.0;
        const int fit = iters;
        const int dmi = (int)std::max(1.0, fit * ratio * (32.0 * 2.0 * CHAINS) / (4.0 * 2.0 * 8 * 8 * 4));
        float ms = best_ms([&] { fp64_mixed_kernel<<<blocks, threads>>>(scratch, dmi, fit); }, 5);
        const double half_warps = warps / 2.0;
        const double flops = half_warps * 4.0 * dmi * (2.0 * 8 * 8 * 4) + half_warps * 32.0 * 2.0 * CHAINS * fit;
        out->fp64_mixed_tflops = flops / (ms * 1e-3) / 1e12;
    }
    {
        float ms = best_ms([&] { imma_peak_kernel<<<blocks, threads>>>((int *)scratch, dit); }, 5);
        out->imma_s8_tops = 4.0 * dit * warps * (2.0 * 16 * 8 * 32) / (ms * 1e-3) / 1e12;
    }
    {
        // tcgen05: one CTA per SM; a wait that gave up leaves a nonzero word
        int *err = reinterpret_cast<int *>(scratch) + 2048;
        cudaMemset(err, 0, sizeof(int));
        const int tit = 4096;
        cudaFuncSetAttribute(tc_peak_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM);
        cudaFuncSetAttribute(tc_peak_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM);
        const double per_cta = 4.0 * tit * 2.0 * TCP_M * TCP_N;
        float ms = best_ms([&] { tc_peak_kernel<0><<<sms, 128, TCP_SMEM>>>(tit, err); }, 5);
        out->tc_bf16_tflops = per_cta * 16 * sms / (ms * 1e-3) / 1e12;
        ms = best_ms([&] { tc_peak_kernel<1><<<sms, 128, TCP_SMEM>>>(tit, err); }, 5);
        out->tc_e4m3_tflops = per_cta * 32 * sms / (ms * 1e-3) / 1e12;
        int word = 0;
        cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost);
        if (word) out->tc_bf16_tflops = out->tc_e4m3_tflops = 0;  // a wait gave up: no figure
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

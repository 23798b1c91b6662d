/*
 * gett_bench.h -- measurement entry points of the xGETT library (no
 * counterpart in the thesis, which reports no performance).
 */
#ifndef GETT_BENCH_H
#define GETT_BENCH_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Throughput of the arithmetic pipes and HBM on the current device,
 * best of several runs timed with CUDA events.  TFLOP/s count a fused
 * multiply-add as 2 flops; copy_gbs counts bytes read + written. */
typedef struct gett_peaks {
    double dfma_tflops;          /* FP64 FMA on CUDA cores                 */
    double dmma_m8n8k4_tflops;   /* mma.sync f64 shapes (FP64 tensor path) */
    double dmma_m16n8k4_tflops;
    double dmma_m16n8k8_tflops;
    double ffma_tflops;          /* FP32 FMA on CUDA cores                 */
    double copy_gbs;             /* device-to-device copy, read + write    */
    int sms;
    double imma_s8_tops;         /* mma.sync s8 -> s32 (INT8 tensor path), */
                                 /* tera-operations/s                      */
    double tc_bf16_tflops;       /* tcgen05.mma kind::f16, bf16 operands,  */
                                 /* 128 x 256 tiles, one CTA per SM        */
    double tc_e4m3_tflops;       /* tcgen05.mma kind::f8f6f4, e4m3 operands */
    double fp64_mixed_tflops;    /* DMMA and DFMA warps side by side (do    */
                                 /* the two FP64 paths add up?)             */
} gett_peaks;

/* Runs the microbenchmarks on the current device (synchronous; allocates
 * 2*copy_bytes of device memory for the copy, skipped when copy_bytes is
 * below 1 MiB).  Returns 0, or a negative gett_status on a CUDA error. */
int gett_measure_peaks(gett_peaks *out, size_t copy_bytes);

#ifdef __cplusplus
}
#endif

#endif /* GETT_BENCH_H */

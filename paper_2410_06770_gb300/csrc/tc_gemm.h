// tc_gemm.h -- host interface of the tensor-core GEMM on packed bf16 data.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace gett {

enum TcMode : int { TC_MODE_F32 = 0, TC_MODE_MOD = 1 };

// Moduli of the split-precision DGETT: pairwise coprime odd numbers <= 255,
// largest first, so symmetric residues fit in [-127, 127] (exact in bf16).
constexpr int OZ_MAX_L = 20;
constexpr int kOzModuli[OZ_MAX_L] = {255, 253, 251, 247, 241, 239, 233, 229, 227, 223,
                                     217, 211, 199, 197, 193, 191, 181, 179, 173, 167};
// K per exact fp32 chunk: 1024 * 127^2 + 2^8 < 2^24.
constexpr int OZ_CHUNK_K = 1024;

struct TcGemmParams {
    int64_t M, N, K;     // D_z is M x N, sum over K
    int tiles_m, tiles_n, tiles_z;  // filled by the launcher (tiles_z = Z)
    int kc_tiles;        // MODE_MOD: 64-wide K tiles per exact fp32 chunk
    int *err;            // device error word (bounded waits)
    // MODE_MOD: slice z is reduced modulo kOzModuli[z]
    int8_t *R;            // [Z][N][M] symmetric residues
    // MODE_F32: C[z * c_slice + rowC[m] + colC[n]] += D_z[m, n]
    float *C;
    const int64_t *rowC, *colC;
    int64_t c_slice;
    // MODE_F32 epilogue: SCALE_ACC adds into C, SCALE_AX writes alpha * D,
    // SCALE_AXPBY writes alpha * D + beta * C (real alpha, beta)
    int smode;
    float alpha, beta;
    // MODE_F32, optional: rows of A / columns of B that hold a value the
    // bf16 pieces cannot carry (Inf, NaN, or beyond the bf16 range); the
    // epilogue leaves their outputs to the non-finite fix-up kernel
    const uint32_t *flagA, *flagB;
    // Operands staged in place (Z == 1): row pitch in elements of the
    // caller's K-major bf16 operand, and its contracted extent (the tensor
    // map's inner dimension; TMA fills k >= K with zeros).  0: packed
    // operand with pitch tc_ld(K) and inner extent K.
    int64_t a_ld, b_ld, a_kdim, b_kdim;
};

// Row pitch (elements) of a packed operand with K columns: multiple of 8
// bf16 so every row starts on a 16-byte boundary (TMA requirement).
int64_t tc_ld(int64_t K);

// Ap: [Z][M][tc_ld(K)] bf16, Bp: [Z][N][tc_ld(K)] bf16, both 16-byte aligned.
cudaError_t launch_tc_gemm(int mode, const void *Ap, const void *Bp, int64_t Z, const TcGemmParams &p,
                           cudaStream_t s);

// Failure-detection check (see gett_check_wait_timeout).
cudaError_t launch_wait_timeout_probe(int *err, long long limit_cycles, cudaStream_t s);

}  // namespace gett

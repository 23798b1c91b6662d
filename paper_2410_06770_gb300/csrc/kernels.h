// kernels.h -- host-side launchers of the xGETT kernel families.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gett {

// ---- dense tiled GETT on CUDA cores (k_dense.cu) ----
constexpr int DENSE_NUM_CONFIGS = 3;
bool dense_config_valid(DType t, int cfg);
void dense_tile_shape(int cfg, int *bm, int *bn, int *bk);
size_t dense_workspace_bytes(const Plan &p, DType t, int cfg, int split_k);
int dense_effective_split(const Plan &p, int cfg, int split_k);
// CTAs of the configuration resident on one SM (occupancy query, cached).
int dense_ctas_per_sm(DType t, int cfg);
cudaError_t launch_dense(const Plan &p, DType t, const void *A, const void *B, void *C, int cfg,
                         int split_k, void *ws, cudaStream_t s);

// Offset tables of the three classes: rowA/rowC [M], colB/colC [N], kA/kB [K].
cudaError_t launch_build_tables(const Plan &p, int64_t *rowA, int64_t *rowC, int64_t *colB, int64_t *colC,
                                int64_t *kA, int64_t *kB, cudaStream_t s);

// ---- streaming kernels (k_stream.cu) ----
// OUTER: no contracted mode of extent > 1 (K == 1), or a short sum.
cudaError_t launch_outer(const Plan &p, DType t, const void *A, const void *B, void *C, int num_sms,
                         cudaStream_t s);
// OUTER also covers short sums: K <= OUTER_MAX_SUM.
constexpr int OUTER_MAX_SUM = 8;
// SKINNY: one free class of at most 8 indices, K > 1.
bool skinny_applicable(const Plan &p);
size_t skinny_workspace_bytes(const Plan &p, DType t, int num_sms);
cudaError_t launch_skinny(const Plan &p, DType t, const void *A, const void *B, void *C, int num_sms, void *ws,
                          cudaStream_t s);
// REDUCE: few outputs (M*N small), long sums; deterministic two-pass.
size_t reduce_workspace_bytes(const Plan &p, DType t, int num_sms);
cudaError_t launch_reduce(const Plan &p, DType t, const void *A, const void *B, void *C, int num_sms,
                          void *ws, cudaStream_t s);

// C <- beta * C over the planned output (the scaled form with alpha == 0 or
// an empty sum); uses p.sc's beta.
cudaError_t launch_scale_c(const Plan &p, DType t, void *C, int num_sms, cudaStream_t s);

// ---- transpose and the reduction's unit operand (k_aux.cu) ----
// Transpose: the planned contraction with no contracted and no B-free modes
// (C[rowC[m]] <- A[rowA[m]] under p.sc).  Tiled through shared memory when A's
// and C's fastest modes differ.
bool transpose_tiled(const Plan &p);
cudaError_t launch_transpose(const Plan &p, DType t, const void *A, void *C, int num_sms, cudaStream_t s);
// Device address of one element of value 1 of type t (the B of a reduction).
cudaError_t unit_operand(DType t, const void **out);
// Conjugated copy of a complex operand in planned order: dst[r + R k] =
// conj(src[rowT[r] + kT[k]]) for r < R, k < K (c and z only).
cudaError_t launch_conj_pack(DType t, const void *src, const int64_t *rowT, const int64_t *kT, int64_t R, int64_t K,
                             void *dst, int num_sms, cudaStream_t s);

// ---- tensor-core forms ----
// s / bf16 inputs: packed bf16 pieces + one tcgen05 GEMM (k_tcpack.cu)
int tc_split_blocks(int algo);
// Which operands of a bf16 tensor-core call TMA reads in place (bit 0 A,
// bit 1 B; the others are packed first).
int tc_in_place_mask(const Plan &p, DType t, int algo, const void *A, const void *B);
size_t tc_split_workspace_bytes(const Plan &p, int algo);
cudaError_t launch_tc_split(const Plan &p, DType t, int algo, const void *A, const void *B, void *C, void *ws,
                            int num_sms, int *err, cudaStream_t s);
// d: split-precision modular form (k_ozaki.cu)
int ozaki_moduli_for(int64_t K, int want);
int ozaki_bits_for(int64_t K, int L);
size_t ozaki_workspace_bytes(const Plan &p, int L);
cudaError_t launch_ozaki(const Plan &p, int L, const void *A, const void *B, void *C, void *ws, int num_sms,
                         int *err, cudaStream_t s);
// z: the same on the real form of the complex contraction (2M rows, 2K sums)
size_t ozaki_complex_workspace_bytes(const Plan &p, int L);
cudaError_t launch_ozaki_complex(const Plan &p, int L, const void *A, const void *B, void *C, void *ws,
                                 int num_sms, int *err, cudaStream_t s);

}  // namespace gett

// batch_common.cuh -- descriptors shared by the batched launch's kernels
// (k_batch.cu: gathered tiles and short sums; k_batch_pack.cu: packed
// operands, packed tiles and the skinny warp kernel).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "common.cuh"

namespace gett {

constexpr int BT = 256;  // threads per CTA of the tile kernels
constexpr int NSHAPE = 4;
struct BCfg {
    int bm, bn, bk, tm, tn;
};
// Tile shapes (all 256 threads, at most 4x4 accumulators a thread).
constexpr BCfg kB[NSHAPE] = {{64, 64, 16, 4, 4}, {32, 64, 16, 2, 4}, {32, 32, 16, 2, 2}, {64, 32, 16, 4, 2}};

// How a problem of the batch is computed.  A configuration id names a
// method and, for the tile methods, a shape:
//   0..3  GATHER: tiles read the strided operands through the class offset
//         tables (the planner's logical mode fusion only);
//   4..7  PACK: the operands are first copied into tile-blocked dense
//         matrices (each class's modes physically fused into one contiguous
//         index, [K][bm] blocks of A, [K][bn] of B), then the tiles stream
//         them with bulk copies;
//   8     SKINNY: one free class of at most 8 indices; warp items, lanes
//         along the long free class or along the sum;
//   9     TC (bf16 operands only): packed into 128 x 64 bf16 tiles laid out
//         as the tensor core reads them, multiplied by tcgen05 (128 x 128
//         output tiles, fp32 accumulators in TMEM).
enum BatchMethod : int { BM_GATHER = 0, BM_PACK = 1, BM_SKINNY = 2, BM_TC = 3 };
constexpr int NCFG = 2 * NSHAPE + 2;
constexpr int CFG_SKINNY = 2 * NSHAPE;
constexpr int CFG_TC = 2 * NSHAPE + 1;
constexpr int SKINNY_MAX_SHORT = 8;
// tensor-core method: output tile, K tile (one 128-byte swizzled row of bf16)
constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;
constexpr int TC_TILE_ELEMS = 128 * TC_BK;  // one packed 128 x 64 tile

__host__ __device__ constexpr int cfg_method(int cfg)
{
    return cfg == CFG_TC ? BM_TC : (cfg == CFG_SKINNY ? BM_SKINNY : cfg / NSHAPE);
}
__host__ __device__ constexpr int cfg_shape(int cfg) { return cfg >= CFG_SKINNY ? 0 : cfg % NSHAPE; }

struct BatchProb {
    const void *A;
    const void *B;
    float *C;
    int64_t M, N, K;
    int64_t tab;  // offset of this problem's tables in the table buffer
    int tiles_m, tiles_n;
    int cfg, dtype;   // cfg: the configuration id above; dtype 0 f32, 1 bf16
    int shape;        // tile shape (kB index) of the tile methods
    int bm, bn;       // its tile extents
    int method;
    int a_m_fast, b_n_fast, c_m_fast;
    int splits;       // K slices (1: the result is added into C directly)
    int64_t kps;      // K per slice (multiple of the tile's BK)
    float *partial;   // splits > 1: [splits][M*N] partial results
    int tpi;          // tiles per work item (short sums: several; else 1)
    // PACK: tile-blocked operands, block t of A at pA + t * Kp * bm
    const float *pA, *pB;
    int64_t Kp;       // K rounded up to the tile's BK
    // SKINNY: the long free class is A's (M) when long_is_a, else B's (N);
    // lanes_k: lanes run along the sum (L, S <= 4), else along the long class
    int long_is_a, lanes_k;
    int64_t kslice;   // contracted indices per warp item
    // TC: packed bf16 tiles, tile (t, kt) of A at tA + (t * nkt + kt) *
    // TC_TILE_ELEMS (B the same with tB), nkt = K tiles of 64
    const uint16_t *tA, *tB;
    int nkt;
};

// Offset tables of problem pr: rowA, rowC [M], colB, colC [N], kA, kB [K].
struct BatchTables {
    const int64_t *rowA, *rowC, *colB, *colC, *kA, *kB;
};
__device__ __forceinline__ BatchTables batch_tables(const BatchProb &pr, const int64_t *tables)
{
    const int64_t *t = tables + pr.tab;
    BatchTables r;
    r.rowA = t;
    r.rowC = t + pr.M;
    r.colB = t + 2 * pr.M;
    r.colC = t + 2 * pr.M + pr.N;
    r.kA = t + 2 * pr.M + 2 * pr.N;
    r.kB = t + 2 * pr.M + 2 * pr.N + pr.K;
    return r;
}

// Work items of the packing kernel: problem, operand (0 A, 1 B), block of
// bm (bn) rows, chunk of 64 contracted indices.
struct PackItem {
    int prob, operand, block, chunk;
};
// Warp items of the skinny kernel: problem, K slice, first long index.
struct SkinnyItem {
    int prob, slice;
    int64_t l0;
};

// Launchers of k_batch_pack.cu.  `err`: the device error word of bounded
// waits (the packed tile kernel's bulk-copy waits).
void launch_batch_pack(int blocks, cudaStream_t s, const BatchProb *probs, const PackItem *items, int64_t n,
                       int64_t wrap, const int64_t *tables);
void launch_batch_packed_tiles(int cps, int ctas, cudaStream_t s, const BatchProb *probs, const uint2 *work,
                               int64_t nwork, int64_t wrap, const int64_t *tables, int *err);
void launch_batch_skinny(int blocks, cudaStream_t s, const BatchProb *probs, const SkinnyItem *items, int64_t n,
                         int64_t wrap, const int64_t *tables);
// Resident CTAs per SM of the packed tile kernel (shared-memory bound).
int batch_packed_ctas_per_sm();

// Tensor-core method (k_batch_tc.cu).  Packing items: problem, operand,
// 128-row block, K tile of 64 (one packed tile).  Tile kernel: one CTA per
// SM, items (problem, 128 x 128 output tile) dealt statically.
struct TcPackItem {
    int prob, operand, block, ktile;
};
void launch_batch_tc_pack(int blocks, cudaStream_t s, const BatchProb *probs, const TcPackItem *items, int64_t n,
                          int64_t wrap, const int64_t *tables);
cudaError_t launch_batch_tc_tiles(int ctas, cudaStream_t s, const BatchProb *probs, const uint2 *work, int64_t nwork,
                                  int64_t wrap, const int64_t *tables, int *err);

}  // namespace gett

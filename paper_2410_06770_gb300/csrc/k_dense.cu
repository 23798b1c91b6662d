// k_dense.cu -- tiled GETT on CUDA cores for every element type.
//
// The planner reduces any contraction to C[m,n] += sum_k A[m,k] B[k,n] over
// multi-mode index sets M, N, K (Sec. 2.2 / Alg. 1 computed tile by tile
// instead of element by element).  A setup kernel turns each class's mode
// list into offset tables (the element offset of every flat m, n, k in the
// tensors that carry that class), so the tiled kernel can gather a BM x BK
// tile of A and a BK x BN tile of B through arbitrary increments -- padded,
// negative, zero or non-unit -- and scatter the BM x BN result into C through
// INCC/PERM.
//
// Staging: each thread prefetches its share of the next K tile into
// registers while the current tile is multiplied from shared memory (double
// buffered).  Threads walk the tile along whichever index has the smaller
// increment so global loads coalesce.  The epilogue maps lanes along the
// index with C's smaller increment so the read-modify-write of C coalesces.
//
// Split-K: with S > 1 slices each CTA sums one slice of K into a workspace
// tile and a second kernel adds the S partial tiles into C in slice order,
// so results do not depend on scheduling.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "dense_tile.cuh"
#include "kernels.h"

namespace gett {

namespace {

__global__ void build_tables_kernel(ModeList L, int64_t count, int64_t *t0, int64_t *t1)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a, b;
        decode2(L, i, a, b);
        t0[i] = a;
        t1[i] = b;
    }
}

struct DenseParams {
    const void *A;
    const void *B;
    void *C;
    const int64_t *rowA, *rowC, *colB, *colC, *kA, *kB;
    int64_t M, N, K;
    int64_t k_per_split;
    int tiles_m, tiles_n;
    int a_m_fast, b_n_fast, c_m_fast;
    void *partial;  // split-K partial tiles (Acc), null when S == 1
    Scale sc;       // how the sum meets C
};

template <class T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
dense_kernel(DenseParams p)
{
    using Acc = typename Tr<T>::Acc;
    __shared__ Acc sA[2 * BK * BM];
    __shared__ Acc sB[2 * BK * BN];
    __shared__ int64_t sRowA[BM];
    __shared__ int64_t sColB[BN];
    // column tiles fastest: the CTAs that share one row block of A run
    // together, so A is fetched from DRAM about once
    const int tile = blockIdx.x;
    const int tile_n = tile % p.tiles_n;
    const int tile_m = tile / p.tiles_n;
    const int split = blockIdx.y;
    TileArgs a;
    a.A = p.A;
    a.B = p.B;
    a.C = p.C;
    a.rowA = p.rowA; a.rowC = p.rowC; a.colB = p.colB; a.colC = p.colC; a.kA = p.kA; a.kB = p.kB;
    a.M = p.M;
    a.N = p.N;
    a.m0 = (int64_t)tile_m * BM;
    a.n0 = (int64_t)tile_n * BN;
    a.kbeg = split * p.k_per_split;
    a.kend = min(p.K, a.kbeg + p.k_per_split);
    a.a_m_fast = p.a_m_fast;
    a.b_n_fast = p.b_n_fast;
    a.c_m_fast = p.c_m_fast;
    a.partial = p.partial ? static_cast<Acc *>(p.partial) + (int64_t)split * p.M * p.N : nullptr;
    a.sc = p.sc;
    dense_tile<T, BM, BN, BK, TM, TN>(a, sA, sB, sRowA, sColB);
}

template <class T>
__global__ void splitk_reduce_kernel(DenseParams p, int S)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    const Acc *P = static_cast<const Acc *>(p.partial);
    Out *C = static_cast<Out *>(p.C);
    const int64_t MN = p.M * p.N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MN;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m, n;
        if (p.c_m_fast) { m = i % p.M; n = i / p.M; }
        else { n = i % p.N; m = i / p.N; }
        Acc s = P[i];
        for (int t = 1; t < S; ++t) s = R::add(s, P[(int64_t)t * MN + i]);
        epi_store<R>(C + p.rowC[m] + p.colC[n], s, p.sc);
    }
}

struct TileCfg {
    int bm, bn, bk;
};
constexpr TileCfg kCfg[DENSE_NUM_CONFIGS] = {{128, 128, 8}, {64, 64, 8}, {32, 32, 16}};

template <class T>
bool cfg_allowed(int cfg)
{
    // complex double at 128x128 would need 256 accumulator registers a thread
    return !(sizeof(T) == 16 && cfg == 0);
}

template <class T>
cudaError_t launch_typed(const DenseParams &p, int cfg, int S, cudaStream_t s)
{
    dim3 grid(p.tiles_m * p.tiles_n, S);
    switch (cfg) {
    case 0:
        if constexpr (sizeof(T) != 16) {
            dense_kernel<T, 128, 128, 8, 8, 8><<<grid, 256, 0, s>>>(p);
            break;
        }
        return cudaErrorInvalidValue;
    case 1:
        dense_kernel<T, 64, 64, 8, 4, 4><<<grid, 256, 0, s>>>(p);
        break;
    case 2:
        dense_kernel<T, 32, 32, 16, 2, 2><<<grid, 256, 0, s>>>(p);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || S == 1) return e;
    int64_t MN = p.M * p.N;
    int blocks = (int)std::min<int64_t>((MN + 255) / 256, 4096);
    splitk_reduce_kernel<T><<<blocks, 256, 0, s>>>(p, S);
    return cudaGetLastError();
}

size_t acc_size(DType t)
{
    switch (t) {
    case DT_F32: case DT_BF16: return 4;
    case DT_F64: return 8;
    case DT_C32: return 8;
    case DT_C64: return 16;
    }
    return 0;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

cudaError_t launch_build_tables(const Plan &pl, int64_t *rowA, int64_t *rowC, int64_t *colB, int64_t *colC,
                                int64_t *kA, int64_t *kB, cudaStream_t s)
{
    auto build = [&](const ModeList &L, int64_t count, int64_t *t0, int64_t *t1) {
        int blocks = (int)std::min<int64_t>((count + 255) / 256, 2048);
        if (blocks < 1) blocks = 1;
        build_tables_kernel<<<blocks, 256, 0, s>>>(L, count, t0, t1);
    };
    build(pl.m, pl.M, rowA, rowC);
    build(pl.n, pl.N, colB, colC);
    build(pl.k, pl.K, kA, kB);
    return cudaGetLastError();
}

bool dense_config_valid(DType t, int cfg)
{
    if (cfg < 0 || cfg >= DENSE_NUM_CONFIGS) return false;
    return !(t == DT_C64 && cfg == 0);
}

namespace {

template <class T>
int occupancy_of(int cfg)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (cfg) {
    case 0:
        if constexpr (sizeof(T) != 16)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dense_kernel<T, 128, 128, 8, 8, 8>, 256, 0);
        break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dense_kernel<T, 64, 64, 8, 4, 4>, 256, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dense_kernel<T, 32, 32, 16, 2, 2>, 256, 0); break;
    default: break;
    }
    return e == cudaSuccess && n > 0 ? n : 1;
}

}  // namespace

int dense_ctas_per_sm(DType t, int cfg)
{
    // resident CTAs of each (type, configuration), asked once
    static int cache[5][DENSE_NUM_CONFIGS] = {};
    static std::mutex mu;
    if (!dense_config_valid(t, cfg)) return 1;
    std::lock_guard<std::mutex> lk(mu);
    int &c = cache[t][cfg];
    if (c == 0) {
        switch (t) {
        case DT_F32: c = occupancy_of<float>(cfg); break;
        case DT_F64: c = occupancy_of<double>(cfg); break;
        case DT_C32: c = occupancy_of<cf>(cfg); break;
        case DT_C64: c = occupancy_of<zd>(cfg); break;
        case DT_BF16: c = occupancy_of<uint16_t>(cfg); break;
        }
    }
    return c;
}

void dense_tile_shape(int cfg, int *bm, int *bn, int *bk)
{
    *bm = kCfg[cfg].bm;
    *bn = kCfg[cfg].bn;
    *bk = kCfg[cfg].bk;
}

size_t dense_workspace_bytes(const Plan &p, DType t, int cfg, int split_k)
{
    size_t tables = align256(sizeof(int64_t) * 2 * (size_t)(p.M + p.N + p.K));
    size_t partial = split_k > 1 ? align256(acc_size(t) * (size_t)split_k * p.M * p.N) : 0;
    (void)cfg;
    return tables + partial;
}

cudaError_t launch_dense(const Plan &pl, DType t, const void *A, const void *B, void *C, int cfg,
                         int split_k, void *ws, cudaStream_t s)
{
    if (!dense_config_valid(t, cfg)) return cudaErrorInvalidValue;
    int64_t *tab = static_cast<int64_t *>(ws);
    int64_t *rowA = tab, *rowC = rowA + pl.M, *colB = rowC + pl.M, *colC = colB + pl.N;
    int64_t *kA = colC + pl.N, *kB = kA + pl.K;
    cudaError_t te = launch_build_tables(pl, rowA, rowC, colB, colC, kA, kB, s);
    if (te != cudaSuccess) return te;

    const TileCfg c = kCfg[cfg];
    DenseParams p{};
    size_t esz = dtype_size(t);
    p.A = static_cast<const char *>(A) + pl.offA * (int64_t)esz;
    p.B = static_cast<const char *>(B) + pl.offB * (int64_t)esz;
    size_t csz = (t == DT_BF16) ? 4 : esz;
    p.C = static_cast<char *>(C) + pl.offC * (int64_t)csz;
    p.rowA = rowA; p.rowC = rowC; p.colB = colB; p.colC = colC; p.kA = kA; p.kB = kB;
    p.M = pl.M; p.N = pl.N; p.K = pl.K;
    int S = split_k < 1 ? 1 : split_k;
    int64_t kps = (pl.K + S - 1) / S;
    kps = (kps + c.bk - 1) / c.bk * c.bk;
    S = (int)((pl.K + kps - 1) / kps);
    p.k_per_split = kps;
    p.tiles_m = (int)((pl.M + c.bm - 1) / c.bm);
    p.tiles_n = (int)((pl.N + c.bn - 1) / c.bn);
    // coalescing choices: the index with the smaller increment runs fastest
    auto first = [](const ModeList &L, const int64_t *s) { return L.n ? (s[0] < 0 ? -s[0] : s[0]) : 0; };
    int64_t am = first(pl.m, pl.m.s0), ak = first(pl.k, pl.k.s0);
    int64_t bn = first(pl.n, pl.n.s0), bk = first(pl.k, pl.k.s1);
    int64_t cm = first(pl.m, pl.m.s1), cn = first(pl.n, pl.n.s1);
    p.a_m_fast = (am != 0 && (ak == 0 || am <= ak)) ? 1 : 0;
    p.b_n_fast = (bn != 0 && (bk == 0 || bn <= bk)) ? 1 : 0;
    p.c_m_fast = (cm != 0 && (cn == 0 || cm <= cn)) ? 1 : 0;
    p.sc = pl.sc;
    p.partial = S > 1 ? static_cast<char *>(ws) + align256(sizeof(int64_t) * 2 * (size_t)(pl.M + pl.N + pl.K))
                      : nullptr;
    if ((int64_t)p.tiles_m * p.tiles_n > (int64_t)INT32_MAX || S > 65535) return cudaErrorInvalidValue;
    switch (t) {
    case DT_F32: return launch_typed<float>(p, cfg, S, s);
    case DT_F64: return launch_typed<double>(p, cfg, S, s);
    case DT_C32: return launch_typed<cf>(p, cfg, S, s);
    case DT_C64: return launch_typed<zd>(p, cfg, S, s);
    case DT_BF16: return launch_typed<uint16_t>(p, cfg, S, s);
    }
    return cudaErrorInvalidValue;
}

int dense_effective_split(const Plan &pl, int cfg, int split_k)
{
    const TileCfg c = kCfg[cfg];
    int S = split_k < 1 ? 1 : split_k;
    int64_t kps = (pl.K + S - 1) / S;
    kps = (kps + c.bk - 1) / c.bk * c.bk;
    return (int)((pl.K + kps - 1) / kps);
}

}  // namespace gett

// k_tcpack.cu -- the tensor-core forms of SGETT (fp32 split into bf16
// pieces) and of the bf16-input contraction: gather the strided operands into
// packed K-major bf16 matrices, then one tcgen05 GEMM whose epilogue adds the
// fp32 result into C through INCC/PERM.
//
// Split forms.  x = hi + mid + lo with hi = bf16(x), mid = bf16(x - hi),
// lo = bf16(x - hi - mid).  BF16X3 keeps two pieces and the products
// hi*hi + hi*mid + mid*hi; BF16X6 keeps three pieces and the six products
// whose piece ranks sum to at most 2.  The products are laid side by side
// along K (A' = [hi | hi | mid], B' = [hi | mid | hi] for BF16X3), so one
// GEMM over K' = 3K (6K) sums all of them into the same fp32 accumulator.
//
// Packing reads a 32 x 64 (row x k) tile through shared memory along
// whichever index has the unit increment and writes packed rows along k.
//
// Values the pieces cannot carry -- Inf, NaN, and finite fp32 values beyond
// the bf16 range, whose hi piece would round to Inf -- are packed as zeros and
// their row of A (column of B) is marked.  The GEMM epilogue skips every
// output in a marked row or column, and a fix-up kernel computes those outputs
// by the definition (the fp32 products summed in k order, as the plain form
// does), so Inf and NaN reach C as Alg. 1's arithmetic makes them.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace gett {

namespace {

constexpr int TR = 64, TKP = 64, PT = 256;

__device__ __forceinline__ uint16_t f2bf_bits(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t *>(&b);
}

__device__ __forceinline__ float bf_bits2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

template <class T>
__device__ __forceinline__ float load_as_float(const T *p);
template <>
__device__ __forceinline__ float load_as_float<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_as_float<uint16_t>(const uint16_t *p) { return bf_bits2f(__ldg(p)); }

// pieces[j] for block j of the packed K axis: 0 = hi, 1 = mid, 2 = lo
struct PieceMap {
    int nblocks;
    int piece[8];
};

// Writes, for every row, nblocks blocks of Kb (>= K, multiple of 64) packed
// values; block b holds piece pm.piece[b] of the row's K values followed by
// zeros up to Kb, so every 64-wide K tile belongs to exactly one block.
//
// A CTA takes 64 x 64 tiles: the tile's row and K offsets (one round trip),
// then its 16 loads a thread, all issued before the first store to shared
// memory, along whichever index has the smaller increment; then each thread
// splits 8 consecutive k of one row into pieces and writes every block's
// 8 bf16 values as one 16-byte store (the packed pitch, Kb and the tile
// start are multiples of 8 elements, the buffer 256-byte aligned).
template <class T>
__global__ void __launch_bounds__(PT, 4) pack_pieces_kernel(const T *__restrict__ src, const int64_t *__restrict__ rowT,
                                                        const int64_t *__restrict__ kT, int64_t rows, int64_t K,
                                                        int64_t Kb, int row_fast, PieceMap pm,
                                                        uint16_t *__restrict__ out, int64_t ld,
                                                        uint32_t *__restrict__ flags, uint32_t *__restrict__ any)
{
    static_assert(TR == 64 && TKP == 64 && PT == 256, "index split below");
    __shared__ float tile[TR][TKP + 1];
    __shared__ int64_t srow[TR];
    __shared__ int64_t sk[TKP];
    const int64_t tiles_k = (Kb + TKP - 1) / TKP;
    const int64_t ntiles = ((rows + TR - 1) / TR) * tiles_k;
    const int tid = threadIdx.x;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = (t / tiles_k) * TR, k0 = (t % tiles_k) * TKP;
        __syncthreads();
        if (tid < TR) srow[tid] = r0 + tid < rows ? rowT[r0 + tid] : 0;
        else if (tid < TR + TKP) sk[tid - TR] = k0 + (tid - TR) < K ? kT[k0 + (tid - TR)] : 0;
        __syncthreads();
        constexpr int NV = TR * TKP / PT;
        float v[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int e = tid + j * PT;
            const int r = row_fast ? (e & (TR - 1)) : (e >> 6), k = row_fast ? (e >> 6) : (e & (TKP - 1));
            v[j] = r0 + r < rows && k0 + k < K ? load_as_float<T>(src + srow[r] + sk[k]) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int e = tid + j * PT;
            const int r = row_fast ? (e & (TR - 1)) : (e >> 6), k = row_fast ? (e >> 6) : (e & (TKP - 1));
            tile[r][k] = v[j];
        }
        __syncthreads();
        // thread: k8 = 8 (tid & 7), rows tid >> 3 and 32 + (tid >> 3)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = (tid >> 3) + 32 * h, k8 = (tid & 7) * 8;
            if (r0 + r >= rows) continue;
            uint32_t hw[4], mw[4], lw[4];
            bool bad = false;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float x = tile[r][k8 + q];  // zero for k >= K
                uint16_t hb = f2bf_bits(x);
                if ((hb & 0x7F80u) == 0x7F80u) {
                    // Inf / NaN, or beyond the bf16 range: mark the row, pack zeros
                    bad = true;
                    x = 0.f;
                    hb = 0;
                }
                const float r1 = x - bf_bits2f(hb);
                const uint16_t mb = f2bf_bits(r1);
                const float r2 = r1 - bf_bits2f(mb);
                const uint16_t lb = f2bf_bits(r2);
                const int sh = (q & 1) * 16;
                if ((q & 1) == 0) hw[q >> 1] = mw[q >> 1] = lw[q >> 1] = 0u;
                hw[q >> 1] |= (uint32_t)hb << sh;
                mw[q >> 1] |= (uint32_t)mb << sh;
                lw[q >> 1] |= (uint32_t)lb << sh;
            }
            if (bad) {
                // plain stores of one value: the races are benign
                flags[r0 + r] = 1u;
                *any = 1u;
            }
            const uint4 vh = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            const uint4 vm = make_uint4(mw[0], mw[1], mw[2], mw[3]);
            const uint4 vl = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            uint16_t *o = out + (r0 + r) * ld + k0 + k8;
            for (int b = 0; b < pm.nblocks; ++b) {
                const int pc = pm.piece[b];
                *reinterpret_cast<uint4 *>(o + b * Kb) = pc == 0 ? vh : (pc == 1 ? vm : vl);
            }
        }
    }
}

// Outputs of marked rows of A / columns of B (see above): the products in
// fp32 summed in k order from zero, then met with C under the call's scale.
// Returns at once when the packing marked nothing.
template <class T>
__global__ void __launch_bounds__(256) tc_nonfinite_fixup_kernel(const T *__restrict__ A, const T *__restrict__ B,
                                                                 const int64_t *__restrict__ rowA,
                                                                 const int64_t *__restrict__ colB,
                                                                 const int64_t *__restrict__ kA,
                                                                 const int64_t *__restrict__ kB,
                                                                 const int64_t *__restrict__ rowC,
                                                                 const int64_t *__restrict__ colC, float *C,
                                                                 int64_t M, int64_t N, int64_t K,
                                                                 const uint32_t *__restrict__ flagA,
                                                                 const uint32_t *__restrict__ flagB,
                                                                 const uint32_t *__restrict__ any, int smode,
                                                                 float alpha, float beta)
{
    if (*any == 0u) return;
    const int64_t MN = M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i % M, n = i / M;
        if (!flagA[m] && !flagB[n]) continue;
        const T *a = A + rowA[m];
        const T *b = B + colB[n];
        float acc = 0.f;
        for (int64_t k = 0; k < K; ++k) acc = fmaf(load_as_float<T>(a + kA[k]), load_as_float<T>(b + kB[k]), acc);
        float *dst = C + rowC[m] + colC[n];
        if (smode == SCALE_ACC) *dst = *dst + acc;
        else if (smode == SCALE_AX) *dst = alpha * acc;
        else *dst = alpha * acc + beta * *dst;
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

void pieces_for(int algo, bool is_a, PieceMap *pm)
{
    if (algo == GETT_ALGO_BF16X3) {
        static const int A[3] = {0, 0, 1}, B[3] = {0, 1, 0};
        pm->nblocks = 3;
        for (int i = 0; i < 3; ++i) pm->piece[i] = is_a ? A[i] : B[i];
    } else if (algo == GETT_ALGO_BF16X6) {
        static const int A[6] = {0, 0, 1, 1, 0, 2}, B[6] = {0, 1, 0, 1, 2, 0};
        pm->nblocks = 6;
        for (int i = 0; i < 6; ++i) pm->piece[i] = is_a ? A[i] : B[i];
    } else {
        pm->nblocks = 1;
        pm->piece[0] = 0;
    }
}

// In-place staging (TMA over the caller's tensor instead of a packed copy):
// a bf16 operand whose contracted class is one mode of increment 1 and whose
// row class is at most one mode with a positive increment of whole 16-byte
// units, at a 16-byte-aligned address.  The planner has fused and flipped the
// modes, so e.g. a column-major operand with its contracted modes first
// qualifies.  *ld receives the row pitch in elements.
bool stage_in_place(const ModeList &rows, const int64_t *row_inc, const ModeList &ks, const int64_t *k_inc,
                    const void *base, int64_t K, int64_t *ld)
{
    if (ks.n != 1 || k_inc[0] != 1 || rows.n > 1) return false;
    if (reinterpret_cast<uintptr_t>(base) & 15) return false;
    const int64_t r = rows.n ? row_inc[0] : (K + 7) / 8 * 8;
    if (r <= 0 || (r & 7)) return false;
    *ld = r;
    return true;
}

}  // namespace

int tc_in_place_mask(const Plan &pl, DType t, int algo, const void *A, const void *B)
{
    if (t != DT_BF16 || algo == GETT_ALGO_BF16X3 || algo == GETT_ALGO_BF16X6) return 0;
    int64_t ld = 0;
    const char *Ab = static_cast<const char *>(A) + pl.offA * 2;
    const char *Bb = static_cast<const char *>(B) + pl.offB * 2;
    return (stage_in_place(pl.m, pl.m.s0, pl.k, pl.k.s0, Ab, pl.K, &ld) ? 1 : 0) |
           (stage_in_place(pl.n, pl.n.s0, pl.k, pl.k.s1, Bb, pl.K, &ld) ? 2 : 0);
}

int tc_split_blocks(int algo)
{
    return algo == GETT_ALGO_BF16X3 ? 3 : (algo == GETT_ALGO_BF16X6 ? 6 : 1);
}

int64_t block_len(int64_t K) { return (K + 63) / 64 * 64; }

size_t tc_split_workspace_bytes(const Plan &p, int algo)
{
    const int64_t Kp = block_len(p.K) * tc_split_blocks(algo);
    const int64_t ld = tc_ld(Kp);
    return a256(sizeof(int64_t) * 2 * (size_t)(p.M + p.N + p.K)) + a256(2 * (size_t)p.M * ld) +
           a256(2 * (size_t)p.N * ld) + a256(4 * (size_t)(p.M + p.N + 1));
}

cudaError_t launch_tc_split(const Plan &pl, DType t, int algo, const void *A, const void *B, void *C, void *ws,
                            int num_sms, int *err, cudaStream_t s)
{
    if (t != DT_F32 && t != DT_BF16) return cudaErrorInvalidValue;
    // the packed operands start 256-byte aligned (16-byte vector stores)
    if (reinterpret_cast<uintptr_t>(ws) & 255) return cudaErrorInvalidValue;
    char *w = static_cast<char *>(ws);
    int64_t *rowA = reinterpret_cast<int64_t *>(w);
    int64_t *rowC = rowA + pl.M, *colB = rowC + pl.M, *colC = colB + pl.N, *kA = colC + pl.N, *kB = kA + pl.K;
    w += a256(sizeof(int64_t) * 2 * (size_t)(pl.M + pl.N + pl.K));
    const int nb = t == DT_BF16 ? 1 : tc_split_blocks(algo);
    const int64_t Kb = block_len(pl.K), Kp = Kb * nb, ld = tc_ld(Kp);
    uint16_t *Ap = reinterpret_cast<uint16_t *>(w);
    w += a256(2 * (size_t)pl.M * ld);
    uint16_t *Bp = reinterpret_cast<uint16_t *>(w);
    w += a256(2 * (size_t)pl.N * ld);
    // marks of rows of A and columns of B the pieces cannot carry, and a
    // word that is nonzero when any is marked
    uint32_t *flagA = reinterpret_cast<uint32_t *>(w);
    uint32_t *flagB = flagA + pl.M;
    uint32_t *any = flagB + pl.N;

    cudaError_t e = launch_build_tables(pl, rowA, rowC, colB, colC, kA, kB, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(flagA, 0, 4 * (size_t)(pl.M + pl.N + 1), s);
    if (e != cudaSuccess) return e;
    const size_t esz = dtype_size(t);
    const char *Ab = static_cast<const char *>(A) + pl.offA * (int64_t)esz;
    const char *Bb = static_cast<const char *>(B) + pl.offB * (int64_t)esz;
    float *Cb = static_cast<float *>(C) + pl.offC;
    auto first = [](const ModeList &L, const int64_t *st) { return L.n ? (st[0] < 0 ? -st[0] : st[0]) : 0; };
    const int a_row_fast = first(pl.m, pl.m.s0) != 0 && first(pl.m, pl.m.s0) <= first(pl.k, pl.k.s0) ? 1 : 0;
    const int b_row_fast = first(pl.n, pl.n.s0) != 0 && first(pl.n, pl.n.s0) <= first(pl.k, pl.k.s1) ? 1 : 0;
    PieceMap pa, pb;
    const int split_algo = t == DT_BF16 ? GETT_ALGO_NATIVE : algo;
    pieces_for(split_algo, true, &pa);
    pieces_for(split_algo, false, &pb);
    auto blocks_for = [&](int64_t rows) {
        // four resident CTAs an SM (64 registers a thread), each looping over tiles
        int64_t n = ((rows + TR - 1) / TR) * ((Kb + TKP - 1) / TKP);
        return (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms * 4));
    };
    // bf16 operands that TMA can read where they are skip the packing copy
    // (their Inf / NaN then meet the tensor core's IEEE arithmetic directly)
    int64_t a_ld = 0, b_ld = 0;
    const bool a_direct = t == DT_BF16 && stage_in_place(pl.m, pl.m.s0, pl.k, pl.k.s0, Ab, pl.K, &a_ld);
    const bool b_direct = t == DT_BF16 && stage_in_place(pl.n, pl.n.s0, pl.k, pl.k.s1, Bb, pl.K, &b_ld);
    if (t == DT_F32) {
        pack_pieces_kernel<float><<<blocks_for(pl.M), PT, 0, s>>>((const float *)Ab, rowA, kA, pl.M, pl.K,
                                                                   Kb, a_row_fast, pa, Ap, ld, flagA, any);
        pack_pieces_kernel<float><<<blocks_for(pl.N), PT, 0, s>>>((const float *)Bb, colB, kB, pl.N, pl.K,
                                                                   Kb, b_row_fast, pb, Bp, ld, flagB, any);
    } else {
        if (!a_direct)
            pack_pieces_kernel<uint16_t><<<blocks_for(pl.M), PT, 0, s>>>((const uint16_t *)Ab, rowA, kA, pl.M, pl.K,
                                                                          Kb, a_row_fast, pa, Ap, ld, flagA, any);
        if (!b_direct)
            pack_pieces_kernel<uint16_t><<<blocks_for(pl.N), PT, 0, s>>>((const uint16_t *)Bb, colB, kB, pl.N, pl.K,
                                                                          Kb, b_row_fast, pb, Bp, ld, flagB, any);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TcGemmParams p{};
    p.M = pl.M;
    p.N = pl.N;
    p.K = Kp;
    // one accumulation chunk per piece block (at most 1024 K): every piece
    // product is summed in its own accumulator and the chunk sums are added
    // in registers
    {
        const int64_t tiles = Kb / 64;
        int kc = 1;
        for (int d = 16; d >= 1; --d)
            if (tiles % d == 0) {
                kc = d;
                break;
            }
        p.kc_tiles = kc;
    }
    p.err = err;
    p.C = Cb;
    p.rowC = rowC;
    p.colC = colC;
    p.c_slice = 0;
    p.smode = pl.sc.mode;
    p.alpha = (float)pl.sc.ar;
    p.beta = (float)pl.sc.br;
    p.flagA = flagA;
    p.flagB = flagB;
    if (a_direct) {
        p.a_ld = a_ld;
        p.a_kdim = pl.K;
    }
    if (b_direct) {
        p.b_ld = b_ld;
        p.b_kdim = pl.K;
    }
    e = launch_tc_gemm(TC_MODE_F32, a_direct ? static_cast<const void *>(Ab) : Ap,
                       b_direct ? static_cast<const void *>(Bb) : Bp, 1, p, s);
    if (e != cudaSuccess) return e;
    const int fblocks = (int)std::max<int64_t>(1, std::min<int64_t>((pl.M * pl.N + 255) / 256, (int64_t)num_sms * 8));
    if (t == DT_F32)
        tc_nonfinite_fixup_kernel<float><<<fblocks, 256, 0, s>>>((const float *)Ab, (const float *)Bb, rowA, colB, kA,
                                                                 kB, rowC, colC, Cb, pl.M, pl.N, pl.K, flagA, flagB,
                                                                 any, p.smode, p.alpha, p.beta);
    else
        tc_nonfinite_fixup_kernel<uint16_t><<<fblocks, 256, 0, s>>>((const uint16_t *)Ab, (const uint16_t *)Bb, rowA,
                                                                    colB, kA, kB, rowC, colC, Cb, pl.M, pl.N, pl.K,
                                                                    flagA, flagB, any, p.smode, p.alpha, p.beta);
    return cudaGetLastError();
}

}  // namespace gett

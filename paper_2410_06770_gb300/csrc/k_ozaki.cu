// k_ozaki.cu -- split-precision DGETT on bf16 tensor cores (modular
// "Ozaki scheme II" form), with fp64 used only for the scaling, the integer
// conversion of the inputs and the final recombination into C.
//
// For the canonical problem C[m,n] += sum_k A[m,k] B[k,n]:
//  1. scale scan: for every row m of A the largest |A[m,k]| over K, for every
//     column n of B the largest |B[k,n]| over K (bit patterns, atomicMax);
//  2. integer conversion: A'[m,k] = round(A[m,k] * 2^{s_m}) with s_m chosen so
//     |A'| <= 2^{ka}; B' likewise with t_n and kb bits.  ka + kb is fixed by
//     the moduli: P = p_1 ... p_L must exceed 2 K 2^{ka+kb}, so the exact
//     integer product A'B' is determined by its residues modulo the p_l;
//  3. residues: A' mod p_l, symmetric in [-(p_l-1)/2, (p_l-1)/2] (|.| <= 127,
//     exact in bf16), packed K-major, one slice per modulus;
//  4. one tensor-core GEMM per modulus (all moduli in one launch), exact
//     because K is consumed in chunks whose partial sums stay below 2^24 and
//     are reduced modulo p_l after every chunk (the MODE_MOD epilogue);
//  5. recombination: Garner's mixed-radix form of the residues, sign from a
//     digit comparison with (P-1)/2, exact integer Horner evaluation in three
//     64-bit limbs, one correctly rounded conversion to fp64, scaling by
//     2^{-(s_m+t_n)} and C[m,n] += value.  When the exact sum fits in 53 bits
//     (integer data, for instance) the added value is exact.
// Non-finite inputs.  Alg. 1 forms every product in the operand type, so an
// Inf or NaN in A[m, :] or B[:, n] reaches C[m, n] as IEEE arithmetic makes
// it.  The integer form cannot carry them, so the scale scan marks such a row
// or column (kNonFinite in its maximum); the marked rows and columns get
// all-zero residues, and the recombination computes every output in a marked
// row or column by the definition instead (the fp64 sum over k in order,
// read through the same offset tables), so those outputs propagate Inf and
// NaN exactly as the plain form does.  Unmarked outputs are unaffected.
// Moduli: pairwise coprime odd numbers <= 255 (largest first).  The error
// per element is at most about 2^-ka |A_m|max sum_k |B[k,n]| + 2^-kb
// sum_k |A[m,k]| |B_n|max (the rounding of A' and B'), far below fp64
// accuracy loss of a plain product for the default ka, kb >= 50.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "tc_gemm.h"

namespace gett {

namespace {

constexpr int TR = 32, TKP = 64, PT = 256;

struct OzConsts {
    int L;
    int ka, kb;
    int p[OZ_MAX_L];
    float pf[OZ_MAX_L];
    float invp[OZ_MAX_L];
    float c13[OZ_MAX_L], c26[OZ_MAX_L], c39[OZ_MAX_L];  // 2^13, 2^26, 2^39 mod p, symmetric
    float wpre[OZ_MAX_L][OZ_MAX_L];         // (p_0 ... p_{j-1}) mod p_i, symmetric (j < i)
    float ipre[OZ_MAX_L];                   // (p_0 ... p_{i-1})^{-1} mod p_i
    int half[OZ_MAX_L];                     // mixed-radix digits of (P-1)/2
    float halff[OZ_MAX_L];
    // the residue kernel's constants as f32x2 pairs (the same value twice)
    uint64_t k13[OZ_MAX_L], k26[OZ_MAX_L], k39[OZ_MAX_L], kinv[OZ_MAX_L], knegp[OZ_MAX_L];
};

// Packed pairs of fp32 (Blackwell f32x2): each lane is rounded exactly as
// the scalar .rn instruction, so results equal the per-element code.
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__host__ __device__ constexpr uint64_t pair_bits(uint32_t lo, uint32_t hi) { return ((uint64_t)hi << 32) | lo; }

// Nearest integer of x * r for |x * r| < 2^22, with two full-rate fp32 ops:
// adding 1.5 * 2^23 leaves no fraction bits, so the fused multiply-add rounds
// the product to an integer (round to nearest even), and subtracting the
// constant again is exact.  Replaces rintf, which runs on a slower pipe.
__device__ __forceinline__ float round_mul(float x, float r)
{
    const float magic = 12582912.0f;  // 1.5 * 2^23
    return __fadd_rn(__fmaf_rn(x, r, magic), -magic);
}

// floor(log2(v)) of a positive finite double given its bit pattern
__device__ __forceinline__ int ilog2_bits(uint64_t bits)
{
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e != 0) return e - 1023;
    const uint64_t mant = bits & ((1ull << 52) - 1);
    return -1074 + (63 - __clzll((long long)mant));
}

// Row maximum of a row or column holding an Inf or NaN: above every finite
// |x| pattern, so atomicMax keeps it.
constexpr unsigned long long kNonFinite = 1ull << 63;

// shift s such that max * 2^s lies in [2^(k-1), 2^k); 0 for an all-zero row
__device__ __forceinline__ int shift_for(uint64_t maxbits, int k)
{
    return maxbits == 0 ? 0 : (k - 1 - ilog2_bits(maxbits));
}

// the residue kernel's shift: a marked row gets one that rounds every value
// to zero (scaled_int returns 0 for a shift below -1100)
__device__ __forceinline__ int residue_shift(uint64_t maxbits, int k)
{
    return (maxbits & kNonFinite) ? -4096 : shift_for(maxbits, k);
}

// round(|x| * 2^s) for |x| * 2^s < 2^53 (bit manipulation, no fp64 math)
__device__ __forceinline__ uint64_t scaled_int(uint64_t bits, int s)
{
    const int e = (int)((bits >> 52) & 0x7FF);
    if (e == 0x7FF) return 0;  // inf/nan: not supported by the split forms
    const uint64_t mant = (bits & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    const int eff = e ? e : 1;
    const int sh = eff - 1075 + s;  // value = mant * 2^sh
    if (sh >= 0) return mant << (sh > 11 ? 11 : sh);  // only reachable for k = 53 edge cases
    const int rs = -sh;
    if (rs >= 60) return 0;
    return (mant + (1ull << (rs - 1))) >> rs;
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gmem), "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Gathered tiles of the scan and residue kernels: OZ_STAGES buffers of TR x
// (TKP + 1) doubles (the scan) or RTR x (RTKP + 1) (the residues) in dynamic
// shared memory, OZ_STAGES - 1 tiles in flight.
constexpr int RTR = 32, RTKP = 64;
constexpr int OZ_STAGES = 3;
constexpr size_t OZ_SMEM = (size_t)OZ_STAGES *
                           (TR * (TKP + 1) > RTR * (RTKP + 1) ? TR * (TKP + 1) : RTR * (RTKP + 1)) * sizeof(uint64_t);

// Element offset of (row r, k) in the operand: through the offset tables, or
// AFF (one mode per class after fusion) r * sr + k * sk.
template <bool AFF>
__device__ __forceinline__ int64_t oz_off(const int64_t *rowT, const int64_t *kT, int64_t sr, int64_t sk, int64_t r,
                                          int64_t k)
{
    return AFF ? r * sr + k * sk : rowT[r] + kT[k];
}

// Row maxima of |x| (as bit patterns) over K, for the scaling.  Tiles of 32
// rows x 64 k are gathered with cp.async through OZ_STAGES buffers; each warp
// reduces its values in registers / with shuffles before one shared atomic.
template <int ROW_FAST, bool AFF>
__global__ void __launch_bounds__(PT) oz_maxbits_kernel(const double *__restrict__ src,
                                                       const int64_t *__restrict__ rowT,
                                                       const int64_t *__restrict__ kT, int64_t sr, int64_t sk,
                                                       int64_t rows, int64_t K,
                                                       unsigned long long *__restrict__ maxbits)
{
    extern __shared__ __align__(16) uint64_t oz_dyn[];
    auto tile = [&](int b, int r, int k) -> uint64_t & { return oz_dyn[(b * TR + r) * (TKP + 1) + k]; };
    __shared__ unsigned long long smax[TR];
    const int64_t tiles_k = (K + TKP - 1) / TKP;
    const int64_t ntiles = ((rows + TR - 1) / TR) * tiles_k;
    auto issue = [&](int64_t t, int buf) {
        const int64_t r0 = (t / tiles_k) * TR, k0 = (t % tiles_k) * TKP;
#pragma unroll
        for (int j = 0; j < TR * TKP / PT; ++j) {
            const int e = threadIdx.x + j * PT;
            int r, k;
            if (ROW_FAST) { r = e % TR; k = e / TR; }
            else { k = e % TKP; r = e / TKP; }
            const bool valid = r0 + r < rows && k0 + k < K;
            const double *g = valid ? src + oz_off<AFF>(rowT, kT, sr, sk, r0 + r, k0 + k) : src;
            cp_async8(&tile(buf, r, k), g, valid);
        }
        cp_async_commit();
    };
    int64_t t = blockIdx.x;
#pragma unroll
    for (int st = 0; st < OZ_STAGES - 1; ++st) {
        const int64_t ts = t + (int64_t)st * gridDim.x;
        if (ts < ntiles) issue(ts, st);
        else cp_async_commit();  // empty groups keep the group count uniform
    }
    int buf = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int64_t tn = t + (int64_t)(OZ_STAGES - 1) * gridDim.x;
        if (tn < ntiles) issue(tn, (buf + OZ_STAGES - 1) % OZ_STAGES);
        else cp_async_commit();
        if (threadIdx.x < TR) smax[threadIdx.x] = 0;
        cp_async_wait<OZ_STAGES - 1>();
        __syncthreads();
        const int64_t r0 = (t / tiles_k) * TR;
        // row-fast mapping: a thread's elements share one row; otherwise a warp
        // covers 32 k of one row per step
        unsigned long long mine = 0;
        int myrow = 0;
#pragma unroll
        for (int j = 0; j < TR * TKP / PT; ++j) {
            const int e = threadIdx.x + j * PT;
            int r, k;
            if (ROW_FAST) { r = e % TR; k = e / TR; }
            else { k = e % TKP; r = e / TKP; }
            unsigned long long b = tile(buf, r, k) & 0x7FFFFFFFFFFFFFFFull;
            if ((b >> 52) == 0x7FF) b = kNonFinite;  // inf / nan mark the row
            if (ROW_FAST) {
                mine = b > mine ? b : mine;
                myrow = r;
            } else {
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    const unsigned long long o = __shfl_down_sync(0xffffffffu, b, d);
                    b = o > b ? o : b;
                }
                if ((threadIdx.x & 31) == 0 && b) atomicMax(&smax[r], b);
            }
        }
        if (ROW_FAST && mine) atomicMax(&smax[myrow], mine);
        __syncthreads();
        if (threadIdx.x < TR && r0 + threadIdx.x < rows && smax[threadIdx.x])
            atomicMax(&maxbits[r0 + threadIdx.x], smax[threadIdx.x]);
        __syncthreads();
        buf = (buf + 1) % OZ_STAGES;
    }
}

// Row maxima for one mode per class with rows contiguous (|sr| = 1): no
// staging; a CTA owns 32 rows (lanes) and one slice of K, its 8 warps take
// interleaved k with 4 loads in flight each, and the warps' maxima meet in
// shared memory before one atomic per row.
__global__ void __launch_bounds__(256) oz_maxbits_rows_kernel(const double *__restrict__ src, int64_t sr,
                                                             int64_t sk, int64_t rows, int64_t K, int64_t kslice,
                                                             unsigned long long *__restrict__ maxbits)
{
    __shared__ unsigned long long red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    const int64_t k0 = (int64_t)blockIdx.y * kslice, k1 = min(K, k0 + kslice);
    unsigned long long mine = 0;
    if (r < rows) {
        const unsigned long long *x = reinterpret_cast<const unsigned long long *>(src) + r * sr;
        int64_t k = k0 + warp;
        for (; k + 24 < k1; k += 32) {
            unsigned long long b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = __ldg(x + (k + 8 * u) * sk) & 0x7FFFFFFFFFFFFFFFull;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned long long v = (b[u] >> 52) == 0x7FF ? kNonFinite : b[u];  // inf / nan mark the row
                mine = v > mine ? v : mine;
            }
        }
        for (; k < k1; k += 8) {
            const unsigned long long b = __ldg(x + k * sk) & 0x7FFFFFFFFFFFFFFFull;
            const unsigned long long v = (b >> 52) == 0x7FF ? kNonFinite : b;
            mine = v > mine ? v : mine;
        }
    }
    red[warp][lane] = mine;
    __syncthreads();
    if (warp == 0 && r < rows) {
        for (int w = 1; w < 8; ++w) mine = red[w][lane] > mine ? red[w][lane] : mine;
        if (mine) atomicMax(&maxbits[r], mine);
    }
}

// residues of round(x * 2^shift) for every modulus, packed [L][rows][ld] bf16.
// Tiles of RTR rows x RTKP k are gathered with cp.async through OZ_STAGES
// buffers, so the next tiles' loads are in flight while one is converted.
// Each thread converts two neighbouring k of one row and stores both bf16
// residues of a modulus with one 32-bit store (ld is even, k0 a multiple of
// RTKP); a warp covers 64 k of a row, 128 bytes of every plane.
template <int ROW_FAST, bool AFF, int L>
__global__ void __launch_bounds__(PT) oz_residue_kernel(const double *__restrict__ src,
                                                       const int64_t *__restrict__ rowT,
                                                       const int64_t *__restrict__ kT, int64_t sr, int64_t sk,
                                                       int64_t rows, int64_t K,
                                                       const unsigned long long *__restrict__ maxbits, int kbits,
                                                       OzConsts c, uint16_t *__restrict__ out, int64_t ld,
                                                       int64_t plane, int64_t neg_from)
{
    extern __shared__ __align__(16) uint64_t oz_dyn[];
    auto tile = [&](int b, int r, int k) -> uint64_t & { return oz_dyn[(b * RTR + r) * (RTKP + 1) + k]; };
    __shared__ int sshift[OZ_STAGES][RTR];
    const int64_t tiles_k = (K + RTKP - 1) / RTKP;
    const int64_t ntiles = ((rows + RTR - 1) / RTR) * tiles_k;
    auto issue = [&](int64_t t, int buf) {
        const int64_t r0 = (t / tiles_k) * RTR, k0 = (t % tiles_k) * RTKP;
        if (threadIdx.x < RTR)
            sshift[buf][threadIdx.x] = r0 + threadIdx.x < rows ? residue_shift(maxbits[r0 + threadIdx.x], kbits) : 0;
#pragma unroll
        for (int j = 0; j < RTR * RTKP / PT; ++j) {
            const int e = threadIdx.x + j * PT;
            int r, k;
            if (ROW_FAST) { r = e % RTR; k = e / RTR; }
            else { k = e % RTKP; r = e / RTKP; }
            const bool valid = r0 + r < rows && k0 + k < K;
            const double *g = valid ? src + oz_off<AFF>(rowT, kT, sr, sk, r0 + r, k0 + k) : src;
            cp_async8(&tile(buf, r, k), g, valid);
        }
        cp_async_commit();
    };
    int64_t t = blockIdx.x;
#pragma unroll
    for (int st = 0; st < OZ_STAGES - 1; ++st) {
        const int64_t ts = t + (int64_t)st * gridDim.x;
        if (ts < ntiles) issue(ts, st);
        else cp_async_commit();  // empty groups keep the group count uniform
    }
    int buf = 0;
    for (; t < ntiles; t += gridDim.x) {
        const int64_t tn = t + (int64_t)(OZ_STAGES - 1) * gridDim.x;
        if (tn < ntiles) issue(tn, (buf + OZ_STAGES - 1) % OZ_STAGES);
        else cp_async_commit();
        cp_async_wait<OZ_STAGES - 1>();
        __syncthreads();
        const int64_t r0 = (t / tiles_k) * RTR, k0 = (t % tiles_k) * RTKP;
        // a thread takes 8 consecutive k of one row (four f32x2 pairs) and
        // writes each plane's 8 residues as one 16-byte store (the pitch,
        // the plane pitch and the tile start are multiples of 8 elements,
        // the planes 16-byte aligned: checked by the launcher)
        static_assert(RTR * RTKP == 8 * PT, "one group of 8 a thread");
        {
            const int r = threadIdx.x >> 3, k = (threadIdx.x & 7) * 8;
            if (r0 + r < rows && k0 + k < K) {
                constexpr uint64_t kNeg2p23 = pair_bits(0xCB000000u, 0xCB000000u);  // -2^23
                uint64_t limb[4][4];  // [pair][limb]
#pragma unroll
                for (int pq = 0; pq < 4; ++pq) {
                    // four 13-bit limbs of the scaled integer, sign applied to the
                    // limbs, converted to float through the 2^23 mantissa (no
                    // conversion op); the two elements travel as one f32x2 pair
                    uint32_t lb[4][2], sgb[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int kk = k + 2 * pq + u;
                        const uint64_t bits = tile(buf, r, kk);
                        const uint64_t v = scaled_int(bits & 0x7FFFFFFFFFFFFFFFull, sshift[buf][r]);
                        // k >= neg_from: the value enters negated (the -Im block of
                        // the real form of a complex matrix)
                        const bool neg = ((bits >> 63) != 0) != (k0 + kk >= neg_from);
                        sgb[u] = neg ? 0xBF800000u : 0x3F800000u;  // -1.0f / 1.0f
                        lb[0][u] = 0x4B000000u | (uint32_t)(v & 0x1FFF);
                        lb[1][u] = 0x4B000000u | (uint32_t)((v >> 13) & 0x1FFF);
                        lb[2][u] = 0x4B000000u | (uint32_t)((v >> 26) & 0x1FFF);
                        lb[3][u] = 0x4B000000u | (uint32_t)(v >> 39);
                    }
                    const uint64_t sg = pair_bits(sgb[0], sgb[1]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) limb[pq][q] = mul2(add2(pair_bits(lb[q][0], lb[q][1]), kNeg2p23), sg);
                }
                constexpr uint64_t kMagic = pair_bits(0x4B400000u, 0x4B400000u);     // 1.5 * 2^23
                constexpr uint64_t kNegMagic = pair_bits(0xCB400000u, 0xCB400000u);
                uint4 *o = reinterpret_cast<uint4 *>(out + (r0 + r) * ld + k0 + k);
                const int64_t plane16 = plane / 8;  // plane pitch in 16-byte units
#pragma unroll
                for (int l = 0; l < L; ++l, o += plane16) {
                    uint32_t w[4];
#pragma unroll
                    for (int pq = 0; pq < 4; ++pq) {
                        // |s| <= 127 * 3 * 8191 + 8192 < 2^22: exact; nearest
                        // rounding of s / p is exact for odd p, so the residue
                        // lies in [-(p-1)/2, (p-1)/2]
                        uint64_t sum = fma2(limb[pq][1], c.k13[l], limb[pq][0]);
                        sum = fma2(limb[pq][2], c.k26[l], sum);
                        sum = fma2(limb[pq][3], c.k39[l], sum);
                        const uint64_t q = add2(fma2(sum, c.kinv[l], kMagic), kNegMagic);
                        const uint64_t x = fma2(q, c.knegp[l], sum);
                        // |x| <= 127 has at most 7 significant bits: its bf16
                        // pattern is the upper half of the fp32 pattern
                        w[pq] = __byte_perm((uint32_t)x, (uint32_t)(x >> 32), 0x7632);
                    }
                    *o = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        __syncthreads();
        buf = (buf + 1) % OZ_STAGES;
    }
}

// Dynamic shared memory above 48 KB needs the per-kernel opt-in, once per
// kernel (the template parameter is the kernel itself).
template <auto KERNEL>
cudaError_t oz_smem_optin()
{
    static const cudaError_t e =
        cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM);
    return e;
}

template <int ROW_FAST, bool AFF>
cudaError_t launch_maxbits(const double *src, const int64_t *rowT, const int64_t *kT, int64_t sr, int64_t sk,
                           int64_t rows, int64_t K, unsigned long long *maxbits, int blocks, cudaStream_t s)
{
    cudaError_t e = oz_smem_optin<oz_maxbits_kernel<ROW_FAST, AFF>>();
    if (e != cudaSuccess) return e;
    oz_maxbits_kernel<ROW_FAST, AFF><<<blocks, PT, OZ_SMEM, s>>>(src, rowT, kT, sr, sk, rows, K, maxbits);
    return cudaGetLastError();
}

template <int ROW_FAST, bool AFF>
cudaError_t launch_residues(const double *src, const int64_t *rowT, const int64_t *kT, int64_t sr, int64_t sk,
                            int64_t rows, int64_t K, const unsigned long long *maxbits, int kbits,
                            const OzConsts &c, uint16_t *out, int64_t ld, int blocks, cudaStream_t s,
                            int64_t plane = -1, int64_t neg_from = -1)
{
    if (plane < 0) plane = rows * ld;
    if (neg_from < 0) neg_from = K;
    // 16-byte stores of 8 residues: the planes, the pitch and the plane pitch
    // must keep every group of 8 on a 16-byte boundary
    if ((reinterpret_cast<uintptr_t>(out) & 15) || (ld & 7) || (plane & 7)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
#define CASE(LL)                                                                                          \
    case LL:                                                                                              \
        e = oz_smem_optin<oz_residue_kernel<ROW_FAST, AFF, LL>>();                                          \
        if (e != cudaSuccess) return e;                                                                   \
        oz_residue_kernel<ROW_FAST, AFF, LL><<<blocks, PT, OZ_SMEM, s>>>(src, rowT, kT, sr, sk, rows, K, maxbits, \
                                                                         kbits, c, out, ld, plane, neg_from); \
        break;
    switch (c.L) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
        CASE(14) CASE(15) CASE(16) CASE(17) CASE(18) CASE(19) CASE(20)
    default: return cudaErrorInvalidValue;
    }
#undef CASE
    return cudaGetLastError();
}

// n = i / M for 32-bit i through a precomputed multiplier (Granlund and
// Montgomery's round-up method, 1994): the multiplier is m = 2^32 + mul =
// ceil(2^(32 + shift) / M) with shift = ceil(log2 M).  Its excess m M -
// 2^(32 + shift) is below M <= 2^shift, which is their condition for
// floor(m i / 2^(32 + shift)) = floor(i / M) at every i < 2^32; shift <= 31
// keeps 2^(32 + shift) within 64 bits, so M <= 2^31 (the launcher asks for
// M < 2^31).
struct Div32 {
    uint32_t d, mul, shift;
};
inline Div32 make_div32(uint32_t d)
{
    Div32 r{d, 0, 0};
    uint32_t sh = 0;
    while ((1ull << sh) < d) ++sh;
    r.shift = sh;
    r.mul = (uint32_t)((((1ull << (32 + sh)) + d - 1) / d) & 0xFFFFFFFFull);
    return r;
}
__device__ __forceinline__ uint32_t div32(const Div32 &q, uint32_t i)
{
    // (2^32 + mul) * i >> (32 + shift), the 2^32 term as i itself
    const uint64_t t = (uint64_t)__umulhi(i, q.mul) + i;
    return (uint32_t)(t >> q.shift);
}

// The operands as the residue kernels read them, for the outputs of marked
// (non-finite) rows and columns: row r of the (real-form) A is
// A[rowA[r] + kA_r[k]] with kA_r = kA0 for r < split_row and kA1 above (the
// im-rows of a complex real form), negated for k >= neg_from when r <
// split_row; column n of B is B[colB[n] + kB[k]].
struct OzNative {
    const double *A, *B;
    const int64_t *rowA, *kA0, *kA1, *colB, *kB;
    int64_t K, split_row, neg_from;
};

// C[m, n] of a marked row or column by the definition: the products summed
// in fp64 in k order, so Inf and NaN propagate as in the plain form.
__device__ __noinline__ double oz_native_value(const OzNative &nv, int64_t m, int64_t n)
{
    const bool lower = m < nv.split_row;
    const int64_t *kA = lower ? nv.kA0 : nv.kA1;
    const double *a = nv.A + nv.rowA[m];
    const double *b = nv.B + nv.colB[n];
    double s = 0.0;
    for (int64_t k = 0; k < nv.K; ++k) {
        const double x = a[kA[k]], y = b[nv.kB[k]];
        s = fma((lower && k >= nv.neg_from) ? -x : x, y, s);
    }
    return s;
}

template <int L, bool IDX32>
__global__ void __launch_bounds__(256) oz_crt_kernel(const int8_t *__restrict__ R, int64_t M, int64_t N,
                                                    const unsigned long long *__restrict__ maxA,
                                                    const unsigned long long *__restrict__ maxB,
                                                    const int64_t *__restrict__ rowC,
                                                    const int64_t *__restrict__ colC, double *__restrict__ C,
                                                    OzConsts c, int64_t shift_rows, Scale sc, Div32 divM,
                                                    OzNative nv)
{
    const int64_t MN = M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m, n;
        if (IDX32) {
            n = div32(divM, (uint32_t)i);
            m = i - n * M;
        } else {
            m = i % M;
            n = i / M;
        }
        // row of the scale: m, or m - shift_rows for the imaginary rows of the
        // complex real form (M is shift_rows or twice it)
        const int64_t ms = m >= shift_rows ? m - shift_rows : m;
        const unsigned long long ma = maxA[ms], mb = maxB[n];
        if ((ma | mb) & kNonFinite) {
            const double val = oz_native_value(nv, m, n);
            double *dst = C + rowC[m] + colC[n];
            if (sc.mode == SCALE_ACC) *dst = *dst + val;
            else if (sc.mode == SCALE_AX) *dst = sc.ar * val;
            else *dst = sc.ar * val + sc.br * *dst;
            continue;
        }
        // Garner's mixed-radix digits: X = v_0 + p_0 v_1 + p_0 p_1 v_2 + ...,
        // v_a = (r_a - sum_{b<a} v_b (p_0..p_{b-1} mod p_a)) (p_0..p_{a-1})^{-1} mod p_a.
        // fp32 holds every intermediate exactly: the prefix sum is at most
        // 19 * 254 * 127 < 2^24, the reduced values are below 2^15.
        float v[L];
#pragma unroll
        for (int l = 0; l < L; ++l) {
            // int8 -> float without a conversion instruction: r + 128 in [1, 255]
            // placed in the mantissa of 2^23
            const int r = (int)R[(int64_t)l * MN + i];
            v[l] = __int_as_float(0x4B000000 | (r + 128)) - 8388736.0f;
        }
        v[0] = v[0] < 0.f ? v[0] + c.pf[0] : v[0];
#pragma unroll
        for (int a = 1; a < L; ++a) {
            float sum = v[a];
#pragma unroll
            for (int b = 0; b < a; ++b) sum = fmaf(-v[b], c.wpre[a][b], sum);
            const float pa = c.pf[a], ipa = c.invp[a];
            const float t = fmaf(-round_mul(sum, ipa), pa, sum);      // in [-(pa-1)/2, (pa-1)/2]
            const float x = t * c.ipre[a];                             // |x| < 2^15, exact
            float d = fmaf(-round_mul(x, ipa), pa, x);
            v[a] = d < 0.f ? d + pa : d;
        }
        // sign: compare with (P-1)/2 from the most significant digit
        int cmp = 0;
#pragma unroll
        for (int a = L - 1; a >= 0; --a)
            if (cmp == 0) cmp = v[a] > c.halff[a] ? 1 : (v[a] < c.halff[a] ? -1 : 0);
        const bool negv = cmp > 0;
        // exact Horner evaluation of the mixed-radix digits (|X| < P < 2^160)
        // in five 32-bit limbs, two digits per step: h <- h p_a p_{a-1} +
        // (d_a p_{a-1} + d_{a-1}), with p_a p_{a-1} < 2^16; then one correctly
        // rounded conversion.  Negative values use the digits of P - 1 - X.
        uint32_t dg[L];
#pragma unroll
        for (int a = 0; a < L; ++a) {
            // exact small non-negative integer float -> integer via the 2^23 mantissa
            const float df = negv ? (c.pf[a] - 1.f - v[a]) : v[a];
            dg[a] = (uint32_t)(__float_as_int(df + 8388608.0f) & 0x7FFFFF);
        }
        uint32_t h[5] = {0, 0, 0, 0, 0};
        int a = L - 1;
        if (L % 2) {
            h[0] = dg[L - 1];
            --a;
        }
#pragma unroll
        for (; a > 0; a -= 2) {
            const uint32_t q = (uint32_t)c.p[a] * (uint32_t)c.p[a - 1];
            uint64_t carry = (uint64_t)dg[a] * (uint32_t)c.p[a - 1] + dg[a - 1];
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                const uint64_t prod = (uint64_t)h[t] * q + carry;
                h[t] = (uint32_t)prod;
                carry = prod >> 32;
            }
        }
        uint64_t h0 = ((uint64_t)h[1] << 32) | h[0];
        uint64_t h1 = ((uint64_t)h[3] << 32) | h[2];
        uint64_t h2 = h[4];
        if (negv) {  // value = -(X' + 1)
            h0 += 1;
            if (h0 == 0) {
                h1 += 1;
                if (h1 == 0) h2 += 1;
            }
        }
        // normalise to 64 bits with a sticky bit, convert (round to nearest)
        int drop;
        uint64_t top;
        if (h2) {
            const int lz = __clzll((long long)h2);
            top = (h2 << lz) | (lz ? (h1 >> (64 - lz)) : 0);
            const uint64_t rest_hi = lz ? (h1 << lz) : h1;
            top |= (rest_hi | h0) ? 1 : 0;
            drop = 128 - lz;
        } else if (h1) {
            const int lz = __clzll((long long)h1);
            top = (h1 << lz) | (lz ? (h0 >> (64 - lz)) : 0);
            const uint64_t rest = lz ? (h0 << lz) : h0;
            top |= rest ? 1 : 0;
            drop = 64 - lz;
        } else {
            top = h0;
            drop = 0;
        }
        const double mag = __ull2double_rn(top);
        const int e = drop - (shift_for(ma, c.ka) + shift_for(mb, c.kb));
        // mag * 2^e in two exact power-of-two steps (no overflow of the factors)
        const int e1 = e / 2, e2 = e - e1;
        const double f1 = __longlong_as_double((long long)(e1 + 1023) << 52);
        const double f2 = __longlong_as_double((long long)(e2 + 1023) << 52);
        const double val = negv ? -((mag * f1) * f2) : (mag * f1) * f2;
        double *dst = C + rowC[m] + colC[n];
        if (sc.mode == SCALE_ACC) *dst = *dst + val;
        else if (sc.mode == SCALE_AX) *dst = sc.ar * val;
        else *dst = sc.ar * val + sc.br * *dst;
    }
}

// Complex scaled form with a non-real alpha or beta: the recombination wrote
// the real form's values to T (re-rows m < M, im-rows M + m, column pitch 2M);
// C[rowC[m] + colC[n]] <- alpha * (T_re + i T_im) + beta * C.
__global__ void oz_complex_combine_kernel(const double *__restrict__ T, int64_t M, int64_t N,
                                          const int64_t *__restrict__ rowC, const int64_t *__restrict__ colC,
                                          zd *C, Scale sc)
{
    const int64_t MN = M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i % M, n = i / M;
        const zd v{T[n * 2 * M + m], T[n * 2 * M + M + m]};
        epi_store<Tr<zd>>(C + rowC[m] + colC[n], v, sc);
    }
}

__global__ void iota_kernel(int64_t *t, int64_t n, int64_t step)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = i * step;
}

// Offset tables (in doubles) of the real form of a complex contraction:
//   [C_re; C_im] = [[A_re, -A_im], [A_im, A_re]] [B_re; B_im]
// rows r < M of the real A are re-rows, r >= M im-rows; k' < K selects the
// first block of columns.  Complex element offsets o become 2 o (+1 for the
// imaginary part).
__global__ void oz_complex_tables_kernel(const int64_t *rowA, const int64_t *rowC, const int64_t *colB,
                                         const int64_t *colC, const int64_t *kA, const int64_t *kB, int64_t M,
                                         int64_t N, int64_t K, int64_t *rowA2, int64_t *kAre, int64_t *kAim,
                                         int64_t *colB2, int64_t *kB2, int64_t *rowC2, int64_t *colC2)
{
    const int64_t n_all = max(max(2 * M, 2 * K), N);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_all; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < 2 * M) {
            const int64_t m = i % M, im = i >= M ? 1 : 0;
            rowA2[i] = 2 * rowA[m] + im;
            rowC2[i] = 2 * rowC[m] + im;
        }
        if (i < 2 * K) {
            const int64_t k = i % K, hi = i >= K ? 1 : 0;
            kAre[i] = 2 * kA[k] + hi;   // re-rows: Re then Im (the Im block enters negated)
            kAim[i] = 2 * kA[k] - hi;   // im-rows (offset +1 in rowA2): Im then Re
            kB2[i] = 2 * kB[k] + hi;    // B: Re block over Im block
        }
        if (i < N) {
            colB2[i] = 2 * colB[i];
            colC2[i] = 2 * colC[i];
        }
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int modinv(int a, int m)
{
    int t = 0, nt = 1, r = m, nr = a % m;
    while (nr) {
        int q = r / nr;
        int tmp = t - q * nt;
        t = nt;
        nt = tmp;
        tmp = r - q * nr;
        r = nr;
        nr = tmp;
    }
    return t < 0 ? t + m : t;
}

// Number of moduli and bit budgets for a sum of length K.
void oz_setup(int64_t K, int want_L, OzConsts *c)
{
    const double lk = std::log2((double)(K > 1 ? K : 1));
    int L = want_L;
    if (L <= 0) {
        // smallest L that leaves >= 50 bits per operand
        for (L = 8; L < OZ_MAX_L; ++L) {
            double lp = 0;
            for (int i = 0; i < L; ++i) lp += std::log2((double)kOzModuli[i]);
            if (std::floor((lp - 1.0 - lk - 1e-6) / 2.0) >= 50) break;
        }
    }
    if (L > OZ_MAX_L) L = OZ_MAX_L;
    if (L < 2) L = 2;
    double lp = 0;
    for (int i = 0; i < L; ++i) lp += std::log2((double)kOzModuli[i]);
    int kk = (int)std::floor((lp - 1.0 - lk - 1e-6) / 2.0);
    if (kk > 52) kk = 52;
    if (kk < 1) kk = 1;
    c->L = L;
    c->ka = kk;
    c->kb = kk;
    for (int i = 0; i < L; ++i) {
        const int p = kOzModuli[i];
        c->p[i] = p;
        c->pf[i] = (float)p;
        c->invp[i] = 1.0f / (float)p;
        auto sym = [p](long long r) { r %= p; return (float)(r > (p - 1) / 2 ? r - p : r); };
        const long long m13 = (1LL << 13) % p;
        c->c13[i] = sym(m13);
        c->c26[i] = sym(m13 * m13);
        c->c39[i] = sym(m13 * m13 % p * m13);
        auto pair = [](float f) {
            uint32_t b;
            std::memcpy(&b, &f, 4);
            return pair_bits(b, b);
        };
        c->k13[i] = pair(c->c13[i]);
        c->k26[i] = pair(c->c26[i]);
        c->k39[i] = pair(c->c39[i]);
        c->kinv[i] = pair(c->invp[i]);
        c->knegp[i] = pair(-c->pf[i]);
        long long pre = 1;  // (p_0 ... p_{j-1}) mod p
        for (int j = 0; j < OZ_MAX_L; ++j) {
            long long w = pre % p;
            c->wpre[i][j] = (j < i) ? (float)(w > (p - 1) / 2 ? w - p : w) : 0.f;
            if (j == i) c->ipre[i] = (float)(i == 0 ? 1 : modinv((int)pre, p));
            if (j < i) pre = pre * (kOzModuli[j] % p) % p;
        }
    }
    // digits of (P-1)/2: long division of the digits (p_i - 1) by 2 from the top
    int carry = 0;
    for (int i = L - 1; i >= 0; --i) {
        const int cur = carry * c->p[i] + (c->p[i] - 1);
        c->half[i] = cur / 2;
        c->halff[i] = (float)c->half[i];
        carry = cur % 2;
    }
}

template <int L>
void launch_crt_t(const int8_t *R, int64_t M, int64_t N, const unsigned long long *maxA,
                  const unsigned long long *maxB, const int64_t *rowC, const int64_t *colC, double *C,
                  const OzConsts &c, int num_sms, cudaStream_t s, int64_t shift_rows, const Scale &sc,
                  const OzNative &nv)
{
    const int64_t MN = M * N;
    int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((MN + 255) / 256, (int64_t)num_sms * 16));
    if (MN < (1LL << 32) && M < (1LL << 31)) {
        // every grid-stride index stays below 2^32 + 2^31: i < MN < 2^32 when it is used
        oz_crt_kernel<L, true><<<blocks, 256, 0, s>>>(R, M, N, maxA, maxB, rowC, colC, C, c, shift_rows, sc,
                                                       make_div32((uint32_t)M), nv);
    } else {
        oz_crt_kernel<L, false><<<blocks, 256, 0, s>>>(R, M, N, maxA, maxB, rowC, colC, C, c, shift_rows, sc,
                                                        Div32{1, 0, 0}, nv);
    }
}

cudaError_t launch_crt(const int8_t *R, int64_t M, int64_t N, const unsigned long long *maxA,
                       const unsigned long long *maxB, const int64_t *rowC, const int64_t *colC, double *C,
                       const OzConsts &c, int num_sms, cudaStream_t s, const Scale &sc, const OzNative &nv,
                       int64_t shift_rows = -1)
{
    if (shift_rows <= 0) shift_rows = M;
#define CASE(L)                                                                               \
    case L:                                                                                   \
        launch_crt_t<L>(R, M, N, maxA, maxB, rowC, colC, C, c, num_sms, s, shift_rows, sc, nv); \
        break;
    switch (c.L) {
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12) CASE(13)
        CASE(14) CASE(15) CASE(16) CASE(17) CASE(18) CASE(19) CASE(20)
    default: return cudaErrorInvalidValue;
    }
#undef CASE
    return cudaGetLastError();
}

struct OzLayout {
    int64_t *rowA, *rowC, *colB, *colC, *kA, *kB;
    unsigned long long *maxA, *maxB;
    uint16_t *RA, *RB;
    int8_t *R;
    int64_t ld;
    size_t total;
};

OzLayout oz_layout(const Plan &p, int L, void *ws)
{
    OzLayout o{};
    char *w = static_cast<char *>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *r = w ? w + off : nullptr;
        off += a256(bytes);
        return r;
    };
    o.ld = tc_ld(p.K);
    char *tab = take(sizeof(int64_t) * 2 * (size_t)(p.M + p.N + p.K));
    o.rowA = reinterpret_cast<int64_t *>(tab);
    if (tab) {
        o.rowC = o.rowA + p.M;
        o.colB = o.rowC + p.M;
        o.colC = o.colB + p.N;
        o.kA = o.colC + p.N;
        o.kB = o.kA + p.K;
    }
    o.maxA = reinterpret_cast<unsigned long long *>(take(8 * (size_t)p.M));
    o.maxB = reinterpret_cast<unsigned long long *>(take(8 * (size_t)p.N));
    o.RA = reinterpret_cast<uint16_t *>(take(2 * (size_t)L * p.M * o.ld));
    o.RB = reinterpret_cast<uint16_t *>(take(2 * (size_t)L * p.N * o.ld));
    o.R = reinterpret_cast<int8_t *>(take((size_t)L * p.M * p.N));
    o.total = off;
    return o;
}

}  // namespace

int ozaki_moduli_for(int64_t K, int want)
{
    OzConsts c;
    oz_setup(K, want, &c);
    return c.L;
}

int ozaki_bits_for(int64_t K, int L)
{
    OzConsts c;
    oz_setup(K, L, &c);
    return c.ka;
}

size_t ozaki_workspace_bytes(const Plan &p, int L)
{
    return oz_layout(p, L, nullptr).total;
}

namespace {

cudaError_t oz_maxbits(const double *X, const int64_t *rowT, const int64_t *kT, bool row_fast, bool aff, int64_t sr,
                       int64_t sk, int64_t rows, int64_t K, unsigned long long *mx, int blocks, cudaStream_t s)
{
    if (aff && (sr == 1 || sr == -1) && rows > 0 && K > 0) {
        // enough CTAs for about 16 per SM; each K slice at least 256 long
        const int64_t rb = (rows + 31) / 32;
        const int64_t want = std::max<int64_t>(1, (2LL * blocks + rb - 1) / rb);
        const int64_t slices = std::min<int64_t>(want, std::max<int64_t>(1, K / 256));
        const int64_t kslice = (K + slices - 1) / slices;
        dim3 grid((unsigned)rb, (unsigned)((K + kslice - 1) / kslice));
        oz_maxbits_rows_kernel<<<grid, 256, 0, s>>>(X, sr, sk, rows, K, kslice, mx);
        return cudaGetLastError();
    }
    if (row_fast) return aff ? launch_maxbits<1, true>(X, rowT, kT, sr, sk, rows, K, mx, blocks, s)
                             : launch_maxbits<1, false>(X, rowT, kT, sr, sk, rows, K, mx, blocks, s);
    return aff ? launch_maxbits<0, true>(X, rowT, kT, sr, sk, rows, K, mx, blocks, s)
               : launch_maxbits<0, false>(X, rowT, kT, sr, sk, rows, K, mx, blocks, s);
}

cudaError_t oz_residues(const double *X, const int64_t *rowT, const int64_t *kT, bool row_fast, bool aff, int64_t sr,
                        int64_t sk, int64_t rows, int64_t K, const unsigned long long *mx, int kbits,
                        const OzConsts &c, uint16_t *out, int64_t ld, int blocks, cudaStream_t s, int64_t plane = -1,
                        int64_t neg_from = -1)
{
    if (row_fast)
        return aff ? launch_residues<1, true>(X, rowT, kT, sr, sk, rows, K, mx, kbits, c, out, ld, blocks, s, plane,
                                              neg_from)
                   : launch_residues<1, false>(X, rowT, kT, sr, sk, rows, K, mx, kbits, c, out, ld, blocks, s, plane,
                                               neg_from);
    return aff ? launch_residues<0, true>(X, rowT, kT, sr, sk, rows, K, mx, kbits, c, out, ld, blocks, s, plane,
                                          neg_from)
               : launch_residues<0, false>(X, rowT, kT, sr, sk, rows, K, mx, kbits, c, out, ld, blocks, s, plane,
                                           neg_from);
}

// Scale scan (row maxima) then residue planes of one operand.
cudaError_t oz_scan_and_residues(const double *X, const int64_t *rowT, const int64_t *kT, bool row_fast, bool aff,
                                 int64_t sr, int64_t sk, int64_t rows, int64_t K, unsigned long long *mx, int kbits,
                                 const OzConsts &c, uint16_t *out, int64_t ld, int blocks, cudaStream_t s)
{
    cudaError_t e = oz_maxbits(X, rowT, kT, row_fast, aff, sr, sk, rows, K, mx, blocks, s);
    if (e != cudaSuccess) return e;
    return oz_residues(X, rowT, kT, row_fast, aff, sr, sk, rows, K, mx, kbits, c, out, ld, blocks, s);
}

}  // namespace

cudaError_t launch_ozaki(const Plan &pl, int L_req, const void *A, const void *B, void *C, void *ws, int num_sms,
                         int *err, cudaStream_t s)
{
    OzConsts c;
    oz_setup(pl.K, L_req, &c);
    OzLayout o = oz_layout(pl, c.L, ws);
    cudaError_t e = launch_build_tables(pl, o.rowA, o.rowC, o.colB, o.colC, o.kA, o.kB, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(o.maxA, 0, 8 * (size_t)pl.M, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o.maxB, 0, 8 * (size_t)pl.N, s);
    if (e != cudaSuccess) return e;
    const double *Ab = static_cast<const double *>(A) + pl.offA;
    const double *Bb = static_cast<const double *>(B) + pl.offB;
    double *Cb = static_cast<double *>(C) + pl.offC;
    auto first = [](const ModeList &Lm, const int64_t *st) { return Lm.n ? (st[0] < 0 ? -st[0] : st[0]) : 0; };
    const bool a_row_fast = first(pl.m, pl.m.s0) != 0 && first(pl.m, pl.m.s0) <= first(pl.k, pl.k.s0);
    const bool b_row_fast = first(pl.n, pl.n.s0) != 0 && first(pl.n, pl.n.s0) <= first(pl.k, pl.k.s1);
    auto blocks_for = [&](int64_t rows) {
        int64_t n = ((rows + TR - 1) / TR) * ((pl.K + TKP - 1) / TKP);
        return (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms * 8));
    };
    // one mode per class after fusion: addresses without the offset tables
    const bool a_aff = pl.m.n <= 1 && pl.k.n <= 1, b_aff = pl.n.n <= 1 && pl.k.n <= 1;
    const int64_t a_sr = pl.m.n ? pl.m.s0[0] : 0, a_sk = pl.k.n ? pl.k.s0[0] : 0;
    const int64_t b_sr = pl.n.n ? pl.n.s0[0] : 0, b_sk = pl.k.n ? pl.k.s1[0] : 0;
    e = oz_scan_and_residues(Ab, o.rowA, o.kA, a_row_fast, a_aff, a_sr, a_sk, pl.M, pl.K, o.maxA, c.ka, c, o.RA,
                             o.ld, blocks_for(pl.M), s);
    if (e != cudaSuccess) return e;
    e = oz_scan_and_residues(Bb, o.colB, o.kB, b_row_fast, b_aff, b_sr, b_sk, pl.N, pl.K, o.maxB, c.kb, c, o.RB,
                             o.ld, blocks_for(pl.N), s);
    if (e != cudaSuccess) return e;
    TcGemmParams p{};
    p.M = pl.M;
    p.N = pl.N;
    p.K = pl.K;
    p.err = err;
    p.kc_tiles = OZ_CHUNK_K / 64;
    p.R = o.R;
    e = launch_tc_gemm(TC_MODE_MOD, o.RA, o.RB, c.L, p, s);
    if (e != cudaSuccess) return e;
    const OzNative nv{Ab, Bb, o.rowA, o.kA, o.kA, o.colB, o.kB, pl.K, pl.M, pl.K};
    return launch_crt(o.R, pl.M, pl.N, o.maxA, o.maxB, o.rowC, o.colC, Cb, c, num_sms, s, pl.sc, nv);
}

namespace {

struct OzComplexLayout {
    int64_t *rowA, *rowC, *colB, *colC, *kA, *kB;              // complex element units
    int64_t *rowA2, *kAre, *kAim, *colB2, *kB2, *rowC2, *colC2;  // doubles, real form
    unsigned long long *maxA, *maxB;
    uint16_t *RA, *RB;
    int8_t *R;
    double *T;              // non-real alpha or beta: [N][2M] real-form result
    int64_t *rowT, *colT;   // its offset tables
    int64_t ld;
    size_t total;
};

// A non-real alpha or beta mixes the real and imaginary parts, which the
// recombination writes from different threads: go through T.
bool complex_scale_via_temp(const Scale &sc)
{
    return sc.mode != SCALE_ACC && (sc.ai != 0.0 || sc.bi != 0.0);
}

OzComplexLayout oz_complex_layout(const Plan &p, int L, void *ws)
{
    OzComplexLayout o{};
    char *w = static_cast<char *>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *r = w ? w + off : nullptr;
        off += a256(bytes);
        return r;
    };
    const int64_t M2 = 2 * p.M, K2 = 2 * p.K;
    o.ld = tc_ld(K2);
    auto t64 = [&](int64_t n) { return reinterpret_cast<int64_t *>(take(8 * (size_t)n)); };
    o.rowA = t64(p.M); o.rowC = t64(p.M); o.colB = t64(p.N); o.colC = t64(p.N); o.kA = t64(p.K); o.kB = t64(p.K);
    o.rowA2 = t64(M2); o.kAre = t64(K2); o.kAim = t64(K2); o.colB2 = t64(p.N); o.kB2 = t64(K2);
    o.rowC2 = t64(M2); o.colC2 = t64(p.N);
    o.maxA = reinterpret_cast<unsigned long long *>(take(8 * (size_t)p.M));
    o.maxB = reinterpret_cast<unsigned long long *>(take(8 * (size_t)p.N));
    o.RA = reinterpret_cast<uint16_t *>(take(2 * (size_t)L * M2 * o.ld));
    o.RB = reinterpret_cast<uint16_t *>(take(2 * (size_t)L * p.N * o.ld));
    o.R = reinterpret_cast<int8_t *>(take((size_t)L * M2 * p.N));
    if (complex_scale_via_temp(p.sc)) {
        o.T = reinterpret_cast<double *>(take(8 * (size_t)M2 * p.N));
        o.rowT = t64(M2);
        o.colT = t64(p.N);
    }
    o.total = off;
    return o;
}

}  // namespace

size_t ozaki_complex_workspace_bytes(const Plan &p, int L)
{
    return oz_complex_layout(p, L, nullptr).total;
}

// Complex double (z) split precision: the same scaling, residue, slice-GEMM and
// recombination kernels applied to the real form of the contraction (2M rows,
// 2K contracted indices), reading the interleaved complex buffers in place
// through the real-form offset tables.
cudaError_t launch_ozaki_complex(const Plan &pl, int L_req, const void *A, const void *B, void *C, void *ws,
                                 int num_sms, int *err, cudaStream_t s)
{
    const int64_t M2 = 2 * pl.M, K2 = 2 * pl.K;
    OzConsts c;
    oz_setup(K2, L_req, &c);
    OzComplexLayout o = oz_complex_layout(pl, c.L, ws);
    cudaError_t e = launch_build_tables(pl, o.rowA, o.rowC, o.colB, o.colC, o.kA, o.kB, s);
    if (e != cudaSuccess) return e;
    {
        const int64_t n_all = std::max(std::max(M2, K2), pl.N);
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n_all + 255) / 256, 4096));
        oz_complex_tables_kernel<<<blocks, 256, 0, s>>>(o.rowA, o.rowC, o.colB, o.colC, o.kA, o.kB, pl.M, pl.N, pl.K,
                                                        o.rowA2, o.kAre, o.kAim, o.colB2, o.kB2, o.rowC2, o.colC2);
    }
    e = cudaMemsetAsync(o.maxA, 0, 8 * (size_t)pl.M, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o.maxB, 0, 8 * (size_t)pl.N, s);
    if (e != cudaSuccess) return e;
    const double *Ab = static_cast<const double *>(A) + 2 * pl.offA;
    const double *Bb = static_cast<const double *>(B) + 2 * pl.offB;
    double *Cb = static_cast<double *>(C) + 2 * pl.offC;
    auto first = [](const ModeList &Lm, const int64_t *st) { return Lm.n ? (st[0] < 0 ? -st[0] : st[0]) : 0; };
    const bool a_row_fast = first(pl.m, pl.m.s0) != 0 && first(pl.m, pl.m.s0) <= first(pl.k, pl.k.s0);
    const bool b_row_fast = first(pl.n, pl.n.s0) != 0 && first(pl.n, pl.n.s0) <= first(pl.k, pl.k.s1);
    auto blocks_for = [&](int64_t rows) {
        int64_t n = ((rows + TR - 1) / TR) * ((K2 + TKP - 1) / TKP);
        return (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms * 8));
    };
    // scales: a complex row's maximum over both parts (its re-row covers both)
    e = oz_maxbits(Ab, o.rowA2, o.kAre, a_row_fast, false, 0, 0, pl.M, K2, o.maxA, blocks_for(pl.M), s);
    if (e == cudaSuccess) e = oz_maxbits(Bb, o.colB2, o.kB2, b_row_fast, false, 0, 0, pl.N, K2, o.maxB, blocks_for(pl.N), s);
    if (e != cudaSuccess) return e;
    const int64_t planeA = M2 * o.ld;
    // re-rows: [Re | -Im], im-rows: [Im | Re]
    e = oz_residues(Ab, o.rowA2, o.kAre, a_row_fast, false, 0, 0, pl.M, K2, o.maxA, c.ka, c, o.RA, o.ld,
                    blocks_for(pl.M), s, planeA, pl.K);
    if (e != cudaSuccess) return e;
    e = oz_residues(Ab, o.rowA2 + pl.M, o.kAim, a_row_fast, false, 0, 0, pl.M, K2, o.maxA, c.ka, c,
                    o.RA + pl.M * o.ld, o.ld, blocks_for(pl.M), s, planeA, K2);
    if (e != cudaSuccess) return e;
    e = oz_residues(Bb, o.colB2, o.kB2, b_row_fast, false, 0, 0, pl.N, K2, o.maxB, c.kb, c, o.RB, o.ld,
                    blocks_for(pl.N), s);
    if (e != cudaSuccess) return e;
    TcGemmParams p{};
    p.M = M2;
    p.N = pl.N;
    p.K = K2;
    p.err = err;
    p.kc_tiles = OZ_CHUNK_K / 64;
    p.R = o.R;
    e = launch_tc_gemm(TC_MODE_MOD, o.RA, o.RB, c.L, p, s);
    if (e != cudaSuccess) return e;
    // marked rows and columns: re-rows are [Re | -Im] through kAre, im-rows
    // [Im | Re] through kAim, B is [Re; Im] through kB2
    const OzNative nv{Ab, Bb, o.rowA2, o.kAre, o.kAim, o.colB2, o.kB2, K2, pl.M, pl.K};
    if (!complex_scale_via_temp(pl.sc))  // real alpha and beta act on each part alone
        return launch_crt(o.R, M2, pl.N, o.maxA, o.maxB, o.rowC2, o.colC2, Cb, c, num_sms, s, pl.sc, nv, pl.M);
    {
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((std::max(M2, pl.N) + 255) / 256, 4096));
        iota_kernel<<<blocks, 256, 0, s>>>(o.rowT, M2, 1);
        iota_kernel<<<blocks, 256, 0, s>>>(o.colT, pl.N, M2);
    }
    const Scale store{SCALE_AX, 1.0, 0.0, 0.0, 0.0};
    e = launch_crt(o.R, M2, pl.N, o.maxA, o.maxB, o.rowT, o.colT, o.T, c, num_sms, s, store, nv, pl.M);
    if (e != cudaSuccess) return e;
    const int64_t MN = pl.M * pl.N;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((MN + 255) / 256, (int64_t)num_sms * 16));
    oz_complex_combine_kernel<<<blocks, 256, 0, s>>>(o.T, pl.M, pl.N, o.rowC, o.colC, reinterpret_cast<zd *>(C) + pl.offC,
                                                     pl.sc);
    return cudaGetLastError();
}

}  // namespace gett

// k_aux.cu -- the tensor transpose and the unit operand of the tensor
// reduction (two of the operations the thesis lists as future work for a
// BLAS-like tensor interface, Sec. 9).
//
// Transpose: C[o permuted by PERM] <- alpha * A[o] + beta * C (or C += A).
// It is the contraction with a rank-0 B equal to 1, planned the same way (M =
// A's modes, s0 = A increment, s1 = C increment, ordered by C increment), but
// run by its own kernel: when A's smallest-increment mode is not C's, a
// 32 x 32 tile goes through shared memory so that the reads run along A's
// fastest mode and the writes along C's; otherwise both run along the same
// mode in 128 x 32 blocks over it and the next mode (a streaming copy).  HBM-bound: 8 bytes read + 8 written per double
// (plus 8 read when C is accumulated).
//
// Reduction: the contraction with a B of ones over the reduced modes, all of
// B's increments zero, so B is one element; unit_operand() gives its device
// address for every element type.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace gett {

namespace {

constexpr int TT = 32;  // transpose tile edge

struct TransParams {
    const void *A;
    void *C;
    int64_t e0, e1;   // extents: C's fastest mode, A's fastest mode
    int64_t a0, c0;   // increments of the first in A and C
    int64_t a1, c1;   // and of the second
    ModeList rest;    // all other modes (s0: A, s1: C)
    int64_t t0n, t1n, items;
    int64_t tg, t0g;  // tile kernel: tiles of mode 0 per item, item groups along mode 0
    int wide;         // rows kernel: 1024 x 1 blocks instead of 128 x 32
    Scale sc;
};

template <class R>
__device__ __forceinline__ void trans_store(typename R::Out *c, typename R::Acc v, const Scale &sc)
{
    if (sc.mode == SCALE_AX && sc.ar == 1.0 && sc.ai == 0.0) R::store_c(c, v);
    else epi_store<R>(c, v, sc);
}

// Tiles of TT x TT over (mode 0, mode 1) times the other modes; a CTA of
// 32 x 8 threads reads the tile with lanes along mode 1 (A's fastest) and
// writes it with lanes along mode 0 (C's fastest).  Addresses advance by
// increments (no per-element 64-bit products); UNIT: A's mode-1 and C's
// mode-0 increments are 1.
template <class T, bool UNIT>
__global__ void __launch_bounds__(256) transpose_tile_kernel(TransParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    __shared__ Acc tile[TT][TT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t a1 = UNIT ? 1 : p.a1, c0 = UNIT ? 1 : p.c0;
    const bool plain = p.sc.mode == SCALE_AX && p.sc.ar == 1.0 && p.sc.ai == 0.0;
    // an item is a run of up to tg tiles along mode 0 at one (mode-1 tile,
    // other modes) position: its index arithmetic is shared by the run
    for (int64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const int64_t g0 = item % p.t0g;
        const int64_t r1 = item / p.t0g;
        const int64_t t1 = r1 % p.t1n;
        const int64_t ir = r1 / p.t1n;
        int64_t oa, oc;
        decode2(p.rest, ir, oa, oc);
        const int64_t i1 = t1 * TT;
        const int n1 = (int)min((int64_t)TT, p.e1 - i1);
        const T *abase = static_cast<const T *>(p.A) + oa + (i1 + tx) * a1;
        Out *cbase = static_cast<Out *>(p.C) + oc + (i1 + ty) * p.c1;
        const int64_t tend = min(p.t0n, (g0 + 1) * p.tg);
        for (int64_t t0 = g0 * p.tg; t0 < tend; ++t0) {
            const int64_t i0 = t0 * TT;
            // rows this thread touches: mode-0 index i0 + ty + 8 j when reading,
            // mode-1 index i1 + ty + 8 j when writing
            const int n0 = (int)min((int64_t)TT, p.e0 - i0);
            __syncthreads();  // the previous tile has been written out
            if (tx < n1) {
                const T *src = abase + (i0 + ty) * p.a0;
#pragma unroll
                for (int r = ty; r < TT; r += 8, src += 8 * p.a0)
                    if (r < n0) tile[r][tx] = R::load(src);
            }
            __syncthreads();
            if (tx < n0) {
                Out *dst = cbase + (i0 + tx) * c0;
#pragma unroll
                for (int r = ty; r < TT; r += 8, dst += 8 * p.c1) {
                    if (r >= n1) continue;
                    if (plain) R::store_c(dst, tile[tx][r]);
                    else trans_store<R>(dst, tile[tx][r], p.sc);
                }
            }
        }
    }
}

// A's and C's fastest modes coincide (mode 0): both sides run along mode 0.
// A work item is 128 elements of mode 0 (a warp, 4 per lane) times 32
// indices of mode 1 (8 warps, 4 passes) times one index of the other modes,
// so short fastest modes still keep every thread busy; all 16 loads of a
// thread are issued before its stores.
// WIDE (mode 1 shorter than 32, mode 0 long): 1024 elements of mode 0 (8
// warps side by side) and one index of mode 1 per item instead.
template <class T, bool WIDE>
__global__ void __launch_bounds__(256) transpose_rows_kernel(TransParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    constexpr int UX = 4, UY = WIDE ? 1 : 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool plain = p.sc.mode == SCALE_AX && p.sc.ar == 1.0 && p.sc.ai == 0.0;
    // an item is a run of up to tg blocks along mode 0 (shared index arithmetic)
    for (int64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const int64_t g0 = item % p.t0g;
        const int64_t r1 = item / p.t0g;
        const int64_t t1 = r1 % p.t1n;
        const int64_t ir = r1 / p.t1n;
        int64_t oa, oc;
        decode2(p.rest, ir, oa, oc);
        const int64_t y0 = WIDE ? t1 : t1 * 8 * UY + warp;
        const int64_t tend = min(p.t0n, (g0 + 1) * p.tg);
        for (int64_t t0 = g0 * p.tg; t0 < tend; ++t0) {
            const int64_t x0 = WIDE ? t0 * 8 * 32 * UX + warp * 32 * UX + lane : t0 * 32 * UX + lane;
            const T *src = static_cast<const T *>(p.A) + oa + x0 * p.a0 + y0 * p.a1;
            Out *dst = static_cast<Out *>(p.C) + oc + x0 * p.c0 + y0 * p.c1;
            Acc v[UY][UX];
#pragma unroll
            for (int j = 0; j < UY; ++j)
#pragma unroll
                for (int u = 0; u < UX; ++u)
                    if (x0 + 32 * u < p.e0 && y0 + 8 * j < p.e1) v[j][u] = R::load(src + 32 * u * p.a0 + 8 * j * p.a1);
#pragma unroll
            for (int j = 0; j < UY; ++j)
#pragma unroll
                for (int u = 0; u < UX; ++u) {
                    if (!(x0 + 32 * u < p.e0 && y0 + 8 * j < p.e1)) continue;
                    Out *c = dst + 32 * u * p.c0 + 8 * j * p.c1;
                    if (plain) R::store_c(c, v[j][u]);
                    else trans_store<R>(c, v[j][u], p.sc);
                }
        }
    }
}

// Drop modes i and j (i != j, either may be -1) from a list; the rest is
// ordered by A's increment, so consecutive work items read nearby data.
ModeList without(const ModeList &L, int i, int j)
{
    ModeList r{};
    for (int q = 0; q < L.n; ++q) {
        if (q == i || q == j) continue;
        int at = r.n;
        while (at > 0 && std::llabs(r.s0[at - 1]) > std::llabs(L.s0[q])) {
            r.ext[at] = r.ext[at - 1];
            r.s0[at] = r.s0[at - 1];
            r.s1[at] = r.s1[at - 1];
            --at;
        }
        r.ext[at] = L.ext[q];
        r.s0[at] = L.s0[q];
        r.s1[at] = L.s1[q];
        ++r.n;
    }
    return r;
}

// bytes of one C element (bf16 inputs accumulate into float)
size_t c_bytes(DType t) { return t == DT_BF16 ? 4 : dtype_size(t); }

int64_t count(const ModeList &L)
{
    int64_t n = 1;
    for (int i = 0; i < L.n; ++i) n *= L.ext[i];
    return n;
}

template <class T>
cudaError_t transpose_typed(const TransParams &p, bool tiled, int num_sms, cudaStream_t s)
{
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(p.items, (int64_t)num_sms * 8));
    if (tiled && p.a1 == 1 && p.c0 == 1) transpose_tile_kernel<T, true><<<(unsigned)blocks, 256, 0, s>>>(p);
    else if (tiled) transpose_tile_kernel<T, false><<<(unsigned)blocks, 256, 0, s>>>(p);
    else if (p.wide) transpose_rows_kernel<T, true><<<(unsigned)blocks, 256, 0, s>>>(p);
    else transpose_rows_kernel<T, false><<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// One element of value 1 per element type (B of the reduction).
__device__ __align__(16) float g_one_f32 = 1.0f;
__device__ __align__(16) double g_one_f64 = 1.0;
__device__ __align__(16) float g_one_c32[2] = {1.0f, 0.0f};
__device__ __align__(16) double g_one_c64[2] = {1.0, 0.0};
__device__ __align__(16) uint16_t g_one_bf16 = 0x3F80;  // bfloat16 1.0

struct OnePtrs {
    bool init = false;
    const void *p[5] = {};
};
OnePtrs g_ones[64];
std::mutex g_ones_mu;

}  // namespace

bool transpose_tiled(const Plan &pl)
{
    if (pl.m.n < 2) return false;
    int ia = 0;
    for (int i = 1; i < pl.m.n; ++i)
        if (std::llabs(pl.m.s0[i]) < std::llabs(pl.m.s0[ia])) ia = i;
    return ia != 0;
}

cudaError_t launch_transpose(const Plan &pl, DType t, const void *A, void *C, int num_sms, cudaStream_t s)
{
    const size_t esz = dtype_size(t);
    TransParams p{};
    p.A = static_cast<const char *>(A) + pl.offA * (int64_t)esz;
    p.C = static_cast<char *>(C) + pl.offC * (int64_t)c_bytes(t);
    p.sc = pl.sc;
    // mode 0 of M has C's smallest increment; ia has A's smallest
    int ia = 0;
    for (int i = 1; i < pl.m.n; ++i)
        if (std::llabs(pl.m.s0[i]) < std::llabs(pl.m.s0[ia])) ia = i;
    const bool tiled = transpose_tiled(pl);
    if (pl.m.n == 0) {
        p.e0 = 1;
        p.rest.n = 0;
    } else {
        p.e0 = pl.m.ext[0];
        p.a0 = pl.m.s0[0];
        p.c0 = pl.m.s1[0];
    }
    if (tiled) {
        p.e1 = pl.m.ext[ia];
        p.a1 = pl.m.s0[ia];
        p.c1 = pl.m.s1[ia];
        p.rest = without(pl.m, 0, ia);
        p.t0n = (p.e0 + TT - 1) / TT;
        p.t1n = (p.e1 + TT - 1) / TT;
        p.tg = std::min<int64_t>(p.t0n, 8);
        p.t0g = (p.t0n + p.tg - 1) / p.tg;
        p.items = p.t0g * p.t1n * count(p.rest);
    } else {
        // mode 1: the next mode by C increment (mode 1 of the plan), if any
        if (pl.m.n > 1) {
            p.e1 = pl.m.ext[1];
            p.a1 = pl.m.s0[1];
            p.c1 = pl.m.s1[1];
            p.rest = without(pl.m, 0, 1);
        } else {
            p.e1 = 1;
            p.rest.n = 0;
        }
        p.wide = p.e1 < 32 && p.e0 >= 1024;
        if (p.wide) {  // 1024 x 1 blocks
            p.t0n = (p.e0 + 1023) / 1024;
            p.t1n = p.e1;
        } else {  // 128 x 32 blocks
            p.t0n = (p.e0 + 127) / 128;
            p.t1n = (p.e1 + 31) / 32;
        }
        p.tg = std::min<int64_t>(p.t0n, 8);
        p.t0g = (p.t0n + p.tg - 1) / p.tg;
        p.items = p.t0g * p.t1n * count(p.rest);
    }
    switch (t) {
    case DT_F32: return transpose_typed<float>(p, tiled, num_sms, s);
    case DT_F64: return transpose_typed<double>(p, tiled, num_sms, s);
    case DT_C32: return transpose_typed<cf>(p, tiled, num_sms, s);
    case DT_C64: return transpose_typed<zd>(p, tiled, num_sms, s);
    case DT_BF16: return transpose_typed<uint16_t>(p, tiled, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t unit_operand(DType t, const void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_ones_mu);
    OnePtrs &o = g_ones[dev];
    if (!o.init) {
        void *q[5] = {};
        e = cudaGetSymbolAddress(&q[DT_F32], g_one_f32);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q[DT_F64], g_one_f64);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q[DT_C32], g_one_c32);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q[DT_C64], g_one_c64);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q[DT_BF16], g_one_bf16);
        if (e != cudaSuccess) return e;
        for (int i = 0; i < 5; ++i) o.p[i] = q[i];
        o.init = true;
    }
    *out = o.p[t];
    return cudaSuccess;
}

namespace {

// dst[r + R k] = conj(src[rowT[r] + kT[k]]): the operand's used elements in
// the planned (row, k) order, imaginary parts negated (a sign flip, exact).
template <class T>
__global__ void __launch_bounds__(256) conj_pack_kernel(const T *__restrict__ src, const int64_t *__restrict__ rowT,
                                                        const int64_t *__restrict__ kT, int64_t R, int64_t K,
                                                        T *__restrict__ dst)
{
    const int64_t n = R * K;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % R, k = i / R;
        T v = src[rowT[r] + kT[k]];
        v.im = -v.im;
        dst[i] = v;
    }
}

}  // namespace

cudaError_t launch_conj_pack(DType t, const void *src, const int64_t *rowT, const int64_t *kT, int64_t R, int64_t K,
                             void *dst, int num_sms, cudaStream_t s)
{
    const int64_t n = R * K;
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 16));
    if (t == DT_C32)
        conj_pack_kernel<cf><<<blocks, 256, 0, s>>>(static_cast<const cf *>(src), rowT, kT, R, K, static_cast<cf *>(dst));
    else if (t == DT_C64)
        conj_pack_kernel<zd><<<blocks, 256, 0, s>>>(static_cast<const zd *>(src), rowT, kT, R, K, static_cast<zd *>(dst));
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace gett

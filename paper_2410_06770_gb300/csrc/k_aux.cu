// k_aux.cu -- the tensor transpose and the unit operand of the tensor
// reduction (two of the operations the thesis lists as future work for a
// BLAS-like tensor interface, Sec. 8).
//
// Transpose: C[o permuted by PERM] <- alpha * A[o] + beta * C (or C += A).
// It is the contraction with a rank-0 B equal to 1, planned the same way (M =
// A's modes, s0 = A increment, s1 = C increment, ordered by C increment), but
// run by its own kernel: when A's smallest-increment mode is not C's, a
// 32 x 32 tile goes through shared memory so that the reads run along A's
// fastest mode and the writes along C's; otherwise both run along the same
// mode (a streaming copy).  HBM-bound: 8 bytes read + 8 written per double
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
// writes it with lanes along mode 0 (C's fastest).
template <class T>
__global__ void __launch_bounds__(256) transpose_tile_kernel(TransParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    __shared__ Acc tile[TT][TT + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const int64_t t0 = item % p.t0n;
        const int64_t r1 = item / p.t0n;
        const int64_t t1 = r1 % p.t1n;
        const int64_t ir = r1 / p.t1n;
        int64_t oa, oc;
        decode2(p.rest, ir, oa, oc);
        const T *A = static_cast<const T *>(p.A) + oa;
        Out *C = static_cast<Out *>(p.C) + oc;
        const int64_t i0 = t0 * TT, i1 = t1 * TT;
        __syncthreads();  // the previous tile has been written out
#pragma unroll
        for (int r = ty; r < TT; r += 8) {
            const int64_t x0 = i0 + r, x1 = i1 + tx;
            if (x0 < p.e0 && x1 < p.e1) tile[r][tx] = R::load(A + x0 * p.a0 + x1 * p.a1);
        }
        __syncthreads();
#pragma unroll
        for (int r = ty; r < TT; r += 8) {
            const int64_t x0 = i0 + tx, x1 = i1 + r;
            if (x0 < p.e0 && x1 < p.e1) trans_store<R>(C + x0 * p.c0 + x1 * p.c1, tile[tx][r], p.sc);
        }
    }
}

// A's and C's fastest modes coincide: stream along mode 0 in chunks of
// 256 x 4 elements, one chunk and one index of the other modes per item.
template <class T>
__global__ void __launch_bounds__(256) transpose_stream_kernel(TransParams p)
{
    using R = Tr<T>;
    using Out = typename R::Out;
    constexpr int U = 4, CH = 256 * U;
    for (int64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const int64_t t0 = item % p.t0n;
        const int64_t ir = item / p.t0n;
        int64_t oa, oc;
        decode2(p.rest, ir, oa, oc);
        const T *A = static_cast<const T *>(p.A) + oa;
        Out *C = static_cast<Out *>(p.C) + oc;
        typename R::Acc v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t x = t0 * CH + u * 256 + threadIdx.x;
            if (x < p.e0) v[u] = R::load(A + x * p.a0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t x = t0 * CH + u * 256 + threadIdx.x;
            if (x < p.e0) trans_store<R>(C + x * p.c0, v[u], p.sc);
        }
    }
}

// Drop modes i and j (i != j, either may be -1) from a list.
ModeList without(const ModeList &L, int i, int j)
{
    ModeList r{};
    for (int q = 0; q < L.n; ++q) {
        if (q == i || q == j) continue;
        r.ext[r.n] = L.ext[q];
        r.s0[r.n] = L.s0[q];
        r.s1[r.n] = L.s1[q];
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
    if (tiled) transpose_tile_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(p);
    else transpose_stream_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(p);
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
        p.items = p.t0n * p.t1n * count(p.rest);
    } else {
        if (pl.m.n > 0) p.rest = without(pl.m, 0, -1);
        p.t0n = (p.e0 + 1023) / 1024;
        p.t1n = 1;
        p.items = p.t0n * count(p.rest);
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

}  // namespace gett

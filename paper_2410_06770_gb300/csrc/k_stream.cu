// k_stream.cu -- HBM-streaming kernels for low-intensity contractions.
//
// OUTER: no contracted mode of extent > 1 (the thesis's "nothing
// contraction", Sec. 7): C[m,n] += A[m] * B[n].  Every C element is read and
// written once, so the kernel is bound by HBM bandwidth.  C is walked along
// its smallest-increment mode (the first mode of whichever class holds it),
// in runs of that mode; the operand that varies along the run is read along
// the same index, the other operand is one value per run.
//
// REDUCE: few output elements and long sums (the "scalar contraction" of
// Sec. 7 and its neighbours).  Pass 1 splits the flat contracted index
// space into a fixed number of contiguous ranges, one per CTA, and sums each
// range with a fixed per-thread stride, warp shuffles and a fixed cross-warp
// order; pass 2 adds the per-CTA partials in CTA order and accumulates into
// C.  The result is bitwise reproducible on a given GPU.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gett {

namespace {

struct OuterParams {
    const void *X;  // operand varying along the run
    const void *Y;  // operand fixed along the run
    void *C;
    ModeList xr;    // remaining modes of the run's class (s0: X inc, s1: C inc)
    ModeList y;     // modes of the other class (s0: Y inc, s1: C inc)
    int64_t e0, sx0, sc0;
    int64_t nxr, ny;
    int64_t chunk, nchunks, items;
};

template <class T, int NT>
__global__ void __launch_bounds__(NT) outer_kernel(OuterParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    constexpr int U = 4;
    const T *X = static_cast<const T *>(p.X);
    const T *Y = static_cast<const T *>(p.Y);
    Out *C = static_cast<Out *>(p.C);
    for (int64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        int64_t c = item % p.nchunks;
        int64_t rest = item / p.nchunks;
        int64_t ixr = rest % p.nxr;
        int64_t iy = rest / p.nxr;
        int64_t ox, ocx, oy, ocy;
        decode2(p.xr, ixr, ox, ocx);
        decode2(p.y, iy, oy, ocy);
        const Acc yv = R::load(Y + oy);
        const T *xb = X + ox;
        Out *cb = C + ocx + ocy;
        const int64_t x0 = c * p.chunk;
        const int64_t x1 = min(p.e0, x0 + p.chunk);
        for (int64_t x = x0 + threadIdx.x; x < x1; x += U * NT) {
            Acc xv[U], cv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int64_t xx = x + u * NT;
                if (xx < x1) {
                    xv[u] = R::load(xb + xx * p.sx0);
                    cv[u] = R::load_c(cb + xx * p.sc0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int64_t xx = x + u * NT;
                if (xx < x1) {
                    R::mac(cv[u], xv[u], yv);
                    R::store_c(cb + xx * p.sc0, cv[u]);
                }
            }
        }
    }
}

struct ReduceParams {
    const void *A;
    const void *B;
    void *C;
    ModeList m, n;   // output decode: s0 = operand inc, s1 = C inc
    ModeList kr;     // contracted modes after the first (s0: A inc, s1: B inc)
    int64_t e0, sa0, sb0;
    int64_t K, M, O;
    int G;
    void *partial;   // Acc[O * G]
};

// Sum over the CTA: warp shuffles, then warps in index order (fixed order).
template <class R, int NT>
__device__ __forceinline__ typename R::Acc block_sum(typename R::Acc v, typename R::Acc *red)
{
    using Acc = typename R::Acc;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = R::add(v, shfl_down(v, d));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    Acc s = red[0];
    for (int w = 1; w < NT / 32; ++w) s = R::add(s, red[w]);
    __syncthreads();
    return s;
}

template <class T, int NT>
__global__ void __launch_bounds__(NT) reduce_pass1(ReduceParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    __shared__ Acc red[NT / 32];
    const T *A = static_cast<const T *>(p.A);
    const T *B = static_cast<const T *>(p.B);
    Acc *P = static_cast<Acc *>(p.partial);
    const int g = blockIdx.x;
    const int64_t lo = p.K * g / p.G, hi = p.K * (g + 1) / p.G;
    for (int64_t o = 0; o < p.O; ++o) {
        int64_t oam, ocm, obn, ocn;
        decode2(p.m, o % p.M, oam, ocm);
        decode2(p.n, o / p.M, obn, ocn);
        Acc acc[4] = {R::zero(), R::zero(), R::zero(), R::zero()};
        int64_t k = lo;
        while (k < hi) {
            const int64_t k0 = k % p.e0;
            const int64_t seg = min(hi - k, p.e0 - k0);
            int64_t oa, ob;
            decode2(p.kr, k / p.e0, oa, ob);
            const T *a = A + oam + oa + k0 * p.sa0;
            const T *b = B + obn + ob + k0 * p.sb0;
            for (int64_t j = threadIdx.x; j < seg; j += 4 * NT) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int64_t jj = j + u * NT;
                    if (jj < seg) R::mac(acc[u], R::load(a + jj * p.sa0), R::load(b + jj * p.sb0));
                }
            }
            k += seg;
        }
        Acc v = R::add(R::add(acc[0], acc[1]), R::add(acc[2], acc[3]));
        Acc s = block_sum<R, NT>(v, red);
        if (threadIdx.x == 0) P[o * p.G + g] = s;
    }
}

template <class T, int NT>
__global__ void __launch_bounds__(NT) reduce_pass2(ReduceParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    __shared__ Acc red[NT / 32];
    const Acc *P = static_cast<const Acc *>(p.partial);
    const int64_t o = blockIdx.x;
    Acc v = R::zero();
    for (int i = threadIdx.x; i < p.G; i += NT) v = R::add(v, P[o * p.G + i]);
    Acc s = block_sum<R, NT>(v, red);
    if (threadIdx.x == 0) {
        int64_t oam, ocm, obn, ocn;
        decode2(p.m, o % p.M, oam, ocm);
        decode2(p.n, o / p.M, obn, ocn);
        Out *C = static_cast<Out *>(p.C);
        R::store_add(C + ocm + ocn, s);
    }
}

// Remove the first mode of a list.
ModeList drop_first(const ModeList &L)
{
    ModeList r{};
    r.n = L.n > 0 ? L.n - 1 : 0;
    for (int i = 0; i < r.n; ++i) {
        r.ext[i] = L.ext[i + 1];
        r.s0[i] = L.s0[i + 1];
        r.s1[i] = L.s1[i + 1];
    }
    return r;
}

int64_t prod(const ModeList &L)
{
    int64_t p = 1;
    for (int i = 0; i < L.n; ++i) p *= L.ext[i];
    return p;
}

size_t out_size(DType t) { return t == DT_BF16 ? 4 : dtype_size(t); }

template <class T>
cudaError_t outer_typed(const OuterParams &p, int num_sms, cudaStream_t s)
{
    constexpr int NT = 256;
    int64_t blocks = std::min<int64_t>(p.items, (int64_t)num_sms * 8);
    if (blocks < 1) blocks = 1;
    outer_kernel<T, NT><<<(unsigned)blocks, NT, 0, s>>>(p);
    return cudaGetLastError();
}

template <class T>
cudaError_t reduce_typed(const ReduceParams &p, cudaStream_t s)
{
    constexpr int NT = 256;
    reduce_pass1<T, NT><<<p.G, NT, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_pass2<T, NT><<<(unsigned)p.O, NT, 0, s>>>(p);
    return cudaGetLastError();
}

int reduce_grid(int num_sms) { return num_sms * 4; }

}  // namespace

cudaError_t launch_outer(const Plan &pl, DType t, const void *A, const void *B, void *C, int num_sms,
                         cudaStream_t s)
{
    const size_t esz = dtype_size(t);
    const char *Ab = static_cast<const char *>(A) + pl.offA * (int64_t)esz;
    const char *Bb = static_cast<const char *>(B) + pl.offB * (int64_t)esz;
    char *Cb = static_cast<char *>(C) + pl.offC * (int64_t)out_size(t);
    // the run follows C's smallest increment
    bool run_in_m;
    if (pl.m.n == 0) run_in_m = false;
    else if (pl.n.n == 0) run_in_m = true;
    else run_in_m = pl.m.s1[0] <= pl.n.s1[0];
    OuterParams p{};
    p.C = Cb;
    const ModeList &run = run_in_m ? pl.m : pl.n;
    const ModeList &oth = run_in_m ? pl.n : pl.m;
    p.X = run_in_m ? (const void *)Ab : (const void *)Bb;
    p.Y = run_in_m ? (const void *)Bb : (const void *)Ab;
    if (run.n > 0) {
        p.e0 = run.ext[0];
        p.sx0 = run.s0[0];
        p.sc0 = run.s1[0];
        p.xr = drop_first(run);
    } else {
        p.e0 = 1;
        p.sx0 = 0;
        p.sc0 = 0;
        p.xr.n = 0;
    }
    p.y = oth;
    p.nxr = prod(p.xr);
    p.ny = prod(p.y);
    p.chunk = 8192;
    p.nchunks = (p.e0 + p.chunk - 1) / p.chunk;
    p.items = p.nchunks * p.nxr * p.ny;
    switch (t) {
    case DT_F32: return outer_typed<float>(p, num_sms, s);
    case DT_F64: return outer_typed<double>(p, num_sms, s);
    case DT_C32: return outer_typed<cf>(p, num_sms, s);
    case DT_C64: return outer_typed<zd>(p, num_sms, s);
    case DT_BF16: return outer_typed<uint16_t>(p, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

size_t reduce_workspace_bytes(const Plan &p, DType t, int num_sms)
{
    size_t acc = (t == DT_BF16 || t == DT_F32) ? 4 : (t == DT_C64 ? 16 : 8);
    return acc * (size_t)p.M * p.N * reduce_grid(num_sms) + 256;
}

cudaError_t launch_reduce(const Plan &pl, DType t, const void *A, const void *B, void *C, int num_sms,
                          void *ws, cudaStream_t s)
{
    const size_t esz = dtype_size(t);
    ReduceParams p{};
    p.A = static_cast<const char *>(A) + pl.offA * (int64_t)esz;
    p.B = static_cast<const char *>(B) + pl.offB * (int64_t)esz;
    p.C = static_cast<char *>(C) + pl.offC * (int64_t)out_size(t);
    p.m = pl.m;
    p.n = pl.n;
    if (pl.k.n > 0) {
        p.e0 = pl.k.ext[0];
        p.sa0 = pl.k.s0[0];
        p.sb0 = pl.k.s1[0];
        p.kr = drop_first(pl.k);
    } else {
        p.e0 = 1;
        p.sa0 = p.sb0 = 0;
        p.kr.n = 0;
    }
    p.K = pl.K;
    p.M = pl.M;
    p.O = pl.M * pl.N;
    p.G = reduce_grid(num_sms);
    p.partial = ws;
    switch (t) {
    case DT_F32: return reduce_typed<float>(p, s);
    case DT_F64: return reduce_typed<double>(p, s);
    case DT_C32: return reduce_typed<cf>(p, s);
    case DT_C64: return reduce_typed<zd>(p, s);
    case DT_BF16: return reduce_typed<uint16_t>(p, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gett

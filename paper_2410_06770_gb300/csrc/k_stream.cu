// k_stream.cu -- HBM-streaming kernels for low-intensity contractions.
//
// OUTER: no contracted mode of extent > 1 (the thesis's "nothing
// contraction", Sec. 7): C[m,n] += A[m] * B[n]; also short sums (K <= 8):
// C[m,n] += sum_k A[m,k] B[k,n].  Every C element is read and written once
// (written only, in the scaled form with beta = 0), so the kernel is bound by
// HBM bandwidth.  C is walked along its smallest-increment mode (the first
// mode of whichever class holds it), in chunks of that mode; the operand that
// varies along the run is loaded once per element into registers and serves
// a group of 8 indices of the other class, whose operand values (alpha folded
// in) and C offsets sit in shared memory.
//
// SKINNY: one free class of at most 8 indices and a long sum (matrix-vector
// like).  Each of the (up to 8) short-class outputs of a long-class row is
// accumulated in registers.  When the long operand's contracted index has the
// smaller increment a warp reduces one row (lanes along k, warp shuffles);
// otherwise a CTA owns 32 consecutive rows (lanes along the row index) and its
// warps split the K range.  The CTA stages each chunk of its K range (the
// long operand's offsets and the short operand's values) in shared memory,
// so the inner loop's only global loads are the long operand's, several in
// flight per thread.  The grid also splits K into slices so that about
// sixteen CTAs per SM stream the long operand; slice partials are added into
// C in slice order by a second kernel.  In FP64 on this GPU the kernel is
// bound by the FP64 FMA rate once S >= 2 (2 S flops per 8-byte element).
//
// REDUCE: few output elements and long sums (the "scalar contraction" of
// Sec. 7 and its neighbours).  Pass 1 splits the flat contracted index
// space into 8 contiguous ranges per SM, one per CTA, and sums each range
// with a fixed per-thread stride (4 loads of each operand in flight, unit
// stride specialised), warp shuffles and a fixed cross-warp order; pass 2
// adds the per-CTA partials in CTA order and applies the epilogue to C.  The
// result is bitwise reproducible on a given GPU.
//
// Every kernel here applies the plan's Scale in its epilogue (C += v, or
// alpha v + beta C, or alpha v without reading C).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace gett {

namespace {

constexpr int OUTER_MAX_K = 8;

struct OuterParams {
    const void *X;  // operand varying along the run
    const void *Y;  // operand fixed along the run
    void *C;
    ModeList xr;    // remaining modes of the run's class (s0: X inc, s1: C inc)
    ModeList y;     // modes of the other class (s0: Y inc, s1: C inc)
    int64_t e0, sx0, sc0;
    int64_t nxr, ny;
    int64_t chunk, nchunks, items;
    int nk;                       // contracted length (1 for a pure outer product)
    int64_t kx[OUTER_MAX_K];      // offsets of contracted index k in X
    int64_t ky[OUTER_MAX_K];      // and in Y
    Scale sc;                     // SCALE_AX: C is written without being read
};

// Each work item is one chunk of the run, one index of the run class's other
// modes and a group of OUTER_NY consecutive indices of the other class: the
// run operand's values are loaded once per group (registers), the group's
// operand values and C offsets sit in shared memory.  FP64 arithmetic is
// scarce on this GPU (about 0.6 T operations/s, so the outer product's one
// FMA per element is within 1.5x of the HBM time): the scaled forms cost no
// extra operation per element beyond beta * C.
constexpr int OUTER_NY = 8;

template <class T, int NT, int KM>
__global__ void __launch_bounds__(NT) outer_kernel(OuterParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    constexpr int U = sizeof(Acc) > 8 ? 2 : 4;
    __shared__ Acc sY[OUTER_NY][KM];
    __shared__ int64_t sOcy[OUTER_NY];
    const T *X = static_cast<const T *>(p.X);
    const T *Y = static_cast<const T *>(p.Y);
    Out *C = static_cast<Out *>(p.C);
    const bool acc_c = p.sc.mode == SCALE_ACC;
    for (int64_t item = blockIdx.x; item < p.items; item += gridDim.x) {
        const int64_t c = item % p.nchunks;
        const int64_t rest = item / p.nchunks;
        const int64_t ixr = rest % p.nxr;
        const int64_t g = rest / p.nxr;
        const int nyg = (int)min((int64_t)OUTER_NY, p.ny - g * OUTER_NY);
        int64_t ox, ocx;
        decode2(p.xr, ixr, ox, ocx);
        __syncthreads();  // the previous item's readers are done with sY
        if (threadIdx.x < OUTER_NY) {
            const int j = threadIdx.x;
            int64_t oy = 0, ocy = 0;
            if (j < nyg) decode2(p.y, g * OUTER_NY + j, oy, ocy);
            sOcy[j] = ocy;
            // the scaled forms fold alpha into the staged values, so no
            // per-element multiply by alpha is needed
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                Acc v = (j < nyg && k < p.nk) ? R::load(Y + oy + p.ky[k]) : R::zero();
                sY[j][k] = acc_c ? v : scale_by(v, p.sc.ar, p.sc.ai);
            }
        }
        __syncthreads();
        const T *xb = X + ox;
        Out *cb = C + ocx;
        const int64_t x0 = c * p.chunk;
        const int64_t x1 = min(p.e0, x0 + p.chunk);
        for (int64_t x = x0 + threadIdx.x; x < x1; x += U * NT) {
            Acc xv[U][KM];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t xx = x + u * NT;
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    xv[u][k] = (k < p.nk && xx < x1) ? R::load(xb + xx * p.sx0 + p.kx[k]) : R::zero();
            }
            for (int j = 0; j < nyg; ++j) {
                Out *cj = cb + sOcy[j];
                // C's contribution first: C (accumulate), beta * C, or nothing
                Acc cv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t xx = x + u * NT;
                    cv[u] = R::zero();
                    if (xx < x1 && acc_c) cv[u] = R::load_c(cj + xx * p.sc0);
                    else if (xx < x1 && p.sc.mode == SCALE_AXPBY)
                        cv[u] = scale_by(R::load_c(cj + xx * p.sc0), p.sc.br, p.sc.bi);
                }
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (k >= p.nk) break;
                    const Acc yk = sY[j][k];
#pragma unroll
                    for (int u = 0; u < U; ++u) R::mac(cv[u], xv[u][k], yk);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t xx = x + u * NT;
                    if (xx < x1) R::store_c(cj + xx * p.sc0, cv[u]);
                }
            }
        }
    }
}

constexpr int SKINNY_MAX_S = 8;

struct SkinnyParams {
    const void *X;  // operand of the long free class (R rows)
    const void *Y;  // operand of the short class (S <= 8 columns)
    void *C;
    const int64_t *rowX, *rowC;   // [R] offsets of the long class in X and C
    const int64_t *kX, *kY;       // [K] offsets of the contracted class
    int64_t colY[SKINNY_MAX_S], colC[SKINNY_MAX_S];
    int64_t R, K;
    int S;
    int splits;                   // K slices (grid.y)
    int64_t kps;                  // K per slice
    void *partial;                // splits > 1: Acc[splits][S][R]
    Scale sc;
};

template <class Rt>
__device__ __forceinline__ void skinny_emit(const SkinnyParams &p, int64_t r, int s, typename Rt::Acc v)
{
    using Acc = typename Rt::Acc;
    if (p.splits > 1)
        static_cast<Acc *>(p.partial)[((int64_t)blockIdx.y * p.S + s) * p.R + r] = v;
    else
        epi_store<Rt>(static_cast<typename Rt::Out *>(p.C) + p.rowC[r] + p.colC[s], v, p.sc);
}

// K chunk staged in shared memory by each SKINNY CTA: 2 KB of Acc values
// per short-class column (256 doubles).
template <class Acc>
__host__ __device__ constexpr int skinny_kc()
{
    return (int)(2048 / sizeof(Acc));
}

template <class Acc, int SM>
__host__ __device__ constexpr size_t skinny_smem_bytes(bool with_red)
{
    return (size_t)skinny_kc<Acc>() * (sizeof(int64_t) + SM * sizeof(Acc)) > (with_red ? 8 * SM * 32 * sizeof(Acc) : 0)
               ? (size_t)skinny_kc<Acc>() * (sizeof(int64_t) + SM * sizeof(Acc))
               : 8 * SM * 32 * sizeof(Acc);
}

// Stage k = kc .. kc+n-1 of the slice: koff[i] = offset of k in X, yv[i][s] =
// Y element of short-class column s at k.  The whole CTA loads (coalesced
// reads of the tables), so the inner loops read only X from global memory.
template <class T, int SM>
__device__ __forceinline__ void skinny_stage(const SkinnyParams &p, int64_t kc, int n, int64_t *koff,
                                             typename Tr<T>::Acc *yv)
{
    using Rt = Tr<T>;
    const T *Y = static_cast<const T *>(p.Y);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        koff[i] = p.kX[kc + i];
        const int64_t yk = p.kY[kc + i];
#pragma unroll
        for (int s = 0; s < SM; ++s)
            if (s < p.S) yv[i * SM + s] = Rt::load(Y + p.colY[s] + yk);
    }
}

// Rows contiguous in X: a CTA owns 32 rows (lane = row); its 8 warps take
// interleaved k of each staged chunk of the CTA's K slice, then add their
// sums in warp order.  SM >= S bounds the register-held columns.
template <class T, int SM>
__global__ void __launch_bounds__(256) skinny_rows_kernel(SkinnyParams p)
{
    using Rt = Tr<T>;
    using Acc = typename Rt::Acc;
    constexpr int KC = skinny_kc<Acc>();
    __shared__ __align__(16) unsigned char sbuf[skinny_smem_bytes<Acc, SM>(true)];
    int64_t *koff = reinterpret_cast<int64_t *>(sbuf);
    Acc *yv = reinterpret_cast<Acc *>(sbuf + KC * sizeof(int64_t));
    const T *X = static_cast<const T *>(p.X);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    const bool ok = r < p.R;
    const T *xr = X + (ok ? p.rowX[r] : 0);
    const int64_t k0 = (int64_t)blockIdx.y * p.kps, k1 = min(p.K, k0 + p.kps);
    Acc acc[SM];
#pragma unroll
    for (int s = 0; s < SM; ++s) acc[s] = Rt::zero();
    for (int64_t kc = k0; kc < k1; kc += KC) {
        const int n = (int)min((int64_t)KC, k1 - kc);
        __syncthreads();
        skinny_stage<T, SM>(p, kc, n, koff, yv);
        __syncthreads();
        if (!ok) continue;
        int i = warp;
        for (; i + 24 < n; i += 32) {  // four independent loads in flight
            Acc xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = Rt::load(xr + koff[i + 8 * u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int s = 0; s < SM; ++s)
                    if (s < p.S) Rt::mac(acc[s], xv[u], yv[(i + 8 * u) * SM + s]);
        }
        for (; i < n; i += 8) {
            const Acc xv = Rt::load(xr + koff[i]);
#pragma unroll
            for (int s = 0; s < SM; ++s)
                if (s < p.S) Rt::mac(acc[s], xv, yv[i * SM + s]);
        }
    }
    __syncthreads();
    Acc *red = reinterpret_cast<Acc *>(sbuf);  // [8][SM][32]
#pragma unroll
    for (int s = 0; s < SM; ++s) red[(warp * SM + s) * 32 + lane] = acc[s];
    __syncthreads();
    if (warp == 0 && ok) {
#pragma unroll
        for (int s = 0; s < SM; ++s) {
            if (s >= p.S) break;
            Acc v = red[s * 32 + lane];
            for (int w = 1; w < 8; ++w) v = Rt::add(v, red[(w * SM + s) * 32 + lane]);
            skinny_emit<Rt>(p, r, s, v);
        }
    }
}

// K contiguous in X: one warp per row (8 rows per CTA), lanes along k of each
// staged chunk of the CTA's K slice, warp shuffles.
template <class T, int SM>
__global__ void __launch_bounds__(256) skinny_warp_kernel(SkinnyParams p)
{
    using Rt = Tr<T>;
    using Acc = typename Rt::Acc;
    constexpr int KC = skinny_kc<Acc>();
    __shared__ __align__(16) unsigned char sbuf[skinny_smem_bytes<Acc, SM>(false)];
    int64_t *koff = reinterpret_cast<int64_t *>(sbuf);
    Acc *yv = reinterpret_cast<Acc *>(sbuf + KC * sizeof(int64_t));
    const T *X = static_cast<const T *>(p.X);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 8 + warp;
    const bool ok = r < p.R;
    const T *xr = X + (ok ? p.rowX[r] : 0);
    const int64_t k0 = (int64_t)blockIdx.y * p.kps, k1 = min(p.K, k0 + p.kps);
    Acc acc[SM];
#pragma unroll
    for (int s = 0; s < SM; ++s) acc[s] = Rt::zero();
    for (int64_t kc = k0; kc < k1; kc += KC) {
        const int n = (int)min((int64_t)KC, k1 - kc);
        __syncthreads();
        skinny_stage<T, SM>(p, kc, n, koff, yv);
        __syncthreads();
        if (!ok) continue;
        int i = lane;
        for (; i + 96 < n; i += 128) {
            Acc xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = Rt::load(xr + koff[i + 32 * u]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int s = 0; s < SM; ++s)
                    if (s < p.S) Rt::mac(acc[s], xv[u], yv[(i + 32 * u) * SM + s]);
        }
        for (; i < n; i += 32) {
            const Acc xv = Rt::load(xr + koff[i]);
#pragma unroll
            for (int s = 0; s < SM; ++s)
                if (s < p.S) Rt::mac(acc[s], xv, yv[i * SM + s]);
        }
    }
    if (!ok) return;
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        if (s >= p.S) break;
        Acc v = acc[s];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v = Rt::add(v, shfl_down(v, d));
        if (lane == 0) skinny_emit<Rt>(p, r, s, v);
    }
}

// C <- beta * C over the output index space (the scaled form when alpha == 0
// or the sum is empty); beta == 0 writes zeros without reading C.
template <class T>
__global__ void scale_c_kernel(ModeList m, ModeList n, int64_t M, int64_t MN, typename Tr<T>::Out *C, Scale sc)
{
    using R = Tr<T>;
    const bool zero = sc.br == 0.0 && sc.bi == 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a, cm, b, cn;
        decode2(m, i % M, a, cm);
        decode2(n, i / M, b, cn);
        typename R::Out *c = C + cm + cn;
        if (zero) R::store_c(c, R::zero());
        else R::store_c(c, scale_by(R::load_c(c), sc.br, sc.bi));
    }
}

// C[rowC[r] + colC[s]] += sum of the K-slice partials, slices in order.
template <class T>
__global__ void skinny_reduce_kernel(SkinnyParams p)
{
    using Rt = Tr<T>;
    using Acc = typename Rt::Acc;
    const Acc *P = static_cast<const Acc *>(p.partial);
    const int64_t SR = (int64_t)p.S * p.R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < SR; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % p.R, s = i / p.R;
        Acc v = P[i];
        for (int j = 1; j < p.splits; ++j) v = Rt::add(v, P[(int64_t)j * SR + i]);
        epi_store<Rt>(static_cast<typename Rt::Out *>(p.C) + p.rowC[r] + p.colC[s], v, p.sc);
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
    Scale sc;
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

// UNIT: both operands have increment 1 along the first contracted mode.
// Otherwise the addresses advance by pointer increments (no per-load
// multiply).  Each thread keeps four loads of each operand in flight.
template <class T, int NT, bool UNIT>
__global__ void __launch_bounds__(NT) reduce_pass1(ReduceParams p)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    constexpr int U = 4;
    __shared__ Acc red[NT / 32];
    const T *A = static_cast<const T *>(p.A);
    const T *B = static_cast<const T *>(p.B);
    Acc *P = static_cast<Acc *>(p.partial);
    const int g = blockIdx.x;
    const int64_t lo = p.K * g / p.G, hi = p.K * (g + 1) / p.G;
    const int64_t sa = UNIT ? 1 : p.sa0, sb = UNIT ? 1 : p.sb0;
    for (int64_t o = 0; o < p.O; ++o) {
        int64_t oam, ocm, obn, ocn;
        decode2(p.m, o % p.M, oam, ocm);
        decode2(p.n, o / p.M, obn, ocn);
        Acc acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = R::zero();
        int64_t k = lo;
        while (k < hi) {
            const int64_t k0 = k % p.e0;
            const int64_t seg = min(hi - k, p.e0 - k0);
            int64_t oa, ob;
            decode2(p.kr, k / p.e0, oa, ob);
            const T *a = A + oam + oa + (k0 + threadIdx.x) * sa;
            const T *b = B + obn + ob + (k0 + threadIdx.x) * sb;
            const int64_t da = (int64_t)NT * sa, db = (int64_t)NT * sb;
            for (int64_t j = threadIdx.x; j < seg; j += U * NT) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (j + u * NT < seg) R::mac(acc[u], R::load(a + u * da), R::load(b + u * db));
                a += U * da;
                b += U * db;
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
        epi_store<R>(C + ocm + ocn, s, p.sc);
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
    // KM >= nk bounds the contracted values held per run element
    if (p.nk <= 1) outer_kernel<T, NT, 1><<<(unsigned)blocks, NT, 0, s>>>(p);
    else if (p.nk <= 2) outer_kernel<T, NT, 2><<<(unsigned)blocks, NT, 0, s>>>(p);
    else if (p.nk <= 4) outer_kernel<T, NT, 4><<<(unsigned)blocks, NT, 0, s>>>(p);
    else outer_kernel<T, NT, OUTER_MAX_K><<<(unsigned)blocks, NT, 0, s>>>(p);
    return cudaGetLastError();
}

template <class T>
cudaError_t reduce_typed(const ReduceParams &p, cudaStream_t s)
{
    constexpr int NT = 256;
    if (p.sa0 == 1 && p.sb0 == 1) reduce_pass1<T, NT, true><<<p.G, NT, 0, s>>>(p);
    else reduce_pass1<T, NT, false><<<p.G, NT, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_pass2<T, NT><<<(unsigned)p.O, NT, 0, s>>>(p);
    return cudaGetLastError();
}

int reduce_grid(int num_sms) { return num_sms * 8; }

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
    p.sc = pl.sc;
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
    // contracted offsets (first mode fastest), at most OUTER_MAX_K of them
    if (pl.K > OUTER_MAX_K) return cudaErrorInvalidValue;
    p.nk = (int)pl.K;
    for (int64_t k = 0; k < pl.K; ++k) {
        int64_t r = k, oa = 0, ob = 0;
        for (int i = 0; i < pl.k.n; ++i) {
            const int64_t x = r % pl.k.ext[i];
            r /= pl.k.ext[i];
            oa += x * pl.k.s0[i];
            ob += x * pl.k.s1[i];
        }
        p.kx[k] = run_in_m ? oa : ob;
        p.ky[k] = run_in_m ? ob : oa;
    }
    p.nxr = prod(p.xr);
    p.ny = prod(p.y);
    p.chunk = 8192;
    p.nchunks = (p.e0 + p.chunk - 1) / p.chunk;
    p.items = p.nchunks * p.nxr * ((p.ny + OUTER_NY - 1) / OUTER_NY);
    switch (t) {
    case DT_F32: return outer_typed<float>(p, num_sms, s);
    case DT_F64: return outer_typed<double>(p, num_sms, s);
    case DT_C32: return outer_typed<cf>(p, num_sms, s);
    case DT_C64: return outer_typed<zd>(p, num_sms, s);
    case DT_BF16: return outer_typed<uint16_t>(p, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

// K slices of the SKINNY kernel: enough CTAs for sixteen per SM, each slice
// at least 1024 long.
int skinny_splits(const Plan &p, bool rows_mode, int num_sms)
{
    const int64_t R = std::max(p.M, p.N);
    const int64_t row_tiles = rows_mode ? (R + 31) / 32 : (R + 7) / 8;
    int64_t want = (16LL * num_sms + row_tiles - 1) / row_tiles;
    want = std::min<int64_t>(want, std::max<int64_t>(1, p.K / 1024));
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, 1024));
}

bool skinny_rows_mode(const Plan &pl)
{
    const bool short_is_n = pl.N <= pl.M;
    const ModeList &lg = short_is_n ? pl.m : pl.n;
    const int64_t s_row = lg.n ? (lg.s0[0] < 0 ? -lg.s0[0] : lg.s0[0]) : 0;
    const int64_t s_k0 = pl.k.n ? (short_is_n ? pl.k.s0[0] : pl.k.s1[0]) : 0;
    const int64_t sk = s_k0 < 0 ? -s_k0 : s_k0;
    return !(s_row == 0 || (sk != 0 && sk < s_row));
}

size_t skinny_workspace_bytes(const Plan &p, DType t, int num_sms)
{
    const size_t acc = (t == DT_BF16 || t == DT_F32) ? 4 : (t == DT_C64 ? 16 : 8);
    const int sp = skinny_splits(p, skinny_rows_mode(p), num_sms);
    const int64_t R = std::max(p.M, p.N), S = std::min(p.M, p.N);
    size_t bytes = sizeof(int64_t) * 2 * (size_t)(p.M + p.N + p.K) + 256;
    if (sp > 1) bytes += acc * (size_t)sp * S * R + 256;
    return bytes;
}

bool skinny_applicable(const Plan &p)
{
    return std::min(p.M, p.N) <= SKINNY_MAX_S && p.K > 1;
}

template <class T, int SM>
void skinny_main(const SkinnyParams &p, bool rows_mode, cudaStream_t s)
{
    if (rows_mode) {
        dim3 grid((unsigned)((p.R + 31) / 32), (unsigned)p.splits);
        skinny_rows_kernel<T, SM><<<grid, 256, 0, s>>>(p);
    } else {
        dim3 grid((unsigned)((p.R + 7) / 8), (unsigned)p.splits);
        skinny_warp_kernel<T, SM><<<grid, 256, 0, s>>>(p);
    }
}

template <class T>
cudaError_t skinny_typed(const SkinnyParams &p, bool rows_mode, int num_sms, cudaStream_t s)
{
    if (p.S <= 1) skinny_main<T, 1>(p, rows_mode, s);
    else if (p.S <= 2) skinny_main<T, 2>(p, rows_mode, s);
    else if (p.S <= 4) skinny_main<T, 4>(p, rows_mode, s);
    else skinny_main<T, 8>(p, rows_mode, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || p.splits == 1) return e;
    const int64_t SR = (int64_t)p.S * p.R;
    skinny_reduce_kernel<T><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((SR + 255) / 256, num_sms * 8)), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_skinny(const Plan &pl, DType t, const void *A, const void *B, void *C, int num_sms, void *ws,
                          cudaStream_t s)
{
    if (!skinny_applicable(pl)) return cudaErrorInvalidValue;
    int64_t *tab = static_cast<int64_t *>(ws);
    int64_t *rowA = tab, *rowC = rowA + pl.M, *colB = rowC + pl.M, *colC = colB + pl.N;
    int64_t *kA = colC + pl.N, *kB = kA + pl.K;
    cudaError_t e = launch_build_tables(pl, rowA, rowC, colB, colC, kA, kB, s);
    if (e != cudaSuccess) return e;
    const size_t esz = dtype_size(t);
    const char *Ab = static_cast<const char *>(A) + pl.offA * (int64_t)esz;
    const char *Bb = static_cast<const char *>(B) + pl.offB * (int64_t)esz;
    SkinnyParams p{};
    p.sc = pl.sc;
    p.C = static_cast<char *>(C) + pl.offC * (int64_t)out_size(t);
    p.K = pl.K;
    // the short class becomes the register-held columns
    const bool short_is_n = pl.N <= pl.M;
    const ModeList &sh = short_is_n ? pl.n : pl.m;
    p.S = (int)(short_is_n ? pl.N : pl.M);
    for (int64_t j = 0; j < p.S; ++j) {
        int64_t r = j, a = 0, c = 0;
        for (int i = 0; i < sh.n; ++i) {
            const int64_t x = r % sh.ext[i];
            r /= sh.ext[i];
            a += x * sh.s0[i];
            c += x * sh.s1[i];
        }
        p.colY[j] = a;
        p.colC[j] = c;
    }
    if (short_is_n) {
        p.X = Ab;
        p.Y = Bb;
        p.rowX = rowA;
        p.rowC = rowC;
        p.kX = kA;
        p.kY = kB;
        p.R = pl.M;
    } else {
        p.X = Bb;
        p.Y = Ab;
        p.rowX = colB;
        p.rowC = colC;
        p.kX = kB;
        p.kY = kA;
        p.R = pl.N;
    }
    const bool rows_mode = skinny_rows_mode(pl);
    p.splits = skinny_splits(pl, rows_mode, num_sms);
    p.kps = (pl.K + p.splits - 1) / p.splits;
    p.splits = (int)((pl.K + p.kps - 1) / p.kps);
    p.partial = p.splits > 1 ? static_cast<char *>(ws) + ((sizeof(int64_t) * 2 * (size_t)(pl.M + pl.N + pl.K) + 255) & ~size_t(255))
                             : nullptr;
    switch (t) {
    case DT_F32: return skinny_typed<float>(p, rows_mode, num_sms, s);
    case DT_F64: return skinny_typed<double>(p, rows_mode, num_sms, s);
    case DT_C32: return skinny_typed<cf>(p, rows_mode, num_sms, s);
    case DT_C64: return skinny_typed<zd>(p, rows_mode, num_sms, s);
    case DT_BF16: return skinny_typed<uint16_t>(p, rows_mode, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_scale_c(const Plan &pl, DType t, void *C, int num_sms, cudaStream_t s)
{
    const int64_t MN = pl.M * pl.N;
    if (MN == 0) return cudaSuccess;
    char *Cb = static_cast<char *>(C) + pl.offC * (int64_t)out_size(t);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((MN + 255) / 256, 8LL * num_sms));
    switch (t) {
    case DT_F32: scale_c_kernel<float><<<blocks, 256, 0, s>>>(pl.m, pl.n, pl.M, MN, (float *)Cb, pl.sc); break;
    case DT_F64: scale_c_kernel<double><<<blocks, 256, 0, s>>>(pl.m, pl.n, pl.M, MN, (double *)Cb, pl.sc); break;
    case DT_C32: scale_c_kernel<cf><<<blocks, 256, 0, s>>>(pl.m, pl.n, pl.M, MN, (cf *)Cb, pl.sc); break;
    case DT_C64: scale_c_kernel<zd><<<blocks, 256, 0, s>>>(pl.m, pl.n, pl.M, MN, (zd *)Cb, pl.sc); break;
    case DT_BF16: scale_c_kernel<uint16_t><<<blocks, 256, 0, s>>>(pl.m, pl.n, pl.M, MN, (float *)Cb, pl.sc); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
    p.sc = pl.sc;
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

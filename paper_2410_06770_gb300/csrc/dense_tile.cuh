// dense_tile.cuh -- one BM x BN output tile of C[m,n] += sum_k A[m,k] B[k,n]
// (or the scaled form alpha * sum + beta * C)
// on CUDA cores, with A, B and C addressed through the planner's offset
// tables.  Used by the single-call dense kernel and the batched persistent
// kernel.
//
// Staging: each thread prefetches its share of the next K tile into
// registers while the current tile is multiplied from shared memory (double
// buffered).  Threads walk the tile along whichever index has the smaller
// increment so global loads coalesce.  The epilogue maps lanes along the
// index with C's smaller increment so the read-modify-write of C coalesces.
#pragma once

#include "common.cuh"

namespace gett {

struct TileArgs {
    const void *A;
    const void *B;
    void *C;
    const int64_t *rowA, *rowC, *colB, *colC, *kA, *kB;
    int64_t M, N;
    int64_t m0, n0;      // tile origin
    int64_t kbeg, kend;  // contracted range of this tile
    int a_m_fast, b_n_fast, c_m_fast;
    void *partial;       // if set: write the tile (Acc) here instead of adding into C
    Scale sc;            // how the tile meets C (SCALE_ACC: C += tile)
};

// sA: 2*BK*BM, sB: 2*BK*BN shared arrays; sRowA: BM, sColB: BN.
template <class T, int BM, int BN, int BK, int TM, int TN>
__device__ __forceinline__ void dense_tile(const TileArgs &p, typename Tr<T>::Acc *sA, typename Tr<T>::Acc *sB,
                                           int64_t *sRowA, int64_t *sColB)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    using Out = typename R::Out;
    constexpr int NT = (BM / TM) * (BN / TN);
    constexpr int LA = BM * BK / NT;
    constexpr int LB = BN * BK / NT;
    static_assert(LA * NT == BM * BK && LB * NT == BN * BK, "tile/threads mismatch");

    const int tid = threadIdx.x;
    const int64_t m0 = p.m0, n0 = p.n0, kbeg = p.kbeg, kend = p.kend;

    const T *A = static_cast<const T *>(p.A);
    const T *B = static_cast<const T *>(p.B);

    for (int i = tid; i < BM; i += NT) sRowA[i] = (m0 + i < p.M) ? p.rowA[m0 + i] : 0;
    for (int i = tid; i < BN; i += NT) sColB[i] = (n0 + i < p.N) ? p.colB[n0 + i] : 0;
    __syncthreads();

    Acc ra[LA], rb[LB];
    auto load_tile = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            int e = tid + r * NT;
            int mm, kk;
            if (p.a_m_fast) { mm = e % BM; kk = e / BM; }
            else { kk = e % BK; mm = e / BK; }
            int64_t k = k0 + kk;
            ra[r] = (m0 + mm < p.M && k < kend) ? R::load(A + sRowA[mm] + p.kA[k]) : R::zero();
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            int e = tid + r * NT;
            int nn, kk;
            if (p.b_n_fast) { nn = e % BN; kk = e / BN; }
            else { kk = e % BK; nn = e / BK; }
            int64_t k = k0 + kk;
            rb[r] = (n0 + nn < p.N && k < kend) ? R::load(B + sColB[nn] + p.kB[k]) : R::zero();
        }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            int e = tid + r * NT;
            int mm, kk;
            if (p.a_m_fast) { mm = e % BM; kk = e / BM; }
            else { kk = e % BK; mm = e / BK; }
            sA[(buf * BK + kk) * BM + mm] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            int e = tid + r * NT;
            int nn, kk;
            if (p.b_n_fast) { nn = e % BN; kk = e / BN; }
            else { kk = e % BK; nn = e / BK; }
            sB[(buf * BK + kk) * BN + nn] = rb[r];
        }
    };

    int tm, tn;
    if (p.c_m_fast) { tm = tid % (BM / TM); tn = tid / (BM / TM); }
    else { tn = tid % (BN / TN); tm = tid / (BN / TN); }

    Acc acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = R::zero();

    const int64_t nkt = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
    if (nkt > 0) {
        load_tile(kbeg);
        store_tile(0);
        __syncthreads();
    }
    for (int64_t kt = 0; kt < nkt; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nkt) load_tile(kbeg + (kt + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Acc a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = sA[(cur * BK + kk) * BM + tm + i * (BM / TM)];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = sB[(cur * BK + kk) * BN + tn + j * (BN / TN)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) R::mac(acc[i][j], a[i], b[j]);
        }
        if (kt + 1 < nkt) store_tile(cur ^ 1);
        __syncthreads();
    }

    // epilogue
    if (p.partial) {
        Acc *P = static_cast<Acc *>(p.partial);
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int64_t m = m0 + tm + i * (BM / TM);
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                int64_t n = n0 + tn + j * (BN / TN);
                if (m < p.M && n < p.N) P[p.c_m_fast ? n * p.M + m : m * p.N + n] = acc[i][j];
            }
        }
        return;
    }
    Out *C = static_cast<Out *>(p.C);
    int64_t rc[TM], cc[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int64_t m = m0 + tm + i * (BM / TM);
        rc[i] = m < p.M ? p.rowC[m] : 0;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        int64_t n = n0 + tn + j * (BN / TN);
        cc[j] = n < p.N ? p.colC[n] : 0;
    }
    if (p.sc.mode == SCALE_ACC) {
        // every load of C before any store when a thread's outputs take at
        // most 128 bytes (larger register tiles, whose tiles run long sums,
        // keep the plain loop): a load after a store through another
        // pointer cannot be hoisted above it, so interleaved
        // read-modify-writes would each pay a full round trip; the tile's
        // outputs are distinct (C is injective)
        if constexpr (sizeof(Acc) * TM * TN > 128) {
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                int64_t m = m0 + tm + i * (BM / TM);
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    int64_t n = n0 + tn + j * (BN / TN);
                    if (m < p.M && n < p.N) R::store_add(C + rc[i] + cc[j], acc[i][j]);
                }
            }
        } else {
            Acc cv[TM][TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const bool vm = m0 + tm + i * (BM / TM) < p.M;
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    cv[i][j] = vm && n0 + tn + j * (BN / TN) < p.N ? R::load_c(C + rc[i] + cc[j]) : R::zero();
            }
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const bool vm = m0 + tm + i * (BM / TM) < p.M;
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    if (vm && n0 + tn + j * (BN / TN) < p.N)
                        R::store_c(C + rc[i] + cc[j], R::add(cv[i][j], acc[i][j]));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int64_t m = m0 + tm + i * (BM / TM);
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                int64_t n = n0 + tn + j * (BN / TN);
                if (m < p.M && n < p.N) epi_store<R>(C + rc[i] + cc[j], acc[i][j], p.sc);
            }
        }
    }
}

}  // namespace gett

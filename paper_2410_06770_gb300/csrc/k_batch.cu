// k_batch.cu -- thousands of xGETT contractions in one batched launch.
//
// gett_batch_create plans every problem on the host (validation, squeeze,
// flips, fusion -- the same planner as single calls), picks a configuration
// per problem (heuristic, fixed, caller table, tuning database or learned
// model: a tile shape and a method), decodes the offset tables of all
// problems into one buffer, and builds one work list per method, sorted by
// decreasing cost so long items start first.  This file holds the gathered
// tiles (persistent CTAs taking items from an atomic counter and computing a
// tile through the offset tables), the short sums (their own kernel and
// counter), the ordered reduction of K-slice partials and the launch itself:
// the method chains run as concurrent branches of one stream-ordered (and
// graph-capturable) launch.  Tiles whose K extent would make them far longer
// than a CTA's average share are split into K slices; slices write partial
// tiles that the reduction adds into C in slice order.  Every output element
// is therefore summed in a fixed order and results do not depend on
// scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "batch_common.cuh"
#include "dense_tile.cuh"
#include "gett_batch.h"
#include "internal.h"
#include "learn.h"
#include "select.h"
#include "gett_tune.h"
#include "tunedb.h"

namespace gett {

namespace {

// Resident CTAs per SM: the gather kernel is compiled for 2, 3 and 4 (register caps
// 128, 80 and 64 per thread; the lower caps trade spills for warps in
// flight).  The gathers are latency bound, so warps win: on the 4096-problem
// workload 2 / 3 / 4 CTAs per SM take 8.74 / 7.97 / 7.37 ms.
constexpr int kCtasPerSm = 4;
constexpr int kMaxCtasPerSm = 4;

// A short-sum problem (K <= 8, one slice) takes its outputs straight from
// gathered loads; several of its tiles form one work item so that a few
// tens of thousands of outputs share the item's fixed latency.
__host__ __device__ inline bool batch_direct(const BatchProb &pr) { return pr.K <= 8 && pr.splits == 1; }

// work items of a problem: tile runs (short sums) or tiles x K slices
inline int batch_items(const BatchProb &pr)
{
    const int nt = pr.tiles_m * pr.tiles_n;
    return batch_direct(pr) ? (nt + pr.tpi - 1) / pr.tpi : nt * pr.splits;
}

// K offsets of one slice staged in shared memory (at most kStageK entries per
// operand): a K step then waits for one global round trip (the operands)
// instead of two (the offset table, then the operands).
constexpr int kStageK = 1536;
constexpr int kGatherStages = 2;  // cp.async ring of the float gather tiles (double buffer)

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, bool valid)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Gathered tile of float operands with the K offsets of its slice in shared
// memory: every element's address comes from shared memory, so the tile is
// staged by cp.async gathers (4 bytes each; an element outside the tile or
// the slice is zero-filled) through a ring of kGatherStages buffers, with
// kGatherStages - 1 K steps in flight and no registers holding them.  (bf16
// operands cannot be gathered this way -- cp.async moves 4, 8 or 16 bytes --
// and keep the register-staged tile.)  Same thread-to-output mapping,
// summation order and epilogue as the register-staged tile.
template <int CFG>
__device__ __forceinline__ void gather_tile_async(const BatchProb &pr, const int64_t *tables, int item,
                                                  float *smem_f, int64_t *smem_i, int64_t *skA, int64_t *skB)
{
    constexpr BCfg c = kB[CFG];
    constexpr int BM = c.bm, BN = c.bn, BK = c.bk, TM = c.tm, TN = c.tn, S = kGatherStages;
    constexpr int RM = BM / TM, RN = BN / TN, LA = BM * BK / BT, LB = BN * BK / BT;
    const int tid = threadIdx.x;
    const int tile = item / pr.splits, split = item % pr.splits;
    const int tmi = tile / pr.tiles_n, tni = tile % pr.tiles_n;
    const BatchTables t = batch_tables(pr, tables);
    const int64_t m0 = (int64_t)tmi * BM, n0 = (int64_t)tni * BN;
    const int64_t kbeg = (int64_t)split * pr.kps, kend = min(pr.K, kbeg + pr.kps), n = kend - kbeg;
    int64_t *sRowA = smem_i, *sColB = smem_i + BM;
    for (int64_t i = tid; i < n; i += BT) {
        skA[i] = t.kA[kbeg + i];
        skB[i] = t.kB[kbeg + i];
    }
    for (int i = tid; i < BM; i += BT) sRowA[i] = m0 + i < pr.M ? t.rowA[m0 + i] : 0;
    for (int i = tid; i < BN; i += BT) sColB[i] = n0 + i < pr.N ? t.colB[n0 + i] : 0;
    __syncthreads();
    const float *A = static_cast<const float *>(pr.A);
    const float *B = static_cast<const float *>(pr.B);
    float *sA = smem_f, *sB = smem_f + S * BK * BM;
    const int nkt = (int)((n + BK - 1) / BK);
    auto issue = [&](int kt) {
        const int st = kt % S;
        const int64_t k0 = (int64_t)kt * BK;
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + r * BT;
            int mm, kk;
            if (pr.a_m_fast) { mm = e % BM; kk = e / BM; }
            else { kk = e % BK; mm = e / BK; }
            const bool valid = m0 + mm < pr.M && k0 + kk < n;
            cp_async4(&sA[(st * BK + kk) * BM + mm], valid ? A + sRowA[mm] + skA[k0 + kk] : A, valid);
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int e = tid + r * BT;
            int nn, kk;
            if (pr.b_n_fast) { nn = e % BN; kk = e / BN; }
            else { kk = e % BK; nn = e / BK; }
            const bool valid = n0 + nn < pr.N && k0 + kk < n;
            cp_async4(&sB[(st * BK + kk) * BN + nn], valid ? B + sColB[nn] + skB[k0 + kk] : B, valid);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int q = 0; q < S - 1; ++q) {
        if (q < nkt) issue(q);
        else cp_async_commit();  // empty groups keep the group count uniform
    }
    int tm, tn;
    if (pr.c_m_fast) { tm = tid % RM; tn = tid / RM; }
    else { tn = tid % RN; tm = tid / RN; }
    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    for (int kt = 0; kt < nkt; ++kt) {
        cp_async_wait<S - 2>();
        // stage kt has landed for every thread, and every thread has finished
        // stage kt - 1, whose buffer the next issue refills
        __syncthreads();
        if (kt + S - 1 < nkt) issue(kt + S - 1);
        else cp_async_commit();
        const int cur = kt % S;
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = sA[(cur * BK + kk) * BM + tm + i * RM];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = sB[(cur * BK + kk) * BN + tn + j * RN];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
    }
    cp_async_wait<0>();
    if (pr.splits > 1) {
        float *P = pr.partial + (int64_t)split * pr.M * pr.N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t m = m0 + tm + i * RM;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t nn = n0 + tn + j * RN;
                if (m < pr.M && nn < pr.N) P[pr.c_m_fast ? nn * pr.M + m : m * pr.N + nn] = acc[i][j];
            }
        }
        return;
    }
    // offsets first, then a row's loads of C before its stores: a load that
    // follows a store through another pointer cannot be hoisted above it, so
    // interleaved read-modify-writes would each pay a full round trip (the
    // tile's outputs are distinct: C is injective).  Row by row keeps the
    // 64-register build's live values down.
    int64_t rc[TM], cc[TN];
    bool vm[TM], vn[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        vm[i] = m0 + tm + i * RM < pr.M;
        rc[i] = vm[i] ? t.rowC[m0 + tm + i * RM] : 0;
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        vn[j] = n0 + tn + j * RN < pr.N;
        cc[j] = vn[j] ? t.colC[n0 + tn + j * RN] : 0;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        float cv[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) cv[j] = vm[i] && vn[j] ? pr.C[rc[i] + cc[j]] : 0.f;
#pragma unroll
        for (int j = 0; j < TN; ++j)
            if (vm[i] && vn[j]) pr.C[rc[i] + cc[j]] = cv[j] + acc[i][j];
    }
}

template <class T, int CFG>
__device__ __forceinline__ void run_tile(const BatchProb &pr, const int64_t *tables, int item, float *smem_f,
                                         int64_t *smem_i, int64_t *skA, int64_t *skB)
{
    constexpr BCfg c = kB[CFG];
    if constexpr (sizeof(T) == 4) {
        // float operands: cp.async-staged gathers when the slice's K offsets fit
        if (min(pr.K, (int64_t)(item % pr.splits) * pr.kps + pr.kps) - (int64_t)(item % pr.splits) * pr.kps <=
            kStageK) {
            gather_tile_async<CFG>(pr, tables, item, smem_f, smem_i, skA, skB);
            return;
        }
    }
    const int tile = item / pr.splits, split = item % pr.splits;
    const int tm = tile / pr.tiles_n, tn = tile % pr.tiles_n;
    TileArgs a;
    a.A = pr.A;
    a.B = pr.B;
    a.C = pr.C;
    const int64_t *t = tables + pr.tab;
    a.rowA = t;
    a.rowC = t + pr.M;
    a.colB = t + 2 * pr.M;
    a.colC = t + 2 * pr.M + pr.N;
    a.kA = t + 2 * pr.M + 2 * pr.N;
    a.kB = t + 2 * pr.M + 2 * pr.N + pr.K;
    {
        const int64_t kb = split * pr.kps, n = min(pr.K, kb + pr.kps) - kb;
        if (n <= kStageK) {
            // visible to the tile after its first barrier (the row/column
            // offset staging); the tile indexes kA[k] for k in [kb, kb + n)
            for (int64_t i = threadIdx.x; i < n; i += BT) {
                skA[i] = a.kA[kb + i];
                skB[i] = a.kB[kb + i];
            }
            a.kA = skA - kb;
            a.kB = skB - kb;
        }
    }
    a.M = pr.M;
    a.N = pr.N;
    a.m0 = (int64_t)tm * c.bm;
    a.n0 = (int64_t)tn * c.bn;
    a.kbeg = split * pr.kps;
    a.kend = min(pr.K, a.kbeg + pr.kps);
    a.a_m_fast = pr.a_m_fast;
    a.b_n_fast = pr.b_n_fast;
    a.c_m_fast = pr.c_m_fast;
    a.partial = pr.splits > 1 ? pr.partial + (int64_t)split * pr.M * pr.N : nullptr;
    a.sc = Scale{};
    dense_tile<T, c.bm, c.bn, c.bk, c.tm, c.tn>(a, smem_f, smem_f + 2 * c.bk * c.bm, smem_i, smem_i + c.bm);
}

// Short sums (K <= 8, one K slice): each thread forms its TM x TN outputs
// straight from gathered loads -- no operand staging, no padding of K to the
// tile's BK.  A tile's row and column offsets (rowA, rowC, colB, colC) are
// staged in shared memory, one coalesced load a thread, and so are the
// sum's K offsets: the operand loads of every k then depend on
// shared-memory reads only, and the offsets take no registers.  The offsets
// of the item's next tile are loaded while the current tile's loads are in
// flight and stored into the other half of a double buffer, so a tile costs
// one round trip and one barrier.  Same thread-to-output mapping as the
// staged tile (lanes along C's smaller increment); each output starts from
// C's value and adds the products with k ascending, Alg. 1's order.
template <int CFG>
__device__ __forceinline__ int64_t direct_offset(const BatchProb &pr, const int64_t *tables, int tile)
{
    constexpr int BM = kB[CFG].bm, BN = kB[CFG].bn;
    const int64_t M = pr.M, N = pr.N;
    const int64_t m0 = (int64_t)(tile / pr.tiles_n) * BM, n0 = (int64_t)(tile % pr.tiles_n) * BN;
    const int64_t *rowA = tables + pr.tab;
    const int64_t *rowC = rowA + M, *colB = rowC + M, *colC = colB + N;
    const int tid = threadIdx.x;
    // [0, BM) rowA, [BM, 2 BM) rowC, [2 BM, 2 BM + BN) colB, then colC
    if (tid < 2 * BM) {
        const int r = tid % BM;
        return m0 + r < M ? (tid < BM ? rowA : rowC)[m0 + r] : 0;
    }
    if (tid < 2 * (BM + BN)) {
        const int q = (tid - 2 * BM) % BN;
        return n0 + q < N ? (tid < 2 * BM + BN ? colB : colC)[n0 + q] : 0;
    }
    return 0;
}

constexpr int kDirectOff = 2 * (64 + 64);  // offsets of one tile, largest shape

template <class T, int CFG>
__device__ __forceinline__ void run_direct(const BatchProb &pr, const int64_t *tables, int t0, int t1,
                                           int64_t *s_off, int64_t *s_k)
{
    using R = Tr<T>;
    using Acc = typename R::Acc;
    constexpr BCfg c = kB[CFG];
    constexpr int BM = c.bm, BN = c.bn, TM = c.tm, TN = c.tn, RM = BM / TM, RN = BN / TN;
    static_assert(2 * (BM + BN) <= BT && 2 * (BM + BN) <= kDirectOff, "one offset a thread");
    const int64_t M = pr.M, N = pr.N, K = pr.K;
    const int tid = threadIdx.x;
    {
        const int64_t v = direct_offset<CFG>(pr, tables, t0);
        if (tid < 2 * (BM + BN)) s_off[tid] = v;
        const int64_t *kA = tables + pr.tab + 2 * M + 2 * N;
        if (tid < 16) s_k[tid] = (tid & 7) < K ? kA[(tid < 8 ? 0 : K) + (tid & 7)] : 0;
    }
    __syncthreads();
    int tm, tn;
    if (pr.c_m_fast) { tm = tid % RM; tn = tid / RM; }
    else { tn = tid % RN; tm = tid / RN; }
    const T *A = static_cast<const T *>(pr.A);
    const T *B = static_cast<const T *>(pr.B);
    for (int tile = t0; tile < t1; ++tile) {
        const int64_t *so = s_off + ((tile - t0) & 1) * kDirectOff;
        // the next tile's offset: in flight with this tile's loads
        const int64_t nv = tile + 1 < t1 ? direct_offset<CFG>(pr, tables, tile + 1) : 0;
        const int64_t m0 = (int64_t)(tile / pr.tiles_n) * BM, n0 = (int64_t)(tile % pr.tiles_n) * BN;
        bool vm[TM], vn[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) vm[i] = m0 + tm + i * RM < M;
#pragma unroll
        for (int j = 0; j < TN; ++j) vn[j] = n0 + tn + j * RN < N;
        // C is read before the sum (the batch only accumulates): its loads
        // are in flight together with the operands' instead of after them
        Acc acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                acc[i][j] = (vm[i] && vn[j]) ? pr.C[so[BM + tm + i * RM] + so[2 * BM + BN + tn + j * RN]] : R::zero();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k < K) {
                const int64_t ka = s_k[k], kb = s_k[8 + k];
                Acc a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = vm[i] ? R::load(A + so[tm + i * RM] + ka) : R::zero();
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = vn[j] ? R::load(B + so[2 * BM + tn + j * RN] + kb) : R::zero();
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) R::mac(acc[i][j], a[i], b[j]);
            }
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (vm[i] && vn[j]) pr.C[so[BM + tm + i * RM] + so[2 * BM + BN + tn + j * RN]] = acc[i][j];
        // the other buffer was last read in the previous tile, which every
        // thread finished before the barrier that closed it
        if (tile + 1 < t1 && tid < 2 * (BM + BN)) s_off[(((tile - t0) & 1) ^ 1) * kDirectOff + tid] = nv;
        __syncthreads();
    }
}

// largest shared footprint over the configurations (floats / int64s)
constexpr int smem_floats()
{
    int m = 0;
    for (int i = 0; i < NSHAPE; ++i) m = std::max(m, kGatherStages * kB[i].bk * (kB[i].bm + kB[i].bn));
    return m;
}
constexpr int smem_ints()
{
    int m = 0;
    for (int i = 0; i < NSHAPE; ++i) m = std::max(m, kB[i].bm + kB[i].bn);
    return m;
}

// Work item i is work[i % wrap]; normal launches pass wrap == nwork, the
// autotuner's throughput mode replicates one problem's items to fill the GPU.
template <int CPS>
__global__ void __launch_bounds__(BT, CPS) batch_kernel(const BatchProb *__restrict__ probs, const uint2 *__restrict__ work,
                                                       int64_t nwork, int64_t wrap, const int64_t *__restrict__ tables,
                                                       unsigned long long *counter)
{
    __shared__ float smem_f[smem_floats()];
    __shared__ int64_t smem_i[smem_ints()];
    __shared__ int64_t skA[kStageK], skB[kStageK];
    __shared__ unsigned long long s_item;
    // the item's problem descriptor, copied once by warp 0: fields are read
    // from shared memory instead of living in registers (the build for four
    // resident CTAs has 64 registers a thread)
    __shared__ __align__(16) BatchProb s_pr;
    constexpr int kWords = (int)(sizeof(BatchProb) / 4);
    static_assert(sizeof(BatchProb) % 4 == 0 && kWords <= 64, "descriptor copy by one warp, two words a lane");
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1ull);
    __syncthreads();
    unsigned long long it = s_item;
    while (it < (unsigned long long)nwork) {
        // thread 0 asks for the next item now: the atomic's round trip overlaps
        // this item's tile (most items are a few tens of KFLOP)
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1ull);
        const uint2 w = work[it % (unsigned long long)wrap];
        if (threadIdx.x < 32) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(probs + w.x);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_pr);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (threadIdx.x + 32 * q < kWords) dst[threadIdx.x + 32 * q] = __ldg(src + threadIdx.x + 32 * q);
        }
        __syncthreads();
        const BatchProb &pr = s_pr;
        const int key = pr.shape * 2 + pr.dtype;
        switch (key) {
        case 0: run_tile<float, 0>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 1: run_tile<uint16_t, 0>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 2: run_tile<float, 1>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 3: run_tile<uint16_t, 1>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 4: run_tile<float, 2>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 5: run_tile<uint16_t, 2>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 6: run_tile<float, 3>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        case 7: run_tile<uint16_t, 3>(pr, tables, w.y, smem_f, smem_i, skA, skB); break;
        default: break;
        }
        __syncthreads();  // the tile's shared memory and s_item are free again
        if (threadIdx.x == 0) s_item = next;
        __syncthreads();
        it = s_item;
    }
}

// the instantiation whose register cap lets `cps` CTAs reside on an SM
void launch_batch_kernel(int cps, int ctas, cudaStream_t s, const BatchProb *probs, const uint2 *work,
                         int64_t nwork, int64_t wrap, const int64_t *tables, unsigned long long *counter)
{
    if (cps >= 4) batch_kernel<4><<<ctas, BT, 0, s>>>(probs, work, nwork, wrap, tables, counter);
    else if (cps == 3) batch_kernel<3><<<ctas, BT, 0, s>>>(probs, work, nwork, wrap, tables, counter);
    else batch_kernel<2><<<ctas, BT, 0, s>>>(probs, work, nwork, wrap, tables, counter);
}

// Short sums (K <= 8): items are runs of tiles of one problem, taken from
// their own atomic counter.  Apart from the staged offsets the kernel holds
// no shared memory, so four CTAs of 256 threads share an SM with the other
// branches' kernels.
__global__ void __launch_bounds__(BT, 4) batch_direct_kernel(const BatchProb *__restrict__ probs,
                                                             const uint2 *__restrict__ work, int64_t nwork,
                                                             int64_t wrap, const int64_t *__restrict__ tables,
                                                             unsigned long long *counter)
{
    __shared__ int64_t s_off[2 * kDirectOff], s_k[16];
    __shared__ unsigned long long s_item;
    __shared__ __align__(16) BatchProb s_pr;
    constexpr int kWords = (int)(sizeof(BatchProb) / 4);
    static_assert(sizeof(BatchProb) % 4 == 0 && kWords <= 64, "descriptor copy by one warp, two words a lane");
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1ull);
    __syncthreads();
    unsigned long long it = s_item;
    while (it < (unsigned long long)nwork) {
        unsigned long long next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1ull);
        const uint2 w = work[it % (unsigned long long)wrap];
        if (threadIdx.x < 32) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(probs + w.x);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&s_pr);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (threadIdx.x + 32 * q < kWords) dst[threadIdx.x + 32 * q] = __ldg(src + threadIdx.x + 32 * q);
        }
        __syncthreads();
        const BatchProb &pr = s_pr;
        const int key = pr.shape * 2 + pr.dtype;
        const int t0 = (int)w.y * pr.tpi, t1 = min(pr.tiles_m * pr.tiles_n, t0 + pr.tpi);
        switch (key) {
        case 0: run_direct<float, 0>(pr, tables, t0, t1, s_off, s_k); break;
        case 1: run_direct<uint16_t, 0>(pr, tables, t0, t1, s_off, s_k); break;
        case 2: run_direct<float, 1>(pr, tables, t0, t1, s_off, s_k); break;
        case 3: run_direct<uint16_t, 1>(pr, tables, t0, t1, s_off, s_k); break;
        case 4: run_direct<float, 2>(pr, tables, t0, t1, s_off, s_k); break;
        case 5: run_direct<uint16_t, 2>(pr, tables, t0, t1, s_off, s_k); break;
        case 6: run_direct<float, 3>(pr, tables, t0, t1, s_off, s_k); break;
        case 7: run_direct<uint16_t, 3>(pr, tables, t0, t1, s_off, s_k); break;
        default: break;
        }
        if (threadIdx.x == 0) s_item = next;
        __syncthreads();  // (run_direct ends with a barrier: s_pr is free too)
        it = s_item;
    }
}

void launch_batch_direct(int ctas, cudaStream_t s, const BatchProb *probs, const uint2 *work, int64_t nwork,
                         int64_t wrap, const int64_t *tables, unsigned long long *counter)
{
    batch_direct_kernel<<<ctas, BT, 0, s>>>(probs, work, nwork, wrap, tables, counter);
}

// Adds the K-slice partial tiles of every split problem into C, slices in
// order (deterministic).  One CTA per listed problem at a time.
__global__ void __launch_bounds__(256) batch_reduce_kernel(const BatchProb *__restrict__ probs,
                                                           const int *__restrict__ list, int nlist,
                                                           const int64_t *__restrict__ tables)
{
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        const BatchProb pr = probs[list[li]];
        const int64_t *t = tables + pr.tab;
        const int64_t *rowC = t + pr.M;
        const int64_t *colC = t + 2 * pr.M + pr.N;
        const int64_t MN = pr.M * pr.N;
        // four outputs a thread per pass: their sums and every load of C go
        // before the stores (a load after a store through another pointer
        // cannot be hoisted above it); slices still add in order
        constexpr int U = 4;
        for (int64_t i0 = threadIdx.x; i0 < MN; i0 += U * (int64_t)blockDim.x) {
            int64_t off[U];
            float sum[U], cv[U];
            bool v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x;
                v[u] = i < MN;
                int64_t m = 0, n = 0;
                if (v[u]) {
                    if (pr.c_m_fast) { m = i % pr.M; n = i / pr.M; }
                    else { n = i % pr.N; m = i / pr.N; }
                }
                off[u] = v[u] ? rowC[m] + colC[n] : 0;
                sum[u] = v[u] ? pr.partial[i] : 0.f;
                for (int sp = 1; sp < pr.splits; ++sp)
                    if (v[u]) sum[u] += pr.partial[(int64_t)sp * MN + i];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) cv[u] = v[u] ? pr.C[off[u]] : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (v[u]) pr.C[off[u]] = cv[u] + sum[u];
        }
    }
}

void decode_host(const ModeList &L, int64_t count, int64_t *t0, int64_t *t1)
{
    // first mode fastest; incremental odometer (the order Alg. 2 visits)
    int64_t coord[GETT_MAX_MODES] = {0};
    int64_t a = 0, b = 0;
    for (int64_t i = 0; i < count; ++i) {
        t0[i] = a;
        t1[i] = b;
        for (int d = 0; d < L.n; ++d) {
            coord[d]++;
            a += L.s0[d];
            b += L.s1[d];
            if (coord[d] < L.ext[d]) break;
            a -= L.s0[d] * L.ext[d];
            b -= L.s1[d] * L.ext[d];
            coord[d] = 0;
        }
    }
}

int64_t first_abs(const ModeList &L, const int64_t *s) { return L.n ? (s[0] < 0 ? -s[0] : s[0]) : 0; }

}  // namespace

// The fixed rule: short sums (K <= 8) take the gathered direct path; one
// free class of at most 8 indices the skinny warp kernel; everything else is
// packed.  The tile shape follows M and N.
int batch_shape_rule(int64_t M, int64_t N)
{
    if (M >= 64 && N >= 64) return 0;
    if (M < 64 && N >= 64) return 1;
    if (M >= 64 && N < 64) return 3;
    return 2;
}

bool batch_skinny_shape(int64_t M, int64_t N) { return std::min(M, N) <= SKINNY_MAX_SHORT; }

int batch_heuristic_config(int64_t M, int64_t N, int64_t K, int dtype)
{
    const int shape = batch_shape_rule(M, N);
    if (K <= 8) return shape;
    if (batch_skinny_shape(M, N)) return CFG_SKINNY;
    if (dtype == GETT_BATCH_BF16 && K >= 256 && M >= 128 && N >= 128) return CFG_TC;
    return NSHAPE + shape;
}

// A configuration is valid for a problem unless it asks for the skinny
// kernel on a problem without a free class of at most 8 indices, or for the
// tensor cores with float operands.
bool batch_config_valid(int cfg, int64_t M, int64_t N, int dtype)
{
    if (cfg < 0 || cfg >= NCFG) return false;
    if (cfg == CFG_SKINNY) return batch_skinny_shape(M, N);
    if (cfg == CFG_TC) return dtype == GETT_BATCH_BF16;
    return true;
}

}  // namespace gett

struct gett_batch {
    int n = 0;
    int nonempty = 0;
    int64_t nwork = 0;        // gathered tiles (work items of the gather kernel)
    int64_t npacked = 0;      // packed tile items
    int64_t npack = 0;        // packing items
    int64_t nskinny = 0;      // skinny warp items
    double flops = 0;
    int config_count[GETT_BATCH_MAX_CONFIGS] = {};
    int fallbacks = 0;
    int tuned_hits = 0;
    int ctas = 0;
    int sms = 0;
    int cps = 4;  // gather kernel instantiation (resident CTAs per SM it is compiled for)
    gett::BatchProb *d_probs = nullptr;
    uint2 *d_work = nullptr;
    uint2 *d_packed_work = nullptr;
    gett::PackItem *d_pack = nullptr;
    gett::SkinnyItem *d_skinny = nullptr;
    gett::SkinnyItem *d_skinny_by_problem = nullptr;
    uint2 *d_tc_work = nullptr;              // tensor-core tiles (sorted)
    uint2 *d_tc_work_by_problem = nullptr;
    gett::TcPackItem *d_tc_pack = nullptr;   // their packing items (grouped by problem)
    uint16_t *d_tiles16 = nullptr;           // packed bf16 tiles of the TC method
    int64_t ntc = 0, ntcpack = 0;
    int64_t *d_tables = nullptr;
    float *d_packed = nullptr;           // tile-blocked operands of packed problems
    unsigned long long *d_counter = nullptr;  // work counters: [0] gathered tiles, [1] short sums
    // every list again grouped by problem (the autotuner times one problem)
    uint2 *d_work_by_problem = nullptr;
    uint2 *d_direct = nullptr;               // short-sum tile runs (sorted) and grouped by problem
    uint2 *d_direct_by_problem = nullptr;
    int64_t ndirect = 0;
    uint2 *d_packed_by_problem = nullptr;
    float *d_partial = nullptr;          // K-slice partials of split problems
    int *d_reduce = nullptr;             // indices (into the descriptor table) of split problems
    int *d_err = nullptr;                // device error word (bounded waits)
    int nreduce = 0;
    std::vector<int> reduce_of;          // per user index: descriptor index if split, else -1
    // per user index: start and count in each by-problem list
    std::vector<int64_t> gw_start, gw_count, pw_start, pw_count, pk_start, pk_count, sk_start, sk_count;
    std::vector<int64_t> tw_start, tw_count, tk_start, tk_count, dw_start, dw_count;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;
    // concurrent branches of a launch: the method chains other than the
    // packed one run on these streams, forked from and joined back into the
    // launch stream (created with the handle unless `serial`)
    bool serial = false;
    cudaStream_t branch[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[4] = {nullptr, nullptr, nullptr, nullptr};
};

using namespace gett;

extern "C" int gett_batch_num_configs(void) { return NCFG; }

extern "C" int gett_batch_config_shape(int config, int *bm, int *bn)
{
    if (config < 0 || config >= NCFG) return GETT_ERR_ARG;
    const int m = cfg_method(config);
    if (bm) *bm = m == BM_SKINNY ? 0 : kB[cfg_shape(config)].bm;
    if (bn) *bn = m == BM_SKINNY ? 0 : kB[cfg_shape(config)].bn;
    return GETT_OK;
}

extern "C" int gett_batch_config_method(int config)
{
    if (config < 0 || config >= NCFG) return GETT_ERR_ARG;
    return cfg_method(config);
}

extern "C" int gett_batch_heuristic_config(int RANKA, const int64_t *EXTA, const int64_t *INCA, int RANKB,
                                           const int64_t *EXTB, const int64_t *INCB, int CONTS, const int *CONTA,
                                           const int *CONTB, const int *PERM, const int64_t *INCC, int dtype,
                                           int *config)
{
    if (!config) return GETT_ERR_ARG;
    Args a{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC};
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(bad);
    if (rc != GETT_OK) return rc;
    *config = p.empty ? 0 : batch_heuristic_config(p.M, p.N, p.K, dtype);
    return GETT_OK;
}

extern "C" int gett_batch_config_valid(int RANKA, const int64_t *EXTA, const int64_t *INCA, int RANKB,
                                       const int64_t *EXTB, const int64_t *INCB, int CONTS, const int *CONTA,
                                       const int *CONTB, const int *PERM, const int64_t *INCC, int dtype, int config)
{
    Args a{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC};
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(bad);
    if (rc != GETT_OK) return rc;
    return batch_config_valid(config, p.M, p.N, dtype) ? 1 : 0;
}

namespace {

// Limits of one batch's host-side planning (checked before allocating):
// indices per class and offset-table entries over all problems (2^31
// entries = 16 GB of int64 tables), packed operand floats (2^30 = 4 GB; a
// problem whose packed operands would pass it is gathered instead).
constexpr int64_t kMaxClassIndices = (int64_t)1 << 31;
constexpr int64_t kMaxTableEntries = (int64_t)1 << 31;
constexpr int64_t kMaxPackedFloats = (int64_t)1 << 30;
constexpr int64_t kMaxTcElems = (int64_t)1 << 30;  // bf16 tiles of the TC method (2 GB)
constexpr int64_t kSkinnyLaneSlice = 256;   // K per warp item, lanes along the long class
constexpr int64_t kSkinnySumSlice = 2048;   // K per warp item, lanes along the sum

int64_t a64(int64_t x) { return (x + 63) & ~int64_t(63); }

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &v)
{
    cudaError_t e = cudaMalloc(dst, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

// items sorted by decreasing cost (long items first), stable
template <class T>
std::vector<T> by_cost(const std::vector<T> &items, const std::vector<double> &cost)
{
    std::vector<size_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<T> out(items.size());
    for (size_t i = 0; i < order.size(); ++i) out[i] = items[order[i]];
    return out;
}

int batch_create_impl(int n, const gett_problem_desc *probs, const gett_batch_options *opt, gett_batch **out,
                      int *bad_index)
{
    if (bad_index) *bad_index = -1;
    if (!out || n < 0 || (n > 0 && !probs)) return GETT_ERR_ARG;
    *out = nullptr;
    gett_batch_options o{};
    if (opt) o = *opt;
    if (o.select < GETT_BATCH_SELECT_HEURISTIC || o.select > GETT_BATCH_SELECT_TUNED) return GETT_ERR_ARG;
    if (o.select == GETT_BATCH_SELECT_FIXED && (o.config < 0 || o.config >= NCFG)) return GETT_ERR_ARG;
    if (o.select == GETT_BATCH_SELECT_TABLE && !o.configs) return GETT_ERR_ARG;
    if (o.serial != 0 && o.serial != 1) return GETT_ERR_ARG;

    std::vector<Plan> plans(n);
    std::vector<BatchProb> hp;
    std::vector<int> hp_index;
    int64_t table_len = 0;
    struct Span {
        __int128 lo, hi;  // byte range; 128-bit so broadcast spans cannot wrap
        int idx;
    };
    std::vector<Span> cspans, inspans;
    int fallbacks = 0, tuned_hits = 0;
    for (int i = 0; i < n; ++i) {
        const gett_problem_desc &d = probs[i];
        if (d.dtype != GETT_BATCH_F32 && d.dtype != GETT_BATCH_BF16) {
            if (bad_index) *bad_index = i;
            set_last_error_arg(0);
            return GETT_ERR_ARG;
        }
        Args a{d.RANKA, d.EXTA, d.INCA, d.RANKB, d.EXTB, d.INCB, d.CONTS, d.CONTA, d.CONTB, d.PERM, d.INCC};
        int bad = 0;
        int rc = make_plan(a, &plans[i], &bad);
        if (rc != GETT_OK) {
            set_last_error_arg(bad);
            if (bad_index) *bad_index = i;
            return rc;
        }
        const Plan &p = plans[i];
        if (p.empty) continue;
        // host and device offset tables hold 2 (M + N + K) entries per problem
        // and a problem's tiles are counted in 32 bits: bound both before any
        // allocation (a class may count up to 2^62 indices through broadcast
        // modes, which the address spans do not bound)
        if (p.M > kMaxClassIndices || p.N > kMaxClassIndices || p.K > kMaxClassIndices ||
            table_len + 2 * (p.M + p.N + p.K) > kMaxTableEntries) {
            set_last_error_arg(0);
            if (bad_index) *bad_index = i;
            return GETT_ERR_UNSUPPORTED;
        }
        const size_t esz = d.dtype == GETT_BATCH_F32 ? 4 : 2;
        if (!d.A || !d.B || !d.C) {
            set_last_error_arg(!d.A ? 4 : (!d.B ? 8 : 14));
            if (bad_index) *bad_index = i;
            return GETT_ERR_ARG;
        }
        auto span = [](const void *ptr, int64_t lo, int64_t hi, size_t e, int idx) {
            const __int128 b = reinterpret_cast<intptr_t>(ptr);
            return Span{b + (__int128)lo * (int64_t)e, b + ((__int128)hi + 1) * (int64_t)e, idx};
        };
        cspans.push_back(span(d.C, p.c_lo, p.c_hi, 4, i));
        inspans.push_back(span(d.A, p.a_lo, p.a_hi, esz, i));
        inspans.push_back(span(d.B, p.b_lo, p.b_hi, esz, i));
        // the choice chain: learned model -> tuning database -> heuristic
        // (SELECT_LEARNED), database -> heuristic (SELECT_TUNED)
        int cfg = -1;
        if (o.select == GETT_BATCH_SELECT_FIXED) cfg = o.config;
        else if (o.select == GETT_BATCH_SELECT_TABLE) cfg = o.configs[i];
        else if (o.select == GETT_BATCH_SELECT_LEARNED) {
            bool valid[NCFG];
            for (int c = 0; c < NCFG; ++c) valid[c] = batch_config_valid(c, p.M, p.N, d.dtype);
            cfg = learned_batch_config(p, d.dtype, NCFG, valid);
        }
        if ((o.select == GETT_BATCH_SELECT_TUNED || o.select == GETT_BATCH_SELECT_LEARNED) &&
            !batch_config_valid(cfg, p.M, p.N, d.dtype)) {
            int v0 = -1, v1 = 0, v2 = 0;
            if (tune_db_lookup(GETT_TUNE_BATCH, d.dtype, p, &v0, &v1, &v2) &&
                batch_config_valid(v0, p.M, p.N, d.dtype)) {
                cfg = v0;
                ++tuned_hits;
            }
        }
        if (!batch_config_valid(cfg, p.M, p.N, d.dtype)) {
            if (o.select != GETT_BATCH_SELECT_HEURISTIC) ++fallbacks;
            cfg = batch_heuristic_config(p.M, p.N, p.K, d.dtype);
        }
        BatchProb b{};
        b.A = static_cast<const char *>(d.A) + p.offA * (int64_t)esz;
        b.B = static_cast<const char *>(d.B) + p.offB * (int64_t)esz;
        b.C = d.C + p.offC;
        b.M = p.M;
        b.N = p.N;
        b.K = p.K;
        b.tab = table_len;
        b.cfg = cfg;
        b.dtype = d.dtype;
        b.shape = cfg_shape(cfg);
        b.bm = kB[b.shape].bm;
        b.bn = kB[b.shape].bn;
        // short sums take the gathered direct path whatever the tile method
        b.method = (p.K <= 8 && cfg_method(cfg) == BM_PACK) ? BM_GATHER : cfg_method(cfg);
        {
            const int tbm = b.method == BM_TC ? TC_BM : b.bm, tbn = b.method == BM_TC ? TC_BN : b.bn;
            const int64_t tm = (p.M + tbm - 1) / tbm, tn = (p.N + tbn - 1) / tbn;
            if (tm * tn > (int64_t)INT32_MAX) {  // M, N <= 2^31 each: the product fits int64
                set_last_error_arg(0);
                if (bad_index) *bad_index = i;
                return GETT_ERR_UNSUPPORTED;
            }
            b.tiles_m = (int)tm;
            b.tiles_n = (int)tn;
        }
        const int64_t am = first_abs(p.m, p.m.s0), ak = first_abs(p.k, p.k.s0);
        const int64_t bnn = first_abs(p.n, p.n.s0), bk = first_abs(p.k, p.k.s1);
        const int64_t cm = first_abs(p.m, p.m.s1), cn = first_abs(p.n, p.n.s1);
        b.a_m_fast = (am != 0 && (ak == 0 || am <= ak)) ? 1 : 0;
        b.b_n_fast = (bnn != 0 && (bk == 0 || bnn <= bk)) ? 1 : 0;
        b.c_m_fast = (cm != 0 && (cn == 0 || cm <= cn)) ? 1 : 0;
        table_len += 2 * (p.M + p.N + p.K);
        hp.push_back(b);
        hp_index.push_back(i);
    }
    // C of different problems must not overlap each other or any input
    std::sort(cspans.begin(), cspans.end(), [](const Span &x, const Span &y) { return x.lo < y.lo; });
    for (size_t i = 1; i < cspans.size(); ++i)
        if (cspans[i].lo < cspans[i - 1].hi) {
            if (bad_index) *bad_index = cspans[i].idx;
            return GETT_ERR_ALIAS;
        }
    for (const Span &s : inspans) {
        auto it = std::upper_bound(cspans.begin(), cspans.end(), s.lo,
                                   [](__int128 v, const Span &c) { return v < c.lo; });
        if (it != cspans.begin() && std::prev(it)->hi > s.lo) {
            if (bad_index) *bad_index = s.idx;
            return GETT_ERR_ALIAS;
        }
        if (it != cspans.end() && it->lo < s.hi) {
            if (bad_index) *bad_index = s.idx;
            return GETT_ERR_ALIAS;
        }
    }

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    const int cps = o.ctas_per_sm > 0 ? o.ctas_per_sm : kCtasPerSm;
    const int ctas = sms * cps;

    // K slices.  Tiles (gathered or packed): a tile whose work is far above
    // the average share of a CTA is split along K so the longest work item
    // stays short (tail effects), and so is any tile with more than kMaxSteps
    // K steps whatever its area (a small tile with a long sum is a chain of
    // dependent steps).  Skinny warp items cover kSkinnyLaneSlice (lanes along
    // the long class) or kSkinnySumSlice (lanes along the sum) contracted
    // indices.  Slices of one problem are added into C in slice order by a
    // second kernel.
    constexpr int64_t kMaxSteps = 96, kMaxSplits = 512;  // kMaxSteps * BK <= kStageK
    double total_cost = 0;
    for (const BatchProb &pr : hp)
        if (pr.method != BM_SKINNY && pr.method != BM_TC)
            total_cost += (double)pr.tiles_m * pr.tiles_n * pr.bm * pr.bn * (double)pr.K;
    const double target = std::max(total_cost / (2.0 * ctas), 1.0);
    int64_t partial_floats = 0, packed_floats = 0, tc_elems = 0;
    std::vector<int64_t> partial_off(hp.size(), -1), packed_off(hp.size(), -1), tc_off(hp.size(), -1);
    for (size_t j = 0; j < hp.size(); ++j) {
        BatchProb &pr = hp[j];
        int64_t S = 1, kps = pr.K;
        if (pr.method == BM_TC) {
            // one slice (the tensor cores make long sums short); 128 x 64 tiles
            pr.nkt = (int)((pr.K + TC_BK - 1) / TC_BK);
            const int64_t ea = (int64_t)pr.tiles_m * pr.nkt * TC_TILE_ELEMS;
            const int64_t eb = (int64_t)pr.tiles_n * pr.nkt * TC_TILE_ELEMS;
            if (tc_elems + ea + eb > kMaxTcElems) {
                // the tile buffer is full: gather this one instead
                pr.method = BM_GATHER;
                pr.tiles_m = (int)((pr.M + pr.bm - 1) / pr.bm);
                pr.tiles_n = (int)((pr.N + pr.bn - 1) / pr.bn);
            } else {
                tc_off[j] = tc_elems;
                tc_elems += ea + eb;
                pr.splits = 1;
                pr.kps = pr.K;
                pr.tpi = 1;
                continue;
            }
        }
        if (pr.method == BM_SKINNY) {
            const int64_t L = std::max(pr.M, pr.N), Sh = std::min(pr.M, pr.N);
            pr.long_is_a = pr.M >= pr.N ? 1 : 0;
            pr.lanes_k = (L <= 4 && Sh <= 4) ? 1 : 0;
            pr.kslice = pr.lanes_k ? kSkinnySumSlice : kSkinnyLaneSlice;
            S = (pr.K + pr.kslice - 1) / pr.kslice;
            if (S > 1 && partial_floats + S * pr.M * pr.N > (int64_t)(1 << 28)) {
                pr.kslice = pr.K;  // one slice: long warp items, no partials
                S = 1;
            }
            kps = pr.kslice;
        } else {
            const int bk = kB[pr.shape].bk;
            const double tile_cost = (double)pr.bm * pr.bn * (double)pr.K;
            const int64_t steps = (pr.K + bk - 1) / bk;
            S = std::max<int64_t>((int64_t)std::ceil(tile_cost / target), (steps + kMaxSteps - 1) / kMaxSteps);
            S = std::min<int64_t>(S, kMaxSplits);
            S = std::min<int64_t>(S, std::max<int64_t>(1, pr.K / 128));
            if (S < 1) S = 1;
            kps = (pr.K + S - 1) / S;
            kps = (kps + bk - 1) / bk * bk;
            S = (pr.K + kps - 1) / kps;
            if (S > 1 && partial_floats + S * pr.M * pr.N > (int64_t)(1 << 28)) S = 1, kps = pr.K;
        }
        pr.splits = (int)S;
        pr.kps = S > 1 ? kps : pr.K;
        pr.tpi = 1;
        if (batch_direct(pr))
            pr.tpi = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)pr.tiles_m * pr.tiles_n,
                                                                   32768 / (pr.bm * pr.bn)));
        if (S > 1) {
            partial_off[j] = partial_floats;
            partial_floats += S * pr.M * pr.N;
        }
        if (pr.method == BM_PACK) {
            // packed K is zero-padded to whole 16-steps: one slice covers Kp
            pr.Kp = (pr.K + 15) / 16 * 16;
            pr.kps = pr.splits > 1 ? std::min(pr.kps, pr.Kp) : pr.Kp;
            const int64_t fa = a64(pr.Kp * pr.bm * (int64_t)pr.tiles_m), fb = a64(pr.Kp * pr.bn * (int64_t)pr.tiles_n);
            if (packed_floats + fa + fb > kMaxPackedFloats) {
                pr.method = BM_GATHER;  // the packed buffer is full: gather this one
            } else {
                packed_off[j] = packed_floats;
                packed_floats += fa + fb;
            }
        }
    }

    gett_batch *b = new gett_batch();
    b->n = n;
    b->nonempty = (int)hp.size();
    b->fallbacks = fallbacks;
    b->tuned_hits = tuned_hits;
    b->sms = sms;
    std::vector<int64_t> tables((size_t)std::max<int64_t>(table_len, 1));
    // per-problem lists (grouped) and their costs
    std::vector<uint2> gwork, pwork, twork, dwork;
    std::vector<PackItem> pack;
    std::vector<TcPackItem> tpack;
    std::vector<SkinnyItem> skinny;
    std::vector<double> gcost, pcost, scost, tcost, dcost;
    b->gw_start.assign(n, 0); b->gw_count.assign(n, 0);
    b->pw_start.assign(n, 0); b->pw_count.assign(n, 0);
    b->pk_start.assign(n, 0); b->pk_count.assign(n, 0);
    b->sk_start.assign(n, 0); b->sk_count.assign(n, 0);
    b->tw_start.assign(n, 0); b->tw_count.assign(n, 0);
    b->tk_start.assign(n, 0); b->tk_count.assign(n, 0);
    b->dw_start.assign(n, 0); b->dw_count.assign(n, 0);
    for (size_t j = 0; j < hp.size(); ++j) {
        const Plan &p = plans[hp_index[j]];
        BatchProb &pr = hp[j];
        const int ui = hp_index[j];
        int64_t *t = tables.data() + pr.tab;
        decode_host(p.m, p.M, t, t + p.M);
        decode_host(p.n, p.N, t + 2 * p.M, t + 2 * p.M + p.N);
        decode_host(p.k, p.K, t + 2 * p.M + 2 * p.N, t + 2 * p.M + 2 * p.N + p.K);
        b->flops += 2.0 * (double)p.M * (double)p.N * (double)p.K;
        b->config_count[pr.cfg]++;
        const double tile_area = (double)pr.bm * pr.bn;
        if (pr.method == BM_GATHER) {
            // short sums go to their own kernel
            const bool dir = batch_direct(pr);
            std::vector<uint2> &lst = dir ? dwork : gwork;
            std::vector<double> &cst = dir ? dcost : gcost;
            (dir ? b->dw_start : b->gw_start)[ui] = (int64_t)lst.size();
            const int nitems = batch_items(pr);
            for (int tt = 0; tt < nitems; ++tt) {
                lst.push_back(make_uint2((unsigned)j, (unsigned)tt));
                cst.push_back(tile_area * (double)pr.kps * pr.tpi);
            }
            (dir ? b->dw_count : b->gw_count)[ui] = nitems;
        } else if (pr.method == BM_PACK) {
            b->pw_start[ui] = (int64_t)pwork.size();
            const int nitems = pr.tiles_m * pr.tiles_n * pr.splits;
            for (int tt = 0; tt < nitems; ++tt) {
                pwork.push_back(make_uint2((unsigned)j, (unsigned)tt));
                pcost.push_back(tile_area * (double)pr.kps);
            }
            b->pw_count[ui] = nitems;
            b->pk_start[ui] = (int64_t)pack.size();
            const int chunks = (int)((pr.Kp + 63) / 64);
            for (int op = 0; op < 2; ++op) {
                const int blocks = op == 0 ? pr.tiles_m : pr.tiles_n;
                for (int bl = 0; bl < blocks; ++bl)
                    for (int ch = 0; ch < chunks; ++ch) pack.push_back(PackItem{(int)j, op, bl, ch});
            }
            b->pk_count[ui] = (int64_t)pack.size() - b->pk_start[ui];
        } else if (pr.method == BM_TC) {
            b->tw_start[ui] = (int64_t)twork.size();
            const int nitems = pr.tiles_m * pr.tiles_n;
            for (int tt = 0; tt < nitems; ++tt) {
                twork.push_back(make_uint2((unsigned)j, (unsigned)tt));
                tcost.push_back((double)pr.nkt);
            }
            b->tw_count[ui] = nitems;
            b->tk_start[ui] = (int64_t)tpack.size();
            for (int op = 0; op < 2; ++op) {
                const int blocks = op == 0 ? pr.tiles_m : pr.tiles_n;
                for (int bl = 0; bl < blocks; ++bl)
                    for (int kt = 0; kt < pr.nkt; ++kt) tpack.push_back(TcPackItem{(int)j, op, bl, kt});
            }
            b->tk_count[ui] = (int64_t)tpack.size() - b->tk_start[ui];
        } else {
            b->sk_start[ui] = (int64_t)skinny.size();
            const int64_t L = std::max(pr.M, pr.N);
            const int64_t lblocks = pr.lanes_k ? 1 : (L + 31) / 32;
            for (int sl = 0; sl < pr.splits; ++sl)
                for (int64_t lb = 0; lb < lblocks; ++lb) {
                    skinny.push_back(SkinnyItem{(int)j, sl, lb * 32});
                    scost.push_back((double)std::min(pr.kslice, pr.K - (int64_t)sl * pr.kslice));
                }
            b->sk_count[ui] = (int64_t)skinny.size() - b->sk_start[ui];
        }
    }
    b->reduce_of.assign(n, -1);
    std::vector<int> reduce_list;
    for (size_t j = 0; j < hp.size(); ++j)
        if (hp[j].splits > 1) {
            b->reduce_of[hp_index[j]] = (int)reduce_list.size();
            reduce_list.push_back((int)j);
        }
    b->nreduce = (int)reduce_list.size();
    const std::vector<uint2> gsorted = by_cost(gwork, gcost), psorted = by_cost(pwork, pcost);
    const std::vector<SkinnyItem> ssorted = by_cost(skinny, scost);
    const std::vector<uint2> tsorted = by_cost(twork, tcost);
    const std::vector<uint2> dsorted = by_cost(dwork, dcost);
    b->ndirect = (int64_t)dsorted.size();
    b->ntc = (int64_t)tsorted.size();
    b->ntcpack = (int64_t)tpack.size();
    b->nwork = (int64_t)gsorted.size();
    b->npacked = (int64_t)psorted.size();
    b->npack = (int64_t)pack.size();
    b->nskinny = (int64_t)ssorted.size();
    b->ctas = ctas;
    b->cps = std::min(cps, kMaxCtasPerSm);

    e = cudaMalloc(&b->d_partial, sizeof(float) * (size_t)std::max<int64_t>(partial_floats, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_packed, sizeof(float) * (size_t)std::max<int64_t>(packed_floats, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles16, sizeof(uint16_t) * (size_t)std::max<int64_t>(tc_elems, 1));
    if (e == cudaSuccess)
        for (size_t j = 0; j < hp.size(); ++j)
            if (tc_off[j] >= 0) {
                hp[j].tA = b->d_tiles16 + tc_off[j];
                hp[j].tB = b->d_tiles16 + tc_off[j] + (int64_t)hp[j].tiles_m * hp[j].nkt * TC_TILE_ELEMS;
            }
    if (e == cudaSuccess)
        for (size_t j = 0; j < hp.size(); ++j) {
            hp[j].partial = partial_off[j] >= 0 ? b->d_partial + partial_off[j] : nullptr;
            if (packed_off[j] >= 0) {
                hp[j].pA = b->d_packed + packed_off[j];
                hp[j].pB = b->d_packed + packed_off[j] + a64(hp[j].Kp * hp[j].bm * (int64_t)hp[j].tiles_m);
            }
        }
    if (e == cudaSuccess) e = upload(&b->d_reduce, reduce_list);
    if (e == cudaSuccess) e = upload(&b->d_probs, hp);
    if (e == cudaSuccess) e = upload(&b->d_work, gsorted);
    if (e == cudaSuccess) e = upload(&b->d_packed_work, psorted);
    if (e == cudaSuccess) e = upload(&b->d_pack, pack);
    if (e == cudaSuccess) e = upload(&b->d_skinny, ssorted);
    if (e == cudaSuccess) e = upload(&b->d_tables, tables);
    if (e == cudaSuccess) e = upload(&b->d_work_by_problem, gwork);
    if (e == cudaSuccess) e = upload(&b->d_packed_by_problem, pwork);
    if (e == cudaSuccess) e = upload(&b->d_skinny_by_problem, skinny);
    if (e == cudaSuccess) e = upload(&b->d_tc_work, tsorted);
    if (e == cudaSuccess) e = upload(&b->d_tc_work_by_problem, twork);
    if (e == cudaSuccess) e = upload(&b->d_tc_pack, tpack);
    if (e == cudaSuccess) e = upload(&b->d_direct, dsorted);
    if (e == cudaSuccess) e = upload(&b->d_direct_by_problem, dwork);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 2 * sizeof(unsigned long long));
    b->serial = o.serial != 0;
    if (e == cudaSuccess && !b->serial) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
        }
    }
    if (e == cudaSuccess) b->d_err = device_error_word();
    if (e == cudaSuccess && !b->d_err) e = cudaErrorInitializationError;
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        gett_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? GETT_ERR_NOMEM : GETT_ERR_CUDA;
    }
    *out = b;
    return GETT_OK;
}

}  // namespace

// The planning above uses host containers: a failed host allocation maps to
// GETT_ERR_NOMEM instead of an exception crossing the C boundary.
extern "C" int gett_batch_create(int n, const gett_problem_desc *probs, const gett_batch_options *opt,
                                 gett_batch **out, int *bad_index)
{
    try {
        return batch_create_impl(n, probs, opt, out, bad_index);
    } catch (const std::bad_alloc &) {
        return GETT_ERR_NOMEM;
    } catch (const std::length_error &) {
        return GETT_ERR_NOMEM;
    }
}

namespace {

// Item ranges of one launch: the whole batch, or one problem's items (the
// autotuner), each list repeated `copies` times through the kernels' wrap.
struct Ranges {
    const uint2 *gw;
    int64_t gn;
    const uint2 *pw;
    int64_t pn;
    const PackItem *pk;
    int64_t kn;
    const SkinnyItem *sk;
    int64_t sn;
    const int *red;
    int nred;
    int64_t copies;
    const uint2 *tw;
    int64_t tn;
    const TcPackItem *tk;
    int64_t tkn;
    const uint2 *dw;  // short-sum tile runs
    int64_t dn;
};

// The method chains of a launch touch disjoint outputs (every problem runs
// one method, and problems' C regions do not overlap) and disjoint
// workspaces, so they are independent: (1) packing + packed tiles,
// (2) tensor-core packing + tensor-core tiles, (3) gathered tiles, (4) skinny
// warp items, (5) short sums.  The ordered reduction of K-slice partials
// runs after all of them.  Unless the launch is serial, chains 2-5 run on
// branch streams that wait for an event recorded on the launch stream, and
// the launch stream waits for each branch's join event before the
// reduction; the same calls build a forked graph under stream capture.
// Each chain's kernels are persistent and sized to the whole GPU, so a
// branch mostly fills the SMs the others leave idle (ramps, tails,
// latency-bound stretches).
cudaError_t enqueue_ranges(gett_batch *b, const Ranges &r, cudaStream_t s, bool concurrent)
{
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t c = r.copies;
    const bool has[4] = {r.tkn > 0 || r.tn > 0, r.gn > 0, r.sn > 0, r.dn > 0};
    const bool fork = concurrent && b->fork;
    cudaStream_t bs[4] = {s, s, s, s};
    if (fork) {
        e = cudaEventRecord(b->fork, s);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i)
            if (has[i]) {
                bs[i] = b->branch[i];
                e = cudaStreamWaitEvent(bs[i], b->fork, 0);
            }
        if (e != cudaSuccess) return e;
    }
    // issue order as in a serial launch: packing (chain 1), tensor-core
    // packing and tiles (chain 2), packed tiles (chain 1), gathered tiles
    // (chain 3; the work counters were reset on the launch stream before the
    // fork), skinny items (chain 4), short sums (chain 5)
    if (r.kn > 0)
        launch_batch_pack((int)std::min<int64_t>(r.kn * c, (int64_t)b->sms * 8), s, b->d_probs, r.pk, r.kn * c, r.kn,
                          b->d_tables);
    if (r.tkn > 0)
        launch_batch_tc_pack((int)std::min<int64_t>(r.tkn * c, (int64_t)b->sms * 8), bs[0], b->d_probs, r.tk,
                             r.tkn * c, r.tkn, b->d_tables);
    if (r.tn > 0) {
        e = launch_batch_tc_tiles((int)std::min<int64_t>(b->sms, r.tn * c), bs[0], b->d_probs, r.tw, r.tn * c,
                                  r.tn, b->d_tables, b->d_err);
        if (e != cudaSuccess) return e;
    }
    if (r.pn > 0) {
        const int ctas = (int)std::min<int64_t>((int64_t)b->sms * batch_packed_ctas_per_sm(), r.pn * c);
        launch_batch_packed_tiles(batch_packed_ctas_per_sm(), ctas, s, b->d_probs, r.pw, r.pn * c, r.pn, b->d_tables,
                                  b->d_err);
    }
    if (r.gn > 0) {
        const int ctas = (int)std::min<int64_t>(b->ctas, r.gn * c);
        launch_batch_kernel(b->cps, ctas, bs[1], b->d_probs, r.gw, r.gn * c, r.gn, b->d_tables, b->d_counter);
    }
    if (r.sn > 0)
        launch_batch_skinny((int)std::min<int64_t>((r.sn * c + 7) / 8, (int64_t)b->sms * 4), bs[2], b->d_probs, r.sk,
                            r.sn * c, r.sn, b->d_tables);
    if (r.dn > 0)
        launch_batch_direct((int)std::min<int64_t>((int64_t)b->sms * 4, r.dn * c), bs[3], b->d_probs, r.dw, r.dn * c,
                            r.dn, b->d_tables, b->d_counter + 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (fork) {
        for (int i = 0; i < 4 && e == cudaSuccess; ++i)
            if (has[i]) {
                e = cudaEventRecord(b->join[i], bs[i]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[i], 0);
            }
        if (e != cudaSuccess) return e;
    }
    if (r.nred > 0)
        batch_reduce_kernel<<<std::min(r.nred, b->ctas), 256, 0, s>>>(b->d_probs, r.red, r.nred, b->d_tables);
    return cudaGetLastError();
}

}  // namespace

static cudaError_t enqueue(gett_batch *b, cudaStream_t s)
{
    const Ranges r{b->d_work, b->nwork, b->d_packed_work, b->npacked, b->d_pack, b->npack,
                   b->d_skinny, b->nskinny, b->d_reduce, b->nreduce, 1,
                   b->d_tc_work, b->ntc, b->d_tc_pack, b->ntcpack, b->d_direct, b->ndirect};
    return enqueue_ranges(b, r, s, !b->serial);
}

extern "C" int gett_batch_launch(gett_batch *b, void *stream)
{
    if (!b) return GETT_ERR_ARG;
    cudaError_t e = enqueue(b, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return GETT_OK;
}

extern "C" int gett_batch_launch_graph(gett_batch *b, void *stream)
{
    if (!b) return GETT_ERR_ARG;
    cudaError_t e = cudaSuccess;
    if (!b->exec) {
        if (!b->cap) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue(b, b->cap);
            e = cudaStreamEndCapture(b->cap, &b->graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return GETT_OK;
}

extern "C" int gett_batch_profile(gett_batch *b, int reps, int mode, float *ms_out)
{
    if (!b || reps <= 0 || !ms_out || (mode != 0 && mode != 1)) return GETT_ERR_ARG;
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        ms_out[i] = 0.f;
        const int64_t cnt = b->gw_count[i] + b->pw_count[i] + b->sk_count[i] + b->tw_count[i] + b->dw_count[i];
        if (cnt == 0) continue;
        // throughput mode: enough copies of the problem's items to give every
        // persistent CTA (skinny: every warp; tensor cores: every SM) several,
        // so the time reflects its cost in a full GPU
        const int64_t slots = b->sk_count[i] > 0 ? (int64_t)b->sms * 32
                              : (b->tw_count[i] > 0 ? (int64_t)b->sms : (int64_t)b->ctas);
        const int64_t copies = mode == 1 ? std::min<int64_t>(64, std::max<int64_t>(1, (4 * slots + cnt - 1) / cnt)) : 1;
        const int red = b->reduce_of[i];
        const Ranges r{b->d_work_by_problem + b->gw_start[i], b->gw_count[i],
                       b->d_packed_by_problem + b->pw_start[i], b->pw_count[i],
                       b->d_pack + b->pk_start[i], b->pk_count[i],
                       b->d_skinny_by_problem + b->sk_start[i], b->sk_count[i],
                       red >= 0 ? b->d_reduce + red : nullptr, red >= 0 ? 1 : 0, copies,
                       b->d_tc_work_by_problem + b->tw_start[i], b->tw_count[i],
                       b->d_tc_pack + b->tk_start[i], b->tk_count[i],
                       b->d_direct_by_problem + b->dw_start[i], b->dw_count[i]};
        // one problem runs one method: its chain needs no branch streams (and
        // every configuration is timed on the same single stream)
        e = enqueue_ranges(b, r, s, false);  // warm-up
        cudaEventRecord(e0, s);
        for (int rr = 0; rr < reps && e == cudaSuccess; ++rr) e = enqueue_ranges(b, r, s, false);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms_out[i] = ms / reps / (float)copies;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return GETT_OK;
}

extern "C" int gett_batch_get_info(const gett_batch *b, gett_batch_info *info)
{
    if (!b || !info) return GETT_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n = b->n;
    info->nonempty = b->nonempty;
    info->tiles = b->nwork + b->npacked + b->nskinny + b->ntc + b->ndirect;
    info->flops = b->flops;
    for (int i = 0; i < GETT_BATCH_MAX_CONFIGS; ++i) info->config_count[i] = b->config_count[i];
    info->fallbacks = b->fallbacks;
    info->gather_items = b->nwork + b->ndirect;
    info->packed_items = b->npacked;
    info->pack_items = b->npack;
    info->skinny_items = b->nskinny;
    info->tuned_hits = b->tuned_hits;
    info->tc_items = b->ntc;
    info->tc_pack_items = b->ntcpack;
    return GETT_OK;
}

extern "C" int gett_batch_destroy(gett_batch *b)
{
    if (!b) return GETT_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int i = 0; i < 4; ++i) {
        if (b->branch[i]) cudaStreamDestroy(b->branch[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    void *bufs[] = {b->d_probs, b->d_work, b->d_packed_work, b->d_pack, b->d_skinny, b->d_skinny_by_problem,
                    b->d_tables, b->d_packed, b->d_counter, b->d_work_by_problem, b->d_packed_by_problem,
                    b->d_partial, b->d_reduce, b->d_tc_work, b->d_tc_work_by_problem, b->d_tc_pack,
                    b->d_tiles16, b->d_direct, b->d_direct_by_problem};
    for (void *p : bufs)
        if (p) cudaFree(p);
    delete b;
    return GETT_OK;
}

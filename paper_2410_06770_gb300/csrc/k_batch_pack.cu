// k_batch_pack.cu -- the batched launch's PACK and SKINNY methods.
//
// PACK.  A problem's operands are copied once into tile-blocked dense
// matrices: block t of A holds rows [t bm, (t+1) bm) of the M x K operand as
// [Kp][bm] floats (the A-free modes fused into one contiguous index, the
// contracted modes into another; zeros beyond M and K), block t of B the same
// for [Kp][bn].  This is the physical counterpart of the planner's mode
// fusion: after it every K step of a tile is one contiguous run of bytes, so
// the tile kernel stages its operands with bulk copies (cp.async.bulk, an
// mbarrier per stage) through a ring of PSTAGES shared-memory stages instead
// of chains of gathered loads.  bf16 operands are widened exactly to fp32
// while packing.  Within a K step the block's rows are interleaved -- row w
// at position (w % 16) T + w / 16, T = bw / 16 the register tile's height --
// so the T rows one thread multiplies are adjacent and arrive as one vector
// read from shared memory.
//
// The packing kernel reads a 64 x bm (bn) block of the strided operand along
// whichever of its two indices has the smaller increment, transposes it
// through shared memory and writes packed rows along the block's row index.
//
// SKINNY.  One free class of at most 8 indices (S outputs per long index),
// a sum of more than 8 terms: GEMV- and dot-like problems.  A warp item is a
// K slice of 32 long indices (lanes along the long class, each lane S running
// sums) or, when the outputs are few (L, S <= 4), a K slice with lanes
// along the sum followed by a fixed shuffle tree.  K slices write partial
// results that the batch's ordered reduction adds into C.
#include <cuda_runtime.h>

#include "batch_common.cuh"
#include "tc_common.cuh"

namespace gett {

namespace {

__device__ __forceinline__ float load_f(const void *base, int64_t off, int dtype)
{
    return dtype ? bf16_bits_to_float(__ldg(static_cast<const uint16_t *>(base) + off))
                 : __ldg(static_cast<const float *>(base) + off);
}

// ---------------------------------------------------------------------------
// packing
// ---------------------------------------------------------------------------
constexpr int PK = 64;  // contracted indices per packing item

__global__ void __launch_bounds__(256, 4) batch_pack_kernel(const BatchProb *__restrict__ probs,
                                                         const PackItem *__restrict__ items, int64_t n,
                                                         int64_t wrap, const int64_t *__restrict__ tables)
{
    __shared__ float tile[PK][65];
    __shared__ int64_t srow[64], sk[PK];
    const int tid = threadIdx.x;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const PackItem it = items[i % wrap];
        const BatchProb &pr = probs[it.prob];
        const BatchTables t = batch_tables(pr, tables);
        const bool isA = it.operand == 0;
        const int bw = isA ? pr.bm : pr.bn;
        const int64_t rows = isA ? pr.M : pr.N, K = pr.K, Kp = pr.Kp;
        const int64_t *rowT = isA ? t.rowA : t.colB;
        const int64_t *kT = isA ? t.kA : t.kB;
        const void *src = isA ? pr.A : pr.B;
        const int fast = isA ? pr.a_m_fast : pr.b_n_fast;
        const int dtype = pr.dtype;
        const int64_t r0 = (int64_t)it.block * bw, k0 = (int64_t)it.chunk * PK;
        const int klen = (int)(Kp - k0 < PK ? Kp - k0 : PK);
        float *dst = const_cast<float *>(isA ? pr.pA : pr.pB) + r0 * Kp + k0 * bw;
        __syncthreads();  // the previous item's tile has been written out
        if (tid < bw) srow[tid] = r0 + tid < rows ? rowT[r0 + tid] : 0;
        else if (tid >= 64 && tid < 64 + klen) sk[tid - 64] = k0 + (tid - 64) < K ? kT[k0 + (tid - 64)] : 0;
        __syncthreads();
        // the block's 64 x bw elements, 16 a thread, every load issued before
        // the first store to shared memory (one round trip, not one per
        // element); bw is 32 or 64, so the index split is shifts and masks:
        // along w first when that is the operand's smaller increment, else
        // along k (64 wide), with out-of-block lanes idle
        const int lbw = bw == 64 ? 6 : 5;
        constexpr int NV = PK * 64 / 256;
        float v[NV];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = tid + u * 256;
            const int w = fast ? (e & (bw - 1)) : (e >> 6), kk = fast ? (e >> lbw) : (e & (PK - 1));
            v[u] = w < bw && kk < klen && r0 + w < rows && k0 + kk < K ? load_f(src, srow[w] + sk[kk], dtype) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = tid + u * 256;
            const int w = fast ? (e & (bw - 1)) : (e >> 6), kk = fast ? (e >> lbw) : (e & (PK - 1));
            if (w < bw && kk < klen) tile[kk][w] = v[u];
        }
        __syncthreads();
        // rows interleaved for the tile kernel: row w goes to position
        // (w % 16) T + w / 16, T = bw / 16 (every shape's register tile),
        // so a thread's T rows w = t + 16 i are adjacent; written in
        // position order (coalesced), read from the row they hold
        const int nel = bw * klen;
        const int T = bw >> 4;
        for (int e = tid; e < nel; e += 256) {
            const int kk = e >> lbw, pos = e & (bw - 1);
            const int w = (pos % T) * 16 + pos / T;
            dst[(int64_t)kk * bw + pos] = tile[kk][w];
        }
    }
}

// ---------------------------------------------------------------------------
// packed tiles
// ---------------------------------------------------------------------------
// T consecutive floats of shared memory (T = 2 or 4, aligned to T floats)
template <int T>
__device__ __forceinline__ void load_run(const float *p, float (&v)[T])
{
    static_assert(T == 2 || T == 4, "register tile of 2 or 4");
    if constexpr (T == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        v[0] = x.x; v[1] = x.y;
    }
}
constexpr int PSTAGES = 6;
constexpr int PBK = 16;  // every shape's BK
constexpr int PSTAGE_FLOATS = PBK * 128;  // largest bm + bn is 128
constexpr size_t PSMEM = (size_t)PSTAGES * PSTAGE_FLOATS * sizeof(float);
constexpr int kPackedWaitError = 5;  // device error code of a bulk-copy wait that gave up

__device__ __forceinline__ void bulk_load(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}

// One work item (tile x K slice) of a packed problem.  `g` counts the stages
// this CTA consumed before (stage u uses slot u % PSTAGES with phase parity
// (u / PSTAGES) & 1).  Returns false when a wait gave up (every thread
// agrees, through the vote of the per-step barrier).
// Stage p of one work item: the A and B runs of K steps [16 p, 16 p + 16)
// of its slice, into slot (g + p) % PSTAGES.  Issued by one thread.
template <int CFG>
struct PackedItemView {
    static constexpr int BM = kB[CFG].bm, BN = kB[CFG].bn;
    static constexpr uint32_t A_STAGE = PBK * BM * 4, B_STAGE = PBK * BN * 4;
    const float *Ab, *Bb;
    int nk, tmi, tni, split;
    __device__ __forceinline__ PackedItemView(const BatchProb &pr, int item)
    {
        const int tile = item / pr.splits;
        split = item % pr.splits;
        tmi = tile / pr.tiles_n;
        tni = tile % pr.tiles_n;
        const int64_t kbeg = (int64_t)split * pr.kps, kend = min(pr.Kp, kbeg + pr.kps);
        nk = (int)((kend - kbeg) / PBK);
        Ab = pr.pA + (int64_t)tmi * pr.Kp * BM + kbeg * BM;
        Bb = pr.pB + (int64_t)tni * pr.Kp * BN + kbeg * BN;
    }
    __device__ __forceinline__ void issue(int p, uint32_t g, float *psm, uint64_t *full) const
    {
        const int s = (int)((g + (uint32_t)p) % PSTAGES);
        float *sA = psm + s * PSTAGE_FLOATS;
        tc::mbar_arrive_expect_tx(&full[s], A_STAGE + B_STAGE);
        bulk_load(sA, Ab + (int64_t)p * PBK * BM, A_STAGE, &full[s]);
        bulk_load(sA + PBK * BM, Bb + (int64_t)p * PBK * BN, B_STAGE, &full[s]);
    }
    // the first PSTAGES - 1 stages (the pipeline fill)
    __device__ __forceinline__ void prologue(uint32_t g, float *psm, uint64_t *full) const
    {
        for (int p = 0; p < PSTAGES - 1 && p < nk; ++p) issue(p, g, psm, full);
    }
};

__device__ __forceinline__ void packed_prologue(const BatchProb &pr, int item, uint32_t g, float *psm, uint64_t *full)
{
    switch (pr.shape) {
    case 0: PackedItemView<0>(pr, item).prologue(g, psm, full); break;
    case 1: PackedItemView<1>(pr, item).prologue(g, psm, full); break;
    case 2: PackedItemView<2>(pr, item).prologue(g, psm, full); break;
    default: PackedItemView<3>(pr, item).prologue(g, psm, full); break;
    }
}

// `pre_issued`: the fill was issued before (during the previous item's
// epilogue).  `between` runs on every thread after the K loop and before the
// epilogue (the caller issues the next item's fill there, so its copies fly
// while this item adds its tile into C); `g` then already counts this item.
template <int CFG, class Between>
__device__ __forceinline__ bool packed_tile(const BatchProb &pr, const int64_t *tables, int item, float *psm,
                                            uint64_t *full, uint32_t &g, int *err, int64_t *s_rc, int64_t *s_cc,
                                            bool pre_issued, Between between)
{
    constexpr BCfg c = kB[CFG];
    constexpr int BM = c.bm, BN = c.bn, TM = c.tm, TN = c.tn, RM = BM / TM, RN = BN / TN;
    const int tid = threadIdx.x;
    const PackedItemView<CFG> v(pr, item);
    const int nk = v.nk, tmi = v.tmi, tni = v.tni, split = v.split;
    if (tid == 0 && !pre_issued) v.prologue(g, psm, full);

    // epilogue offsets first (to shared memory; the K loop's barriers publish
    // them): their loads overlap the pipeline fill
    int tm, tn;
    if (pr.c_m_fast) { tm = tid % RM; tn = tid / RM; }
    else { tn = tid % RN; tm = tid / RN; }
    const int64_t m0 = (int64_t)tmi * BM, n0 = (int64_t)tni * BN;
    if (pr.splits == 1) {
        const BatchTables t = batch_tables(pr, tables);
        if (tid < BM) s_rc[tid] = m0 + tid < pr.M ? t.rowC[m0 + tid] : 0;
        else if (tid >= 128 && tid < 128 + BN) s_cc[tid - 128] = n0 + tid - 128 < pr.N ? t.colC[n0 + tid - 128] : 0;
    }

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
    bool ok = true;
    int kt = 0;
    for (; kt < nk; ++kt) {
        // the slot of stage kt + PSTAGES - 1 was read in stage kt - 1, which
        // every thread finished before the barrier that closed it
        if (tid == 0 && kt + PSTAGES - 1 < nk) v.issue(kt + PSTAGES - 1, g, psm, full);
        const uint32_t u = g + (uint32_t)kt;
        const int s = (int)(u % PSTAGES);
        const bool waited = tc::mbar_wait(&full[s], (u / PSTAGES) & 1, err, kPackedWaitError);
        if (waited) {
            const float *sA = psm + s * PSTAGE_FLOATS;
            const float *sB = sA + PBK * BM;
#pragma unroll
            for (int kk = 0; kk < PBK; ++kk) {
                // the packed rows are interleaved (row w at (w % 16) TM + w / 16):
                // a thread's TM rows tm + 16 i sit side by side, one vector read
                float a[TM], b[TN];
                load_run<TM>(sA + kk * BM + tm * TM, a);
                load_run<TN>(sB + kk * BN + tn * TN, b);
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
        }
        if (!__syncthreads_and(waited)) {
            ok = false;
            break;
        }
    }
    if (!ok) {
        // let the copies already issued land before the CTA winds down
        if (tid == 0) {
            const int issued = min(nk, kt + PSTAGES - 1 + 1);
            for (int p = kt; p < issued; ++p) {
                const uint32_t u = g + (uint32_t)p;
                tc::mbar_drain(&full[u % PSTAGES], (u / PSTAGES) & 1);
            }
        }
        __syncthreads();
        return false;
    }
    g += (uint32_t)nk;
    between();

    if (pr.splits > 1) {
        float *P = pr.partial + (int64_t)split * pr.M * pr.N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t m = m0 + tm + i * RM;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t n = n0 + tn + j * RN;
                if (m < pr.M && n < pr.N) P[pr.c_m_fast ? n * pr.M + m : m * pr.N + n] = acc[i][j];
            }
        }
    } else {
        // C <- C + tile in three phases: offsets, every load, every store.
        // Interleaved load/store pairs would serialise: the compiler cannot
        // move a load above a store through another pointer, so each output
        // would pay a full memory round trip.  The outputs of one tile are
        // distinct (C is injective), so the loads may all go first.
        float *rowp[TM];
        int64_t cc[TN];
        bool vm[TM], vn[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            vm[i] = m0 + tm + i * RM < pr.M;
            rowp[i] = pr.C + (vm[i] ? s_rc[tm + i * RM] : 0);
        }
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            vn[j] = n0 + tn + j * RN < pr.N;
            cc[j] = vn[j] ? s_cc[tn + j * RN] : 0;
        }
        float cv[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) cv[i][j] = vm[i] && vn[j] ? rowp[i][cc[j]] : 0.f;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                if (vm[i] && vn[j]) rowp[i][cc[j]] = cv[i][j] + acc[i][j];
    }
    return true;
}

// Work items of the packed tiles are dealt to the CTAs statically in snake
// order (round r: item r C + c for even r, r C + C - 1 - c for odd r, C CTAs;
// the list is sorted by decreasing cost), so every CTA knows its next items:
// warp 0 loads the next round's descriptor into registers while the current
// tile runs (its work entry one round earlier still) and stores it to the
// other shared-memory slot at the end, so no item starts with a chain of
// dependent loads.
constexpr int kProbWords = (int)(sizeof(BatchProb) / 4);
static_assert(sizeof(BatchProb) % 4 == 0 && kProbWords <= 64, "descriptor copy by one warp, two words a lane");

template <int CPS>
__global__ void __launch_bounds__(BT, CPS) batch_packed_kernel(const BatchProb *__restrict__ probs,
                                                              const uint2 *__restrict__ work, int64_t nwork,
                                                              int64_t wrap, const int64_t *__restrict__ tables,
                                                              int *err)
{
    extern __shared__ __align__(128) float psm[];
    __shared__ uint64_t full[PSTAGES];
    __shared__ int64_t s_rc[64], s_cc[64];
    __shared__ __align__(16) BatchProb s_pr[2];
    __shared__ uint2 s_w[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t C = gridDim.x;
    auto item_of = [&](int64_t r) { return r * C + ((r & 1) ? (C - 1 - blockIdx.x) : (int64_t)blockIdx.x); };
    auto load_words = [&](uint32_t (&wd)[2], unsigned prob) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(probs + prob);
#pragma unroll
        for (int q = 0; q < 2; ++q) wd[q] = lane + 32 * q < kProbWords ? __ldg(src + lane + 32 * q) : 0u;
    };
    auto store_words = [&](const uint32_t (&wd)[2], int slot) {
        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_pr[slot]);
#pragma unroll
        for (int q = 0; q < 2; ++q)
            if (lane + 32 * q < kProbWords) dst[lane + 32 * q] = wd[q];
    };
    uint2 w_next = make_uint2(0, 0);  // warp 0: the work entry of the next round
    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; ++s) tc::mbar_init(&full[s], 1);
        tc::fence_barrier_init();
    }
    if (warp == 0 && item_of(0) < nwork) {
        const uint2 w0 = work[item_of(0) % wrap];
        uint32_t wd[2];
        load_words(wd, w0.x);
        store_words(wd, 0);
        if (lane == 0) s_w[0] = w0;
        if (item_of(1) < nwork) w_next = work[item_of(1) % wrap];
    }
    __syncthreads();
    uint32_t g = 0;
    for (int64_t r = 0; item_of(r) < nwork; ++r) {
        const int cur = (int)(r & 1);
        const bool more = item_of(r + 1) < nwork;
        uint32_t wd[2] = {0u, 0u};
        uint2 w_after = make_uint2(0, 0);
        if (warp == 0 && more) {
            load_words(wd, w_next.x);  // used at the end of this round
            if (item_of(r + 2) < nwork) w_after = work[item_of(r + 2) % wrap];
        }
        const BatchProb &pr = s_pr[cur];
        const int item = (int)s_w[cur].y;
        // after this item's K loop: publish the next descriptor, then issue
        // the next item's fill before this item's epilogue
        auto between = [&]() {
            if (warp == 0 && more) {
                store_words(wd, cur ^ 1);
                if (lane == 0) s_w[cur ^ 1] = w_next;
            }
            __syncthreads();
            if (threadIdx.x == 0 && more) packed_prologue(s_pr[cur ^ 1], (int)s_w[cur ^ 1].y, g, psm, full);
        };
        bool ok = true;
        switch (pr.shape) {
        case 0: ok = packed_tile<0>(pr, tables, item, psm, full, g, err, s_rc, s_cc, r > 0, between); break;
        case 1: ok = packed_tile<1>(pr, tables, item, psm, full, g, err, s_rc, s_cc, r > 0, between); break;
        case 2: ok = packed_tile<2>(pr, tables, item, psm, full, g, err, s_rc, s_cc, r > 0, between); break;
        default: ok = packed_tile<3>(pr, tables, item, psm, full, g, err, s_rc, s_cc, r > 0, between); break;
        }
        if (!ok) break;  // a bounded wait gave up; the error word says so
        if (warp == 0 && more) w_next = w_after;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// skinny warp items
// ---------------------------------------------------------------------------
// Lanes along the long class (LANES_K false) or along the sum (true); the
// two are separate kernels so each keeps its own register budget.
template <bool LANES_K>
__global__ void __launch_bounds__(256, 4) batch_skinny_kernel(const BatchProb *__restrict__ probs,
                                                              const SkinnyItem *__restrict__ items, int64_t n,
                                                              int64_t wrap, const int64_t *__restrict__ tables)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nw) {
        const SkinnyItem it = items[i % wrap];
        const BatchProb &pr = probs[it.prob];
        if ((pr.lanes_k != 0) != LANES_K) continue;
        const BatchTables t = batch_tables(pr, tables);
        const bool la = pr.long_is_a != 0;
        const void *X = la ? pr.A : pr.B;
        const void *Y = la ? pr.B : pr.A;
        const int64_t *rowX = la ? t.rowA : t.colB, *kX = la ? t.kA : t.kB;
        const int64_t *rowY = la ? t.colB : t.rowA, *kY = la ? t.kB : t.kA;
        const int64_t L = la ? pr.M : pr.N;
        const int S = (int)(la ? pr.N : pr.M);
        const int dtype = pr.dtype;
        const int64_t k0 = (int64_t)it.slice * pr.kslice, k1 = min(pr.K, k0 + pr.kslice);
        float *P = pr.splits > 1 ? pr.partial + (int64_t)it.slice * pr.M * pr.N : nullptr;
        auto pidx = [&](int64_t l, int s) {
            const int64_t m = la ? l : s, nn = la ? s : l;
            return pr.c_m_fast ? nn * pr.M + m : m * pr.N + nn;
        };
        auto coff = [&](int64_t l, int s) { return la ? t.rowC[l] + t.colC[s] : t.rowC[s] + t.colC[l]; };
        if constexpr (!LANES_K) {
            // lanes along the long class: lane l keeps S running sums over the slice
            const int64_t l = it.l0 + lane;
            const bool valid = l < L;
            const int64_t ox = valid ? rowX[l] : 0;
            int64_t oy[SKINNY_MAX_SHORT];
#pragma unroll
            for (int s = 0; s < SKINNY_MAX_SHORT; ++s) oy[s] = s < S ? rowY[s] : 0;
            float acc[SKINNY_MAX_SHORT];
#pragma unroll
            for (int s = 0; s < SKINNY_MAX_SHORT; ++s) acc[s] = 0.f;
            // the slice's K offsets arrive 32 at a time (one coalesced load a
            // table) and are broadcast by shuffles, so the operand loads of
            // several k are in flight together
            for (int64_t kb = k0; kb < k1; kb += 32) {
                const int64_t kk = kb + lane;
                const int64_t kxl = kk < k1 ? kX[kk] : 0, kyl = kk < k1 ? kY[kk] : 0;
                const int nj = (int)(k1 - kb < 32 ? k1 - kb : 32);
#pragma unroll 4
                for (int j = 0; j < nj; ++j) {
                    const int64_t kx = __shfl_sync(0xffffffffu, kxl, j), ky = __shfl_sync(0xffffffffu, kyl, j);
                    const float x = valid ? load_f(X, ox + kx, dtype) : 0.f;
#pragma unroll
                    for (int s = 0; s < SKINNY_MAX_SHORT; ++s)
                        if (s < S) acc[s] = fmaf(x, load_f(Y, oy[s] + ky, dtype), acc[s]);
                }
            }
            if (valid) {
                if (P) {
#pragma unroll
                    for (int s = 0; s < SKINNY_MAX_SHORT; ++s)
                        if (s < S) P[pidx(l, s)] = acc[s];
                } else {
                    // offsets, then every load, then every store (a load
                    // after a store through another pointer cannot be hoisted)
                    int64_t off[SKINNY_MAX_SHORT];
                    float cv[SKINNY_MAX_SHORT];
#pragma unroll
                    for (int s = 0; s < SKINNY_MAX_SHORT; ++s) off[s] = s < S ? coff(l, s) : 0;
#pragma unroll
                    for (int s = 0; s < SKINNY_MAX_SHORT; ++s) cv[s] = s < S ? pr.C[off[s]] : 0.f;
#pragma unroll
                    for (int s = 0; s < SKINNY_MAX_SHORT; ++s)
                        if (s < S) pr.C[off[s]] = cv[s] + acc[s];
                }
            }
        } else {
            // few outputs (L, S <= 4): lanes along the sum, then a fixed
            // shuffle tree per output
            const int Li = (int)L;
            int64_t ox[4], oy[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ox[q] = q < Li ? rowX[q] : 0;
                oy[q] = q < S ? rowY[q] : 0;
            }
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 2
            for (int64_t k = k0 + lane; k < k1; k += 32) {
                const int64_t kx = kX[k], ky = kY[k];
                float xv[4], yv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    xv[q] = q < Li ? load_f(X, ox[q] + kx, dtype) : 0.f;
                    yv[q] = q < S ? load_f(Y, oy[q] + ky, dtype) : 0.f;
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xv[a], yv[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) acc[a][b] += __shfl_down_sync(0xffffffffu, acc[a][b], d);
            if (lane == 0) {
                if (P) {
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if (a < Li && b < S) P[pidx(a, b)] = acc[a][b];
                } else {
                    int64_t off[4][4];
                    float cv[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) off[a][b] = a < Li && b < S ? coff(a, b) : 0;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) cv[a][b] = a < Li && b < S ? pr.C[off[a][b]] : 0.f;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if (a < Li && b < S) pr.C[off[a][b]] = cv[a][b] + acc[a][b];
                }
            }
        }
    }
}

}  // namespace

void launch_batch_pack(int blocks, cudaStream_t s, const BatchProb *probs, const PackItem *items, int64_t n,
                       int64_t wrap, const int64_t *tables)
{
    if (n > 0) batch_pack_kernel<<<blocks, 256, 0, s>>>(probs, items, n, wrap, tables);
}

// three resident CTAs an SM: 80 registers a thread hold the register tile,
// the read-ahead descriptor and the ring's counters without spilling (at
// four, 64 registers spilled inside the K loop)
int batch_packed_ctas_per_sm() { return 3; }

void launch_batch_packed_tiles(int cps, int ctas, cudaStream_t s, const BatchProb *probs, const uint2 *work,
                               int64_t nwork, int64_t wrap, const int64_t *tables, int *err)
{
    if (nwork <= 0) return;
    (void)cps;
    static const cudaError_t attr =
        cudaFuncSetAttribute(batch_packed_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PSMEM);
    (void)attr;
    batch_packed_kernel<3><<<ctas, BT, PSMEM, s>>>(probs, work, nwork, wrap, tables, err);
}

void launch_batch_skinny(int blocks, cudaStream_t s, const BatchProb *probs, const SkinnyItem *items, int64_t n,
                         int64_t wrap, const int64_t *tables)
{
    if (n <= 0) return;
    // each kernel skips the other's items (a warp-uniform test on the item)
    batch_skinny_kernel<false><<<blocks, 256, 0, s>>>(probs, items, n, wrap, tables);
    batch_skinny_kernel<true><<<blocks, 256, 0, s>>>(probs, items, n, wrap, tables);
}

}  // namespace gett

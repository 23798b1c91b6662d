// k_batch_tc.cu -- the batched launch's TC method: problems with bf16
// operands on the 5th-generation tensor cores.
//
// Packing.  Each operand is cut into 128-row blocks and 64-wide K tiles; a
// tile is 128 x 64 bf16 = 16 KB, stored exactly as the tensor core reads it
// from shared memory: row r at byte r * 128, its 16-byte chunk j at chunk
// position j ^ (r & 7) (the 128-byte swizzle TMA applies to a 64-wide bf16
// box).  A plain bulk copy (cp.async.bulk) of a tile into a 1024-byte aligned
// stage therefore gives the image the UMMA shared-memory descriptor of the
// 128-byte-swizzled K-major layout expects, with no tensor map per problem.
// Rows beyond M (N) and k beyond K are zeros.
//
// Tiles.  One CTA per SM, items (problem, 128 x 128 output tile) dealt to the
// CTAs statically in snake order (the list is sorted by decreasing K).  Warp
// 0 streams the item's K tiles of A and B into a four-stage ring; warp 1 owns
// 256 TMEM columns and issues tcgen05.mma (M = 128, N = 128, K = 16, four per
// stage) from one thread into one of two 128-column fp32 accumulators, which
// alternate between items so the epilogue of one item overlaps the MMAs of
// the next; warps 2..9 read their 32-lane quarter and 64-column half of the
// accumulator with tcgen05.ld and add it into C through the problem's
// row/column offset tables.  Every wait is bounded; on a give-up the roles drain what they
// started before TMEM is released, and the error word records the code.
#include <cuda_runtime.h>

#include "batch_common.cuh"
#include "tc_common.cuh"

namespace gett {

namespace {

__device__ __forceinline__ void tc_bulk_load(void *smem_dst, const void *gmem_src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            tc::smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// packing into swizzled tiles
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) batch_tc_pack_kernel(const BatchProb *__restrict__ probs,
                                                            const TcPackItem *__restrict__ items, int64_t n,
                                                            int64_t wrap, const int64_t *__restrict__ tables)
{
    __shared__ __align__(16) uint16_t tile[128][72];  // rows x k; a 144-byte pitch keeps 16-byte reads aligned
    __shared__ int64_t srow[128], sk[64];
    const int tid = threadIdx.x;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const TcPackItem it = items[i % wrap];
        const BatchProb &pr = probs[it.prob];
        const BatchTables t = batch_tables(pr, tables);
        const bool isA = it.operand == 0;
        const int64_t rows = isA ? pr.M : pr.N, K = pr.K;
        const int64_t *rowT = isA ? t.rowA : t.colB;
        const int64_t *kT = isA ? t.kA : t.kB;
        const uint16_t *src = static_cast<const uint16_t *>(isA ? pr.A : pr.B);
        const int fast = isA ? pr.a_m_fast : pr.b_n_fast;
        const int64_t r0 = (int64_t)it.block * 128, k0 = (int64_t)it.ktile * TC_BK;
        uint16_t *dst = const_cast<uint16_t *>(isA ? pr.tA : pr.tB) +
                        ((int64_t)it.block * pr.nkt + it.ktile) * TC_TILE_ELEMS;
        __syncthreads();  // the previous item's tile has been written out
        if (tid < 128) srow[tid] = r0 + tid < rows ? rowT[r0 + tid] : 0;
        else if (tid < 192) sk[tid - 128] = k0 + (tid - 128) < K ? kT[k0 + (tid - 128)] : 0;
        __syncthreads();
        // 32 elements a thread in two halves of 16 loads, each half's loads
        // all issued before its stores to shared memory
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint16_t v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = tid + (h * 16 + u) * 256;
                const int r = fast ? (e & 127) : (e >> 6), kk = fast ? (e >> 7) : (e & (TC_BK - 1));
                v[u] = (r0 + r < rows && k0 + kk < K) ? __ldg(src + srow[r] + sk[kk]) : (uint16_t)0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = tid + (h * 16 + u) * 256;
                const int r = fast ? (e & 127) : (e >> 6), kk = fast ? (e >> 7) : (e & (TC_BK - 1));
                tile[r][kk] = v[u];
            }
        }
        __syncthreads();
        // 16-byte chunks: chunk j of row r goes to chunk position j ^ (r & 7)
        for (int c = tid; c < 128 * 8; c += 256) {
            const int r = c >> 3, j = c & 7;
            const uint4 v = *reinterpret_cast<const uint4 *>(&tile[r][j * 8]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<char *>(dst) + r * 128 + ((j ^ (r & 7)) << 4)) = v;
        }
    }
}

// ---------------------------------------------------------------------------
// grouped tensor-core tiles
// ---------------------------------------------------------------------------
constexpr int TST = 4;  // stages
constexpr int T_TILE_BYTES = TC_TILE_ELEMS * 2;      // 16 KB
constexpr int T_STAGE = 2 * T_TILE_BYTES;            // A and B tiles
constexpr int T_EPI_WARPS = 8;  // lane quarter x column half of the accumulator
constexpr int T_THREADS = (2 + T_EPI_WARPS) * 32;
constexpr int T_SMEM = TST * T_STAGE + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t T_NCOLS = 2 * TC_BN;              // two accumulators
constexpr int kTcWaitError = 6;

__global__ void __launch_bounds__(T_THREADS, 1) batch_tc_kernel(const BatchProb *__restrict__ probs,
                                                                const uint2 *__restrict__ work, int64_t nwork,
                                                                int64_t wrap, const int64_t *__restrict__ tables,
                                                                int *err)
{
    extern __shared__ uint8_t tsm_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tsm_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(base + TST * T_STAGE);
    uint64_t *empty = full + TST;
    uint64_t *accf = empty + TST;
    uint64_t *acce = accf + 2;
    uint64_t *tdone = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tdone + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t C = gridDim.x;
    auto item_of = [&](int64_t r) { return r * C + ((r & 1) ? (C - 1 - blockIdx.x) : (int64_t)blockIdx.x); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < TST; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accf[b], 1);
            tc::mbar_init(&acce[b], T_EPI_WARPS);
        }
        tc::mbar_init(tdone, 1);
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, T_NCOLS);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;  // K tiles issued by this CTA
            bool ok = true;
            for (int64_t r = 0; ok && item_of(r) < nwork; ++r) {
                const uint2 w = work[item_of(r) % wrap];
                const BatchProb &pr = probs[w.x];
                const int tmi = (int)w.y / pr.tiles_n, tni = (int)w.y % pr.tiles_n;
                const uint16_t *a = pr.tA + (int64_t)tmi * pr.nkt * TC_TILE_ELEMS;
                const uint16_t *b = pr.tB + (int64_t)tni * pr.nkt * TC_TILE_ELEMS;
                for (int kt = 0; kt < pr.nkt; ++kt, ++g) {
                    const int s = (int)(g % TST);
                    if (!tc::mbar_wait(&empty[s], ((g / TST) & 1) ^ 1, err, kTcWaitError)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sa = base + s * T_STAGE;
                    tc::mbar_arrive_expect_tx(&full[s], T_STAGE);
                    tc_bulk_load(sa, a + (int64_t)kt * TC_TILE_ELEMS, T_TILE_BYTES, &full[s]);
                    tc_bulk_load(sa + T_TILE_BYTES, b + (int64_t)kt * TC_TILE_ELEMS, T_TILE_BYTES, &full[s]);
                }
            }
            if (!ok) {
                // let the copies already issued land (clock-bounded; the
                // error word is set)
                for (uint32_t j = g > TST ? g - TST : 0; j < g; ++j) tc::mbar_drain(&full[j % TST], (j / TST) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_BM, TC_BN);
            uint32_t g = 0, itc = 0;
            bool ok = true;
            for (int64_t r = 0; ok && item_of(r) < nwork; ++r, ++itc) {
                const BatchProb &pr = probs[work[item_of(r) % wrap].x];
                const int buf = (int)(itc & 1);
                if (!tc::mbar_wait(&acce[buf], ((itc >> 1) & 1) ^ 1, err, kTcWaitError)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d = tmem_base + buf * TC_BN;
                for (int kt = 0; kt < pr.nkt; ++kt, ++g) {
                    const int s = (int)(g % TST);
                    if (!tc::mbar_wait(&full[s], (g / TST) & 1, err, kTcWaitError)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t sa = tc::smem_u32(base + s * T_STAGE);
                    const uint64_t ad = tc::smem_desc_sw128(sa);
                    const uint64_t bd = tc::smem_desc_sw128(sa + T_TILE_BYTES);
#pragma unroll
                    for (int j = 0; j < TC_BK / 16; ++j)
                        tc::umma_bf16(d, ad + (uint64_t)(j * 2), bd + (uint64_t)(j * 2), idesc,
                                      (kt > 0 || j > 0) ? 1u : 0u);
                    tc::umma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::umma_commit(&accf[buf]);
            }
            if (!ok) {
                // MMAs may still be writing TMEM: wait for all of them
                tc::umma_commit(tdone);
                tc::mbar_drain(tdone, 0);
            }
        }
    } else {
        // epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31
        // and one half of the columns
        const int q = warp & 3, h = (warp - 2) >> 2;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        uint32_t itc = 0;
        for (int64_t r = 0; item_of(r) < nwork; ++r, ++itc) {
            const uint2 w = work[item_of(r) % wrap];
            const BatchProb &pr = probs[w.x];
            const BatchTables t = batch_tables(pr, tables);
            const int tmi = (int)w.y / pr.tiles_n, tni = (int)w.y % pr.tiles_n;
            const int buf = (int)(itc & 1);
            // a warp-uniform give-up: tcgen05.ld and the shuffles below need
            // every lane of the warp
            const bool got = tc::mbar_wait(&accf[buf], (itc >> 1) & 1, err, kTcWaitError);
            if (!__all_sync(0xffffffffu, got)) break;
            tc::tc_fence_after();
            const int64_t m = (int64_t)tmi * TC_BM + q * 32 + lane;
            const bool vm = m < pr.M;
            float *crow = pr.C + (vm ? t.rowC[m] : 0);
#pragma unroll
            for (int cb = 0; cb < TC_BN / 64; ++cb) {
                uint32_t v[32];
                const int col = h * (TC_BN / 2) + cb * 32;
                // the 32 columns' offsets: one coalesced load (lane i holds
                // column col + i), broadcast by shuffles
                const int64_t nl = (int64_t)tni * TC_BN + col + lane;
                const int64_t ccl = nl < pr.N ? t.colC[nl] : 0;
                const int64_t left = pr.N - ((int64_t)tni * TC_BN + col);
                const int ncols = left < 32 ? (int)left : 32;
                int64_t cc[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) cc[i] = __shfl_sync(0xffffffffu, ccl, i);
                // every load of C before any store: interleaved
                // read-modify-writes would serialise (a load after a store
                // through another pointer cannot be hoisted above it); the
                // accumulator is read while those loads are in flight
                float cv[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) cv[i] = vm && i < ncols ? crow[cc[i]] : 0.f;
                tc::tmem_ld_32x32b_x32(tmem_base + lane_addr + buf * TC_BN + col, v);
                tc::tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (vm && i < ncols) crow[cc[i]] = cv[i] + __uint_as_float(v[i]);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[buf]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, T_NCOLS);
    }
}

}  // namespace

void launch_batch_tc_pack(int blocks, cudaStream_t s, const BatchProb *probs, const TcPackItem *items, int64_t n,
                          int64_t wrap, const int64_t *tables)
{
    if (n > 0) batch_tc_pack_kernel<<<blocks, 256, 0, s>>>(probs, items, n, wrap, tables);
}

cudaError_t launch_batch_tc_tiles(int ctas, cudaStream_t s, const BatchProb *probs, const uint2 *work, int64_t nwork,
                                  int64_t wrap, const int64_t *tables, int *err)
{
    if (nwork <= 0) return cudaSuccess;
    static const cudaError_t attr =
        cudaFuncSetAttribute(batch_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, T_SMEM);
    if (attr != cudaSuccess) return attr;
    batch_tc_kernel<<<ctas, T_THREADS, T_SMEM, s>>>(probs, work, nwork, wrap, tables, err);
    return cudaGetLastError();
}

}  // namespace gett

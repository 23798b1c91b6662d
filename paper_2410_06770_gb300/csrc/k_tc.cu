// k_tc.cu -- tensor-core GEMM on packed bf16 operands (tcgen05 + TMA + TMEM).
//
// Every tensor-core form of xGETT first packs its operands into K-major bf16
// matrices (one "slice" per z index: a modulus, a split piece group or a
// batch entry), so this kernel only sees dense matrices:
//     D_z[m, n] = sum_k Ap_z[m, k] * Bp_z[n, k]      (fp32 in TMEM)
// The strided gather, the permutation and the precision logic live in the
// packing kernels and in the epilogues.
//
// Persistent: one CTA per SM walks the 128 x 256 output tiles of every slice
// with a stride of the grid; TMEM, the barriers and the shared-memory ring
// live across its tiles, so the next tile's loads and MMAs run while the
// epilogue finishes the previous one.  Warp 0 issues TMA loads of
// 128x64 (A) and 256x64 (B) bf16 tiles, 128-byte swizzled, into a 4-stage
// shared-memory ring; warp 1 owns the TMEM allocation and issues the
// tcgen05.mma instructions (M=128, N=256, K=16, four per stage) from one
// thread; warps 2..9 are the epilogue: each reads its 32-lane quarter and
// 128-column half of the accumulator with tcgen05.ld.
//
// Epilogue modes:
//  * MODE_MOD (split-precision DGETT): K is processed in chunks short enough
//    that every partial sum of integer residues stays below 2^24 and is
//    therefore exact in fp32; after each chunk the epilogue folds the chunk's
//    accumulator into a running residue modulo p_z held in registers, while
//    the MMA warp already fills the other of two TMEM accumulators.  The
//    final symmetric residues are stored as int8, layout [z][n][m].
//  * MODE_F32: K is processed in chunks of kc_tiles 64-wide tiles; the
//    epilogue adds each chunk's fp32 sum into fp32 running sums held in
//    registers (again overlapping the next chunk's MMAs through the two TMEM
//    accumulators), and finally adds the tile into C through the planner's
//    row/column offset tables (C[rowC[m] + colC[n]]).  Chunking bounds the
//    length of every in-accumulator sum, which keeps long split-precision
//    sums accurate.
//
// Every wait is bounded (tc::mbar_wait); a wait that gives up records an
// error code in the device error word, and all roles fall through to the
// common teardown, which releases TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace gett {

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_EPI_WARPS = 8;
constexpr int NUM_THREADS = (2 + NUM_EPI_WARPS) * 32;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

#define GETT_MF(i) static_cast<float>(kOzModuli[i])
__constant__ float c_moduli[OZ_MAX_L] = {
    GETT_MF(0),  GETT_MF(1),  GETT_MF(2),  GETT_MF(3),  GETT_MF(4),  GETT_MF(5),  GETT_MF(6),
    GETT_MF(7),  GETT_MF(8),  GETT_MF(9),  GETT_MF(10), GETT_MF(11), GETT_MF(12), GETT_MF(13),
    GETT_MF(14), GETT_MF(15), GETT_MF(16), GETT_MF(17), GETT_MF(18), GETT_MF(19)};
#undef GETT_MF

template <int MODE>
__global__ void __launch_bounds__(NUM_THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               TcGemmParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;
    uint64_t *acce = accf + 2;
    uint64_t *tdone = acce + 2;  // teardown: the MMAs issued before a give-up have completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tdone + 1);

    constexpr uint32_t NCOLS = 512;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles t = z * tiles_m * tiles_n + tm * tiles_n + tn, this CTA's being
    // blockIdx.x, blockIdx.x + gridDim.x, ... (the CTAs in flight work on a
    // window of consecutive tiles: row blocks of A shared by their column
    // tiles, one slice of B)
    const int tiles_mn = p.tiles_m * p.tiles_n;
    const int64_t ntile = (int64_t)tiles_mn * p.tiles_z;
    const int nkt = (p.K + BK - 1) / BK;
    const int kc = p.kc_tiles > 0 ? p.kc_tiles : (nkt > 0 ? nkt : 1);
    const int chunks = (nkt + kc - 1) / kc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&accf[b], 1);
            tc::mbar_init(&acce[b], NUM_EPI_WARPS);
        }
        tc::mbar_init(tdone, 1);
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_slot, NCOLS);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            tc::prefetch_tmap(&tmA);
            tc::prefetch_tmap(&tmB);
            // g counts the stage fills of this CTA over all its tiles: fill g
            // uses slot g % STAGES, phase (g / STAGES) & 1, so the ring runs
            // on from one tile into the next
            uint32_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
                const int z = (int)(t / tiles_mn), tl = (int)(t % tiles_mn);
                const int tm = tl / p.tiles_n, tn = tl % p.tiles_n;
                for (int kt = 0; kt < nkt; ++kt, ++g) {
                    const int s = (int)(g % STAGES);
                    if (!tc::mbar_wait(&empty[s], ((g / STAGES) & 1) ^ 1, p.err, tc::ERR_WAIT_EMPTY)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sa = base + s * STAGE_BYTES;
                    tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    tc::tma_load_3d(sa, &tmA, &full[s], kt * BK, tm * BM, z);
                    tc::tma_load_3d(sa + A_BYTES, &tmB, &full[s], kt * BK, tn * BN, z);
                }
            }
            if (!ok) {
                // gave up: let the copies already issued land before the CTA
                // exits (clock-bounded waits; the error word is already set)
                for (uint32_t j = (g > STAGES ? g - STAGES : 0); j < g; ++j)
                    tc::mbar_drain(&full[j % STAGES], (j / STAGES) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, BN);
            bool ok = true;
            uint32_t g = 0;   // stage uses, as the producer counts them
            uint32_t cc = 0;  // accumulator chunks over all tiles: buffer cc & 1
            for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
                for (int c = 0; c < chunks; ++c, ++cc) {
                    const int buf = (int)(cc & 1);
                    if (!tc::mbar_wait(&acce[buf], ((cc >> 1) & 1) ^ 1, p.err, tc::ERR_WAIT_ACC_EMPTY)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t d = tmem_base + buf * BN;
                    const int kbeg = c * kc, kend = min(nkt, (c + 1) * kc);
                    for (int kt = kbeg; kt < kend; ++kt, ++g) {
                        const int s = (int)(g % STAGES);
                        if (!tc::mbar_wait(&full[s], (g / STAGES) & 1, p.err, tc::ERR_WAIT_FULL)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t sa = tc::smem_u32(base + s * STAGE_BYTES);
                        const uint64_t ad = tc::smem_desc_sw128(sa);
                        const uint64_t bd = tc::smem_desc_sw128(sa + A_BYTES);
#pragma unroll
                        for (int j = 0; j < BK / 16; ++j) {
                            // advance 16 bf16 (32 bytes) along K inside the swizzled row
                            tc::umma_bf16(d, ad + (uint64_t)(j * 2), bd + (uint64_t)(j * 2), idesc,
                                          (kt > kbeg || j > 0) ? 1u : 0u);
                        }
                        tc::umma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    tc::umma_commit(&accf[buf]);
                }
            }
            if (!ok) {
                // gave up with MMAs possibly still writing TMEM: one more commit
                // tracks every tcgen05 operation this thread issued; wait for it
                // (clock-bounded) before the common teardown frees TMEM
                tc::umma_commit(tdone);
                tc::mbar_drain(tdone, 0);
            }
        }
    } else {
        // epilogue warps: the same tiles in the same order; the chunk count
        // cc runs on across tiles like the MMA warp's, so while these warps
        // finish a tile (its last fold and its store) the MMAs of the next
        // tile already fill the other accumulator
        const int ew = warp - 2;
        const int q = warp & 3;   // TMEM lane quarter this warp may access
        const int h = ew >> 2;    // 128-column half
        const int row = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        uint32_t cc = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            const int z = (int)(t / tiles_mn), tl = (int)(t % tiles_mn);
            const int tm = tl / p.tiles_n, tn = tl % p.tiles_n;
            const int64_t m = (int64_t)tm * BM + row;
            const float pm = MODE == TC_MODE_MOD ? c_moduli[z] : 1.f;
            const float inv = 1.0f / pm;
            float res[128];
#pragma unroll
            for (int i = 0; i < 128; ++i) res[i] = 0.f;
            for (int c = 0; c < chunks; ++c, ++cc) {
                const int buf = (int)(cc & 1);
                // the give-up is made warp-uniform: tcgen05.ld below (and the
                // shuffles of the store) need every lane of the warp
                const bool got = tc::mbar_wait(&accf[buf], (cc >> 1) & 1, p.err, tc::ERR_WAIT_ACC_FULL);
                if (!__all_sync(0xffffffffu, got)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
#pragma unroll
                for (int cb = 0; cb < 4; ++cb) {
                    uint32_t v[32];
                    tc::tmem_ld_32x32b_x32(tmem_base + lane_addr + buf * BN + h * 128 + cb * 32, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float x = res[cb * 32 + i] + __uint_as_float(v[i]);
                        if (MODE == TC_MODE_MOD) {
                            // exact: |res| <= p/2 + 3 and |chunk sum| < 2^24 - 2^8;
                            // q = nearest integer of x / p via the 1.5 * 2^23 constant
                            const float qq = __fadd_rn(__fmaf_rn(x, inv, 12582912.0f), -12582912.0f);
                            res[cb * 32 + i] = fmaf(-qq, pm, x);
                        } else {
                            res[cb * 32 + i] = x;
                        }
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acce[buf]);
            }
            if (MODE == TC_MODE_MOD) {
                if (ok && m < p.M) {
                    const float half = 0.5f * (pm - 1.f);
                    int8_t *R = p.R + (int64_t)z * p.N * p.M;
#pragma unroll
                    for (int i = 0; i < 128; ++i) {
                        const int64_t n = (int64_t)tn * BN + h * 128 + i;
                        float r = res[i];
                        r = r > half ? r - pm : r;
                        r = r < -half ? r + pm : r;
                        if (n < p.N) R[n * p.M + m] = (int8_t)__float2int_rn(r);
                    }
                }
            } else if (__all_sync(0xffffffffu, ok)) {
                // the warp's 128 columns: lane l loads the offset and mark of
                // columns 32 j + l (j < 4) once, and shuffles broadcast them;
                // then C is read eight columns at a time with every load issued
                // before the group's stores (a load after a store through
                // another pointer cannot be hoisted above it, so one
                // read-modify-write per column would each pay a round trip)
                const int64_t nb = (int64_t)tn * BN + h * 128;
                int64_t ccol[4];
                uint32_t cskip[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t n = nb + 32 * j + lane;
                    ccol[j] = n < p.N ? p.colC[n] : 0;
                    cskip[j] = n < p.N ? (p.flagB ? p.flagB[n] : 0u) : 1u;
                }
                const bool row_ok = m < p.M && !(p.flagA && p.flagA[m]);
                float *crow = p.C + (int64_t)z * p.c_slice + (m < p.M ? p.rowC[m] : 0);
#pragma unroll
                for (int g = 0; g < 128; g += 8) {
                    int64_t off[8];
                    bool st[8];
                    float cv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        // every lane runs both shuffles (a shuffle under a
                        // per-lane condition would pair with other lanes' later
                        // shuffles and return wrong offsets)
                        const int i = g + u;
                        off[u] = __shfl_sync(0xffffffffu, ccol[i >> 5], i & 31);
                        const uint32_t skip = __shfl_sync(0xffffffffu, cskip[i >> 5], i & 31);
                        st[u] = row_ok && skip == 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) cv[u] = st[u] && p.smode != SCALE_AX ? crow[off[u]] : 0.f;
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (st[u]) {
                            const float r = res[g + u];
                            crow[off[u]] = p.smode == SCALE_ACC ? cv[u] + r
                                           : (p.smode == SCALE_AX ? p.alpha * r : p.alpha * r + p.beta * cv[u]);
                        }
                }
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, NCOLS);
    }
}

// Failure-detection check: one thread waits on an mbarrier whose phase
// nothing completes (count 2, a single arrival), with a short limit; the
// bounded wait gives up, records ERR_WAIT_FULL in the error word and the
// kernel returns normally.  No fault, no trap, no endless loop.
__global__ void wait_timeout_probe_kernel(int *err, long long limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 2);
        tc::fence_barrier_init();
        tc::mbar_arrive(&bar);  // one of the two expected arrivals: phase 0 never completes
        tc::mbar_wait(&bar, 0, err, tc::ERR_WAIT_FULL, limit);
    }
}

// ---- tensor maps ---------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

// 3-D map over a packed operand [Z][rows][ld] of bf16: box 64 (K) x box_rows.
bool make_map(CUtensorMap *map, const void *ptr, int64_t K, int64_t rows, int64_t ld, int64_t Z, int box_rows)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)Z};
    // the slice pitch matters only with several slices (a single slice never
    // steps along z, and its pitch must still be a valid one)
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(Z > 1 ? ld * 2 * rows : ld * 2)};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

int64_t tc_ld(int64_t K) { return (K + 7) / 8 * 8; }

cudaError_t launch_tc_gemm(int mode, const void *Ap, const void *Bp, int64_t Z, const TcGemmParams &prm,
                           cudaStream_t s)
{
    if (prm.M <= 0 || prm.N <= 0 || prm.K <= 0 || Z <= 0) return cudaSuccess;
    if (Z > 65535 || (mode == TC_MODE_MOD && Z > OZ_MAX_L)) return cudaErrorInvalidValue;
    const int64_t ld = tc_ld(prm.K);
    if ((reinterpret_cast<uintptr_t>(Ap) | reinterpret_cast<uintptr_t>(Bp)) & 15) return cudaErrorInvalidValue;
    // in-place operands: one slice, a pitch of whole 16-byte units
    if ((prm.a_ld || prm.b_ld) && Z != 1) return cudaErrorInvalidValue;
    if ((prm.a_ld & 7) || (prm.b_ld & 7) || prm.a_ld < 0 || prm.b_ld < 0) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, Ap, prm.a_ld ? prm.a_kdim : prm.K, prm.M, prm.a_ld ? prm.a_ld : ld, Z, BM) ||
        !make_map(&mb, Bp, prm.b_ld ? prm.b_kdim : prm.K, prm.N, prm.b_ld ? prm.b_ld : ld, Z, BN))
        return cudaErrorInvalidValue;
    TcGemmParams p = prm;
    p.tiles_m = (int)((p.M + BM - 1) / BM);
    p.tiles_n = (int)((p.N + BN - 1) / BN);
    p.tiles_z = (int)Z;
    if ((int64_t)p.tiles_m * p.tiles_n > INT32_MAX) return cudaErrorInvalidValue;
    // persistent: one CTA per SM (its shared memory and 512 TMEM columns
    // allow no second), each walking the tiles with a stride of the grid
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t ntile = (int64_t)p.tiles_m * p.tiles_n * Z;
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ntile, sms)));
    if (mode == TC_MODE_MOD) {
        if (p.kc_tiles < 1 || p.kc_tiles * BK > OZ_CHUNK_K) return cudaErrorInvalidValue;
        e = cudaFuncSetAttribute(tc_gemm_kernel<TC_MODE_MOD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SMEM_BYTES);
        if (e != cudaSuccess) return e;
        tc_gemm_kernel<TC_MODE_MOD><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, p);
    } else {
        e = cudaFuncSetAttribute(tc_gemm_kernel<TC_MODE_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 SMEM_BYTES);
        if (e != cudaSuccess) return e;
        tc_gemm_kernel<TC_MODE_F32><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(ma, mb, p);
    }
    return cudaGetLastError();
}

}  // namespace gett

namespace gett {
cudaError_t launch_wait_timeout_probe(int *err, long long limit_cycles, cudaStream_t s)
{
    wait_timeout_probe_kernel<<<1, 32, 0, s>>>(err, limit_cycles);
    return cudaGetLastError();
}
}  // namespace gett

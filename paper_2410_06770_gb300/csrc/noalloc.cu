// noalloc.cu -- dgett_noalloc: the double-precision contraction on the dense
// CUDA-core kernel, with the kernel's scratch memory (the class offset
// tables) taken from one fixed device array instead of memory allocated for
// the call.
//
// Who needs it: callers that must not enter the CUDA allocator while they
// run.  Examples: a serving process that reserves the device memory it may
// use up front and treats any allocation on its request path as an error;
// latency-critical loops where cudaFree's implicit device-wide
// synchronisation (and the allocator's locks) would stall other streams;
// code embedded in a framework whose own caching allocator owns all device
// memory.  The regular entry points allocate their workspace per call from
// the stream-ordered pool; this one allocates nothing.
//
// The array: g_noalloc_scratch, 2 * GETT_NOALLOC_MAX_INDEX_SUM int64 entries
// (4 MiB), a file-scope __device__ array; every GPU that loads the library
// holds it until the process exits.  Host code only sees a host-side stand-in
// for the symbol, so the device address is looked up with
// cudaGetSymbolAddress once per device (on the first call made with that
// device current) and passed to the kernels.
//
// Sharing: every call uses the same array and the array keeps the previous
// call's contents.  Nothing in it needs to start at zero: the table kernel
// overwrites every entry the contraction kernel reads before it reads it.
// Two calls whose work overlaps on the GPU (different streams, or another
// thread) race on the array and may produce wrong results; callers must
// order their calls (one stream, or events).
#include <cuda_runtime.h>

#include <mutex>

#include "gett.h"
#include "internal.h"
#include "kernels.h"
#include "select.h"

namespace gett {

namespace {

constexpr int64_t kNoallocEntries = 2 * (int64_t)GETT_NOALLOC_MAX_INDEX_SUM;

static __device__ __align__(256) int64_t g_noalloc_scratch[kNoallocEntries];

struct NoallocDev {
    bool init = false;
    int64_t *ptr = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
};
NoallocDev g_noalloc_dev[64];
std::mutex g_noalloc_mu;

int noalloc_device(NoallocDev **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocDev &d = g_noalloc_dev[dev];
    if (!d.init) {
        int64_t *ptr = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_noalloc_scratch);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return GETT_ERR_CUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return GETT_ERR_CUDA;
        }
        d.ptr = ptr;
        d.sms = sms;
        d.init = true;
    }
    *out = &d;
    return GETT_OK;
}

// byte ranges in 128-bit arithmetic: element spans up to 2^62 times 8 bytes
// do not fit 64 bits
bool overlap(const void *p, int64_t lo, int64_t hi, const void *q, int64_t qlo, int64_t qhi)
{
    const __int128 a0 = (__int128)reinterpret_cast<intptr_t>(p) + (__int128)lo * 8;
    const __int128 a1 = (__int128)reinterpret_cast<intptr_t>(p) + ((__int128)hi + 1) * 8;
    const __int128 b0 = (__int128)reinterpret_cast<intptr_t>(q) + (__int128)qlo * 8;
    const __int128 b1 = (__int128)reinterpret_cast<intptr_t>(q) + ((__int128)qhi + 1) * 8;
    return a0 < b1 && b0 < a1;
}

// tile configuration: the heuristic's when it picks the dense kernel,
// otherwise the largest tile that still gives one tile per SM (no split-K:
// its partial tiles would need more scratch)
int noalloc_config(const Plan &p, int sms)
{
    const Choice h = heuristic_choice(p, DT_F64, sms);
    if (h.family == GETT_FAMILY_DENSE && h.split_k == 1) return h.config;
    for (int cfg = 0; cfg < DENSE_NUM_CONFIGS; ++cfg) {
        int bm, bn, bk;
        dense_tile_shape(cfg, &bm, &bn, &bk);
        if (((p.M + bm - 1) / bm) * ((p.N + bn - 1) / bn) >= sms) return cfg;
    }
    return DENSE_NUM_CONFIGS - 1;
}

}  // namespace

}  // namespace gett

extern "C" int dgett_noalloc(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A, int RANKB,
                             const int64_t *EXTB, const int64_t *INCB, const double *B, int CONTS,
                             const int *CONTA, const int *CONTB, const int *PERM, const int64_t *INCC, double *C,
                             void *stream)
{
    using namespace gett;
    Args a{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC};
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(bad);
    if (rc != GETT_OK) return rc;
    if (p.empty) return GETT_OK;
    if (!A || reinterpret_cast<uintptr_t>(A) % 8) { set_last_error_arg(4); return GETT_ERR_ARG; }
    if (!B || reinterpret_cast<uintptr_t>(B) % 8) { set_last_error_arg(8); return GETT_ERR_ARG; }
    if (!C || reinterpret_cast<uintptr_t>(C) % 8) { set_last_error_arg(14); return GETT_ERR_ARG; }
    if (overlap(C, p.c_lo, p.c_hi, A, p.a_lo, p.a_hi) || overlap(C, p.c_lo, p.c_hi, B, p.b_lo, p.b_hi))
        return GETT_ERR_ALIAS;
    // the offset tables of the three classes must fit the fixed array; each
    // class may count up to 2^62 indices (broadcast modes), so the terms are
    // bounded one by one before they are added (the sum then stays below
    // 3 * GETT_NOALLOC_MAX_INDEX_SUM)
    const int64_t lim = (int64_t)GETT_NOALLOC_MAX_INDEX_SUM;
    if (p.M > lim || p.N > lim || p.K > lim || p.M + p.N + p.K > lim) {
        set_last_error_arg(0);
        return GETT_ERR_UNSUPPORTED;
    }
    NoallocDev *d = nullptr;
    rc = noalloc_device(&d);
    if (rc != GETT_OK) return rc;
    const int cfg = noalloc_config(p, d->sms);
    cudaError_t e = launch_dense(p, DT_F64, A, B, C, cfg, 1, d->ptr, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return GETT_OK;
}

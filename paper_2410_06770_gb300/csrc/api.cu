// api.cu -- the exported C ABI: argument checks, family selection, scratch
// memory and dispatch to the kernel families.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "kernels.h"
#include "select.h"
#include "tc_gemm.h"

namespace gett {

namespace {

struct DevState {
    bool init = false;
    int sms = 0;
    int *err = nullptr;  // device error word written by kernels with bounded waits
};
DevState g_dev[64];
std::mutex g_mu;

int dev_state(DevState **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &st = g_dev[dev];
    if (!st.init) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return GETT_ERR_CUDA;
        }
        int *err = nullptr;
        e = cudaMalloc(&err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return GETT_ERR_CUDA;
        }
        // keep memory freed by cudaFreeAsync in the device pool instead of
        // returning it to the driver at every synchronisation
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        st.sms = sms;
        st.err = err;
        st.init = true;
    }
    *out = &st;
    return GETT_OK;
}

size_t out_elem_size(DType t) { return t == DT_BF16 ? 4 : dtype_size(t); }
size_t in_align(DType t) { return t == DT_C64 ? 16 : (t == DT_C32 ? 8 : dtype_size(t)); }
size_t out_align(DType t) { return t == DT_BF16 ? 4 : in_align(t); }

// byte ranges in 128-bit arithmetic (spans of broadcast-heavy layouts may
// exceed 2^63 bytes)
bool ranges_overlap(const void *p, int64_t lo, int64_t hi, size_t esz, const void *q, int64_t qlo,
                    int64_t qhi, size_t qesz)
{
    const __int128 a0 = (__int128)reinterpret_cast<intptr_t>(p) + (__int128)lo * (int64_t)esz;
    const __int128 a1 = (__int128)reinterpret_cast<intptr_t>(p) + ((__int128)hi + 1) * (int64_t)esz;
    const __int128 b0 = (__int128)reinterpret_cast<intptr_t>(q) + (__int128)qlo * (int64_t)qesz;
    const __int128 b1 = (__int128)reinterpret_cast<intptr_t>(q) + ((__int128)qhi + 1) * (int64_t)qesz;
    return a0 < b1 && b0 < a1;
}

cudaError_t run_family(const Plan &p, DType t, const Choice &ch, const void *A, const void *B, void *C,
                       const DevState &st, cudaStream_t s)
{
    size_t ws_bytes = 0;
    if (ch.family == GETT_FAMILY_DENSE) ws_bytes = dense_workspace_bytes(p, t, ch.config, ch.split_k);
    else if (ch.family == GETT_FAMILY_REDUCE) ws_bytes = reduce_workspace_bytes(p, t, st.sms);
    else if (ch.family == GETT_FAMILY_SKINNY) ws_bytes = skinny_workspace_bytes(p, t, st.sms);
    else if (ch.family == GETT_FAMILY_TC)
        ws_bytes = ch.algo != GETT_ALGO_OZAKI_BF16 ? tc_split_workspace_bytes(p, ch.algo)
                   : (t == DT_C64 ? ozaki_complex_workspace_bytes(p, ch.moduli) : ozaki_workspace_bytes(p, ch.moduli));
    void *ws = nullptr;
    cudaError_t e = cudaSuccess;
    if (ws_bytes) {
        e = cudaMallocAsync(&ws, ws_bytes, s);
        if (e != cudaSuccess) return e;
    }
    switch (ch.family) {
    case GETT_FAMILY_DENSE: e = launch_dense(p, t, A, B, C, ch.config, ch.split_k, ws, s); break;
    case GETT_FAMILY_OUTER: e = launch_outer(p, t, A, B, C, st.sms, s); break;
    case GETT_FAMILY_REDUCE: e = launch_reduce(p, t, A, B, C, st.sms, ws, s); break;
    case GETT_FAMILY_SKINNY: e = launch_skinny(p, t, A, B, C, st.sms, ws, s); break;
    case GETT_FAMILY_TC:
        if (ch.algo != GETT_ALGO_OZAKI_BF16) e = launch_tc_split(p, t, ch.algo, A, B, C, ws, st.sms, st.err, s);
        else if (t == DT_C64) e = launch_ozaki_complex(p, ch.moduli, A, B, C, ws, st.sms, st.err, s);
        else e = launch_ozaki(p, ch.moduli, A, B, C, ws, st.sms, st.err, s);
        break;
    default: e = cudaErrorInvalidValue; break;
    }
    if (ws) {
        cudaError_t f = cudaFreeAsync(ws, s);
        if (e == cudaSuccess) e = f;
    }
    return e;
}

// C <- beta * C only (the scaled form with alpha == 0 or an empty sum): A and
// B are not read.
int run_scale_only(DType t, const Plan &p, void *C, cudaStream_t s, bool sync)
{
    if (p.M * p.N == 0) return GETT_OK;
    if (p.sc.br == 1.0 && p.sc.bi == 0.0) return GETT_OK;
    if (!C || reinterpret_cast<uintptr_t>(C) % out_align(t)) {
        set_last_error_arg(14);
        return GETT_ERR_ARG;
    }
    if (!p.c_injective) return GETT_ERR_ALIAS;
    DevState *st = nullptr;
    int rc = dev_state(&st);
    if (rc != GETT_OK) return rc;
    cudaError_t e = launch_scale_c(p, t, C, st->sms, s);
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return GETT_OK;
}

// Conjugated complex operands (gett_options.conj): each is copied, with its
// imaginary parts negated, into workspace in the planned (row, k) order, and
// the plan is rewritten to read the copy: rows at unit increment, k at R
// times the packed increment of its modes.  Only the operand's own class
// increments change; C's and the other operand's stay.
void pack_increments(ModeList &rows, ModeList &ks, int k_slot, int64_t R)
{
    int64_t st = 1;
    for (int i = 0; i < rows.n; ++i) {
        rows.s0[i] = st;
        st *= rows.ext[i];
    }
    st = R;
    for (int i = 0; i < ks.n; ++i) {
        (k_slot == 0 ? ks.s0 : ks.s1)[i] = st;
        st *= ks.ext[i];
    }
}

cudaError_t conj_operands(Plan &p, DType t, int conj, const void **A, const void **B, int sms, cudaStream_t s,
                          void **ws_out)
{
    *ws_out = nullptr;
    const bool ca = (conj & GETT_CONJ_A) != 0, cb = (conj & GETT_CONJ_B) != 0;
    if (!ca && !cb) return cudaSuccess;
    const size_t esz = dtype_size(t);
    auto elems = [](int64_t r, int64_t k) -> __int128 { return (__int128)r * k; };
    const __int128 na = ca ? elems(p.M, p.K) : 0, nb = cb ? elems(p.N, p.K) : 0;
    const __int128 tab = (__int128)16 * (p.M + p.N + p.K);
    const __int128 bytes = tab + 256 + (na + nb) * (__int128)esz + 256;
    if (bytes > ((__int128)1 << 46)) return cudaErrorMemoryAllocation;  // 64 TB: cannot fit
    char *w = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&w), (size_t)bytes, s);
    if (e != cudaSuccess) return e;
    *ws_out = w;
    int64_t *rowA = reinterpret_cast<int64_t *>(w);
    int64_t *rowC = rowA + p.M, *colB = rowC + p.M, *colC = colB + p.N, *kA = colC + p.N, *kB = kA + p.K;
    size_t off = ((size_t)tab + 255) & ~size_t(255);
    e = launch_build_tables(p, rowA, rowC, colB, colC, kA, kB, s);
    if (e != cudaSuccess) return e;
    const char *Ab = static_cast<const char *>(*A) + p.offA * (int64_t)esz;
    const char *Bb = static_cast<const char *>(*B) + p.offB * (int64_t)esz;
    if (ca) {
        void *dst = w + off;
        off += (((size_t)na * esz + 255) & ~size_t(255));
        e = launch_conj_pack(t, Ab, rowA, kA, p.M, p.K, dst, sms, s);
        if (e != cudaSuccess) return e;
        pack_increments(p.m, p.k, 0, p.M);
        p.offA = 0;
        *A = dst;
    }
    if (cb) {
        void *dst = w + off;
        e = launch_conj_pack(t, Bb, colB, kB, p.N, p.K, dst, sms, s);
        if (e != cudaSuccess) return e;
        pack_increments(p.n, p.k, 1, p.N);
        p.offB = 0;
        *B = dst;
    }
    return cudaSuccess;
}

int run(DType t, const Args &a, const void *A, const void *B, void *C, const gett_options *opt,
        gett_report *rep, cudaStream_t s, bool sync, const Scale *scale = nullptr, bool alpha_zero = false)
{
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(bad);
    if (rc != GETT_OK) return rc;
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        rep->family = GETT_FAMILY_NOOP;
    }
    if (scale) {
        p.sc = *scale;
        if (p.zero_sum || (alpha_zero && !p.empty)) {
            if (!p.zero_sum) p.c_injective = true;  // make_plan returned GETT_ERR_ALIAS otherwise
            return run_scale_only(t, p, C, s, sync);
        }
    }
    if (p.empty) return GETT_OK;
    const size_t esz = dtype_size(t), osz = out_elem_size(t);
    if (!A || reinterpret_cast<uintptr_t>(A) % in_align(t)) { set_last_error_arg(4); return GETT_ERR_ARG; }
    if (!B || reinterpret_cast<uintptr_t>(B) % in_align(t)) { set_last_error_arg(8); return GETT_ERR_ARG; }
    if (!C || reinterpret_cast<uintptr_t>(C) % out_align(t)) { set_last_error_arg(14); return GETT_ERR_ARG; }
    if (ranges_overlap(C, p.c_lo, p.c_hi, osz, A, p.a_lo, p.a_hi, esz) ||
        ranges_overlap(C, p.c_lo, p.c_hi, osz, B, p.b_lo, p.b_hi, esz))
        return GETT_ERR_ALIAS;

    if (opt && (opt->conj & ~(GETT_CONJ_A | GETT_CONJ_B))) {
        set_last_error_arg(0);
        return GETT_ERR_ARG;
    }
    DevState *st = nullptr;
    rc = dev_state(&st);
    if (rc != GETT_OK) return rc;
    const int conj = (opt && (t == DT_C32 || t == DT_C64)) ? opt->conj : 0;
    // the report's time: events around every launch and workspace step
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (rep && sync) {
        if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess ||
            cudaEventRecord(ev[0], s) != cudaSuccess) {
            if (ev[0]) cudaEventDestroy(ev[0]);
            if (ev[1]) cudaEventDestroy(ev[1]);
            ev[0] = ev[1] = nullptr;
        }
    }
    auto finish_timing = [&]() {
        if (!ev[0]) return;
        float ms = 0.f;
        if (cudaEventRecord(ev[1], s) == cudaSuccess && cudaEventSynchronize(ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess && rep)
            rep->time_ms = ms;
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        ev[0] = ev[1] = nullptr;
    };
    void *conj_ws = nullptr;
    if (conj) {
        cudaError_t ce = conj_operands(p, t, conj, &A, &B, st->sms, s, &conj_ws);
        if (ce != cudaSuccess) {
            if (conj_ws) cudaFreeAsync(conj_ws, s);
            finish_timing();
            set_last_cuda_error(ce);
            return ce == cudaErrorMemoryAllocation ? GETT_ERR_NOMEM : GETT_ERR_CUDA;
        }
    }
    Choice ch;
    rc = choose(p, t, opt, st->sms, &ch);
    if (rc != GETT_OK) {
        if (conj_ws) cudaFreeAsync(conj_ws, s);
        finish_timing();
        return rc;
    }
    if (rep) {
        rep->family = ch.family;
        // tensor-core family: the configuration reports the in-place staging
        rep->config = (ch.family == GETT_FAMILY_TC && ch.algo != GETT_ALGO_OZAKI_BF16)
                          ? tc_in_place_mask(p, t, ch.algo, A, B) : ch.config;
        rep->split_k = ch.split_k;
        rep->moduli = ch.moduli;
        rep->selector = ch.selector;
        rep->nm = p.m.n;
        rep->nn = p.n.n;
        rep->nk = p.k.n;
        rep->M = p.M;
        rep->N = p.N;
        rep->K = p.K;
        rep->flops = (t == DT_C32 || t == DT_C64 ? 8.0 : 2.0) * (double)p.M * (double)p.N * (double)p.K;
    }
    cudaError_t e = run_family(p, t, ch, A, B, C, *st, s);
    if (conj_ws) {
        const cudaError_t f = cudaFreeAsync(conj_ws, s);
        if (e == cudaSuccess) e = f;
    }
    finish_timing();
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        // the workspace (offset tables, split-K partials, packed operands,
        // residue planes) did not fit
        return e == cudaErrorMemoryAllocation ? GETT_ERR_NOMEM : GETT_ERR_CUDA;
    }
    if (sync && ch.family == GETT_FAMILY_TC) {
        int word = 0;
        e = cudaMemcpy(&word, st->err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return GETT_ERR_CUDA;
        }
        if (word) {
            cudaMemset(st->err, 0, sizeof(int));
            return GETT_ERR_TIMEOUT;
        }
    }
    return GETT_OK;
}

}  // namespace

int device_sms()
{
    DevState *st = nullptr;
    if (dev_state(&st) != GETT_OK) return 0;
    return st->sms;
}

int *device_error_word()
{
    DevState *st = nullptr;
    if (dev_state(&st) != GETT_OK) return nullptr;
    return st->err;
}

}  // namespace gett

using gett::Args;

#define GETT_ARGS_DECL(T)                                                                      \
    int RANKA, const int64_t *EXTA, const int64_t *INCA, const T *A, int RANKB,               \
        const int64_t *EXTB, const int64_t *INCB, const T *B, int CONTS, const int *CONTA,    \
        const int *CONTB, const int *PERM, const int64_t *INCC
#define GETT_ARGS Args{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC}

#define DEFINE_ENTRY(prefix, T, TC, DT)                                                          \
    extern "C" int prefix##gett(GETT_ARGS_DECL(T), TC *C)                                          \
    {                                                                                             \
        return gett::run(gett::DT, GETT_ARGS, A, B, C, nullptr, nullptr, (cudaStream_t)0, true);  \
    }                                                                                             \
    extern "C" int prefix##gett_async(GETT_ARGS_DECL(T), TC *C, void *stream)                      \
    {                                                                                             \
        return gett::run(gett::DT, GETT_ARGS, A, B, C, nullptr, nullptr, (cudaStream_t)stream,   \
                         false);                                                                  \
    }                                                                                             \
    extern "C" int prefix##gett_ex(GETT_ARGS_DECL(T), TC *C, const gett_options *opt,              \
                                   gett_report *rep, void *stream)                                \
    {                                                                                             \
        return gett::run(gett::DT, GETT_ARGS, A, B, C, opt, rep, (cudaStream_t)stream, true);    \
    }

namespace gett {
namespace {
void re_im(const float *x, double *re, double *im) { *re = *x; *im = 0.0; }
void re_im(const double *x, double *re, double *im) { *re = *x; *im = 0.0; }
void re_im(const gett_complex_float *x, double *re, double *im) { *re = x->re; *im = x->im; }
void re_im(const gett_complex_double *x, double *re, double *im) { *re = x->re; *im = x->im; }

// alpha == 1 and beta == 1 is Alg. 1's accumulation; beta == 0 never reads C.
template <class TC>
int scale_of(const TC *alpha, const TC *beta, Scale *sc, bool *alpha_zero, int pos_alpha = 15)
{
    if (!alpha) { set_last_error_arg(pos_alpha); return GETT_ERR_ARG; }
    if (!beta) { set_last_error_arg(pos_alpha + 1); return GETT_ERR_ARG; }
    re_im(alpha, &sc->ar, &sc->ai);
    re_im(beta, &sc->br, &sc->bi);
    *alpha_zero = sc->ar == 0.0 && sc->ai == 0.0;
    if (sc->ar == 1.0 && sc->ai == 0.0 && sc->br == 1.0 && sc->bi == 0.0) sc->mode = SCALE_ACC;
    else if (sc->br == 0.0 && sc->bi == 0.0) sc->mode = SCALE_AX;
    else sc->mode = SCALE_AXPBY;
    return GETT_OK;
}
// Argument positions: an xGETT position of the equivalent contraction ->
// the position in xGETP (1 RANKA, 2 EXTA, 3 INCA, 4 A, 5 PERM, 6 INCC, 7 C)
// or xGETR (1-4, 5 NRED, 6 RED, 7 PERM, 8 INCC, 9 C).
int getp_pos(int pos)
{
    switch (pos) {
    case 12: return 5;
    case 13: return 6;
    case 14: return 7;
    default: return pos <= 4 ? pos : 0;
    }
}
int getr_pos(int pos)
{
    switch (pos) {
    case 9: return 5;
    case 10: case 11: return 6;
    case 12: return 7;
    case 13: return 8;
    case 14: return 9;
    default: return pos <= 4 ? pos : 0;
    }
}

}  // namespace

// Transpose (Sec. 9 future work): the contraction with a rank-0 B of value 1,
// run by the transpose kernel.
int run_transpose(DType t, int RANKA, const int64_t *EXTA, const int64_t *INCA, const void *A, const int *PERM,
                  const int64_t *INCC, void *C, const Scale &sc, bool alpha_zero, cudaStream_t s)
{
    Args a{RANKA, EXTA, INCA, 0, nullptr, nullptr, 0, nullptr, nullptr, PERM, INCC};
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(getp_pos(bad));
    if (rc != GETT_OK) return rc;
    p.sc = sc;
    if (p.empty) return GETT_OK;
    if (alpha_zero) return run_scale_only(t, p, C, s, true);
    if (!A || reinterpret_cast<uintptr_t>(A) % in_align(t)) { set_last_error_arg(4); return GETT_ERR_ARG; }
    if (!C || reinterpret_cast<uintptr_t>(C) % out_align(t)) { set_last_error_arg(7); return GETT_ERR_ARG; }
    if (ranges_overlap(C, p.c_lo, p.c_hi, out_elem_size(t), A, p.a_lo, p.a_hi, dtype_size(t))) return GETT_ERR_ALIAS;
    DevState *st = nullptr;
    rc = dev_state(&st);
    if (rc != GETT_OK) return rc;
    cudaError_t e = launch_transpose(p, t, A, C, st->sms, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return GETT_OK;
}

// Reduction (Sec. 9 future work): the contraction of A with a B of ones over
// the reduced modes (extents EXTA[RED[t]], every increment 0, so B is the one
// element unit_operand gives); the selector and kernels are the contraction's.
int run_reduce(DType t, int RANKA, const int64_t *EXTA, const int64_t *INCA, const void *A, int NRED,
               const int *RED, const int *PERM, const int64_t *INCC, void *C, const Scale &sc, bool alpha_zero,
               cudaStream_t s)
{
    if (RANKA < 0 || RANKA > GETT_MAX_RANK) { set_last_error_arg(1); return GETT_ERR_ARG; }
    if (RANKA > 0 && !EXTA) { set_last_error_arg(2); return GETT_ERR_ARG; }
    if (NRED < 0 || NRED > RANKA) { set_last_error_arg(5); return GETT_ERR_ARG; }
    if (NRED > 0 && !RED) { set_last_error_arg(6); return GETT_ERR_ARG; }
    if (NRED == 0) return run_transpose(t, RANKA, EXTA, INCA, A, PERM, INCC, C, sc, alpha_zero, s);
    int64_t extb[GETT_MAX_RANK], incb[GETT_MAX_RANK];
    int contb[GETT_MAX_RANK];
    for (int i = 0; i < NRED; ++i) {
        if (RED[i] < 0 || RED[i] >= RANKA) { set_last_error_arg(6); return GETT_ERR_ARG; }
        extb[i] = EXTA[RED[i]];
        incb[i] = 0;
        contb[i] = i;
    }
    Args a{RANKA, EXTA, INCA, NRED, extb, incb, NRED, RED, contb, PERM, INCC};
    {
        // report argument errors before any device call
        Plan p;
        int bad = 0;
        const int rc = make_plan(a, &p, &bad);
        if (rc != GETT_OK) {
            set_last_error_arg(getr_pos(bad));
            return rc;
        }
        if (p.empty && !p.zero_sum) return GETT_OK;
    }
    const void *B = nullptr;
    cudaError_t e = unit_operand(t, &B);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    int rc = run(t, a, A, B, C, nullptr, nullptr, s, true, &sc, alpha_zero);
    if (rc == GETT_ERR_ARG) set_last_error_arg(getr_pos(gett_last_error_arg()));
    return rc;
}

}  // namespace gett

#define DEFINE_AUX(prefix, T, TC, DT)                                                                      \
    extern "C" int prefix##getp(int RANKA, const int64_t *EXTA, const int64_t *INCA, const T *A,            \
                                const int *PERM, const int64_t *INCC, TC *C, const TC *alpha, const TC *beta, \
                                void *stream)                                                               \
    {                                                                                                       \
        gett::Scale sc{};                                                                                   \
        bool az = false;                                                                                    \
        int rc = gett::scale_of(alpha, beta, &sc, &az, 8);                                                  \
        if (rc != GETT_OK) return rc;                                                                       \
        return gett::run_transpose(gett::DT, RANKA, EXTA, INCA, A, PERM, INCC, C, sc, az,                   \
                                   (cudaStream_t)stream);                                                   \
    }                                                                                                       \
    extern "C" int prefix##getr(int RANKA, const int64_t *EXTA, const int64_t *INCA, const T *A, int NRED,  \
                                const int *RED, const int *PERM, const int64_t *INCC, TC *C, const TC *alpha, \
                                const TC *beta, void *stream)                                               \
    {                                                                                                       \
        gett::Scale sc{};                                                                                   \
        bool az = false;                                                                                    \
        int rc = gett::scale_of(alpha, beta, &sc, &az, 10);                                                 \
        if (rc != GETT_OK) return rc;                                                                       \
        return gett::run_reduce(gett::DT, RANKA, EXTA, INCA, A, NRED, RED, PERM, INCC, C, sc, az,           \
                                (cudaStream_t)stream);                                                      \
    }

DEFINE_AUX(s, float, float, DT_F32)
DEFINE_AUX(d, double, double, DT_F64)
DEFINE_AUX(c, gett_complex_float, gett_complex_float, DT_C32)
DEFINE_AUX(z, gett_complex_double, gett_complex_double, DT_C64)
DEFINE_AUX(sb, uint16_t, float, DT_BF16)

#define DEFINE_SCALED(prefix, T, TC, DT)                                                             \
    extern "C" int prefix##gett_scaled(GETT_ARGS_DECL(T), TC *C, const TC *alpha, const TC *beta,      \
                                       const gett_options *opt, gett_report *rep, void *stream)        \
    {                                                                                                 \
        gett::Scale sc{};                                                                             \
        bool az = false;                                                                              \
        int rc = gett::scale_of(alpha, beta, &sc, &az);                                               \
        if (rc != GETT_OK) return rc;                                                                 \
        return gett::run(gett::DT, GETT_ARGS, A, B, C, opt, rep, (cudaStream_t)stream, true, &sc, az); \
    }

DEFINE_SCALED(s, float, float, DT_F32)
DEFINE_SCALED(d, double, double, DT_F64)
DEFINE_SCALED(c, gett_complex_float, gett_complex_float, DT_C32)
DEFINE_SCALED(z, gett_complex_double, gett_complex_double, DT_C64)
DEFINE_SCALED(sb, uint16_t, float, DT_BF16)

DEFINE_ENTRY(s, float, float, DT_F32)
DEFINE_ENTRY(d, double, double, DT_F64)
DEFINE_ENTRY(c, gett_complex_float, gett_complex_float, DT_C32)
DEFINE_ENTRY(z, gett_complex_double, gett_complex_double, DT_C64)
DEFINE_ENTRY(sb, uint16_t, float, DT_BF16)

extern "C" void gett_options_init(gett_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->algo = GETT_ALGO_DEFAULT;
    opt->family = GETT_FAMILY_AUTO;
    opt->config = -1;
    opt->split_k = 0;
    opt->moduli = 0;
}

extern "C" const char *gett_status_string(int status)
{
    switch (status) {
    case GETT_OK: return "GETT_OK";
    case GETT_ERR_ARG: return "GETT_ERR_ARG: invalid argument";
    case GETT_ERR_ALIAS: return "GETT_ERR_ALIAS: C overlaps A/B or is not injective";
    case GETT_ERR_UNSUPPORTED: return "GETT_ERR_UNSUPPORTED: beyond compiled limits";
    case GETT_ERR_CUDA: return "GETT_ERR_CUDA: CUDA error";
    case GETT_ERR_TIMEOUT: return "GETT_ERR_TIMEOUT: device wait exceeded its limit";
    case GETT_ERR_NOMEM: return "GETT_ERR_NOMEM: out of device memory";
    }
    return "unknown gett_status";
}

extern "C" int gett_device_status(void)
{
    gett::DevState *st = nullptr;
    int rc = gett::dev_state(&st);
    if (rc != GETT_OK) return rc;
    cudaError_t e = cudaDeviceSynchronize();
    int word = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&word, st->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        gett::set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    if (word) {
        cudaMemset(st->err, 0, sizeof(int));
        return GETT_ERR_TIMEOUT;
    }
    return GETT_OK;
}

extern "C" int gett_check_wait_timeout(long long limit_cycles)
{
    gett::DevState *st = nullptr;
    int rc = gett::dev_state(&st);
    if (rc != GETT_OK) return rc;
    if (limit_cycles <= 0) return GETT_ERR_ARG;
    cudaError_t e = gett::launch_wait_timeout_probe(st->err, limit_cycles, (cudaStream_t)0);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)0);
    if (e != cudaSuccess) {
        gett::set_last_cuda_error(e);
        return GETT_ERR_CUDA;
    }
    return gett_device_status();
}

extern "C" int gett_version(void) { return 100; }

extern "C" int gett_ozaki_params(int64_t K, int moduli_wanted, int *L, int *bits, int *moduli)
{
    static_assert(GETT_OZAKI_MAX_MODULI == gett::OZ_MAX_L, "modulus table size");
    if (K < 0 || moduli_wanted < 0 || moduli_wanted > GETT_OZAKI_MAX_MODULI || !L || !bits) return GETT_ERR_ARG;
    const int l = gett::ozaki_moduli_for(K, moduli_wanted);
    *L = l;
    *bits = gett::ozaki_bits_for(K, l);
    if (moduli)
        for (int i = 0; i < l; ++i) moduli[i] = gett::kOzModuli[i];
    return GETT_OK;
}

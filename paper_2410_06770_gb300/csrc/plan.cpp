// plan.cpp -- argument validation and the mode-classification planner.
//
// Validation follows the interface of Sec. 5.7: ranks, extents, increments,
// the contracted pairs CONTA/CONTB (distinct, in range, equal extents, Sec.
// 4.5), PERM a permutation of the r_C output positions (Sec. 5.6), one INCC
// entry per output mode.
//
// The planner turns the 14 arguments into three mode classes -- A-free modes
// (M), B-free modes (N) and contracted modes (K) -- so every kernel sees the
// contraction as C[m,n] += sum_k A[m,k] B[k,n] over multi-mode index sets.
// It then (i) drops extent-1 modes, (ii) flips modes so the increment the
// kernels stream along is non-negative (an exact re-indexing of one
// coordinate, moving the base pointer to the other end), (iii) fuses two
// modes of a class when the slower one's increment equals the faster one's
// times its extent in every tensor holding them, and (iv) orders each class
// from smallest to largest increment.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "internal.h"

namespace gett {

namespace {

thread_local int tl_bad_arg = 0;
thread_local int tl_cuda_err = 0;

struct Mode {
    int64_t ext, s0, s1;
};

int64_t iabs64(int64_t x) { return x < 0 ? -x : x; }

// lo/hi element offsets reached by a tensor (relative to its pointer).
void span_of(int rank, const int64_t *ext, const int64_t *inc, int64_t *lo, int64_t *hi)
{
    __int128 l = 0, h = 0;
    for (int i = 0; i < rank; ++i) {
        if (ext[i] <= 0) continue;
        __int128 d = (__int128)(ext[i] - 1) * inc[i];
        if (d < 0) l += d; else h += d;
    }
    *lo = (int64_t)l;
    *hi = (int64_t)h;
}

bool span_fits(int rank, const int64_t *ext, const int64_t *inc)
{
    __int128 s = 0;
    for (int i = 0; i < rank; ++i) {
        if (ext[i] <= 0) continue;
        __int128 d = (__int128)(ext[i] - 1) * (inc[i] < 0 ? -(__int128)inc[i] : (__int128)inc[i]);
        s += d;
        if (s > ((__int128)1 << 62)) return false;
    }
    return true;
}

// Sufficient injectivity test: sorted by |inc|, every increment exceeds the
// largest offset the faster modes can reach.
bool injective(int n, const int64_t *ext, const int64_t *inc)
{
    Mode m[GETT_MAX_RANK * 2];
    int k = 0;
    for (int i = 0; i < n; ++i)
        if (ext[i] > 1) m[k++] = Mode{ext[i], iabs64(inc[i]), 0};
    std::sort(m, m + k, [](const Mode &x, const Mode &y) { return x.s0 < y.s0; });
    __int128 reach = 0;
    for (int i = 0; i < k; ++i) {
        if ((__int128)m[i].s0 <= reach) return false;
        reach += (__int128)m[i].s0 * (m[i].ext - 1);
    }
    return true;
}

int fuse_and_sort(Mode *m, int n, bool sort_by_s1_first)
{
    // fuse: mode j can follow mode i when both of its increments are mode i's
    // increments times mode i's extent
    bool merged = true;
    while (merged) {
        merged = false;
        for (int i = 0; i < n && !merged; ++i) {
            for (int j = 0; j < n && !merged; ++j) {
                if (i == j) continue;
                if ((__int128)m[j].s0 == (__int128)m[i].s0 * m[i].ext &&
                    (__int128)m[j].s1 == (__int128)m[i].s1 * m[i].ext) {
                    m[i].ext *= m[j].ext;
                    for (int t = j; t + 1 < n; ++t) m[t] = m[t + 1];
                    --n;
                    merged = true;
                }
            }
        }
    }
    if (sort_by_s1_first)
        std::stable_sort(m, m + n, [](const Mode &x, const Mode &y) {
            if (iabs64(x.s1) != iabs64(y.s1)) return iabs64(x.s1) < iabs64(y.s1);
            return iabs64(x.s0) < iabs64(y.s0);
        });
    else
        std::stable_sort(m, m + n, [](const Mode &x, const Mode &y) {
            if (iabs64(x.s0) != iabs64(y.s0)) return iabs64(x.s0) < iabs64(y.s0);
            return iabs64(x.s1) < iabs64(y.s1);
        });
    return n;
}

}  // namespace

void set_last_error_arg(int pos) { tl_bad_arg = pos; }
void set_last_cuda_error(int err) { tl_cuda_err = err; }

int make_plan(const Args &a, Plan *p, int *bad_arg)
{
    std::memset(p, 0, sizeof(*p));
    p->sc = Scale{SCALE_ACC, 1.0, 0.0, 1.0, 0.0};
    *bad_arg = 0;
#define BAD(pos)              \
    do {                      \
        *bad_arg = (pos);     \
        return GETT_ERR_ARG;  \
    } while (0)
    if (a.RANKA < 0 || a.RANKA > GETT_MAX_RANK) BAD(1);
    if (a.RANKA > 0 && !a.EXTA) BAD(2);
    if (a.RANKA > 0 && !a.INCA) BAD(3);
    if (a.RANKB < 0 || a.RANKB > GETT_MAX_RANK) BAD(5);
    if (a.RANKB > 0 && !a.EXTB) BAD(6);
    if (a.RANKB > 0 && !a.INCB) BAD(7);
    if (a.CONTS < 0 || a.CONTS > a.RANKA || a.CONTS > a.RANKB) BAD(9);
    if (a.CONTS > 0 && !a.CONTA) BAD(10);
    if (a.CONTS > 0 && !a.CONTB) BAD(11);
    for (int i = 0; i < a.RANKA; ++i)
        if (a.EXTA[i] < 0) BAD(2);
    for (int i = 0; i < a.RANKB; ++i)
        if (a.EXTB[i] < 0) BAD(6);
    if (!span_fits(a.RANKA, a.EXTA, a.INCA)) BAD(3);
    if (!span_fits(a.RANKB, a.EXTB, a.INCB)) BAD(7);
    bool conta_used[GETT_MAX_RANK] = {}, contb_used[GETT_MAX_RANK] = {};
    for (int t = 0; t < a.CONTS; ++t) {
        int ma = a.CONTA[t], mb = a.CONTB[t];
        if (ma < 0 || ma >= a.RANKA || conta_used[ma]) BAD(10);
        if (mb < 0 || mb >= a.RANKB || contb_used[mb]) BAD(11);
        conta_used[ma] = contb_used[mb] = true;
        if (a.EXTA[ma] != a.EXTB[mb]) BAD(11);
    }
    const int rc = a.RANKA + a.RANKB - 2 * a.CONTS;
    if (rc > 0 && !a.PERM) BAD(12);
    bool placed[2 * GETT_MAX_RANK] = {};
    for (int q = 0; q < rc; ++q) {
        int v = a.PERM[q];
        if (v < 0 || v >= rc || placed[v]) BAD(12);
        placed[v] = true;
    }
    if (rc > 0 && !a.INCC) BAD(13);
#undef BAD

    // Classify (free index p = A's free modes ascending, then B's; Sec. 5.6).
    Mode mm[GETT_MAX_RANK], nn[GETT_MAX_RANK], kk[GETT_MAX_RANK];
    int nm = 0, nn_ = 0, nk = 0, fp = 0;
    int64_t extc[2 * GETT_MAX_RANK];
    for (int i = 0; i < a.RANKA; ++i) {
        if (conta_used[i]) continue;
        int q = a.PERM[fp++];
        mm[nm++] = Mode{a.EXTA[i], a.INCA[i], a.INCC[q]};
        extc[q] = a.EXTA[i];
    }
    for (int i = 0; i < a.RANKB; ++i) {
        if (contb_used[i]) continue;
        int q = a.PERM[fp++];
        nn[nn_++] = Mode{a.EXTB[i], a.INCB[i], a.INCC[q]};
        extc[q] = a.EXTB[i];
    }
    for (int t = 0; t < a.CONTS; ++t)
        kk[nk++] = Mode{a.EXTA[a.CONTA[t]], a.INCA[a.CONTA[t]], a.INCB[a.CONTB[t]]};

    if (rc > 0 && !span_fits(rc, extc, a.INCC)) {
        *bad_arg = 13;
        return GETT_ERR_ARG;
    }
    span_of(a.RANKA, a.EXTA, a.INCA, &p->a_lo, &p->a_hi);
    span_of(a.RANKB, a.EXTB, a.INCB, &p->b_lo, &p->b_hi);
    span_of(rc, extc, a.INCC, &p->c_lo, &p->c_hi);

    bool no_out = false, no_sum = false;
    for (int i = 0; i < nm; ++i) no_out |= mm[i].ext == 0;
    for (int i = 0; i < nn_; ++i) no_out |= nn[i].ext == 0;
    for (int i = 0; i < nk; ++i) no_sum |= kk[i].ext == 0;
    p->zero_sum = false;
    p->c_injective = true;
    if (no_out) {
        p->empty = true;
        return GETT_OK;
    }
    const bool inj = rc == 0 || injective(rc, extc, a.INCC);
    if (no_sum) {
        // nothing to accumulate; plan m and n only (for beta * C)
        nk = 0;
        p->zero_sum = true;
        p->c_injective = inj;
    } else if (!inj) {
        return GETT_ERR_ALIAS;
    }

    // (i) squeeze extent-1 modes
    auto squeeze = [](Mode *m, int n) {
        int k = 0;
        for (int i = 0; i < n; ++i)
            if (m[i].ext != 1) m[k++] = m[i];
        return k;
    };
    nm = squeeze(mm, nm);
    nn_ = squeeze(nn, nn_);
    nk = squeeze(kk, nk);
    // index counts of the classes: bounded by the spans for modes that move
    // through memory, but broadcast modes (increment 0 in every tensor that
    // holds them) are not, so a class may not count more than 2^62 indices
    auto count_fits = [](const Mode *m, int n) {
        __int128 P = 1;
        for (int i = 0; i < n; ++i) {
            P *= m[i].ext;
            if (P > ((__int128)1 << 62)) return false;
        }
        return true;
    };
    if (!count_fits(mm, nm) || !count_fits(nn, nn_) || !count_fits(kk, nk)) return GETT_ERR_UNSUPPORTED;

    // (ii) flips: free modes get a positive C increment, contracted modes a
    // non-negative A increment (B's if A's is zero)
    int64_t offA = 0, offB = 0, offC = 0;
    for (int i = 0; i < nm; ++i)
        if (mm[i].s1 < 0) {
            offA += mm[i].s0 * (mm[i].ext - 1);
            offC += mm[i].s1 * (mm[i].ext - 1);
            mm[i].s0 = -mm[i].s0;
            mm[i].s1 = -mm[i].s1;
        }
    for (int i = 0; i < nn_; ++i)
        if (nn[i].s1 < 0) {
            offB += nn[i].s0 * (nn[i].ext - 1);
            offC += nn[i].s1 * (nn[i].ext - 1);
            nn[i].s0 = -nn[i].s0;
            nn[i].s1 = -nn[i].s1;
        }
    for (int i = 0; i < nk; ++i)
        if (kk[i].s0 < 0 || (kk[i].s0 == 0 && kk[i].s1 < 0)) {
            offA += kk[i].s0 * (kk[i].ext - 1);
            offB += kk[i].s1 * (kk[i].ext - 1);
            kk[i].s0 = -kk[i].s0;
            kk[i].s1 = -kk[i].s1;
        }

    // (iii) fuse, (iv) order
    nm = fuse_and_sort(mm, nm, true);
    nn_ = fuse_and_sort(nn, nn_, true);
    nk = fuse_and_sort(kk, nk, false);
    if (nm > GETT_MAX_MODES || nn_ > GETT_MAX_MODES || nk > GETT_MAX_MODES)
        return GETT_ERR_UNSUPPORTED;

    auto store = [](ModeList &dst, const Mode *src, int n, int64_t *prod) {
        dst.n = n;
        int64_t P = 1;
        for (int i = 0; i < n; ++i) {
            dst.ext[i] = src[i].ext;
            dst.s0[i] = src[i].s0;
            dst.s1[i] = src[i].s1;
            P *= src[i].ext;
        }
        *prod = P;
    };
    store(p->m, mm, nm, &p->M);
    store(p->n, nn, nn_, &p->N);
    store(p->k, kk, nk, &p->K);
    p->offA = offA;
    p->offB = offB;
    p->offC = offC;
    p->empty = no_sum;
    if (no_sum) p->K = 0;
    return GETT_OK;
}

}  // namespace gett

extern "C" int gett_last_error_arg(void) { return gett::tl_bad_arg; }
extern "C" int gett_last_cuda_error(void) { return gett::tl_cuda_err; }

extern "C" int gett_plan_describe(int RANKA, const int64_t *EXTA, const int64_t *INCA,
                                  int RANKB, const int64_t *EXTB, const int64_t *INCB,
                                  int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                                  const int64_t *INCC, gett_plan_info *out)
{
    using namespace gett;
    Args a{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC};
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(bad);
    if (rc != GETT_OK) return rc;
    if (!out) return GETT_OK;
    std::memset(out, 0, sizeof(*out));
    out->empty = p.empty ? 1 : 0;
    if (p.empty) return GETT_OK;
    out->nm = p.m.n;
    out->nn = p.n.n;
    out->nk = p.k.n;
    out->M = p.M;
    out->N = p.N;
    out->K = p.K;
    for (int i = 0; i < p.m.n; ++i) {
        out->m_ext[i] = p.m.ext[i];
        out->m_inca[i] = p.m.s0[i];
        out->m_incc[i] = p.m.s1[i];
    }
    for (int i = 0; i < p.n.n; ++i) {
        out->n_ext[i] = p.n.ext[i];
        out->n_incb[i] = p.n.s0[i];
        out->n_incc[i] = p.n.s1[i];
    }
    for (int i = 0; i < p.k.n; ++i) {
        out->k_ext[i] = p.k.ext[i];
        out->k_inca[i] = p.k.s0[i];
        out->k_incb[i] = p.k.s1[i];
    }
    out->off_a = p.offA;
    out->off_b = p.offB;
    out->off_c = p.offC;
    return GETT_OK;
}

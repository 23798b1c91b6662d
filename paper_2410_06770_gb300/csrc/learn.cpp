// learn.cpp -- features of a planned contraction and host inference of the
// installed MLP planner model.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "learn.h"

namespace gett {

namespace {

struct Model {
    bool ok = false;
    int nfeat = 0, hidden = 0, nout = 0;
    std::vector<float> params, mean, stdv;
};
Model g_model;
std::mutex g_model_mu;

float lg(double x) { return (float)std::log2(x + 1.0); }

int64_t first_abs(const ModeList &L, const int64_t *s) { return L.n ? (s[0] < 0 ? -s[0] : s[0]) : 0; }

// y = W x + b, optional ReLU; W is [out][in]
void dense(const float *W, const float *b, const float *x, int in, int out, bool relu, float *y)
{
    for (int o = 0; o < out; ++o) {
        double s = b[o];
        const float *w = W + (size_t)o * in;
        for (int i = 0; i < in; ++i) s += (double)w[i] * x[i];
        y[o] = relu ? (s > 0 ? (float)s : 0.f) : (float)s;
    }
}

bool model_forward(const Model &m, const float *raw, float *out)
{
    std::vector<float> x(m.nfeat), h1(m.hidden), h2(m.hidden);
    for (int i = 0; i < m.nfeat; ++i) x[i] = (raw[i] - m.mean[i]) / (m.stdv[i] > 0 ? m.stdv[i] : 1.f);
    const float *p = m.params.data();
    const float *W1 = p, *b1 = W1 + (size_t)m.hidden * m.nfeat;
    const float *W2 = b1 + m.hidden, *b2 = W2 + (size_t)m.hidden * m.hidden;
    const float *W3 = b2 + m.hidden, *b3 = W3 + (size_t)m.nout * m.hidden;
    dense(W1, b1, x.data(), m.nfeat, m.hidden, true, h1.data());
    dense(W2, b2, h1.data(), m.hidden, m.hidden, true, h2.data());
    dense(W3, b3, h2.data(), m.hidden, m.nout, false, out);
    for (int o = 0; o < m.nout; ++o)
        if (!std::isfinite(out[o])) return false;
    return true;
}

}  // namespace

void plan_features(const Plan &p, int dtype, float *f)
{
    std::memset(f, 0, sizeof(float) * GETT_LEARN_NFEAT);
    const int64_t am = first_abs(p.m, p.m.s0), ak = first_abs(p.k, p.k.s0);
    const int64_t bn = first_abs(p.n, p.n.s0), bk = first_abs(p.k, p.k.s1);
    const int64_t cm = first_abs(p.m, p.m.s1), cn = first_abs(p.n, p.n.s1);
    f[0] = lg((double)p.M);
    f[1] = lg((double)p.N);
    f[2] = lg((double)p.K);
    f[3] = lg((double)p.M * (double)p.N * (double)p.K) / 3.f;
    f[4] = (float)p.m.n;
    f[5] = (float)p.n.n;
    f[6] = (float)p.k.n;
    f[7] = lg((double)am);
    f[8] = lg((double)ak);
    f[9] = lg((double)bn);
    f[10] = lg((double)bk);
    f[11] = lg((double)cm);
    f[12] = lg((double)cn);
    f[13] = (am != 0 && (ak == 0 || am <= ak)) ? 1.f : 0.f;
    f[14] = (bn != 0 && (bk == 0 || bn <= bk)) ? 1.f : 0.f;
    f[15] = (cm != 0 && (cn == 0 || cm <= cn)) ? 1.f : 0.f;
    f[16] = lg(p.m.n ? (double)p.m.ext[0] : 1.0);
    f[17] = lg(p.n.n ? (double)p.n.ext[0] : 1.0);
    f[18] = lg(p.k.n ? (double)p.k.ext[0] : 1.0);
    f[19] = (float)dtype;
    f[20] = (float)(p.M % 32) / 32.f;
    f[21] = (float)(p.N % 32) / 32.f;
    f[22] = (float)(p.K % 16) / 16.f;
    f[23] = 1.f;
}

int learned_batch_config(const Plan &p, int dtype, int ncfg, const bool *valid)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!g_model.ok || g_model.nfeat != GETT_LEARN_NFEAT || g_model.nout < ncfg) return -1;
    float f[GETT_LEARN_NFEAT];
    plan_features(p, dtype, f);
    std::vector<float> out(g_model.nout);
    if (!model_forward(g_model, f, out.data())) return -1;
    int best = -1;
    for (int c = 0; c < ncfg; ++c)
        if ((!valid || valid[c]) && (best < 0 || out[c] < out[best])) best = c;
    return best;
}

}  // namespace gett

using namespace gett;

extern "C" int gett_problem_features(int RANKA, const int64_t *EXTA, const int64_t *INCA, int RANKB,
                                     const int64_t *EXTB, const int64_t *INCB, int CONTS, const int *CONTA,
                                     const int *CONTB, const int *PERM, const int64_t *INCC, int dtype,
                                     float *feat)
{
    if (!feat) return GETT_ERR_ARG;
    Args a{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC};
    Plan p;
    int bad = 0;
    int rc = make_plan(a, &p, &bad);
    set_last_error_arg(bad);
    if (rc != GETT_OK) return rc;
    if (p.empty) {
        std::memset(feat, 0, sizeof(float) * GETT_LEARN_NFEAT);
        return GETT_OK;
    }
    plan_features(p, dtype, feat);
    return GETT_OK;
}

extern "C" int gett_learn_install(int nfeat, int hidden, int nout, const float *params, const float *feat_mean,
                                  const float *feat_std)
{
    if (nfeat != GETT_LEARN_NFEAT || hidden <= 0 || nout <= 0 || !params || !feat_mean || !feat_std)
        return GETT_ERR_ARG;
    const size_t np = (size_t)hidden * nfeat + hidden + (size_t)hidden * hidden + hidden + (size_t)nout * hidden + nout;
    Model m;
    m.nfeat = nfeat;
    m.hidden = hidden;
    m.nout = nout;
    m.params.assign(params, params + np);
    m.mean.assign(feat_mean, feat_mean + nfeat);
    m.stdv.assign(feat_std, feat_std + nfeat);
    m.ok = true;
    std::lock_guard<std::mutex> lk(g_model_mu);
    g_model = std::move(m);
    return GETT_OK;
}

extern "C" int gett_learn_clear(void)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    g_model = Model();
    return GETT_OK;
}

extern "C" int gett_learn_predict(const float *feat, float *out)
{
    std::lock_guard<std::mutex> lk(g_model_mu);
    if (!g_model.ok || !feat || !out) return GETT_ERR_ARG;
    return model_forward(g_model, feat, out) ? GETT_OK : GETT_ERR_ARG;
}

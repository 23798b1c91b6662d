// tunedb.cpp -- the signature-keyed tuning database (gett_tune.h): measured
// best configurations for planned problems, consulted by the selection
// chain of single calls and batched launches.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "gett_tune.h"
#include "tunedb.h"

namespace gett {

namespace {

struct Entry {
    int v0, v1, v2;
};
std::map<std::string, Entry> g_db;  // ordered: saved files are stable
std::mutex g_db_mu;

void append_modes(std::string &k, char tag, const ModeList &L)
{
    k += tag;
    for (int i = 0; i < L.n; ++i) {
        k += ':';
        k += std::to_string(L.ext[i]);
        k += ',';
        k += std::to_string(L.s0[i]);
        k += ',';
        k += std::to_string(L.s1[i]);
    }
    k += '/';
}

std::string full_key(int kind, int dtype, const Plan &p)
{
    std::string k = std::to_string(kind) + ' ' + std::to_string(dtype) + ' ';
    k += plan_signature(p);
    return k;
}

bool valid_kind(int kind) { return kind == GETT_TUNE_BATCH || kind == GETT_TUNE_SINGLE; }

}  // namespace

std::string plan_signature(const Plan &p)
{
    std::string k;
    append_modes(k, 'm', p.m);
    append_modes(k, 'n', p.n);
    append_modes(k, 'k', p.k);
    return k;
}

bool tune_db_lookup(int kind, int dtype, const Plan &p, int *v0, int *v1, int *v2)
{
    std::lock_guard<std::mutex> lk(g_db_mu);
    if (g_db.empty()) return false;
    auto it = g_db.find(full_key(kind, dtype, p));
    if (it == g_db.end()) return false;
    *v0 = it->second.v0;
    *v1 = it->second.v1;
    *v2 = it->second.v2;
    return true;
}

}  // namespace gett

using namespace gett;

namespace {

int plan_of(int RANKA, const int64_t *EXTA, const int64_t *INCA, int RANKB, const int64_t *EXTB,
            const int64_t *INCB, int CONTS, const int *CONTA, const int *CONTB, const int *PERM, const int64_t *INCC,
            Plan *p)
{
    Args a{RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC};
    int bad = 0;
    const int rc = make_plan(a, p, &bad);
    set_last_error_arg(bad);
    return rc;
}

}  // namespace

extern "C" int gett_tune_db_put(int kind, int dtype, int RANKA, const int64_t *EXTA, const int64_t *INCA,
                                int RANKB, const int64_t *EXTB, const int64_t *INCB, int CONTS, const int *CONTA,
                                const int *CONTB, const int *PERM, const int64_t *INCC, int v0, int v1, int v2)
{
    if (!valid_kind(kind) || dtype < 0 || dtype > 4) return GETT_ERR_ARG;
    Plan p;
    const int rc = plan_of(RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC, &p);
    if (rc != GETT_OK) return rc;
    if (p.empty) return GETT_OK;
    std::lock_guard<std::mutex> lk(g_db_mu);
    g_db[full_key(kind, dtype, p)] = Entry{v0, v1, v2};
    return GETT_OK;
}

extern "C" int gett_tune_db_get(int kind, int dtype, int RANKA, const int64_t *EXTA, const int64_t *INCA,
                                int RANKB, const int64_t *EXTB, const int64_t *INCB, int CONTS, const int *CONTA,
                                const int *CONTB, const int *PERM, const int64_t *INCC, int *v0, int *v1, int *v2)
{
    if (!valid_kind(kind) || !v0 || !v1 || !v2) return GETT_ERR_ARG;
    Plan p;
    const int rc = plan_of(RANKA, EXTA, INCA, RANKB, EXTB, INCB, CONTS, CONTA, CONTB, PERM, INCC, &p);
    if (rc != GETT_OK) return rc;
    if (p.empty) return 0;
    return tune_db_lookup(kind, dtype, p, v0, v1, v2) ? 1 : 0;
}

extern "C" int gett_tune_db_clear(void)
{
    std::lock_guard<std::mutex> lk(g_db_mu);
    g_db.clear();
    return GETT_OK;
}

extern "C" int gett_tune_db_size(void)
{
    std::lock_guard<std::mutex> lk(g_db_mu);
    return (int)g_db.size();
}

extern "C" int gett_tune_db_save(const char *path)
{
    if (!path) return GETT_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_db_mu);
    std::ofstream f(path);
    if (!f) return GETT_ERR_ARG;
    f << "# xGETT tuning database: kind dtype signature v0 v1 v2\n";
    for (const auto &kv : g_db)
        f << kv.first << ' ' << kv.second.v0 << ' ' << kv.second.v1 << ' ' << kv.second.v2 << '\n';
    return f.good() ? GETT_OK : GETT_ERR_ARG;
}

extern "C" int gett_tune_db_load(const char *path)
{
    if (!path) return GETT_ERR_ARG;
    std::ifstream f(path);
    if (!f) return GETT_ERR_ARG;
    std::map<std::string, Entry> add;
    std::string line;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        int kind = -1, dtype = -1;
        std::string sig;
        Entry e{};
        if (!(is >> kind >> dtype >> sig >> e.v0 >> e.v1 >> e.v2)) return GETT_ERR_ARG;
        std::string rest;
        if (is >> rest) return GETT_ERR_ARG;
        if (!valid_kind(kind) || dtype < 0 || dtype > 4 || sig.empty()) return GETT_ERR_ARG;
        add[std::to_string(kind) + ' ' + std::to_string(dtype) + ' ' + sig] = e;
    }
    std::lock_guard<std::mutex> lk(g_db_mu);
    for (const auto &kv : add) g_db[kv.first] = kv.second;
    return GETT_OK;
}

// select.cpp -- which kernel family runs a planned contraction.
//
// Order: a caller's forced algorithm / family / configuration / split; else
// an entry of the tuning database for the planned signature (gett_tune.h);
// else the fixed heuristic below.
//
// Heuristic (the fixed planner every other selector falls back to):
//  * K == 1 (no contracted extent > 1): OUTER streaming kernel;
//  * at most 32 outputs and K >= 8192: REDUCE streaming kernel;
//  * K <= 8 with at least 2^16 outputs: OUTER (short sums);
//  * one free class of at most 8 indices and max(M, N) * K >= 2^16: SKINNY;
//  * bf16 operands with M, N >= 512 and K >= 256: tcgen05 tensor cores;
//  * otherwise the DENSE tiled kernel with the largest tile that still gives
//    at least one tile per SM (split along K when that fills the last wave
//    of tiles), else the smallest tile plus split-K so the grid covers the
//    SMs.
#include <algorithm>

#include "gett_tune.h"
#include "kernels.h"
#include "select.h"
#include "tunedb.h"

namespace gett {

namespace {

// K slices that fill the last wave of a large tile grid: 1 when the tiles
// already fill their waves to 98 %, else the smallest S <= 32 whose tiles x S
// fill them to 99 %, with slices of at least 512 and at most 4 GB of partial
// tiles (1 if none qualifies).  The slices are added in order by the split-K
// reduce, so the result stays deterministic.
int balance_split(const Plan &p, DType t, int cfg, int64_t tiles, int num_sms)
{
    const int64_t slots = (int64_t)num_sms * dense_ctas_per_sm(t, cfg);
    auto fill = [&](int64_t units) {
        const int64_t waves = (units + slots - 1) / slots;
        return (double)units / (double)(waves * slots);
    };
    if (fill(tiles) >= 0.98) return 1;
    const size_t acc = (t == DT_C64) ? 16 : ((t == DT_F64 || t == DT_C32) ? 8 : 4);
    for (int S = 2; S <= 32; ++S) {
        const int Se = dense_effective_split(p, cfg, S);
        if (Se != S || p.K / S < 512) continue;
        if ((double)acc * S * (double)p.M * (double)p.N > 4e9) break;
        if (fill(tiles * S) >= 0.99) return S;
    }
    return 1;
}

}  // namespace

Choice heuristic_choice(const Plan &p, DType t, int num_sms)
{
    Choice c;
    c.selector = 0;
    if (p.empty) {
        c.family = GETT_FAMILY_NOOP;
        return c;
    }
    if (p.K == 1) {
        c.family = GETT_FAMILY_OUTER;
        return c;
    }
    const int64_t O = p.M * p.N;
    if (O <= 32 && p.K >= 8192) {
        c.family = GETT_FAMILY_REDUCE;
        return c;
    }
    // short sums over a large output stream C at HBM speed
    if (p.K <= OUTER_MAX_SUM && O >= (1 << 16)) {
        c.family = GETT_FAMILY_OUTER;
        return c;
    }
    // matrix-vector like: one free class of at most 8 indices
    if (skinny_applicable(p) && std::max(p.M, p.N) * p.K >= (1 << 16)) {
        c.family = GETT_FAMILY_SKINNY;
        return c;
    }
    // bf16 operands: tensor cores once the packing pays for itself
    if (t == DT_BF16 && p.M >= 512 && p.N >= 512 && p.K >= 256) {
        c.family = GETT_FAMILY_TC;
        c.algo = GETT_ALGO_NATIVE;
        return c;
    }
    c.family = GETT_FAMILY_DENSE;
    for (int cfg = 0; cfg < DENSE_NUM_CONFIGS; ++cfg) {
        if (!dense_config_valid(t, cfg)) continue;
        int bm, bn, bk;
        dense_tile_shape(cfg, &bm, &bn, &bk);
        int64_t tiles = ((p.M + bm - 1) / bm) * ((p.N + bn - 1) / bn);
        if (tiles >= num_sms) {
            c.config = cfg;
            c.split_k = balance_split(p, t, cfg, tiles, num_sms);
            return c;
        }
    }
    const int cfg = DENSE_NUM_CONFIGS - 1;
    int bm, bn, bk;
    dense_tile_shape(cfg, &bm, &bn, &bk);
    int64_t tiles = ((p.M + bm - 1) / bm) * ((p.N + bn - 1) / bn);
    int64_t want = (num_sms + tiles - 1) / tiles;
    int64_t kmax = std::max<int64_t>(1, p.K / (4 * bk));
    c.config = cfg;
    c.split_k = (int)std::max<int64_t>(1, std::min<int64_t>({want, kmax, 64}));
    return c;
}

// A tuning-database entry for single calls, if one exists and fits the
// problem (gett_tune.h: v0 family, v1 configuration, v2 split_k).
bool tuned_choice(const Plan &p, DType t, Choice *out)
{
    int fam = 0, cfg = 0, sk = 0;
    if (!tune_db_lookup(GETT_TUNE_SINGLE, (int)t, p, &fam, &cfg, &sk)) return false;
    Choice c;
    c.family = fam;
    c.config = cfg;
    c.split_k = sk > 0 ? sk : 1;
    c.selector = 1;
    bool ok = false;
    switch (fam) {
    case GETT_FAMILY_DENSE: ok = dense_config_valid(t, cfg); break;
    case GETT_FAMILY_OUTER: ok = p.K <= OUTER_MAX_SUM; break;
    case GETT_FAMILY_SKINNY: ok = skinny_applicable(p); break;
    case GETT_FAMILY_REDUCE: ok = p.M * p.N <= 4096; break;
    case GETT_FAMILY_TC: ok = t == DT_BF16; c.algo = GETT_ALGO_NATIVE; break;
    default: ok = false;
    }
    if (!ok) return false;
    *out = c;
    return true;
}

int choose(const Plan &p, DType t, const gett_options *opt, int num_sms, Choice *out)
{
    Choice c = heuristic_choice(p, t, num_sms);
    // tuned step of the chain: a database entry replaces the heuristic
    // unless the caller forces an algorithm, family, configuration or split
    const bool free_choice = !opt || ((opt->algo == GETT_ALGO_DEFAULT || opt->algo == GETT_ALGO_NATIVE) &&
                                      opt->family == GETT_FAMILY_AUTO && opt->config < 0 && opt->split_k <= 0);
    if (free_choice && !p.empty) {
        Choice tc;
        if (tuned_choice(p, t, &tc)) {
            if (tc.family == GETT_FAMILY_DENSE) tc.split_k = dense_effective_split(p, tc.config, tc.split_k);
            *out = tc;
            return GETT_OK;
        }
    }
    if (opt && opt->algo == GETT_ALGO_OZAKI_BF16) {
        if (t != DT_F64 && t != DT_C64) return GETT_ERR_UNSUPPORTED;
        c = Choice{};
        c.family = GETT_FAMILY_TC;
        c.algo = GETT_ALGO_OZAKI_BF16;
        // the complex form sums 2K real products per element
        c.moduli = ozaki_moduli_for(t == DT_C64 ? 2 * p.K : p.K, opt->moduli);
        c.selector = 3;
        *out = c;
        return GETT_OK;
    }
    if (opt && (opt->algo == GETT_ALGO_BF16X3 || opt->algo == GETT_ALGO_BF16X6)) {
        if (t != DT_F32) return GETT_ERR_UNSUPPORTED;
        c = Choice{};
        c.family = GETT_FAMILY_TC;
        c.algo = opt->algo;
        c.selector = 3;
        *out = c;
        return GETT_OK;
    }
    if (opt && opt->family == GETT_FAMILY_TC) {
        if (t != DT_BF16) return GETT_ERR_UNSUPPORTED;
        c = Choice{};
        c.family = GETT_FAMILY_TC;
        c.algo = GETT_ALGO_NATIVE;
        c.selector = 3;
        *out = c;
        return GETT_OK;
    }
    if (opt) {
        if (opt->algo != GETT_ALGO_DEFAULT && opt->algo != GETT_ALGO_NATIVE)
            return GETT_ERR_UNSUPPORTED;
        if (opt->family != GETT_FAMILY_AUTO) {
            Choice f;
            f.family = opt->family;
            f.selector = 3;
            f.config = opt->config >= 0 ? opt->config
                                        : (c.family == GETT_FAMILY_DENSE ? c.config : DENSE_NUM_CONFIGS - 1);
            f.split_k = opt->split_k > 0 ? opt->split_k : 1;
            bool ok = false;
            switch (f.family) {
            case GETT_FAMILY_DENSE: ok = dense_config_valid(t, f.config); break;
            case GETT_FAMILY_OUTER: ok = p.K <= OUTER_MAX_SUM; break;
            case GETT_FAMILY_SKINNY: ok = skinny_applicable(p); break;
            case GETT_FAMILY_REDUCE: ok = p.M * p.N <= 4096; break;
            default: ok = false;
            }
            if (!ok) {
                set_last_error_arg(0);
                return GETT_ERR_UNSUPPORTED;
            }
            c = f;
        } else if (c.family == GETT_FAMILY_DENSE) {
            if (opt->config >= 0 && dense_config_valid(t, opt->config)) {
                c.config = opt->config;
                c.selector = 3;
            }
            if (opt->split_k > 0) {
                c.split_k = opt->split_k;
                c.selector = 3;
            }
        }
    }
    if (c.family == GETT_FAMILY_DENSE) c.split_k = dense_effective_split(p, c.config, c.split_k);
    *out = c;
    return GETT_OK;
}

}  // namespace gett

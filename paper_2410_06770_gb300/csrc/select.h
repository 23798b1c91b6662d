// select.h -- kernel-family and configuration choice for one planned problem.
#pragma once

#include "internal.h"

namespace gett {

struct Choice {
    int family = GETT_FAMILY_NOOP;
    int config = 0;
    int split_k = 1;
    int moduli = 0;
    int algo = GETT_ALGO_NATIVE;
    int selector = 0;  // 0 heuristic, 1 tuning table, 2 learned model, 3 forced by caller
};

// Picks family/config for a non-empty plan.  Honours a caller's forced
// family/config (gett_options) when it is valid for the problem.
int choose(const Plan &p, DType t, const gett_options *opt, int num_sms, Choice *out);

// The fixed heuristic alone (the fallback of the other selectors).
Choice heuristic_choice(const Plan &p, DType t, int num_sms);

int device_sms();
// The current device's error word (bounded waits record a code there; read
// and cleared by gett_device_status), or NULL without a usable device.
int *device_error_word();

}  // namespace gett

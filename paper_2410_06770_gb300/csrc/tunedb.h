// tunedb.h -- internal access to the tuning database (gett_tune.h).
#pragma once

#include <string>

#include "internal.h"

namespace gett {

// Canonical signature of a planned problem: every class mode's extent and
// its two increments (no spaces; the database key without kind and dtype).
std::string plan_signature(const Plan &p);

// The entry of (kind, dtype, planned problem), if any.
bool tune_db_lookup(int kind, int dtype, const Plan &p, int *v0, int *v1, int *v2);

}  // namespace gett

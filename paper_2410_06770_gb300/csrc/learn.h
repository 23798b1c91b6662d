// learn.h -- learned planner internals shared by the batch planner.
#pragma once

#include "gett_learn.h"
#include "internal.h"

namespace gett {

// Feature vector (GETT_LEARN_NFEAT floats) of a planned problem.
void plan_features(const Plan &p, int dtype, float *f);

// Configuration chosen by the installed model: argmin of the predicted
// times over the first ncfg outputs among those `valid` marks (all when
// NULL), or -1 without a model / for a non-finite prediction.
int learned_batch_config(const Plan &p, int dtype, int ncfg, const bool *valid = nullptr);

}  // namespace gett

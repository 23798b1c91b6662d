// learn.h -- learned planner internals shared by the batch planner.
#pragma once

#include "gett_learn.h"
#include "internal.h"

namespace gett {

// Feature vector (GETT_LEARN_NFEAT floats) of a planned problem.
void plan_features(const Plan &p, int dtype, float *f);

// Tile configuration chosen by the installed model (argmin of predicted
// times over the first ncfg outputs), or -1 without a model / for a
// non-finite prediction.
int learned_batch_config(const Plan &p, int dtype, int ncfg);

}  // namespace gett

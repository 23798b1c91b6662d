// internal.h -- shared declarations of the xGETT library (host side).
#pragma once

#include <cstddef>
#include <cstdint>

#include "gett.h"

namespace gett {

enum DType : int { DT_F32 = 0, DT_F64 = 1, DT_C32 = 2, DT_C64 = 3, DT_BF16 = 4 };

inline size_t dtype_size(DType t)
{
    switch (t) {
    case DT_F32: return 4;
    case DT_F64: return 8;
    case DT_C32: return 8;
    case DT_C64: return 16;
    case DT_BF16: return 2;
    }
    return 0;
}

// One class of modes after planning.  For M: s0 = INCA, s1 = INCC.  For N:
// s0 = INCB, s1 = INCC.  For K: s0 = INCA, s1 = INCB.  Modes are ordered
// from fastest (index 0) to slowest; a flat class index i decodes with the
// first mode fastest (the same mixed-radix order Alg. 2 visits).
struct ModeList {
    int n;
    int64_t ext[GETT_MAX_MODES];
    int64_t s0[GETT_MAX_MODES];
    int64_t s1[GETT_MAX_MODES];
};

// Canonical problem: C[offC + m.s1 + n.s1] += sum_k A[offA + m.s0 + k.s0] *
// B[offB + n.s0 + k.s1].
struct Plan {
    ModeList m, n, k;
    int64_t M, N, K;
    int64_t offA, offB, offC;  // element offsets applied to the user pointers
    bool empty;                // M*N == 0 or K == 0: nothing to do
    // address spans (elements, relative to the user pointers) for alias checks
    int64_t a_lo, a_hi, b_lo, b_hi, c_lo, c_hi;
};

struct Args {
    int RANKA; const int64_t *EXTA; const int64_t *INCA;
    int RANKB; const int64_t *EXTB; const int64_t *INCB;
    int CONTS; const int *CONTA; const int *CONTB; const int *PERM;
    const int64_t *INCC;
};

// Validates the 14 arguments (without pointers) and builds the plan.
// Returns GETT_OK, GETT_ERR_ARG (bad_arg = 1-based position), GETT_ERR_ALIAS
// (C not injective) or GETT_ERR_UNSUPPORTED.
int make_plan(const Args &a, Plan *p, int *bad_arg);

// Thread-local diagnostics.
void set_last_error_arg(int pos);
void set_last_cuda_error(int err);

}  // namespace gett

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

// How a kernel's result v meets C (the scaled form follows xGEMM's ALPHA and
// BETA, Sec. 2.3.1: C <- alpha * A.B + beta * C).  SCALE_ACC is Alg. 1's
// accumulation C <- C + v and the default (a zero-initialised Scale);
// SCALE_AXPBY writes alpha * v + beta * C; SCALE_AX writes alpha * v without
// reading C (beta == 0).  alpha = ar + i ai, beta = br + i bi (the imaginary
// parts are ignored for real types; float types round them to float).
enum ScaleMode : int { SCALE_ACC = 0, SCALE_AXPBY = 1, SCALE_AX = 2 };
struct Scale {
    int mode;
    double ar, ai, br, bi;
};

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
    bool empty;                // M*N == 0 or K == 0: nothing to accumulate
    // K == 0 with M*N > 0: the sum is empty but m and n are planned (the
    // scaled form still writes beta * C); c_injective records whether C's
    // layout passed the injectivity test in that case
    bool zero_sum;
    bool c_injective;
    // how the sum meets C; make_plan sets SCALE_ACC (Alg. 1), the scaled
    // entry points overwrite it
    Scale sc;
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

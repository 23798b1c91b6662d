/*
 * gett_tune.h -- the tuned step of the configuration choice: a database of
 * measured best configurations keyed by the contraction's planned signature
 * (extension; the thesis has no planner or tuning, Sec. 6).
 *
 * Choice order.  Batched launches with GETT_BATCH_SELECT_LEARNED ask the
 * learned model first, then this database, then the fixed heuristic; with
 * GETT_BATCH_SELECT_TUNED the database, then the heuristic.  Single calls
 * (xgett, xgett_async, xgett_ex and xgett_scaled without a forced family,
 * configuration or split) use a database entry when one exists
 * (gett_report.selector = 1), else the heuristic (selector = 0).
 *
 * Key.  The planned problem (Sec. 5.7 arguments after dropping extent-1
 * modes, flipping negative increments and fusing stride-compatible modes):
 * every class mode's extent and its increments in the two tensors holding
 * it, plus the operand type.  Two calls whose layouts plan to the same
 * canonical problem share one entry.  Pointers and offsets are not part of
 * the key.
 *
 * Kinds and values:
 *   GETT_TUNE_BATCH  (dtype 0 float, 1 bfloat16 operands): v0 = batched
 *                    configuration id (gett_batch.h); v1, v2 unused.
 *   GETT_TUNE_SINGLE (dtype: 0 s, 1 d, 2 c, 3 z, 4 sb): v0 = gett_family,
 *                    v1 = configuration within the family, v2 = split_k.
 * An entry that does not fit the problem when it is used (a family the
 * problem cannot run, an invalid configuration) is ignored and the next step
 * of the order decides.
 *
 * File format (gett_tune_db_save / gett_tune_db_load): one entry a line,
 * "kind dtype key v0 v1 v2", with the key a single token; lines starting
 * with '#' are comments.  Loading merges into the current database (a later
 * line for the same key replaces the earlier one).
 *
 * Thread safety: all calls lock one process-wide mutex.  Host only: no call
 * here touches a device.
 */
#ifndef GETT_TUNE_H
#define GETT_TUNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GETT_TUNE_BATCH 0
#define GETT_TUNE_SINGLE 1

/* Records (or replaces) the entry of the problem given by the 11 index
 * arguments of xGETT (no pointers).  GETT_ERR_ARG for invalid arguments or
 * kind; argument errors of the 11 report their positions as xgett does.
 * An empty problem (nothing to compute) is accepted and not stored. */
int gett_tune_db_put(int kind, int dtype, int RANKA, const int64_t *EXTA, const int64_t *INCA,
                     int RANKB, const int64_t *EXTB, const int64_t *INCB,
                     int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                     const int64_t *INCC, int v0, int v1, int v2);
/* 1 and the values if an entry exists, 0 if not, negative on errors. */
int gett_tune_db_get(int kind, int dtype, int RANKA, const int64_t *EXTA, const int64_t *INCA,
                     int RANKB, const int64_t *EXTB, const int64_t *INCB,
                     int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                     const int64_t *INCC, int *v0, int *v1, int *v2);
int gett_tune_db_clear(void);
int gett_tune_db_size(void);
/* GETT_ERR_ARG for a NULL path or a file that cannot be opened, or (load) a
 * malformed line, in which case nothing of the file is merged. */
int gett_tune_db_save(const char *path);
int gett_tune_db_load(const char *path);

#ifdef __cplusplus
}
#endif

#endif /* GETT_TUNE_H */

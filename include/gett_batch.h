/*
 * gett_batch.h -- many xGETT contractions in one persistent launch
 * (extension; the thesis defines single calls only, Sec. 5.7).
 *
 * Each problem is a full xGETT call (the 14 arguments of Sec. 5.7, same
 * meaning as in gett.h) with float C and either float or bfloat16 A and B;
 * products are accumulated in float.  gett_batch_create validates and plans
 * every problem on the host, chooses a tile configuration per problem,
 * uploads one descriptor table, one offset-table buffer and one tile work
 * list, and returns an opaque handle.  gett_batch_launch runs every tile of
 * every problem in ONE persistent kernel (one CTA per SM slot, tiles taken
 * from an atomic work counter); gett_batch_launch_graph does the same through
 * a CUDA graph captured on first use and replayed afterwards.
 *
 * Ownership: the EXT/INC/CONT/PERM arrays are read during create only; the
 * device pointers A, B, C must stay valid while the handle is launched.  Each
 * C must be injective (the same sufficient test as single calls), and the C
 * of one problem may overlap neither another problem's C nor any problem's A
 * or B (address ranges; GETT_ERR_ALIAS).  Operands may be shared.
 * Launches of one handle are stream ordered; concurrent launches of the same
 * handle on different streams race on its work counter.
 */
#ifndef GETT_BATCH_H
#define GETT_BATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gett_batch_dtype { GETT_BATCH_F32 = 0, GETT_BATCH_BF16 = 1 } gett_batch_dtype;

typedef struct gett_problem_desc {
    int dtype;                /* gett_batch_dtype of A and B; C is float  */
    int RANKA;
    const int64_t *EXTA, *INCA;
    const void *A;
    int RANKB;
    const int64_t *EXTB, *INCB;
    const void *B;
    int CONTS;
    const int *CONTA, *CONTB, *PERM;
    const int64_t *INCC;
    float *C;
} gett_problem_desc;

typedef enum gett_batch_select {
    GETT_BATCH_SELECT_HEURISTIC = 0,  /* fixed rule on M, N, K                  */
    GETT_BATCH_SELECT_FIXED = 1,      /* every problem uses `config`            */
    GETT_BATCH_SELECT_TABLE = 2,      /* per-problem configs given in `configs` */
    GETT_BATCH_SELECT_LEARNED = 3     /* the loaded MLP planner (gett_learn.h)  */
} gett_batch_select;

typedef struct gett_batch_options {
    int select;               /* gett_batch_select                          */
    int config;               /* for SELECT_FIXED                           */
    const int *configs;       /* for SELECT_TABLE: n entries (-1 = heuristic) */
    int ctas_per_sm;          /* persistent CTAs per SM (0 = 4); 1-2, 3 and
                                 4 use kernels compiled for 2, 3 and 4
                                 resident CTAs (128, 80, 64 registers a
                                 thread), more than 4 the 4 one            */
} gett_batch_options;

typedef struct gett_batch gett_batch;

typedef struct gett_batch_info {
    int n;                    /* problems                                   */
    int nonempty;             /* problems with work                         */
    int64_t tiles;            /* work items of one launch                   */
    double flops;             /* 2*M*N*K summed over problems               */
    int config_count[8];      /* problems per tile configuration            */
    int fallbacks;            /* learned/table choices replaced by the heuristic */
} gett_batch_info;

/* Number of tile configurations of the batched kernel and their shapes. */
int gett_batch_num_configs(void);
int gett_batch_config_shape(int config, int *bm, int *bn);

/* The fixed heuristic's tile configuration for one problem (14 xGETT
 * arguments without pointers) -- the fallback of the other selectors. */
int gett_batch_heuristic_config(int RANKA, const int64_t *EXTA, const int64_t *INCA,
                                int RANKB, const int64_t *EXTB, const int64_t *INCB,
                                int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                                const int64_t *INCC, int *config);

/* Returns GETT_OK or the first failing problem's status; *bad_index (may be
 * NULL) receives that problem's index and gett_last_error_arg() its
 * argument position (1..14 as in gett.h; 0 for an unknown dtype).
 * GETT_ERR_ARG also for a NULL out, n < 0, SELECT_FIXED with a config
 * outside [0, gett_batch_num_configs()) or SELECT_TABLE without configs.
 * Validation touches no device; GETT_ERR_CUDA / GETT_ERR_NOMEM come from
 * the uploads that follow it. */
int gett_batch_create(int n, const gett_problem_desc *probs, const gett_batch_options *opt,
                      gett_batch **out, int *bad_index);
int gett_batch_launch(gett_batch *b, void *stream);
int gett_batch_launch_graph(gett_batch *b, void *stream);
int gett_batch_get_info(const gett_batch *b, gett_batch_info *info);
/* Autotuner measurement: times every problem of the batch on its own
 * (`reps` back-to-back launches of the persistent kernel between two CUDA
 * events on an internal stream) and writes the mean milliseconds to
 * ms_out[i] (0 for problems with nothing to compute).  mode 0: the problem's
 * tiles alone (latency).  mode 1: the problem's tiles repeated until every
 * persistent CTA gets several, time divided by the repeat count (its cost
 * inside a full batch).  Synchronous; C buffers are updated each run. */
int gett_batch_profile(gett_batch *b, int reps, int mode, float *ms_out);
int gett_batch_destroy(gett_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* GETT_BATCH_H */

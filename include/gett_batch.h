/*
 * gett_batch.h -- many xGETT contractions in one batched launch
 * (extension; the thesis defines single calls only, Sec. 5.7).
 *
 * Each problem is a full xGETT call (the 14 arguments of Sec. 5.7, same
 * meaning as in gett.h) with float C and either float or bfloat16 A and B;
 * products are accumulated in float.  gett_batch_create validates and plans
 * every problem on the host, chooses a configuration per problem (a method
 * and a tile shape, below), uploads one descriptor table, one offset-table
 * buffer and the work lists, and returns an opaque handle.
 * gett_batch_launch enqueues the whole batch as per-method chains of
 * persistent kernels -- packing + packed tiles, tensor-core packing +
 * tensor-core tiles, gathered tiles, skinny warp items, short sums -- which
 * run as concurrent branches forked from the launch stream (or in order on
 * it, with options.serial), then the ordered addition of K-slice partials;
 * the gathered tiles and the short sums take items from atomic work
 * counters, the others deal them to the CTAs statically.
 * gett_batch_launch_graph does the same through a CUDA graph captured on
 * first use and replayed afterwards.
 *
 * Configurations (gett_batch_num_configs() of them):
 *   0..3  GATHER with tile shape 0..3: tiles read A and B through the
 *         planner's class offset tables (its logical mode fusion only);
 *         sums of at most 8 terms form their outputs straight from gathered
 *         loads (a kernel of their own);
 *   4..7  PACK with tile shape 0..3: A and B are first copied into
 *         tile-blocked dense matrices (each class's modes physically fused
 *         into one contiguous index; bf16 widened to float), which the tiles
 *         then stream with bulk copies;
 *   8     SKINNY: for a problem with a free class of at most 8 indices;
 *         warp items along the long class or along the sum;
 *   9     TC: for bf16 operands; A and B are packed into 128 x 64 tiles laid
 *         out as the tensor core reads them and multiplied by tcgen05 into
 *         128 x 128 float tiles (fp32 accumulation in TMEM).
 * gett_batch_config_shape and gett_batch_config_method describe an id.
 *
 * Ownership: the EXT/INC/CONT/PERM arrays are read during create only; the
 * device pointers A, B, C must stay valid while the handle is launched.  Each
 * C must be injective (the same sufficient test as single calls), and the C
 * of one problem may overlap neither another problem's C nor any problem's A
 * or B (address ranges; GETT_ERR_ALIAS).  Operands may be shared.
 * Launches of one handle are stream ordered (a launch's internal branches
 * wait for the work enqueued before it and the launch stream waits for them);
 * concurrent launches of the same handle on different streams race on its
 * work counter and its branch streams.
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
    GETT_BATCH_SELECT_LEARNED = 3,    /* the loaded MLP planner (gett_learn.h),
                                         then the tuning database, then the
                                         heuristic                              */
    GETT_BATCH_SELECT_TUNED = 4       /* the tuning database (gett_tune.h), then
                                         the heuristic                          */
} gett_batch_select;

typedef struct gett_batch_options {
    int select;               /* gett_batch_select                          */
    int config;               /* for SELECT_FIXED                           */
    const int *configs;       /* for SELECT_TABLE: n entries (-1 = heuristic) */
    int ctas_per_sm;          /* persistent CTAs per SM (0 = 4); 1-2, 3 and
                                 4 use kernels compiled for 2, 3 and 4
                                 resident CTAs (128, 80, 64 registers a
                                 thread), more than 4 the 4 one            */
    int serial;               /* 0: the independent method chains of a launch
                                 (packing + packed tiles, tensor-core packing
                                 + tiles, gathered tiles, skinny items) run
                                 as concurrent branches on internal streams
                                 forked from and joined back into the
                                 launch stream before the reduction; 1: all
                                 kernels in order on the launch stream      */
} gett_batch_options;

typedef struct gett_batch gett_batch;

#define GETT_BATCH_MAX_CONFIGS 16

typedef struct gett_batch_info {
    int n;                    /* problems                                   */
    int nonempty;             /* problems with work                         */
    int64_t tiles;            /* tile and warp work items of one launch     */
    double flops;             /* 2*M*N*K summed over problems               */
    int config_count[GETT_BATCH_MAX_CONFIGS]; /* problems per configuration */
    int fallbacks;            /* learned/table choices replaced by the heuristic */
    int64_t gather_items;     /* work items of each kernel of a launch
                                 (gathered tiles and short-sum tile runs)   */
    int64_t packed_items;
    int64_t pack_items;
    int64_t skinny_items;
    int tuned_hits;           /* problems configured by the tuning database */
    int64_t tc_items;         /* tensor-core output tiles of one launch     */
    int64_t tc_pack_items;    /* their packing items (128 x 64 tiles)       */
} gett_batch_info;

/* Number of configurations, the tile shape of an id (0 x 0 for SKINNY) and
 * its method (0 GATHER, 1 PACK, 2 SKINNY); GETT_ERR_ARG for an unknown id. */
int gett_batch_num_configs(void);
int gett_batch_config_shape(int config, int *bm, int *bn);
int gett_batch_config_method(int config);
/* 1 if `config` can run the problem (14 xGETT arguments without pointers,
 * dtype a gett_batch_dtype), 0 if not (SKINNY without a free class of at
 * most 8 indices, TC with float operands), or a negative status for invalid
 * arguments.  Host only.  A table or learned choice that is not valid is
 * replaced by the heuristic's (a fallback). */
int gett_batch_config_valid(int RANKA, const int64_t *EXTA, const int64_t *INCA,
                            int RANKB, const int64_t *EXTB, const int64_t *INCB,
                            int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                            const int64_t *INCC, int dtype, int config);

/* The fixed heuristic's configuration for one problem (14 xGETT arguments
 * without pointers, dtype a gett_batch_dtype) -- the fallback of the other
 * selectors: sums of at most 8 terms GATHER (direct), a free class of at
 * most 8 indices SKINNY, bf16 operands with M, N >= 128 and K >= 256 TC, everything
 * else PACK; the shape follows M and N. */
int gett_batch_heuristic_config(int RANKA, const int64_t *EXTA, const int64_t *INCA,
                                int RANKB, const int64_t *EXTB, const int64_t *INCB,
                                int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                                const int64_t *INCC, int dtype, int *config);

/* Returns GETT_OK or the first failing problem's status; *bad_index (may be
 * NULL) receives that problem's index and gett_last_error_arg() its
 * argument position (1..14 as in gett.h; 0 for an unknown dtype).
 * GETT_ERR_ARG also for a NULL out, n < 0, an unknown select, SELECT_FIXED with a config
 * outside [0, gett_batch_num_configs()) or SELECT_TABLE without configs.
 * Validation touches no device; GETT_ERR_CUDA / GETT_ERR_NOMEM come from
 * the uploads that follow it.  GETT_ERR_UNSUPPORTED: a class of more than
 * 2^31 indices, offset tables beyond 2^31 entries in all, or more than 2^31
 * tiles in one problem.  A packed problem whose operands would take the
 * packed buffer past 2^30 floats is gathered instead.  The packed tiles'
 * bulk-copy waits are bounded; one that gives up records a code that
 * gett_device_status() reports as GETT_ERR_TIMEOUT. */
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

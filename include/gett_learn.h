/*
 * gett_learn.h -- the learned planner: a 3-layer MLP that maps a
 * contraction signature to predicted log run times of the batched kernel's
 * tile configurations (extension; the thesis has no planner, Sec. 6).
 *
 * Features are computed from the planned problem (after squeezing, flips
 * and fusion): log2 of M, N, K and of the leading increments of A, B and C
 * per class, mode counts, coalescing flags, leading extents, raggedness and
 * the operand type (gett_problem_features, GETT_LEARN_NFEAT floats).
 *
 * The network: nfeat -> hidden -> hidden -> nout, ReLU, fp32.  Its
 * parameters are trained on the GPU by the library's own forward, backward
 * and Adam kernels (gett_mlp_*), on targets = normalised log times measured
 * by the autotuner.  gett_learn_install makes a parameter set the model that
 * gett_batch_create uses with GETT_BATCH_SELECT_LEARNED (host inference,
 * argmin of the predicted times); without an installed model, or when a
 * prediction is not finite, the batch falls back to the fixed heuristic.
 *
 * Parameter layout (floats): W1[hidden][nfeat], b1[hidden],
 * W2[hidden][hidden], b2[hidden], W3[nout][hidden], b3[nout].
 */
#ifndef GETT_LEARN_H
#define GETT_LEARN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GETT_LEARN_NFEAT 24

/* Feature vector of one xGETT problem (same 14 arguments as xgett, no
 * pointers).  dtype: 0 = float operands, 1 = bfloat16 operands. */
int gett_problem_features(int RANKA, const int64_t *EXTA, const int64_t *INCA,
                          int RANKB, const int64_t *EXTB, const int64_t *INCB,
                          int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                          const int64_t *INCC, int dtype, float *feat);

typedef struct gett_mlp gett_mlp;

int gett_mlp_create(int nfeat, int hidden, int nout, unsigned long long seed, gett_mlp **out);
int gett_mlp_destroy(gett_mlp *m);
int gett_mlp_num_params(const gett_mlp *m);
int gett_mlp_get_params(const gett_mlp *m, float *host);
int gett_mlp_set_params(gett_mlp *m, const float *host);

/* Loss and gradients on one batch of n samples (host arrays X[n][nfeat],
 * Y[n][nout], mask[n][nout] in {0,1}); loss = sum(mask (pred - Y)^2) /
 * sum(mask).  grads has the parameter layout. */
int gett_mlp_loss_grad(gett_mlp *m, const float *X, const float *Y, const float *mask, int n,
                       float *loss, float *grads);

/* Adam training: `epochs` passes over n samples in shuffled minibatches of
 * `batch` (seeded), learning rate lr; *final_loss = mean loss of the last
 * epoch.  Runs on the current device. */
int gett_mlp_fit(gett_mlp *m, const float *X, const float *Y, const float *mask, int n, int epochs,
                 int batch, float lr, unsigned long long seed, float *final_loss);

/* GPU forward pass: Y[n][nout] = network(X[n][nfeat]). */
int gett_mlp_predict(gett_mlp *m, const float *X, int n, float *Y);

/* Install a parameter set (with the feature normalisation it was trained
 * with: x' = (x - mean) / std) as the planner's learned model. */
int gett_learn_install(int nfeat, int hidden, int nout, const float *params, const float *feat_mean,
                       const float *feat_std);
int gett_learn_clear(void);
/* Host inference with the installed model: predicted outputs for one
 * feature vector (raw, un-normalised).  Returns GETT_ERR_ARG if none. */
int gett_learn_predict(const float *feat, float *out);

#ifdef __cplusplus
}
#endif

#endif /* GETT_LEARN_H */

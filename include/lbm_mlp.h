/*
 * Warm-start network: a 4 -> 64 -> 64 -> 5 multilayer perceptron with GELU activations,
 * trained and evaluated on the GPU by the library's own kernels.
 *
 * The paper has no learned component.  The network maps the parameters of a run, (a,
 * T/T_c, sigma, viscosity ratio), to the five equilibrium quantities that lbm_warm.h
 * turns into an initial density field: coexistence densities and the tanh interface
 * profile of Eq. 31, plus the Laplace coefficient.
 *
 * Numerics.  The master weights, the Adam moments and all accumulations are FP32; the
 * forward and backward passes read a BF16 copy of the weights (round to nearest even),
 * refreshed after every update.  GELU is the exact form x Phi(x) with
 * Phi(x) = erfc(-x / sqrt 2) / 2.  Loss: mean over rows and outputs of the squared error
 * of standardised outputs.  Adam follows Kingma & Ba (2015), Algorithm 1.
 *
 * Parameter packing (LBM_MLP_NPARAMS floats): W1 (64 x 4), b1 (64), W2 (64 x 64),
 * b2 (64), W3 (5 x 64), b3 (5), each W stored (out, in) row-major.
 *
 * Inputs and targets are standardised inside the kernels with the scaling set by
 * lbm_mlp_set_scaling: x_n = (x - in_mean) / in_scale, t_n = (t - out_mean) / out_scale;
 * predictions are returned in physical units, out_mean + out_scale * y_n.
 *
 * Determinism: every reduction (over hidden units, over rows, of the loss) runs in a
 * fixed order, so results are bitwise repeatable for the same inputs.
 *
 * Errors: functions return LBM_OK (0) or a negative LBM_E* code of lbm.h; the message is
 * available from lbm_mlp_last_error.  All calls are synchronous unless stated otherwise.
 */
#ifndef LBM_MLP_H
#define LBM_MLP_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MLP_IN 4
#define LBM_MLP_HIDDEN 64
#define LBM_MLP_OUT 5
#define LBM_MLP_NPARAMS 4805

typedef struct lbm_mlp lbm_mlp;

typedef struct {
  double lr;     /* learning rate (step size alpha) */
  double beta1;  /* first-moment decay (0.9) */
  double beta2;  /* second-moment decay (0.999) */
  double eps;    /* denominator guard (1e-8) */
} lbm_adam;

/*
 * Create a network on `device` (-1: the current device) whose kernels run on `stream`
 * (a cudaStream_t; NULL for the legacy default stream).
 *   params    host, LBM_MLP_NPARAMS floats: the initial master weights (the caller draws
 *             them; the library draws no random numbers).  Copied.
 *   max_rows  the largest row count of any later set_data / predict call (>= 1).
 * The Adam moments start at zero and the update counter at 0.  Scaling starts as the
 * identity (means 0, scales 1).  Returns LBM_EINVAL for bad sizes, LBM_ECUDA without a
 * usable device.
 */
int lbm_mlp_create(lbm_mlp** out, const float* params, int max_rows, void* stream,
                   int device);

/* Free the network (NULL is ignored).  Synchronises its stream first. */
void lbm_mlp_destroy(lbm_mlp* h);

/* Message of the last error on this handle ("" if none).  Owned by the handle. */
const char* lbm_mlp_last_error(const lbm_mlp* h);

/*
 * Set the standardisation.  Scales must be finite and > 0 (LBM_EINVAL otherwise).
 */
int lbm_mlp_set_scaling(lbm_mlp* h, const double in_mean[4], const double in_scale[4],
                        const double out_mean[5], const double out_scale[5]);

/*
 * Set the standardisation from data: per-column mean and population standard deviation
 * (1 where a column is constant) of x (n x 4) and t (n x 5), host, row-major doubles.
 */
int lbm_mlp_fit_scaling(lbm_mlp* h, const double* x, const double* t, int n);

/*
 * Upload the training set: x (n x 4) and t (n x 5), host, row-major, doubles (rounded to
 * FP32 on upload).  1 <= n <= max_rows.  Replaces any previous set.
 */
int lbm_mlp_set_data(lbm_mlp* h, const double* x, const double* t, int n);

/*
 * `steps` full-batch Adam updates on the uploaded set.  Each update runs two kernels
 * (rows: forward and backward per row; parameters: gradient sums over rows in order and
 * the Adam update); runs of updates are replayed from a CUDA graph.
 *   losses  host, `steps` floats or NULL: losses[k] = the loss at the weights used by
 *           update k (before it is applied).
 * Returns LBM_EINVAL without data, or for steps < 0 or a non-positive learning rate.
 */
int lbm_mlp_train(lbm_mlp* h, int steps, const lbm_adam* opt, float* losses);

/*
 * Loss and gradient of the loss with respect to the master parameters at the current
 * weights (BF16 copy), without updating anything: grad (host, LBM_MLP_NPARAMS floats,
 * may be NULL), loss (host, may be NULL).  Requires uploaded data.
 */
int lbm_mlp_gradient(lbm_mlp* h, float* grad, float* loss);

/*
 * Predictions in physical units for x (n x 4, host doubles), written to y (n x 5, host
 * doubles).  1 <= n <= max_rows.
 */
int lbm_mlp_predict(lbm_mlp* h, const double* x, int n, double* y);

/*
 * Read or replace one of the parameter-sized arrays (host, LBM_MLP_NPARAMS floats):
 *   which 0 = master weights, 1 = the BF16 copy (widened to FP32; read only),
 *         2 = Adam first moment, 3 = Adam second moment.
 * Writing the master weights refreshes the BF16 copy.
 */
int lbm_mlp_get_params(lbm_mlp* h, int which, float* out);
int lbm_mlp_set_params(lbm_mlp* h, int which, const float* in);

/* Number of Adam updates applied since create. */
long long lbm_mlp_update_count(const lbm_mlp* h);

#ifdef __cplusplus
}
#endif
#endif

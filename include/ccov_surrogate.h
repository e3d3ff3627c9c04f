/*
 * ccov surrogate: a learned per-camera predictor of the 9x9 covariance blocks
 * of include/ccov.h, trained on blocks that the exact method computes.
 *
 * The paper has no learned component.  Its uses of camera covariances
 * (Sec. 1: choosing the next best view, detecting wrongly added cameras,
 * filtering unconstrained cameras) only need a fast, approximate screen,
 * with the exact method kept as the fallback and as the reference for its error.
 *
 * Per camera i (after ccov_information):
 *   Z_ii     the 9x9 diagonal block of the reduced camera matrix of Sec. 4.2
 *   d        sqrt(diag Z_ii): the block's Jacobi scale
 *   L_z      the Cholesky factor of Z_ii (the `scale` arrays, 9 x 9 row-major,
 *            zero above the diagonal); Z_ii^-1 is the camera's covariance with
 *            every other camera held fixed
 *   features 64 floats: [0,36) Z_kl / (d_k d_l) for k < l row by row,
 *            [36,45) log d_k, 45 log(observations of the camera),
 *            46 mean log track length of its points, 47 fraction of its
 *            points seen twice, 48 10/sqrt(n), 49 distance of the camera centre
 *            -R^T t from the mean centre over the RMS of those distances,
 *            [50,64) zero
 *   target   45 floats, the Cholesky factor L of the whitened exact block
 *            S = L_z^T Sigma_i L_z: [0,9) log L_kk, [9,45) L_kl for k > l
 *            row by row (all zero when Sigma_i = Z_ii^-1)
 * Network: 64 -> 256 -> 256 -> 256 -> 45, ReLU on the hidden layers, every
 * product on the tensor cores with bf16 operands and fp32 accumulation;
 * inputs and targets standardised by per-column mean and deviation.
 * Prediction: Sigma_hat_i = L_z^-T L_hat L_hat^T L_z^-1.
 *
 * Gauge term of the base.  Z_ii^-1 holds every other camera fixed and so
 * also pins the datum; in the similarity gauge of Sec. 4.1 the camera moves
 * with the datum, along its rows H_i of the nullspace (9 x 7, Sec. 4.1).  On
 * exact blocks Sigma_i - Z_ii^-1 lies almost entirely in their span, and in
 * the scene's metric one 7 x 7 matrix M, nearly independent of the scene's
 * size, accounts for it:
 *   Q_i  H_i L_c, L_c the Cholesky factor of (sum_i H_i^T Z_ii H_i)^-1
 *   B_i  Z_ii^-1 + Q_i M Q_i^T, the base covariance
 *   T_i  the Cholesky factor of B_i^-1 (T_i = L_z when M = 0)
 * M is fitted by least squares on exact training blocks.  Passing T_i as
 * the `scale` of ccov_surrogate_targets and ccov_surrogate_predict (in place
 * of L_z) makes the network learn, and predict, the remainder around B_i.
 *
 * Parameters (CCOV_SURR_PARAMS floats, host order): W1 (256 x 64), b1 (256),
 * W2 (256 x 256), b2, W3 (256 x 256), b3, W4 (45 x 256), b4 (45); every W
 * row-major with one row per output.  Normalisation (CCOV_SURR_NORM floats):
 * feature mean (64), feature deviation (64), target mean (45), target
 * deviation (45).
 *
 * Arrays marked "device" are device pointers; "host" are host pointers.
 * Every call runs on the model's stream (or the context's, for
 * ccov_surrogate_features) and returns after that stream has finished it.
 */
#ifndef CCOV_SURROGATE_H
#define CCOV_SURROGATE_H

#include "ccov.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CCOV_SURR_FEATURES 64
#define CCOV_SURR_OUTPUTS 45
#define CCOV_SURR_HIDDEN 256
#define CCOV_SURR_PARAMS 159789
#define CCOV_SURR_NORM 218

typedef struct ccov_surrogate ccov_surrogate;

/* Features and scales of every camera of a context that has run
 * ccov_information.  Z_ii is accumulated from the information blocks
 * (U_i - sum_j W_ij A_j^-1 W_ij^T), so neither the dense Z of ccov_schur nor
 * step (d) is needed.  features: device n x 64 float32; scale: device n x 81
 * float64 (L_z).  DEGENERATE if a block Z_ii is not positive definite. */
CCOV_API ccov_status ccov_surrogate_features(ccov_ctx* ctx, float* features, double* scale);

/* Gauge rows of the base for every camera of a context that has run
 * ccov_information and ccov_nullspace: scale device n x 81 float64 (L_z from
 * ccov_surrogate_features), q device n x 63 float64 (Q_i = H_i L_c, 9 x 7
 * row-major).  The scene sum sum_i H_i^T Z_ii H_i runs in a fixed order (the
 * same bits on every run).  INVALID_ARG before those calls or for cameras of
 * CCOV_CAMERA_CENTRE8; DEGENERATE if the scene sum is not positive
 * definite. */
CCOV_API ccov_status ccov_surrogate_gauge_rows(ccov_ctx* ctx, const double* scale, double* q);

/* Training targets from exact covariance blocks: sigma device n x 81
 * float64 (ccov_covariance output), scale device n x 81 float64 (a lower
 * whitening factor: L_z from ccov_surrogate_features, or T_i from
 * ccov_surrogate_apply_gauge), targets device n x 45 float32.  stream: a
 * cudaStream_t or NULL.  DEGENERATE if a block is not positive definite. */
CCOV_API ccov_status ccov_surrogate_targets(int64_t n, const double* scale, const double* sigma, float* targets,
                                            void* stream);

/* A model with the given parameters (host, CCOV_SURR_PARAMS floats), unit
 * normalisation, zero Adam moments, and workspace for batches of up to
 * max_batch rows (1 <= max_batch <= 65536).  stream: a cudaStream_t or NULL
 * (the model then creates its own).  On failure *out may still hold a model:
 * read ccov_surrogate_last_error, then ccov_surrogate_destroy it. */
CCOV_API ccov_status ccov_surrogate_create(const float* params, int64_t max_batch, void* stream,
                                           ccov_surrogate** out);

/* Normalisation from a training set (device features n x 64, targets
 * n x 45): column means and population deviations, a deviation below 1e-6
 * replaced by 1. */
CCOV_API ccov_status ccov_surrogate_fit_normalization(ccov_surrogate* s, const float* features,
                                                      const float* targets, int64_t n);
CCOV_API ccov_status ccov_surrogate_set_normalization(ccov_surrogate* s, const float* norm);
CCOV_API ccov_status ccov_surrogate_get_normalization(const ccov_surrogate* s, float* norm);
CCOV_API ccov_status ccov_surrogate_set_params(ccov_surrogate* s, const float* params);
CCOV_API ccov_status ccov_surrogate_get_params(const ccov_surrogate* s, float* params);

/* Gradient of the mean squared error (over the batch and the 45
 * standardised outputs) on the rows idx[0..batch) of (features n x 64,
 * targets n x 45), all device arrays (idx int32; 1 <= batch <= max_batch).
 * The gradient stays in the model for ccov_surrogate_get_grads and
 * ccov_surrogate_adam; loss: host float or NULL.  An index outside [0, n) is
 * caught on the device: INVALID_ARG. */
CCOV_API ccov_status ccov_surrogate_backward(ccov_surrogate* s, const float* features, const float* targets,
                                             int64_t n, const int32_t* idx, int64_t batch, float* loss);
CCOV_API ccov_status ccov_surrogate_get_grads(const ccov_surrogate* s, float* grads);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the gradient in the
 * model; the step count that the bias correction uses grows by one. */
CCOV_API ccov_status ccov_surrogate_adam(ccov_surrogate* s, float lr);

/* `steps` training steps, step k on the rows idx[k*batch .. (k+1)*batch)
 * (device int32, steps x batch): backward and Adam, recorded once as a CUDA
 * graph and replayed.  losses: host array of `steps` floats (the loss of
 * each step before its update) or NULL. */
CCOV_API ccov_status ccov_surrogate_train(ccov_surrogate* s, const float* features, const float* targets,
                                          int64_t n, const int32_t* idx, int64_t batch, int steps, float lr,
                                          float* losses);

/* Sigma_hat for n cameras: features device n x 64, scale device n x 81
 * (the factor the model's targets were taken with: L_z, or T_i), sigma
 * device n x 81 float64 (row-major 9 x 9 blocks). */
CCOV_API ccov_status ccov_surrogate_predict(ccov_surrogate* s, const float* features, const double* scale,
                                            int64_t n, double* sigma);

/* The model's gauge matrix M (host, 49 float64, row-major, symmetric;
 * zero in a new model, so that the base is Z_ii^-1).  set: INVALID_ARG
 * unless finite and exactly symmetric. */
CCOV_API ccov_status ccov_surrogate_set_gauge(ccov_surrogate* s, const double* M);
CCOV_API ccov_status ccov_surrogate_get_gauge(const ccov_surrogate* s, double* M);

/* Fit of M by least squares over n training cameras (of any number of
 * scenes, each q from its own scene's ccov_surrogate_gauge_rows): the
 * symmetric M minimising
 *   sum_i |L_z^T (Sigma_i - Z_ii^-1) L_z - L_z^T Q_i M Q_i^T L_z|_F^2
 * (scale device n x 81 L_z, q device n x 63, sigma device n x 81 exact
 * blocks), through its 28 x 28 normal equations, summed in a fixed order
 * and solved by Cholesky on the device.  The result replaces the model's M.
 * DEGENERATE if the normal equations are not positive definite (too few
 * cameras or cameras whose rows do not determine M). */
CCOV_API ccov_status ccov_surrogate_fit_gauge(ccov_surrogate* s, const double* scale, const double* q,
                                              const double* sigma, int64_t n);

/* The base factor T_i = chol((Z_ii^-1 + Q_i M Q_i^T)^-1) for n cameras with
 * the model's M: scale device n x 81 (L_z), q device n x 63, base device
 * n x 81 float64 (lower triangular, row-major), to be passed as the `scale`
 * of ccov_surrogate_targets and ccov_surrogate_predict.  DEGENERATE if a B_i
 * is not positive definite (its T_i is then zero). */
CCOV_API ccov_status ccov_surrogate_apply_gauge(ccov_surrogate* s, const double* scale, const double* q, int64_t n,
                                                double* base);

CCOV_API void ccov_surrogate_destroy(ccov_surrogate* s);
CCOV_API const char* ccov_surrogate_last_error(const ccov_surrogate* s);

#ifdef __cplusplus
}
#endif

#endif /* CCOV_SURROGATE_H */

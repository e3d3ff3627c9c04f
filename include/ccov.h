/*
 * ccov: camera covariance propagation for bundle-adjusted reconstructions on
 * one NVIDIA GB300 (sm_103a).
 *
 * Method: Polic, Foerstner, Pajdla, "Fast and Accurate Camera Covariance
 * Computation for Large 3D Reconstruction".  Given the estimated cameras and
 * points, the index set S of observations and the image-point covariance
 * Sigma_u (Sec. 3), the library returns the 9x9 camera blocks of the natural
 * covariance, i.e. the camera part of the inverse of the bordered information
 * matrix [M H; H^T 0] (Sec. 3, Eq. inversion-of-extended-information-matrix),
 * which equals the camera part of the Moore-Penrose inverse of M.
 *
 * Camera model (9 values per camera, row-major n x 9):
 *   P_i = {r (angle-axis, 3), t (3), f, k1, k2},  X_c = R(r) X + t,
 *   u_hat = f (1 + k1 rho^2 + k2 rho^4) (X_c[0], X_c[1]) / X_c[2],
 *   rho^2 = (X_c[0]^2 + X_c[1]^2) / X_c[2]^2.
 * This is the translation form of the projection of Sec. 4.1 with two radial
 * distortion terms.  Output blocks use the same parameter order.
 *
 * Call order on one context: ccov_create -> ccov_information -> ccov_schur ->
 * ccov_nullspace -> ccov_covariance.  ccov_nullspace may come anywhere before
 * ccov_covariance.  A call made out of order returns CCOV_ERR_INVALID_ARG.
 * Each call runs on the context's CUDA stream and returns after that stream
 * has finished the call's work, so its status covers device-side checks.
 *
 * Ownership: the caller owns every buffer it passes; ccov_create copies the
 * inputs; outputs are written into caller-allocated buffers.  The library
 * allocates its own device workspace in ccov_create (with cudaMalloc) and
 * frees it in ccov_destroy.  No global state: one context per thread.
 * Errors: every entry point returns a ccov_status; after a failure the
 * context stays valid for ccov_destroy and ccov_last_error.
 */
#ifndef CCOV_H
#define CCOV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CCOV_API __attribute__((visibility("default")))
#else
#define CCOV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccov_ctx ccov_ctx;

/* One observation u_ij of point `pt` in camera `cam` (24 bytes, packed as
 * int32, int32, float64[2]).  The observed u does not enter the covariance
 * (M depends on theta, S and Sigma_u only, Sec. 3); it is validated as finite. */
typedef struct {
    int32_t cam;
    int32_t pt;
    double u[2];
} ccov_obs;

typedef enum {
    CCOV_OK = 0,
    CCOV_ERR_INVALID_ARG = 1,   /* bad size, index, pointer, order of calls */
    CCOV_ERR_DEGENERATE = 2,    /* track < 2, camera < 2 obs, point behind a camera,
                                   singular point block A_j or W7, matrix not SPD */
    CCOV_ERR_NOT_CONVERGED = 3,
    CCOV_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    CCOV_ERR_OOM = 5,           /* device allocation failed */
    CCOV_ERR_CUDA = 6           /* any other CUDA runtime error */
} ccov_status;

enum { CCOV_PREC_FP64 = 0, CCOV_PREC_MIXED = 1 };
enum { CCOV_MEM_HOST = 0, CCOV_MEM_DEVICE = 1 };
enum { CCOV_NULL_PAPER = 0, CCOV_NULL_CLOSED = 1 };
enum { CCOV_GAUGE_NATURAL = 0, CCOV_GAUGE_ZPINV = 1, CCOV_GAUGE_FIXED3 = 2 };
enum { CCOV_CAMERA_RT9 = 0, CCOV_CAMERA_CENTRE8 = 1 };

typedef struct {
    int precision;        /* CCOV_PREC_FP64 (default): every sum in FP64;
                             CCOV_PREC_MIXED: step (d) as exact digit products on the
                             tensor cores (int64 fixed point, mixed_slices digits) and the
                             Schur sums of step (b) in double-single arithmetic (about 44
                             bits, above the digits' 39) */
    int mixed_slices;     /* MIXED only: 8-bit digit slices per operand, 4..6; 0 = 5 for
                             the natural gauge with the 9-value camera, 6 for
                             CCOV_GAUGE_ZPINV / _FIXED3 and CCOV_CAMERA_CENTRE8, whose
                             Jacobi-scaled matrices have condition numbers near 2e6
                             (2e4 otherwise) */
    int nullspace_route;  /* CCOV_NULL_PAPER: rotation rows from J_r H_r = B (Sec. 4.1,
                             Eq. rotation-nullspace-equation), default;
                             CCOV_NULL_CLOSED: -J_r^-1(r) in closed form */
    int input_memory;     /* where ccov_create's / ccov_load's arrays live:
                             CCOV_MEM_HOST (default) or CCOV_MEM_DEVICE */
    int profile;          /* 1: bracket every dense trailing-update GEMM with CUDA
                             events and report their time in ccov_stats */
    int est_cameras;      /* cameras sampled by the error estimate of ccov_covariance
                             (only when its est_rel_err is not NULL): 1..16, 0 = 4 */
    int gauge;            /* CCOV_GAUGE_NATURAL (default): the method of the paper, the
                             camera block of the natural covariance [M+]_PP;
                             CCOV_GAUGE_ZPINV: Alg. 4 of Table 2, the Moore-Penrose
                             inverse of the reduced camera matrix Z (projected onto the
                             complement of the similarity nullspace, which leaves it
                             unchanged); CCOV_GAUGE_FIXED3: Alg. 5 of Table 2, three
                             points taken out of the parameters, the inverse of the
                             full-rank Schur complement of the others (computed exactly) */
    int fixed_points[3];  /* CCOV_GAUGE_FIXED3: the three point indices; all three -1 (or
                             all 0): the point farthest from the centroid of the points,
                             the point farthest from it, the point farthest from the line
                             through those two (ties: the smaller index) */
    int camera_model;     /* CCOV_CAMERA_RT9 (default): 9 values per camera, as above;
                             CCOV_CAMERA_CENTRE8: the paper's camera of Sec. 3 and
                             Sec. 4.1, 8 values {r, C, c, k} with X_c = R(r) (X - C),
                             u = c (1 + k rho^2) (X_c[0], X_c[1]) / X_c[2]; `cameras` is
                             then n x 8 (ccov_create, ccov_load), and each returned 9x9
                             block holds the 8x8 covariance of (r, C, c, k) in its
                             top-left corner, its 9th row and column those of an
                             uncorrelated dummy value of variance 1 (a unit prior on a
                             parameter that no observation sees) */
    int reserved[1];      /* set to zero */
} ccov_options;

/* Per-context counters of the last calls (device times from CUDA events). */
typedef struct {
    int64_t n, m, t, N, N_pad;
    double ms_information, ms_schur, ms_nullspace, ms_covariance;
    double ms_factor, ms_inverse;       /* parts of ms_covariance */
    int64_t bytes_device;               /* device workspace held by the context */
    int64_t launches;                   /* kernels launched by the last four calls */
    double ms_gemm;                     /* profile = 1: summed device time of the
                                           trailing-update GEMMs of the last ccov_covariance */
    double gemm_flops;                  /* their executed flops: the MIXED path counts
                                           every kept 128 x 64 tile times its s(s+1)/2
                                           digit products, the FP64 path 2 M N K per
                                           update (lower-triangle updates counted once) */
    int64_t gemm_launches;
    /* error estimate of the last ccov_covariance that asked for one (est_rel_err
     * not NULL): the sampled cameras and, per sampled camera, the estimated
     * relative Frobenius error of its block and the same after the scaling
     * diag(Sigma_i)^-1/2; est_cameras = 0 when no estimate was made */
    int64_t est_cameras;
    int64_t est_index[16];
    double est_rel[16];
    double est_norm[16];
    /* the last ccov_update_observations: device time and kernels launched */
    double ms_update;
    int64_t update_launches;
} ccov_stats;

/* Create a context for one scene and copy its inputs to the device.
 *   cameras  n x 9 float64, row-major, parameter order (r, t, f, k1, k2)
 *   points   m x 3 float64, row-major
 *   obs      t records sorted by point index (non-decreasing `pt`); each
 *            (cam, pt) pair at most once; every point needs >= 2 observations
 *            and every camera >= 2
 *   sigma    isotropic image-point standard deviation in pixels (> 0); used
 *            when obs_cov is NULL, Sigma_u = sigma^2 I (Sec. 3)
 *   obs_cov  NULL, or t x 4 float64: per-observation 2x2 SPD covariance
 *            Sigma_u_ij, row-major (Sec. 3, block-diagonal Sigma_u)
 *   opt      NULL for defaults
 *   stream   a cudaStream_t, or NULL for a stream the context creates
 * Errors: INVALID_ARG for sizes, indices, ordering or non-finite values;
 * DEGENERATE for tracks or cameras with fewer than two observations;
 * OOM when the device workspace (about 2 (9n)^2 x 8 bytes) does not fit. */
CCOV_API ccov_status ccov_create(const double* cameras, int64_t n, const double* points, int64_t m,
                        const ccov_obs* obs, int64_t t, double sigma, const double* obs_cov,
                        const ccov_options* opt, void* stream, ccov_ctx** out);

/* Replace the inputs of an existing context by a scene of the same n, m, t
 * and the same index set S (same cam/pt columns of `obs`).  `memory` says
 * where the arrays live (CCOV_MEM_HOST or CCOV_MEM_DEVICE).  Resets the call
 * sequence to "created". */
CCOV_API ccov_status ccov_load(ccov_ctx* ctx, const double* cameras, const double* points,
                      const ccov_obs* obs, const double* obs_cov, int memory);

/* Step (a), Sec. 3 Eq. normal-equation-system: analytic reprojection
 * Jacobians of every observation, whitened by Sigma_u^-1/2, and the blocks of
 * M = J^T Sigma_u^-1 J: U_i (camera), A_j^-1 (point, inverted) and W_ij.
 * DEGENERATE if a point lies behind a camera or a point block is singular. */
CCOV_API ccov_status ccov_information(ccov_ctx* ctx);

/* Step (b), Sec. 4.2 Eq. schur-complement-inversion: eliminate the 3x3 point
 * blocks.  Builds the dense reduced camera matrix Z = U - W A^-1 W^T
 * (9n x 9n, FP64, lower triangle), the border part -W A^-1 H_X of G and
 * W7 = H_X^T A^-1 H_X, i.e. Z_p = [Z, G; G^T, -W7] of Eq. block-inversion-Qp
 * for the unconditioned system. */
CCOV_API ccov_status ccov_schur(ccov_ctx* ctx);

/* Step (c), Sec. 4.1: the camera rows H_P (n x 9 x 7, columns [T, omega, mu])
 * of the similarity nullspace.  Translation and scale columns in closed form
 * (Eq. transformation-conditions); rotation rows from J_r H_r = B per camera
 * (Eq. rotation-nullspace-equation), least squares over the camera's rows.
 * H_P_out: NULL, or a host buffer of n*63 float64 (row-major 9 x 7 blocks). */
CCOV_API ccov_status ccov_nullspace(ccov_ctx* ctx, double* H_P_out);

/* Step (d), Sec. 4.2: Sigma_P = top-left block of Z_p^-1 =
 * (Z + G W7^-1 G^T)^-1 (block inversion of Z_p), computed as Jacobi scaling,
 * Cholesky factorisation, triangular inverse and the 9x9 diagonal blocks of
 * the inverse.  out: n*81 float64 (row-major 9 x 9 blocks) on the host
 * (out_memory = CCOV_MEM_HOST) or the device (CCOV_MEM_DEVICE).
 * est_rel_err: NULL, or n doubles receiving an a-posteriori estimate of each
 * block's relative Frobenius error against the exact inverse.  It is computed
 * (at extra cost O(N^2 k)) for k sampled cameras (ccov_options.est_cameras,
 * default 4): those with the largest diagonal entry of their Jacobi-scaled
 * block, i.e. the most ill-determined parameters.  For a sampled camera i the
 * estimate is the first-order error y^T R of its block, from the residual
 * R = Z_s y - E_i of the computed columns y = X^T X E_i against a copy of the
 * scaled matrix Z_s taken before the factorisation (double-single arithmetic
 * for the MIXED path, FP64 for the FP64 path, where it is an upper estimate
 * at the residual's own rounding level).  Every other camera receives the
 * largest of the sampled estimates (the error of a block varies from camera
 * to camera by up to about 30x at the same conditioning, so this is a
 * scene-level figure for them).  ccov_stats lists the sampled cameras.
 * DEGENERATE if the scaled reduced matrix is not positive definite;
 * NOT_CONVERGED if the MIXED path's fixed-point range is exceeded (a scene too
 * ill-conditioned for it: an entry of L^-1 beyond 2^19, or a scaled entry
 * beyond 2), in which case precision FP64 is the remedy. */
CCOV_API ccov_status ccov_covariance(ccov_ctx* ctx, double* out, int out_memory, double* est_rel_err);

/* Copies of intermediate results for checking (host buffers, NULL to skip):
 *   U     n x 81 camera blocks of M          A_inv  m x 9 inverted point blocks
 *   W     t x 27 (9 x 3 per observation, in observation order)
 *   Z     (9n) x (9n) after ccov_schur: lower triangle valid, upper undefined
 *   G     (9n) x 7 after ccov_schur and ccov_nullspace (H_P - W A^-1 H_X)
 *   W7    7 x 7 */
CCOV_API ccov_status ccov_get_blocks(ccov_ctx* ctx, double* U, double* A_inv, double* W);
CCOV_API ccov_status ccov_get_schur(ccov_ctx* ctx, double* Z, double* G, double* W7);

/* Selected 9 x 9 blocks Z_ij of the reduced camera matrix (Sec. 4.2, Eq.
 * schur-complement-inversion: Z = M_PP - M_PX A^-1 M_XP), for checking a
 * large scene on sampled blocks without copying all of Z.  Valid between
 * ccov_schur and ccov_covariance (which consumes Z in place; afterwards the
 * call returns INVALID_ARG until ccov_schur runs again).
 *   ij       nblocks pairs (i, j) of camera indices with 0 <= j <= i < n
 *            (the stored lower triangle; Z_ji = Z_ij^T), host memory
 *   nblocks  >= 0
 *   out      nblocks x 81 float64, row-major blocks, host memory (caller's);
 *            a diagonal block (i = j) holds its lower triangle, the entries
 *            above its diagonal are undefined
 * INVALID_ARG for a pair outside the lower triangle or before ccov_schur. */
CCOV_API ccov_status ccov_get_schur_blocks(ccov_ctx* ctx, const int64_t* ij, int64_t nblocks, double* out);

CCOV_API ccov_status ccov_get_stats(const ccov_ctx* ctx, ccov_stats* out);

/* Batched form, Sec. 5 (uncertainty for sub-reconstructions): the camera
 * covariances of k independent scenes, e.g. the neighbourhoods of 100-300
 * cameras into which a large reconstruction is decomposed.  Each ctxs[i] is a
 * created context (its own scene, options and stream); the call runs steps
 * (a)-(d) of every context without host synchronisation between them, so the
 * scenes proceed concurrently on their streams, then waits for all of them.
 *   ctxs        k contexts (k >= 1), each used by this call alone
 *   outs        k buffers of n_i*81 float64, on the host or the device as
 *               `out_memory` says
 * Returns the first failing status in context order; every context's own
 * status is left in its ccov_last_error.  Afterwards each context is in the
 * state ccov_information leaves (its Z has been consumed). */
CCOV_API ccov_status ccov_batch_covariance(ccov_ctx* const* ctxs, int k, double* const* outs, int out_memory);

/* The same batch recorded once as a CUDA graph and replayed by ccov_batch_run
 * with a single graph launch.  ccov_batch_create runs the batch once directly
 * (validating the scenes and preparing every kernel), then captures steps
 * (a)-(d) of all k contexts, forked from one stream onto the contexts' streams
 * and joined back.  outs_device: k device buffers of n_i*81 float64 that each
 * replay writes.  The contexts, their streams and the buffers must outlive the
 * batch; between create and destroy the contexts belong to the batch (a direct
 * call on one of them in between is allowed, but changes nothing in the
 * graph).  Inputs may be replaced with ccov_load (same sizes, device copies
 * happen on the context stream) and are picked up by the next replay.
 * ccov_batch_run: stream = a cudaStream_t or NULL for the batch's own stream;
 * returns after the replay has finished, with the first failing status. */
typedef struct ccov_batch ccov_batch;
CCOV_API ccov_status ccov_batch_create(ccov_ctx* const* ctxs, int k, double* const* outs_device, ccov_batch** out);
CCOV_API ccov_status ccov_batch_run(ccov_batch* batch, void* stream);
CCOV_API void ccov_batch_destroy(ccov_batch* batch);

/* Form of a recorded batch.
 *   CCOV_BATCH_GROUPED: every step of steps (a)-(d) is one launch for all
 *     scenes (the scenes concatenated for (a)-(c); for (d), per sub-panel
 *     pair of the blocked factorisation and inverse, one launch per sub-step
 *     over the scenes that have it, the trailing-update GEMMs as one
 *     persistent tensor-core kernel over the tiles of all of them); the
 *     graph holds a few hundred kernels.  Needs MIXED precision with the same
 *     mixed_slices, nullspace_route and image-point model (the same sigma, or
 *     per-observation covariances) in every context.  The contexts' inputs
 *     are read at every replay (so ccov_load applies); their own workspaces
 *     are not used.  A device-side failure is reported for the batch as a
 *     whole.  When the batch is created, an autotuner times the whole batch
 *     under a few launch shapes of the grouped GEMMs (persistent CTA count,
 *     pipeline depth) and keeps the fastest.
 *   CCOV_BATCH_PER_SCENE: every context's own steps, forked onto the
 *     contexts' streams and joined back (any precision, any options).
 *   CCOV_BATCH_AUTO: grouped when the contexts allow it, else per scene. */
enum { CCOV_BATCH_AUTO = 0, CCOV_BATCH_PER_SCENE = 1, CCOV_BATCH_GROUPED = 2,
       CCOV_BATCH_NO_TUNE = 8 /* or-ed into the form: keep the default launch shape, no tuning passes */ };
CCOV_API ccov_status ccov_batch_create_ex(ccov_ctx* const* ctxs, int k, double* const* outs_device, int form,
                                          ccov_batch** out);

typedef struct {
    int form;               /* CCOV_BATCH_PER_SCENE or CCOV_BATCH_GROUPED */
    int gemm_ctas;          /* grouped: persistent CTAs of the GEMMs chosen by the autotuner */
    int gemm_stages;        /* grouped: their pipeline depth */
    int64_t launches;       /* kernels per replay */
    double tune_ms;         /* grouped: the batch time of the chosen shape while tuning */
} ccov_batch_info;
CCOV_API ccov_status ccov_batch_get_info(const ccov_batch* batch, ccov_batch_info* out);

/* Uncertainty from sub-reconstructions, Sec. 5: a camera's uncertainty is
 * evaluated from a sub-reconstruction of the cameras and points around it;
 * each evaluation bounds it from above; the scene is decomposed several times
 * and per camera the covariance with the smallest trace is kept (Sec. 6 uses
 * the 100 neighbours of a camera in the view graph).
 *   view graph  cameras i, k adjacent, weight = the number of points both see
 *   neighbourhood of a seed camera: grown one camera at a time, adding the
 *               camera with the largest total weight to those chosen (ties:
 *               the smaller index), until cams_per_sub cameras or none left
 *   decomposition d: cameras tried as seeds in the order seed_order[d][.];
 *               a camera already in a neighbourhood of d is skipped, so each
 *               decomposition covers every camera
 *   sub-reconstruction: the neighbourhood's cameras, the points at least two
 *               of them see and those observations, then cameras and points
 *               with fewer than two observations dropped until none is left
 *   merge:      per camera, the 9x9 block of smallest trace over the
 *               sub-reconstructions that hold it */
typedef struct {
    int cams_per_sub;           /* cameras per neighbourhood, >= 2 */
    int decompositions;         /* >= 1 */
    const int32_t* seed_order;  /* host, decompositions x n: each row a permutation of 0..n-1 */
} ccov_subrecon_options;

/* The camera sets of the sub-reconstructions, in order (decomposition by
 * decomposition), as CSR: sub s holds sub_cams[sub_ptr[s] .. sub_ptr[s+1]),
 * ascending.  obs as for ccov_create (sorted by point).  *nsub and *total are
 * always written; INVALID_ARG (nothing else written) if max_subs or max_total
 * is too small (NULL buffers with 0 capacities: a size query). */
CCOV_API ccov_status ccov_subrecon_plan(const ccov_obs* obs, int64_t t, int64_t n, int64_t m,
                                        const ccov_subrecon_options* sopt, int64_t max_subs, int64_t max_total,
                                        int32_t* sub_ptr, int32_t* sub_cams, int64_t* nsub, int64_t* total);

/* The whole pipeline: plan, extraction, the covariances of all
 * sub-reconstructions as one batch (grouped launches for precision MIXED),
 * merge.  Inputs as for ccov_create, host memory; opt applies to every
 * sub-reconstruction.  out: host n x 81, the merged blocks (NaN for a camera
 * that no usable sub-reconstruction holds); cover: NULL or n int32, how many
 * sub-reconstructions held each camera; nsub: NULL or the number solved.
 * A degenerate sub-reconstruction is skipped. */
CCOV_API ccov_status ccov_subrecon_covariance(const double* cameras, int64_t n, const double* points, int64_t m,
                                              const ccov_obs* obs, int64_t t, double sigma, const double* obs_cov,
                                              const ccov_options* opt, const ccov_subrecon_options* sopt,
                                              double* out, int32_t* cover, int64_t* nsub);

/* Camera covariances after adding observations (Sec. 5: M_{i+1} = M_i +
 * M_Delta and the Woodbury identity), from the factorisation of the last
 * ccov_covariance on this context, without a new factorisation.  Exact up to
 * rounding: the result is the natural covariance of the scene with the added
 * observations, as ccov_covariance of that scene would return it.  Adding
 * observations changes the point blocks A as well as Z; the identity is taken
 * on the whole regularised information matrix, so its rank is 2k (two rows per
 * observation) whatever the number of cameras that see the points.  Cost
 * O(N^2 k + N k^2 + k^3) against O(N^3) for a new step (d).
 *   ctx       after a successful ccov_covariance (natural gauge, either camera
 *             model); ccov_load / ccov_information / ccov_schur / a batch on
 *             it end that state.  The context is not changed: it keeps the
 *             scene it holds, and further calls evaluate other additions
 *             against the same factorisation (a next-best-view loop).
 *   add       host, k observations of existing cameras and points (the same
 *             record as ccov_create; the pair need not be new)
 *   k         0 <= k <= 4096; 0 returns the blocks of the last ccov_covariance
 *   add_cov   host, k x 4 per-observation 2x2 covariances (row-major), or NULL
 *             for sigma^2 I; must be NULL/non-NULL as for ccov_create
 *   out       n x 81 doubles on out_memory (CCOV_MEM_HOST or CCOV_MEM_DEVICE),
 *             written
 * Returns INVALID_ARG for a bad index, k, pointer, gauge or order of calls,
 * DEGENERATE for an added observation behind its camera. */
CCOV_API ccov_status ccov_update_observations(ccov_ctx* ctx, const ccov_obs* add, int64_t k, const double* add_cov,
                                              double* out, int out_memory);

/* Allocation-free entry point (the paper has no counterpart).  For callers that
 * cannot call cudaMalloc: a real-time loop that must not allocate, or code in a
 * process whose device memory is owned by another allocator (a framework's
 * caching allocator that has reserved it), where a cudaMalloc may fail or stall
 * the device.  Returns the 9x9 diagonal blocks of A^-1 for a symmetric positive
 * definite A with the FP64 kernels of step (d) (Jacobi scaling, blocked Cholesky,
 * triangular inverse, diagonal Gram blocks); all workspace lives in one static
 * device array of the library (7.9 MB, held on every GPU that loads the library
 * until the process exits).  Nothing is allocated by the call.
 *   A       device, N x N row-major, leading dimension lda >= N; only the lower
 *           triangle is read; not modified
 *   N       a multiple of 9 and at most 576 (64 camera blocks); a larger N is
 *           rejected with CCOV_ERR_INVALID_ARG
 *   blocks  device, (N / 9) x 81 doubles (row-major 9 x 9 blocks), written
 *   stream  a cudaStream_t, or NULL for the legacy default stream; the call
 *           returns after the stream has finished its work
 * The first call on a device (that device current) takes the array's address
 * with cudaGetSymbolAddress and sets kernel attributes.  Every call shares the
 * array and first clears what must start at zero, so a call that failed
 * part-way leaves nothing the next call depends on; calls that overlap on the
 * GPU race on it.  DEGENERATE if A is not positive definite. */
CCOV_API ccov_status ccov_spd_inverse_blocks_noalloc(const double* A, int64_t lda, int64_t N, double* blocks,
                                                     void* stream);
CCOV_API void ccov_destroy(ccov_ctx* ctx);
CCOV_API const char* ccov_status_string(ccov_status s);
/* Message of the last failure on this context ("" if none). */
CCOV_API const char* ccov_last_error(const ccov_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CCOV_H */

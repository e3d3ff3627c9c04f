// Internal declarations shared by the ccov translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/ccov.h"
#include "group.cuh"

namespace ccov {

constexpr int kNB = 128;         // dense block size: panel width and K of every trailing update
constexpr int kCamPrep = 25;     // doubles per prepared camera: R(9) t(3) f k1 k2 (3) J_l(9) model(1)
constexpr int kEstMaxCams = 16;  // sampled cameras of the a-posteriori error estimate, at most
constexpr int kEstDefaultCams = 4;

// Device-side error codes written with atomicMax into ctx->d_flag[0].
enum DevErr : int {
    DEV_OK = 0,
    DEV_BEHIND = 1,       // point behind a camera
    DEV_SINGULAR_A = 2,   // point block A_j not positive definite
    DEV_NOT_SPD = 3,      // reduced camera matrix not positive definite
    DEV_SINGULAR_W7 = 4,
    DEV_SINGULAR_JR = 5,  // J_r^T J_r of a camera singular (nullspace solve)
    DEV_TIMEOUT = 6,      // a bounded spin-wait gave up
    DEV_BAD_INDEX = 7,    // a sample index outside the training set (surrogate)
    DEV_SMEM_ALIGN = 8,   // dynamic shared memory window not 1024-byte aligned (GEMM)
    DEV_RANGE = 9,        // a value left the range of the mixed path's fixed-point formats
};

struct MixedState;  // emulated-FP64 tensor-core path, k_mixed.cu

struct Ctx {
    int64_t n = 0, m = 0, t = 0, N = 0, Np = 0;
    ccov_options opt{};
    double sigma = 1.0;
    bool has_cov = false;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int stage = 0;            // 1 created, 2 information, 3 schur; nullspace tracked apart
    bool null_done = false;
    std::string err;

    // inputs
    double* d_cams = nullptr;     // n x 9
    double* d_pts = nullptr;      // m x 3
    ccov_obs* d_obs = nullptr;    // t
    double* d_obscov = nullptr;   // t x 4 or null
    int* d_pt_ptr = nullptr;      // m + 1
    int* d_cam_ptr = nullptr;     // n + 1
    int* d_cam_perm = nullptr;    // t: observation ids grouped by camera
    // step (a)
    double* d_camprep = nullptr;  // n x kCamPrep
    double* d_W = nullptr;        // t x 27
    double* d_Ainv = nullptr;     // m x 6 (xx xy xz yy yz zz)
    double* d_U = nullptr;        // n x 45 (lower triangle, row by row)
    // step (b), (c)
    double* d_V = nullptr;        // t x 27: W A^-1 per observation (step (a): scratch)
    double* d_J = nullptr;        // t x 24: unwhitened Jc (2 x 9), Jp (2 x 3) per observation, from step (a)
    int4* d_pair_desc = nullptr;  // blocks Z_ik with shared points: (i, k, first entry, entries)
    int2* d_pair_ent = nullptr;   // per block, the observation pairs (o_i, o_k) in point order
    int64_t npairs = 0, nent = 0;
    double* d_w7part = nullptr;   // fixed-order partial sums of W7 and H_X^T H_X
    // several scenes in one context (the grouped batch): per camera its scene,
    // per scene the offset and leading dimension of its Z, its first camera and
    // its point range; W7 holds 128 doubles per scene
    const int* d_cam_scene = nullptr;
    const int64_t* d_scene_zo = nullptr;
    const int64_t* d_scene_ld = nullptr;
    const int* d_scene_co = nullptr;
    const int* d_scene_po = nullptr;
    const int64_t* d_scene_wpo = nullptr;   // several scenes: prefix of their W7 warp counts
    int nscenes = 1, w7_wps = 0;            // one scene: its W7 warp count (w7_warps_for(m))
    int64_t w7_total = 0;                   // several scenes: all their W7 warps
    double* d_Z = nullptr;        // Np x Np row-major, lower triangle
    double* d_Gp = nullptr;       // N x 7: -W A^-1 H_X
    double* d_W7 = nullptr;       // 7 x 7
    double* d_HP = nullptr;       // n x 63
    // step (d)
    double* d_R = nullptr;        // Np x Np: triangular inverse workspace
    double* d_P = nullptr;        // Np x kNB panel copy
    double* d_Linv = nullptr;     // (Np / kNB) x kNB x kNB diagonal-block inverses
    double* d_F = nullptr;        // N x 7: G W7^-1
    double* d_G = nullptr;        // N x 7
    double* d_D = nullptr;        // Np Jacobi scale
    double* d_Sig = nullptr;      // n x 81 scaled, then unscaled blocks
    double* d_small = nullptr;    // 64: W7^-1 and scratch
    double* d_sgauge = nullptr;   // surrogate gauge rows: kSurrGaugeBlocks x 28 partial sums, then L_c (49)
    int* d_flag = nullptr;        // [0] error code, [1] detail
    int64_t bytes = 0;
    int64_t launches = 0;
    MixedState* mixed = nullptr;
    bool mixed_bad_launch = false;  // a GEMM launch was refused (odd tile count)
    bool capturing = false;         // launches are being captured into a graph: no timing events

    // a-posteriori error estimate (k_estimate.cu), allocated on first request
    bool est_on = false;
    int est_k = 0, est_cap = 0;
    void* d_Zkeep = nullptr;        // Np x Np: copy of the scaled matrix that is factorised
    void* d_estW = nullptr;         // Np x 9k each (double or double-single)
    void* d_estY = nullptr;
    void* d_estR = nullptr;
    int* d_est_idx = nullptr;       // sampled cameras
    double* d_est_dS = nullptr;     // k x 81 scaled error blocks
    double* d_est_out = nullptr;    // k x 3: relative, scaled-relative, camera

    // covariance after added observations (ccov_update.cu): set by a
    // successful ccov_covariance, cleared by anything that changes the scene
    bool cov_ready = false;
    bool upd_norm_ok = false;       // ||X||_inf and ||X||_1 of the current factor measured
    double upd_norm[2] = {0.0, 0.0};
    void* d_upd = nullptr;          // one workspace block, grown on demand
    size_t upd_bytes = 0;

    cudaEvent_t ev[8] = {};
    ccov_stats stats{};
    // profile = 1: event pairs around the dense trailing-update GEMMs
    std::vector<cudaEvent_t> prof_ev;
    size_t prof_used = 0;
    double prof_flops = 0.0;
};

// Bracket one GEMM launch with events when profiling (see ccov_options.profile).
void prof_begin(Ctx& c);
void prof_end(Ctx& c, double flops);

// ---- launchers (k_sparse.cu) ----
void launch_cam_prep(Ctx& c);
void launch_point_info(Ctx& c);
void launch_cam_info(Ctx& c);
void launch_schur(Ctx& c);
void launch_nullspace(Ctx& c, bool kept_jacobians);
int w7_warps_for(int64_t m);                      // warps of a scene's W7 partial sums (<= 2048)   // kept: step (a) ran on the current inputs

// ---- launchers (k_dense64.cu) ----
void launch_form_scaled(Ctx& c);           // G, W7^-1, F, D, Z_s = D (Z + F G^T) D
cudaError_t setup_dense64();               // function attributes (large shared memory)
void launch_potrf_diag(Ctx& c, int64_t k0);
void launch_gemm64(Ctx& c, bool nt, bool lower, int64_t M, int64_t N, int64_t K, double alpha,
                   const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                   double* C, int64_t ldc, int64_t row0, int64_t col0);
void launch_copy_panel(Ctx& c, int64_t k0);
void launch_init_identity(Ctx& c, double* X, int64_t ld);
void launch_trtri_row(Ctx& c, int64_t k0);
void launch_extract(Ctx& c);
void spd_factor_inverse64(Ctx& c);         // c.d_Z = L L^T, c.d_R = L^-1 (c.n = 0: no Gram blocks)
void launch_upd_obs(Ctx& c, int64_t k, const ccov_obs* add, const double* add_cov, int64_t ldphi, double* Jc,
                    double* Jp, double* JA, double* Psi, double* Phi);  // k_sparse.cu

// ---- surrogate features (k_surrogate.cu) ----
void surr_launch_features(Ctx& c, float* feat, double* scale);
constexpr int kSurrGaugeBlocks = 152;
constexpr int kGroupDigitK = 512;   // digit columns per row of the grouped batch's digit buffers
// Sub-panels per group of the mixed step (d): four (trailing updates with
// K = 512) for scenes of at least 64 sub-panels of 128 columns and at most
// five digits, else two (K = 256): below that size the in-group launches
// cost more than the longer K saves.  The single-scene path and the grouped
// batch take the same groups, so their results agree bit for bit.
constexpr int64_t kGroup4MinBlocks = 64;
inline int64_t mixed_group_max(int s, int64_t nb) { return s <= 5 && nb >= kGroup4MinBlocks ? 4 : 2; }
void surr_launch_gauge_rows(Ctx& c, const double* scale, double* q);

// ---- mixed path (k_mixed.cu) ----
cudaError_t mixed_alloc(Ctx& c);
void mixed_free(Ctx& c);
cudaError_t mixed_factor_inverse(Ctx& c);
const long long* mixed_inverse_factor(const Ctx& c);   // X = L^-1, Q42, after mixed_factor_inverse
// Y = X^T X V on the tensor cores with X of the last mixed step (d); V and Y
// Np x ld FP64 (ncols <= ld columns used).  With q = mixed_xtxv_ld(ncols):
// Vq / Wq / Yq int64 workspaces of Np x q, Sq q x q, ecol q ints, cmax q
// 64-bit words, norms 2 + 2 Np doubles.  Also Sq = -V'^T X^T X V' in Q(*FS)
// for the columns scaled to V' = V diag(2^-ecol).  The first call after a
// step (d) measures the norms of X and synchronises the stream once.
int64_t mixed_xtxv_ld(int64_t ncols);
cudaError_t mixed_xtxv(Ctx& c, int64_t ncols, const double* V, int64_t ld, double* Y, long long* Vq, long long* Wq,
                       long long* Yq, long long* Sq, int* ecol, unsigned long long* cmax, double* norms, int* FS);
// P = Y_s X_S^T for the update (after mixed_xtxv on the same columns): Yq and
// ecol from mixed_xtxv, X_S ldq x ldq FP64 with |X_S| <= 1; emax one int,
// XSq ldq x ldq and Pq Np x ldq int64 workspaces; P: N x ld FP64.
cudaError_t mixed_update_p(Ctx& c, int64_t ncols, const long long* Yq, const double* XS, const int* ecol,
                           int* emax, long long* XSq, long long* Pq, double* P, int64_t ld);
cudaError_t mixed_setup();                             // kernel attributes, SM count
bool mixed_make_c_map(CUtensorMap* map, long long* buf, int64_t rows, int64_t cols, int64_t ld);
bool mixed_make_b_map(CUtensorMap* map, __nv_bfloat16* buf, int s, int64_t Np);
int mixed_stages(int s);

// ---- grouped launches of the batched form (one launch per step for many
// scenes; parameter records and block prefixes in device memory) ----
int64_t grp_slice_rows_blocks(int K, int rows);
int64_t grp_slice_cols_blocks(int ncols);
int64_t grp_gram_blocks(int64_t ncols);
void grp_slice_rows(cudaStream_t st, int K, const SliceRowsP* P, const int64_t* pre, int k, int64_t blocks, int* flag);
void grp_slice_cols(cudaStream_t st, int K, const SliceColsP* P, const int64_t* pre, int k, int64_t blocks, int* flag);
void grp_potrf(cudaStream_t st, const PotrfP* P, int k, int* flag);
void grp_gram(cudaStream_t st, const GramP* P, const int64_t* pre, int k, int64_t blocks);
void grp_zscale(cudaStream_t st, const ZscaleP* P, const int64_t* pre, int k, int64_t blocks, int* flag);
void grp_identity(cudaStream_t st, const IdentP* P, const int64_t* pre, int k, int64_t blocks);
cudaError_t grp_gemm(cudaStream_t st, int s, int K, const GemmProblem* probs, int nprobs, int64_t total_pairs,
                     int* flag, int max_ctas, int stages);
int64_t mixed_tile_pairs(int M, int N, int lower);   // tile pairs of one GEMM (M, N multiples of 128)
void launch_g(Ctx& c);                               // G = G_part + H_P
ccov_status device_status(Ctx& c, const char* where);  // wait for the stream, map the device flag
void grp_gauge(cudaStream_t st, const GaugeP* P, int k, int* flag);
void grp_fd(cudaStream_t st, const FdP* P, const int64_t* pre, int k, int64_t blocks, int* flag);
void grp_extract(cudaStream_t st, const ExtractP* P, const int64_t* pre, int k, int64_t blocks);

// ---- a-posteriori error estimate (k_estimate.cu) ----
cudaError_t est_alloc(Ctx& c, int k);
void est_free(Ctx& c);
void est_keep_fp64(Ctx& c);                  // after the FP64 scaling: keep Z_s
void est_launch(Ctx& c, const long long* Xq);  // after the inverse, before the extraction
void est_launch_final(Ctx& c);               // after the extraction
// Y = X^T (X V) for g groups of nine columns (Np x 9g FP64, device), X the
// inverse factor of the last step (d); s0..s2 scratch of 8 Np 9g bytes each
void est_xtxv(Ctx& c, int g, const double* V, double* Y, void* s0, void* s1, void* s2);

// ---- covariance after added observations (ccov_update.cu) ----
constexpr int64_t kUpdMaxObs = 4096;
cudaError_t update_enqueue(Ctx& c, const ccov_obs* add, int64_t k, const double* add_cov, double* out,
                           int out_memory);
void update_free(Ctx& c);

// ---- the batched form as grouped launches (ccov_group.cu) ----
struct GroupPlan;
bool group_eligible(Ctx* const* ctxs, int k);
cudaError_t group_create(Ctx* const* ctxs, double* const* outs, int k, GroupPlan** out);
cudaError_t group_enqueue(GroupPlan& P, cudaStream_t main);
cudaError_t group_autotune(GroupPlan& P, cudaStream_t st, int reps, float* best_ms);
ccov_status group_status(GroupPlan& P, cudaStream_t st, const char* where);
void group_free(GroupPlan* P);
int64_t group_launches(const GroupPlan& P);
void group_shape(const GroupPlan& P, int* cap, int* stages);

}  // namespace ccov

#define CCOV_LAUNCH_CHECK(c) do { (c).launches++; } while (0)

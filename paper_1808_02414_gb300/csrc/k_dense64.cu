// Step (d) in FP64.  The camera block of Z_p^-1 (Sec. 4.2, Eq.
// block-inversion-Qp) is reached through the gauge-regularised camera matrix
// Z' = Z + G (Lambda^-1 + W7)^-1 G^T and Sigma_P = Z'^-1 - H_P C H_P^T (see
// gauge_kernel); Lambda -> infinity is the plain block inversion
// (Z + G W7^-1 G^T)^-1, which is far worse conditioned.  Z' is SPD; it is
// Jacobi-scaled (the conditioning of Sec. 4.2), factorised by a blocked
// right-looking Cholesky, inverted as a lower-triangular matrix X = L^-1 by a
// blocked right-looking substitution, and the 9x9 diagonal blocks of
// Z'^-1 = X^T X are accumulated from the rows of X as they are finished.
// Every trailing update is a rank-128 GEMM; in this FP64 path it runs on the
// FP64 pipe (the mixed path replaces it by tensor-core GEMMs).
#include "ccov_internal.cuh"
#include "group.cuh"

namespace ccov {
namespace {

__device__ __forceinline__ void set_flag(int* flag, int code, int detail) {
    if (atomicMax(flag, code) < code) flag[1] = detail;
}

// Symmetric 7x7 inverse: Jacobi-scaled Gauss-Jordan with partial pivoting.
// Returns false if a pivot vanishes.
__device__ bool inv7(const double* Ain, double* Aout) {
    double a[7][14];
    double s[7];
    for (int p = 0; p < 7; ++p) {
        if (!(Ain[7 * p + p] > 0.0)) return false;
        s[p] = 1.0 / sqrt(Ain[7 * p + p]);
    }
    for (int p = 0; p < 7; ++p)
        for (int q = 0; q < 7; ++q) {
            a[p][q] = Ain[7 * p + q] * s[p] * s[q];
            a[p][7 + q] = (p == q) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 7; ++col) {
        int piv = col;
        for (int r = col + 1; r < 7; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (!(fabs(a[piv][col]) > 1e-300)) return false;
        if (piv != col)
            for (int q = 0; q < 14; ++q) { double t = a[col][q]; a[col][q] = a[piv][q]; a[piv][q] = t; }
        double inv = 1.0 / a[col][col];
        for (int q = 0; q < 14; ++q) a[col][q] *= inv;
        for (int r = 0; r < 7; ++r) {
            if (r == col) continue;
            double f = a[r][col];
            for (int q = 0; q < 14; ++q) a[r][q] -= f * a[col][q];
        }
    }
    for (int p = 0; p < 7; ++p)
        for (int q = 0; q < 7; ++q) Aout[7 * p + q] = s[p] * a[p][7 + q] * s[q];
    return true;
}

// G = G_part + H_P (the border column block of Z_p); Gp null: G = H_P.
__global__ void g_kernel(int64_t N, const double* __restrict__ Gp, const double* __restrict__ HP,
                         double* __restrict__ G) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < 7 * N) G[e] = (Gp ? Gp[e] : 0.0) + HP[e];
}

// Gauge weight and the 7x7 matrices of the regularised route.  With span H =
// null M and any SPD Lambda, (M + H Lambda H^T)^-1 = M^+ + H (H^T H)^-1
// Lambda^-1 (H^T H)^-1 H^T; eliminating the points of M + H Lambda H^T gives
// the camera matrix Z' = Z + G (Lambda^-1 + W7)^-1 G^T, so
// Sigma_P = Z'^-1 - H_P C H_P^T with C = (H^T H)^-1 Lambda^-1 (H^T H)^-1.
// Lambda = alpha diag(1 / |D_z G_q|^2), D_z = diag(Z)^-1/2, keeps the gauge
// directions of Z' at the scale of the rest after Jacobi scaling.
// One CTA of 256 threads.  Output (small): K = (Lambda^-1 + W7)^-1 at [0, 49),
// C at [49, 98).  W7 (upper) at W7s[0, 49), H_X^T H_X (upper) at W7s[49, 98).
constexpr double kGaugeAlpha = 1e-2;
// gauge: CCOV_GAUGE_NATURAL as above; CCOV_GAUGE_ZPINV (Alg. 4) with G = H_P,
// W7 = 0 and H^T H = H_P^T H_P, the same identity for Z, whose nullspace is
// span(H_P): (Z + H_P Lambda H_P^T)^-1 = Z+ + H_P (H_P^T H_P)^-1 Lambda^-1
// (H_P^T H_P)^-1 H_P^T; CCOV_GAUGE_FIXED3 (Alg. 5): Z is of full rank, K = C = 0.
__device__ __forceinline__ void gauge_body(int64_t N, const double* __restrict__ G, const double* __restrict__ HP,
                                           const double* __restrict__ Z, int64_t ldz, const double* __restrict__ W7s,
                                           double* __restrict__ small, int* flag, int gauge) {
    if (gauge == CCOV_GAUGE_FIXED3) {
        for (int e = threadIdx.x; e < 98; e += blockDim.x) small[e] = 0.0;
        return;
    }
    __shared__ double red[35][33];
    double acc[35];
#pragma unroll
    for (int e = 0; e < 35; ++e) acc[e] = 0.0;
    for (int64_t r = threadIdx.x; r < N; r += blockDim.x) {
        double dz = 1.0 / Z[r * ldz + r];
        const double* g = G + 7 * r;
        const double* h = HP + 7 * r;
#pragma unroll
        for (int q = 0; q < 7; ++q) acc[q] += g[q] * g[q] * dz;
        int e = 7;
#pragma unroll
        for (int p = 0; p < 7; ++p)
#pragma unroll
            for (int q = p; q < 7; ++q, ++e) acc[e] += h[p] * h[q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < 35; ++e) {
        double v = acc[e];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[e][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot[35];
    for (int e = 0; e < 35; ++e) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[e][w];
        tot[e] = v;
    }
    double lam_inv[7], M7[49], HtH[49], K[49], HtHi[49];
    for (int q = 0; q < 7; ++q) lam_inv[q] = tot[q] / kGaugeAlpha;
    int e = 7;
    for (int p = 0; p < 7; ++p)
        for (int q = p; q < 7; ++q, ++e) {
            double hh = tot[e] + (gauge == CCOV_GAUGE_ZPINV ? 0.0 : W7s[49 + 7 * p + q]);
            HtH[7 * p + q] = hh; HtH[7 * q + p] = hh;
            double w = gauge == CCOV_GAUGE_ZPINV ? 0.0 : W7s[7 * p + q];
            M7[7 * p + q] = w; M7[7 * q + p] = w;
        }
    for (int q = 0; q < 7; ++q) M7[8 * q] += lam_inv[q];
    if (!inv7(M7, K) || !inv7(HtH, HtHi)) { set_flag(flag, DEV_SINGULAR_W7, 0); return; }
    for (int p = 0; p < 49; ++p) small[p] = K[p];
    for (int p = 0; p < 7; ++p)
        for (int q = 0; q < 7; ++q) {
            double v = 0.0;
            for (int k = 0; k < 7; ++k) v += HtHi[7 * p + k] * lam_inv[k] * HtHi[7 * k + q];
            small[49 + 7 * p + q] = v;
        }
}

__global__ void __launch_bounds__(256)
gauge_kernel(int64_t N, const double* __restrict__ G, const double* __restrict__ HP,
             const double* __restrict__ Z, int64_t ldz, const double* __restrict__ W7s,
             double* __restrict__ small, int* flag, int gauge) {
    gauge_body(N, G, HP, Z, ldz, W7s, small, flag, gauge);
}

// F = G K, D_r = (Z_rr + F_r . G_r)^-1/2 (row r of Z').
__device__ __forceinline__ void fd_body(int64_t N, int64_t Np, const double* __restrict__ K,
                                        const double* __restrict__ Z, const double* __restrict__ G,
                                        double* __restrict__ F, double* __restrict__ D, int* flag, int64_t r) {
    if (r >= Np) return;
    if (r >= N) { D[r] = 1.0; return; }
    const double* g = G + 7 * r;
    double d = Z[r * Np + r];
    for (int q = 0; q < 7; ++q) {
        double v = 0.0;
        for (int p = 0; p < 7; ++p) v += g[p] * K[7 * p + q];
        F[7 * r + q] = v;
        d += v * g[q];
    }
    if (!(d > 0.0)) { set_flag(flag, DEV_NOT_SPD, (int)r); d = 1.0; }
    D[r] = 1.0 / sqrt(d);
}

__global__ void fd_kernel(int64_t N, int64_t Np, const double* __restrict__ K,
                          const double* __restrict__ Z, const double* __restrict__ G,
                          double* __restrict__ F, double* __restrict__ D, int* flag) {
    fd_body(N, Np, K, Z, G, F, D, flag, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// Lower triangle of Z_s = D (Z + F G^T) D in place; padded rows/columns get
// the identity.  One thread per element of a 32 x 32 tile.
__global__ void zscale_kernel(int64_t N, int64_t Np, double* __restrict__ Z,
                              const double* __restrict__ F, const double* __restrict__ G,
                              const double* __restrict__ D) {
    int64_t bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    int64_t i = bi * 32 + threadIdx.y, j = bj * 32 + threadIdx.x;
    if (i >= Np || j > i) return;
    double* z = Z + i * Np + j;
    if (i >= N || j >= N) { *z = (i == j) ? 1.0 : 0.0; return; }
    double v = *z;
    const double* fi = F + 7 * i;
    const double* gj = G + 7 * j;
#pragma unroll
    for (int q = 0; q < 7; ++q) v += fi[q] * gj[q];
    *z = D[i] * v * D[j];
}

// Cholesky of the 128 x 128 diagonal block at (k0, k0) in shared memory
// (packed lower triangle), written back in place, and its inverse Linv
// (full 128 x 128, zero above the diagonal).
constexpr int kPD = kNB;
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void __launch_bounds__(512)
potrf_diag_kernel(double* __restrict__ Z, int64_t ld, int64_t k0, double* __restrict__ Linv,
                  int* flag) {
    extern __shared__ __align__(16) double sh[];
    double* S = sh;                         // packed L
    double* Xs = sh + kPD * (kPD + 1) / 2;  // packed inverse
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int e = tid; e < kPD * kPD; e += nt) {
        int i = e / kPD, j = e % kPD;
        if (j <= i) S[pk(i, j)] = Z[(k0 + i) * ld + k0 + j];
    }
    __syncthreads();
    for (int j = 0; j < kPD; ++j) {
        if (tid == 0) {
            double d = S[pk(j, j)];
            if (!(d > 0.0)) { set_flag(flag, DEV_NOT_SPD, (int)(k0 + j)); d = 1.0; }
            S[pk(j, j)] = sqrt(d);
        }
        __syncthreads();
        double inv = 1.0 / S[pk(j, j)];
        for (int i = j + 1 + tid; i < kPD; i += nt) S[pk(i, j)] *= inv;
        __syncthreads();
        for (int i = j + 1 + warp; i < kPD; i += nw) {
            double lij = S[pk(i, j)];
            for (int l = j + 1 + lane; l <= i; l += 32) S[pk(i, l)] -= lij * S[pk(l, j)];
        }
        __syncthreads();
    }
    for (int e = tid; e < kPD * kPD; e += nt) {
        int i = e / kPD, j = e % kPD;
        if (j <= i) Z[(k0 + i) * ld + k0 + j] = S[pk(i, j)];
    }
    // inverse: column c by forward substitution, one thread per column
    if (tid < kPD) {
        const int c = tid;
        Xs[pk(c, c)] = 1.0 / S[pk(c, c)];
        for (int i = c + 1; i < kPD; ++i) {
            double s = 0.0;
            for (int k = c; k < i; ++k) s += S[pk(i, k)] * Xs[pk(k, c)];
            Xs[pk(i, c)] = -s / S[pk(i, i)];
        }
    }
    __syncthreads();
    for (int e = tid; e < kPD * kPD; e += nt) {
        int i = e / kPD, j = e % kPD;
        Linv[e] = (j <= i) ? Xs[pk(i, j)] : 0.0;
    }
}

// C[M x N] = beta C + alpha A[M x K] op(B); op(B) = Bt^T for NT (B given as
// N x K row-major) or B (K x N row-major) for NN.  With `lower`, tiles whose
// first column lies right of their last row (relative to row0, col0) are
// skipped.  64 x 64 tile, K step 16, 256 threads of 4 x 4.
template <bool NT>
__global__ void __launch_bounds__(256)
gemm64_kernel(int64_t M, int64_t N, int64_t K, double alpha, const double* __restrict__ A,
              int64_t lda, const double* __restrict__ B, int64_t ldb, double beta,
              double* __restrict__ C, int64_t ldc, int lower, int64_t row0, int64_t col0) {
    const int64_t bm = blockIdx.y * 64, bn = blockIdx.x * 64;
    if (lower && (col0 + bn) > (row0 + bm + 63)) return;
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int e = tid + 256 * s;        // 0..1023
            int r = e / 16, kk = e % 16;  // A tile: row r, k kk
            int64_t gr = bm + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : 0.0;
            if (NT) {
                int64_t gc = bn + r;
                Bs[kk][r] = (gc < N && gk < K) ? B[gc * ldb + gk] : 0.0;
            } else {
                int kb = e / 64, c = e % 64;
                int64_t gk2 = k0 + kb, gc = bn + c;
                Bs[kb][c] = (gc < N && gk2 < K) ? B[gk2 * ldb + gc] : 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int64_t gr = bm + ty * 4 + u;
        if (gr >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int64_t gc = bn + tx * 4 + v;
            if (gc >= N) continue;
            double* c = C + gr * ldc + gc;
            *c = (beta == 0.0 ? 0.0 : beta * *c) + alpha * acc[u][v];
        }
    }
}

__global__ void copy_panel_kernel(int64_t rows, const double* __restrict__ src, int64_t ld,
                                  double* __restrict__ dst) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * kNB) return;
    int64_t r = e / kNB, c = e % kNB;
    dst[e] = src[r * ld + c];
}

__global__ void identity_diag_kernel(int64_t Np, double* X, int64_t ld) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < Np) X[i * ld + i] = 1.0;
}

// Row block k of X = L^-1: X[k, cols] = Linv_k R[k, cols] in place, then the
// camera Gram blocks Sig_c += X[k, c]^T X[k, c] of the 8 cameras whose 72
// columns this CTA owns.  288 threads: column c = tid % 72, rows rg + 4 s.
constexpr int kCW = 72;
__global__ void __launch_bounds__(288)
trtri_row_kernel(int64_t n, int64_t Np, int64_t k0, int64_t ncols, double* __restrict__ R,
                 const double* __restrict__ Linv, double* __restrict__ Sig) {
    extern __shared__ __align__(16) double sh[];
    double* T = sh;                    // 128 x 72
    double* Ls = sh + kNB * kCW;       // 128 x 128
    const int tid = threadIdx.x;
    const int64_t c0 = blockIdx.x * (int64_t)kCW;
    for (int e = tid; e < kNB * kNB; e += 288) Ls[e] = Linv[e];
    for (int e = tid; e < kNB * kCW; e += 288) {
        int r = e / kCW, c = e % kCW;
        int64_t gc = c0 + c;
        T[e] = (gc < ncols) ? R[(k0 + r) * Np + gc] : 0.0;
    }
    __syncthreads();
    const int c = tid % kCW, rg = tid / kCW;
    double out[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        int i = rg + 4 * s;
        double v = 0.0;
        for (int k = 0; k <= i; ++k) v += Ls[i * kNB + k] * T[k * kCW + c];
        out[s] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        int i = rg + 4 * s;
        T[i * kCW + c] = out[s];
        int64_t gc = c0 + c;
        if (gc < ncols) R[(k0 + i) * Np + gc] = out[s];
    }
    __syncthreads();
    for (int e = tid; e < 8 * 81; e += 288) {
        int g = e / 81, ab = e % 81, a = ab / 9, b = ab % 9;
        int64_t cam = (c0 / 9) + g;
        if (cam >= n || c0 + 9 * g >= ncols) continue;
        double v = 0.0;
        for (int r = 0; r < kNB; ++r) v += T[r * kCW + 9 * g + a] * T[r * kCW + 9 * g + b];
        Sig[81 * cam + ab] += v;
    }
}

// Sigma_c = D_c S_c D_c - H_Pc C H_Pc^T for camera c.
__device__ __forceinline__ void extract_body(int64_t n, const double* __restrict__ D, const double* __restrict__ HP,
                                             const double* __restrict__ Cg, double* __restrict__ Sig, int64_t e) {
    if (e >= n * 81) return;
    int64_t cam = e / 81;
    int ab = (int)(e % 81), a = ab / 9, b = ab % 9;
    const double* ha = HP + 63 * cam + 7 * a;
    const double* hb = HP + 63 * cam + 7 * b;
    double g = 0.0;
    for (int p = 0; p < 7; ++p) {
        double v = 0.0;
        for (int q = 0; q < 7; ++q) v += Cg[7 * p + q] * hb[q];
        g += ha[p] * v;
    }
    Sig[e] = Sig[e] * D[9 * cam + a] * D[9 * cam + b] - g;
}

__global__ void extract_kernel(int64_t n, const double* __restrict__ D, const double* __restrict__ HP,
                               const double* __restrict__ Cg, double* __restrict__ Sig) {
    extract_body(n, D, HP, Cg, Sig, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

// ---- grouped forms: the same step of many scenes in one launch ----
__global__ void __launch_bounds__(256) gauge_grouped(const GaugeP* __restrict__ P, int* flag) {
    const GaugeP& a = P[blockIdx.x];
    gauge_body(a.N, a.G, a.HP, a.Z, a.ldz, a.W7s, a.small, flag, CCOV_GAUGE_NATURAL);
}

__global__ void fd_grouped(const FdP* __restrict__ P, const int64_t* __restrict__ pre, int k, int* flag) {
    const int q = find_group(pre, k, blockIdx.x);
    const FdP& a = P[q];
    fd_body(a.N, a.Np, a.K, a.Z, a.G, a.F, a.D, flag, (blockIdx.x - pre[q]) * (int64_t)blockDim.x + threadIdx.x);
}

__global__ void extract_grouped(const ExtractP* __restrict__ P, const int64_t* __restrict__ pre, int k) {
    const int q = find_group(pre, k, blockIdx.x);
    const ExtractP& a = P[q];
    extract_body(a.n, a.D, a.HP, a.Cg, a.Sig, (blockIdx.x - pre[q]) * (int64_t)blockDim.x + threadIdx.x);
}

}  // namespace

cudaError_t setup_dense64() {
    cudaError_t e = cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * kPD * (kPD + 1)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(trtri_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * (kNB * kCW + kNB * kNB)));
}

void launch_g(Ctx& c) {
    g_kernel<<<(int)((7 * c.N + 255) / 256), 256, 0, c.stream>>>(c.N, c.d_Gp, c.d_HP, c.d_G);
    c.launches++;
}

void launch_form_scaled(Ctx& c) {
    g_kernel<<<(int)((7 * c.N + 255) / 256), 256, 0, c.stream>>>(
        c.N, c.opt.gauge == CCOV_GAUGE_ZPINV ? nullptr : c.d_Gp, c.d_HP, c.d_G);
    gauge_kernel<<<1, 256, 0, c.stream>>>(c.N, c.d_G, c.d_HP, c.d_Z, c.Np, c.d_W7, c.d_small, c.d_flag,
                                          c.opt.gauge);
    fd_kernel<<<(int)((c.Np + 255) / 256), 256, 0, c.stream>>>(c.N, c.Np, c.d_small, c.d_Z, c.d_G, c.d_F,
                                                                c.d_D, c.d_flag);
    c.launches += 3;
    if (c.opt.precision == CCOV_PREC_FP64) {
        // the mixed path writes Z_s as fixed point itself
        int64_t nt = (c.Np + 31) / 32;
        zscale_kernel<<<dim3((unsigned)nt, (unsigned)nt), dim3(32, 32), 0, c.stream>>>(c.N, c.Np, c.d_Z,
                                                                                      c.d_F, c.d_G, c.d_D);
        c.launches++;
    }
}

// Blocked Cholesky c.d_Z = L L^T (lower triangle, c.Np a multiple of kNB) and
// X = L^-1 into c.d_R: the FP64 path's steps on a plain SPD matrix, without
// the camera Gram blocks (c.n = 0).  Stream-ordered, no synchronisation.
void spd_factor_inverse64(Ctx& c) {
    const int64_t Np = c.Np, nb = Np / kNB;
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB;
        launch_potrf_diag(c, k0);
        if (rem > 0) {
            launch_copy_panel(c, k0);
            launch_gemm64(c, true, false, rem, kNB, kNB, 1.0, c.d_P, kNB, c.d_Linv + kb * kNB * kNB, kNB, 0.0,
                          c.d_Z + (k0 + kNB) * Np + k0, Np, 0, 0);
            const double* L21 = c.d_Z + (k0 + kNB) * Np + k0;
            launch_gemm64(c, true, true, rem, rem, kNB, -1.0, L21, Np, L21, Np, 1.0,
                          c.d_Z + (k0 + kNB) * Np + k0 + kNB, Np, 0, 0);
        }
    }
    cudaMemsetAsync(c.d_R, 0, sizeof(double) * Np * Np, c.stream);
    launch_init_identity(c, c.d_R, Np);
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB;
        launch_trtri_row(c, k0);
        if (rem > 0)
            launch_gemm64(c, false, false, rem, k0 + kNB, kNB, -1.0, c.d_Z + (k0 + kNB) * Np + k0, Np,
                          c.d_R + k0 * Np, Np, 1.0, c.d_R + (k0 + kNB) * Np, Np, 0, 0);
    }
}

void launch_potrf_diag(Ctx& c, int64_t k0) {
    potrf_diag_kernel<<<1, 512, sizeof(double) * kPD * (kPD + 1), c.stream>>>(
        c.d_Z, c.Np, k0, c.d_Linv + (k0 / kNB) * kNB * kNB, c.d_flag);
    c.launches++;
}

void launch_gemm64(Ctx& c, bool nt, bool lower, int64_t M, int64_t N, int64_t K, double alpha,
                   const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                   double* C, int64_t ldc, int64_t row0, int64_t col0) {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    if (nt)
        gemm64_kernel<true><<<grid, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                        lower ? 1 : 0, row0, col0);
    else
        gemm64_kernel<false><<<grid, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                         lower ? 1 : 0, row0, col0);
    c.launches++;
}

void launch_copy_panel(Ctx& c, int64_t k0) {
    int64_t rows = c.Np - k0 - kNB;
    copy_panel_kernel<<<(int)((rows * kNB + 255) / 256), 256, 0, c.stream>>>(
        rows, c.d_Z + (k0 + kNB) * c.Np + k0, c.Np, c.d_P);
    c.launches++;
}

void launch_init_identity(Ctx& c, double* X, int64_t ld) {
    identity_diag_kernel<<<(int)((c.Np + 255) / 256), 256, 0, c.stream>>>(c.Np, X, ld);
    c.launches++;
}

void launch_trtri_row(Ctx& c, int64_t k0) {
    int64_t ncols = k0 + kNB;
    int grid = (int)((ncols + kCW - 1) / kCW);
    trtri_row_kernel<<<grid, 288, sizeof(double) * (kNB * kCW + kNB * kNB), c.stream>>>(
        c.n, c.Np, k0, ncols, c.d_R, c.d_Linv + (k0 / kNB) * kNB * kNB, c.d_Sig);
    c.launches++;
}

void grp_gauge(cudaStream_t st, const GaugeP* P, int k, int* flag) { gauge_grouped<<<k, 256, 0, st>>>(P, flag); }

void grp_fd(cudaStream_t st, const FdP* P, const int64_t* pre, int k, int64_t blocks, int* flag) {
    fd_grouped<<<(unsigned)blocks, 256, 0, st>>>(P, pre, k, flag);
}

void grp_extract(cudaStream_t st, const ExtractP* P, const int64_t* pre, int k, int64_t blocks) {
    extract_grouped<<<(unsigned)blocks, 256, 0, st>>>(P, pre, k);
}

void launch_extract(Ctx& c) {
    extract_kernel<<<(int)((c.n * 81 + 255) / 256), 256, 0, c.stream>>>(c.n, c.d_D, c.d_HP, c.d_small + 49,
                                                                      c.d_Sig);
    c.launches++;
}

}  // namespace ccov

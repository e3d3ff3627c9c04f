// Camera covariances after adding observations, by the Woodbury identity
// (Sec. 5: M_{i+1} = M_i + M_Delta), from the factorisation that the last
// step (d) left behind, without a new factorisation.
//
// Step (d) factorised D Z' D = L L^T and kept X = L^-1, where Z' = Z + G K G^T
// is the reduced camera matrix of the regularised M' = M + H Lambda H^T
// (K = (Lambda^-1 + W7)^-1), and returned Sigma = Z'^-1 - H_P C H_P^T.
// Added observations with whitened Jacobian J (2k rows, J = [J_P, J_X]) give
// M'_new = M' + J^T J.  The projections do not change under the similarity
// (J H = 0), so H stays the nullspace of M_new, Lambda may stay as it was,
// and the gauge term H_P C H_P^T is the same as before.  Woodbury on the
// whole of M' then gives, on the camera blocks,
//   Sigma_new = Sigma - Y S^-1 Y^T,
//   Vt  = J_P^T - B' A'^-1 J_X^T = J_P^T - M_PX A^-1 J_X^T - G Phi,
//   Phi = K Psi^T,  Psi = J_X A^-1 H_X,
//   Y   = Z'^-1 Vt = D X^T X D Vt,
//   S   = I + J_X A'^-1 J_X^T + Vt^T Y,
//   J_X A'^-1 J_X^T = J_X A^-1 J_X^T - Psi K Psi^T,
// with B' = M'_PX and A' = M'_XX = A + H_X Lambda H_X^T, whose inverse is
// taken by Woodbury on its rank-7 term (B' A'^-1 = M_PX A^-1 + G K H_X^T A^-1).
// The paper writes the identity on the Schur complement (Z_{i+1} = Z_i +
// Z_Delta); taking it on M' is the same update with the change of the point
// blocks A included, and its rank is 2k, however many cameras see the
// points of the added observations.
//
// Cost: the two triangular products of X with the 2k columns of Vt, O(N^2 k),
// and O(N k^2 + k^3) for S, against O(N^3) for a new step (d).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ccov_internal.cuh"

namespace ccov {
namespace {

constexpr int64_t kAlign = 256;

int64_t up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Vt columns 2o, 2o + 1 of added observation o (thread per o, so that every
// column has one writer): + Jc^T on the rows of its camera, and on the rows
// of every camera i that already observes its point j, -W_ij A_j^-1 Jp^T
// (the stored V_o' = W_o' A_j^-1 of that observation o').
__global__ void upd_scatter_kernel(int64_t k, const ccov_obs* __restrict__ add, const int* __restrict__ pt_ptr,
                                   const ccov_obs* __restrict__ obs, const double* __restrict__ V,
                                   const double* __restrict__ Jc, const double* __restrict__ Jp, int64_t ld,
                                   double* __restrict__ Vt) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= k) return;
    const int cam = add[o].cam, pt = add[o].pt;
    for (int row = 0; row < 2; ++row) {
        const int64_t col = 2 * o + row;
        const double* jc = Jc + 18 * o + 9 * row;
        const double* jp = Jp + 6 * o + 3 * row;
        for (int a = 0; a < 9; ++a) Vt[(9 * (int64_t)cam + a) * ld + col] += jc[a];
        for (int q = pt_ptr[pt]; q < pt_ptr[pt + 1]; ++q) {
            const int64_t i = obs[q].cam;
            const double* v = V + 27 * (int64_t)q;
            for (int a = 0; a < 9; ++a)
                Vt[(9 * i + a) * ld + col] -= v[3 * a] * jp[0] + v[3 * a + 1] * jp[1] + v[3 * a + 2] * jp[2];
        }
    }
}

// Vt <- D (Vt - G Phi) on the first N rows and 2k columns, zero elsewhere.
__global__ void upd_dense_kernel(int64_t N, int64_t Np, int64_t ld, int64_t r, const double* __restrict__ G,
                                 const double* __restrict__ Phi, const double* __restrict__ D,
                                 double* __restrict__ Vt) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= Np * ld) return;
    const int64_t row = e / ld, col = e % ld;
    if (row >= N || col >= r) { Vt[e] = 0.0; return; }
    double v = Vt[e];
    const double* g = G + 7 * row;
#pragma unroll
    for (int q = 0; q < 7; ++q) v -= g[q] * Phi[q * ld + col];
    Vt[e] = D[row] * v;
}

// Split-K partial products part[z] = A[rows of chunk z]^T B[rows of chunk z]
// for A, B of `rows` x ld (row-major): a 32 x 32 tile of the ld x ld result
// per CTA, 256 threads of four entries each.
__global__ void __launch_bounds__(256)
upd_atb_kernel(int64_t rows, int64_t ld, int64_t chunk, const double* __restrict__ A,
               const double* __restrict__ B, double* __restrict__ part) {
    __shared__ double As[32][33];
    __shared__ double Bs[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t a0 = blockIdx.y * 32, b0 = blockIdx.x * 32, z = blockIdx.z;
    const int64_t r0 = z * chunk, r1 = std::min(rows, r0 + chunk);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t rb = r0; rb < r1; rb += 32) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int rr = ty + 8 * s;
            const int64_t gr = rb + rr;
            As[rr][tx] = (gr < r1 && a0 + tx < ld) ? A[gr * ld + a0 + tx] : 0.0;
            Bs[rr][tx] = (gr < r1 && b0 + tx < ld) ? B[gr * ld + b0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const double b = Bs[kk][tx];
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[s] += As[kk][ty + 8 * s] * b;
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t a = a0 + ty + 8 * s, b = b0 + tx;
        if (a < ld && b < ld) part[(z * ld + a) * ld + b] = acc[s];
    }
}

// S (rp x rp): I + J_X A^-1 J_X^T (observations of one point) - Psi K Psi^T
// + Vt^T Y on the 2k x 2k block, the identity elsewhere.  Vt^T Y is either
// the split-K partials summed in order, or (Sq not null, the tensor-core
// form) -Sq[a][b] 2^(e_a + e_b - FS).  Column a is row a & 1 of added
// observation a >> 1.
__global__ void upd_s_kernel(int64_t r, int64_t ld, int64_t rp, int nsplit, const double* __restrict__ part,
                             const long long* __restrict__ Sq, int64_t ldq, const int* __restrict__ ecol, int FS,
                             const ccov_obs* __restrict__ add, const double* __restrict__ JA,
                             const double* __restrict__ Jp, const double* __restrict__ Psi,
                             const double* __restrict__ K, double* __restrict__ S) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rp * rp) return;
    const int64_t a = e / rp, b = e % rp;
    if (a >= r || b >= r) { S[e] = (a == b) ? 1.0 : 0.0; return; }
    double v = 0.0;
    if (Sq)
        v = -ldexp((double)Sq[a * ldq + b], ecol[a] + ecol[b] - FS);
    else
        for (int z = 0; z < nsplit; ++z) v += part[((int64_t)z * ld + a) * ld + b];
    if (a == b) v += 1.0;
    const int64_t oa = a >> 1, ob = b >> 1;
    const int ra = (int)(a & 1), rb = (int)(b & 1);
    if (add[oa].pt == add[ob].pt) {
        const double* x = JA + 6 * oa + 3 * ra;
        const double* y = Jp + 6 * ob + 3 * rb;
        v += x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
    }
    const double* pa = Psi + 14 * oa + 7 * ra;
    const double* pb = Psi + 14 * ob + 7 * rb;
    for (int p = 0; p < 7; ++p) {
        double w = 0.0;
        for (int q = 0; q < 7; ++q) w += K[7 * p + q] * pb[q];
        v -= pa[p] * w;
    }
    S[e] = v;
}

// out_i = Sigma_i - D_i (P_i P_i^T) D_i, P = Y_s X_S^T (rows 9i .. 9i + 8 of
// camera i, `r` columns): CTA per camera, columns staged 256 at a time.
__global__ void __launch_bounds__(128)
upd_diag_kernel(int64_t ld, int64_t r, const double* __restrict__ P, const double* __restrict__ D,
                const double* __restrict__ Sig, double* __restrict__ out) {
    __shared__ double T[9][257];
    const int64_t i = blockIdx.x;
    const int tid = threadIdx.x, a = tid / 9, b = tid % 9;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < r; j0 += 256) {
        for (int q = tid; q < 9 * 256; q += 128) {
            const int row = q / 256, jj = q % 256;
            T[row][jj] = (j0 + jj < r) ? P[(9 * i + row) * ld + j0 + jj] : 0.0;
        }
        __syncthreads();
        if (tid < 81)
            for (int jj = 0; jj < 256; ++jj) acc += T[a][jj] * T[b][jj];
        __syncthreads();
    }
    if (tid < 81) out[81 * i + tid] = Sig[81 * i + tid] - D[9 * i + a] * D[9 * i + b] * acc;
}

struct Layout {
    int64_t r = 0, g = 0, ld = 0, rp = 0, nsplit = 1, chunk = 0;
    int64_t ldq = 0;   // columns of the scratch blocks (the tensor-core products pad to 128)
    size_t add = 0, cov = 0, Jc = 0, Jp = 0, JA = 0, Psi = 0, Phi = 0, Vt = 0, Ys = 0, s0 = 0, s1 = 0, s2 = 0,
           S = 0, RS = 0, PS = 0, LS = 0, part = 0, out = 0, ecol = 0, norms = 0, Sq = 0, cmax = 0, emax = 0,
           total = 0;
};

Layout layout(const Ctx& c, int64_t k) {
    Layout L;
    L.r = 2 * k;
    L.g = (L.r + 8) / 9;
    L.ld = 9 * L.g;
    L.rp = up(L.ld, kNB);
    const int64_t tiles = ((L.ld + 31) / 32) * ((L.ld + 31) / 32);
    L.nsplit = std::max<int64_t>(1, std::min<int64_t>(64, (4 * 152 + tiles - 1) / tiles));
    L.chunk = up((c.N + L.nsplit - 1) / L.nsplit, 32);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += up((int64_t)bytes, kAlign); return o; };
    L.ldq = mixed_xtxv_ld(L.ld);
    const size_t d = sizeof(double), thin = d * (size_t)c.Np * L.ld, wide = d * (size_t)c.Np * L.ldq;
    L.add = take(sizeof(ccov_obs) * k);
    L.cov = take(d * 4 * k);
    L.Jc = take(d * 18 * k);
    L.Jp = take(d * 6 * k);
    L.JA = take(d * 6 * k);
    L.Psi = take(d * 14 * k);
    L.Phi = take(d * 7 * L.ld);
    L.Vt = take(thin);
    L.Ys = take(thin);
    L.s0 = take(wide);
    L.s1 = take(wide);
    L.s2 = take(wide);
    L.S = take(d * L.rp * L.rp);
    L.RS = take(d * L.rp * L.rp);
    L.PS = take(d * L.rp * kNB);
    L.LS = take(d * L.rp * kNB);
    L.part = take(d * L.nsplit * L.ld * L.ld);
    L.out = take(d * 81 * c.n);
    L.ecol = take(sizeof(int) * L.ldq);
    L.norms = take(d * (2 + 2 * (size_t)c.Np));
    L.Sq = take(sizeof(long long) * (size_t)L.ldq * L.ldq);
    L.cmax = take(sizeof(unsigned long long) * (size_t)L.ldq);
    L.emax = take(sizeof(int));
    L.total = off;
    return L;
}

}  // namespace

cudaError_t update_enqueue(Ctx& c, const ccov_obs* add, int64_t k, const double* add_cov, double* out,
                           int out_memory) {
    const Layout L = layout(c, k);
    cudaError_t e;
    if (c.upd_bytes < L.total) {
        if (c.d_upd) { cudaFree(c.d_upd); c.bytes -= (int64_t)c.upd_bytes; c.d_upd = nullptr; c.upd_bytes = 0; }
        if ((e = cudaMalloc(&c.d_upd, L.total)) != cudaSuccess) return e;
        c.upd_bytes = L.total;
        c.bytes += (int64_t)L.total;
    }
    char* base = static_cast<char*>(c.d_upd);
    auto at = [&](size_t off) { return reinterpret_cast<double*>(base + off); };
    ccov_obs* d_add = reinterpret_cast<ccov_obs*>(base + L.add);
    double* d_cov = add_cov ? at(L.cov) : nullptr;
    double *Jc = at(L.Jc), *Jp = at(L.Jp), *JA = at(L.JA), *Psi = at(L.Psi), *Phi = at(L.Phi);
    double *Vt = at(L.Vt), *Ys = at(L.Ys), *S = at(L.S), *RS = at(L.RS), *part = at(L.part);
    double* res = at(L.out);
    const int64_t N = c.N, Np = c.Np, ld = L.ld;
    if ((e = cudaMemsetAsync(c.d_flag, 0, 2 * sizeof(int), c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(d_add, add, sizeof(ccov_obs) * k, cudaMemcpyHostToDevice, c.stream)) != cudaSuccess)
        return e;
    if (d_cov && (e = cudaMemcpyAsync(d_cov, add_cov, sizeof(double) * 4 * k, cudaMemcpyHostToDevice,
                                      c.stream)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(Phi, 0, sizeof(double) * 7 * ld, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Vt, 0, sizeof(double) * Np * ld, c.stream)) != cudaSuccess) return e;
    // per added observation: Jacobian rows, Psi, Phi; then the columns of Vt
    launch_upd_obs(c, k, d_add, d_cov, ld, Jc, Jp, JA, Psi, Phi);
    upd_scatter_kernel<<<(unsigned)((k + 127) / 128), 128, 0, c.stream>>>(k, d_add, c.d_pt_ptr, c.d_obs, c.d_V, Jc,
                                                                          Jp, ld, Vt);
    upd_dense_kernel<<<(unsigned)((Np * ld + 255) / 256), 256, 0, c.stream>>>(N, Np, ld, L.r, c.d_G, Phi, c.d_D,
                                                                              Vt);
    c.launches += 2;
    // Y_s = X^T X (D Vt): on the tensor cores for the mixed form (digit-split
    // GEMMs over panels of X), else in FP64 (or where the operand buffers of
    // the mixed form are too short for the columns)
    const bool tensor = c.opt.precision == CCOV_PREC_MIXED && L.ldq <= Np;
    long long* Sq = tensor ? reinterpret_cast<long long*>(base + L.Sq) : nullptr;
    int* ecol = reinterpret_cast<int*>(base + L.ecol);
    int FS = 0;
    if (tensor) {
        if ((e = mixed_xtxv(c, L.ld, Vt, ld, Ys, reinterpret_cast<long long*>(base + L.s0),
                            reinterpret_cast<long long*>(base + L.s1), reinterpret_cast<long long*>(base + L.s2), Sq,
                            ecol, reinterpret_cast<unsigned long long*>(base + L.cmax), at(L.norms), &FS)) !=
            cudaSuccess)
            return e;
    } else {
        est_xtxv(c, (int)L.g, Vt, Ys, base + L.s0, base + L.s1, base + L.s2);
    }
    // S = I + ... + (D Vt)^T Y_s
    {
        if (!tensor) {
            const unsigned t = (unsigned)((ld + 31) / 32);
            upd_atb_kernel<<<dim3(t, t, (unsigned)L.nsplit), 256, 0, c.stream>>>(N, ld, L.chunk, Vt, Ys, part);
            c.launches++;
        }
        upd_s_kernel<<<(unsigned)((L.rp * L.rp + 255) / 256), 256, 0, c.stream>>>(
            L.r, ld, L.rp, (int)L.nsplit, part, Sq, L.ldq, ecol, FS, d_add, JA, Jp, Psi, c.d_small, S);
        c.launches++;
    }
    // S = L_S L_S^T, X_S = L_S^-1 (the FP64 blocked path on the small matrix)
    {
        Ctx s;
        s.n = 0;
        s.N = s.Np = L.rp;
        s.stream = c.stream;
        s.d_Z = S;
        s.d_R = RS;
        s.d_P = at(L.PS);
        s.d_Linv = at(L.LS);
        s.d_flag = c.d_flag;
        spd_factor_inverse64(s);
        c.launches += s.launches;
    }
    // P = Y_s X_S^T, then the camera blocks.  Tensor-core form: from the
    // fixed-point Y of mixed_xtxv (s2), with X_S in Q60 (s0) and P in int64
    // (s1), P itself into Vt (no longer needed)
    double* P = at(L.s2);
    if (tensor) {
        P = Vt;
        if ((e = mixed_update_p(c, ld, reinterpret_cast<const long long*>(base + L.s2), RS, ecol,
                                reinterpret_cast<int*>(base + L.emax), reinterpret_cast<long long*>(base + L.s0),
                                reinterpret_cast<long long*>(base + L.s1), P, ld)) != cudaSuccess)
            return e;
    } else {
        launch_gemm64(c, true, false, N, ld, ld, 1.0, Ys, ld, RS, L.rp, 0.0, P, ld, 0, 0);
    }
    upd_diag_kernel<<<(unsigned)c.n, 128, 0, c.stream>>>(ld, ld, P, c.d_D, c.d_Sig, res);
    c.launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (out) {
        const cudaMemcpyKind kind = out_memory == CCOV_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if ((e = cudaMemcpyAsync(out, res, sizeof(double) * 81 * c.n, kind, c.stream)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void update_free(Ctx& c) {
    if (c.d_upd) cudaFree(c.d_upd);
    c.d_upd = nullptr;
    c.upd_bytes = 0;
}

}  // namespace ccov

// A-posteriori error estimate of the camera blocks of step (d), on sampled
// cameras.
//
// Step (d) factorises the Jacobi-scaled matrix Z_s = L L^T and inverts the
// factor, X ~ L^-1, so that the scaled camera block i of the result is
// E_i^T X^T X E_i (E_i: the nine unit columns of camera i).  Let
// y = X^T (X E_i), the nine computed columns of Z_s^-1 that this block
// belongs to, and R = Z_s y - E_i their residual against the matrix that was
// factorised (a copy kept before the factorisation).  Then
// y - Z_s^-1 E_i = Z_s^-1 R exactly, and the error of the computed block is
//   E_i^T (y - Z_s^-1 E_i) = (Z_s^-1 E_i)^T R = y^T R - (y - Z_s^-1 E_i)^T R,
// i.e. y^T R up to a term of second order in the error.  Unscaled with the
// Jacobi scale D_i of the camera, it estimates the error of the returned
// block; the gauge term subtracted afterwards is the same in both.
//
// Cost: three products of a triangular N x N matrix with the 9k columns of the
// k sampled cameras (X^T (X E), and Z_s y by its lower triangle and the
// transpose of its strict lower triangle), O(N^2 k).  The residual must be far
// more accurate than the error it measures (about 1e-9 relative for the mixed
// form), so the mixed path computes it in double-single arithmetic (about 48
// bits) on the FP32 pipes; the FP64 path, whose own error is near FP64
// rounding, computes it in FP64 (its estimate is then an upper estimate at
// the rounding level of the residual itself).
//
// The sampled cameras are those whose scaled blocks have the largest
// diagonal entry: the variance inflation of a parameter, (Z_s^-1)_aa, is
// largest where the parameter is nearly determined by the others, which is
// where the inverse loses the most digits.
#include <cuda_runtime.h>

#include "ccov_internal.cuh"
#include "ds_arith.cuh"

namespace ccov {
namespace {

__device__ __forceinline__ void est_flag(int* flag, int code, int detail) {
    if (atomicMax(flag, code) < code) flag[1] = detail;
}

template <class T>
struct Ar;

template <>
struct Ar<double> {
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double fma(double acc, double a, double b) { return __fma_rn(a, b, acc); }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double load(const double* p, float) { return *p; }
    static __device__ __forceinline__ double to_double(double a) { return a; }
    static __device__ __forceinline__ double from_double(double a) { return a; }
    static __device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
};

template <>
struct Ar<dsf> {
    static __device__ __forceinline__ dsf zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ dsf fma(dsf acc, dsf a, dsf b) { return ds_fma(acc, a, b); }
    static __device__ __forceinline__ dsf add(dsf a, dsf b) { return ds_add(a, b); }
    static __device__ __forceinline__ dsf load(const long long* p, float scale) { return ds_from_fixed(*p, scale); }
    static __device__ __forceinline__ double to_double(dsf a) { return (double)a.h + (double)a.l; }
    static __device__ __forceinline__ dsf from_double(double a) { return ds_from_double(a); }
    static __device__ __forceinline__ dsf shfl_xor(dsf v, int o) {
        return {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    }
};

// The k sampled cameras: repeatedly the camera with the largest diagonal
// entry of its scaled block (ties: the lower index), excluding those taken.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024)
est_select_kernel(int64_t n, const double* __restrict__ Sig, int k, int* __restrict__ idx) {
    __shared__ double bv[32];
    __shared__ int bi[32];
    __shared__ int chosen[kEstMaxCams];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < k; ++j) {
        double best = -1.0;
        int bidx = 0x7fffffff;
        for (int64_t i = tid; i < n; i += 1024) {
            bool taken = false;
            for (int q = 0; q < j; ++q) taken |= chosen[q] == (int)i;
            if (taken) continue;
            double v = 0.0;
            for (int a = 0; a < 9; ++a) v = fmax(v, Sig[81 * i + 10 * a]);
            if (v > best || (v == best && (int)i < bidx)) { best = v; bidx = (int)i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
        }
        if (lane == 0) { bv[warp] = best; bi[warp] = bidx; }
        __syncthreads();
        if (tid == 0) {
            double b = -1.0;
            int bj = 0x7fffffff;
            for (int w = 0; w < 32; ++w)
                if (bv[w] > b || (bv[w] == b && bi[w] < bj)) { b = bv[w]; bj = bi[w]; }
            chosen[j] = bj;
            idx[j] = bj;
        }
        __syncthreads();
    }
}

// W[r][9j + a] = X[r][9 idx_j + a] (zero above the diagonal of X).
template <class T, class In>
__global__ void est_gather_kernel(int64_t N, int64_t Np, const In* __restrict__ X, float scale,
                                  const int* __restrict__ idx, int k, T* __restrict__ W) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= Np) return;
    const int ld = 9 * k;
    for (int j = 0; j < k; ++j)
        for (int a = 0; a < 9; ++a) {
            const int64_t col = 9 * (int64_t)idx[j] + a;
            W[r * ld + 9 * j + a] = (r < N && col <= r) ? Ar<T>::load(X + r * Np + col, scale) : Ar<T>::zero();
        }
}

// out[c][9j + a] (+)= sum over r >= c (r > c if strict), r < N, of
// A[r][c] V[r][9j + a]: the transpose of a lower-triangular matrix times the
// nine columns of sampled camera j.  Grid (N / 32, k); a CTA owns 32
// consecutive columns c (one per lane) and one camera; its eight warps take
// the rows r = w (mod 8) and are summed in a fixed order at the end.
template <class T, class In>
__global__ void __launch_bounds__(256)
lt_t_kernel(int64_t N, int64_t Np, const In* __restrict__ A, float scale, int strict, const T* __restrict__ V,
            int k, T* __restrict__ out, int accumulate) {
    __shared__ T part[8][32][9];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.y, ld = 9 * k;
    const int64_t c = blockIdx.x * 32 + lane;
    T acc[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) acc[a] = Ar<T>::zero();
    const int64_t r0 = blockIdx.x * 32;
    for (int64_t r = r0 + warp; r < N; r += 8) {
        if (c >= N || r < c || (strict && r == c)) continue;
        const T x = Ar<T>::load(A + r * Np + c, scale);
        const T* v = V + r * ld + 9 * j;
#pragma unroll
        for (int a = 0; a < 9; ++a) acc[a] = Ar<T>::fma(acc[a], x, v[a]);
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) part[warp][lane][a] = acc[a];
    __syncthreads();
    if (warp == 0 && c < Np) {
        for (int a = 0; a < 9; ++a) {
            T s = part[0][lane][a];
            for (int w = 1; w < 8; ++w) s = Ar<T>::add(s, part[w][lane][a]);
            T* o = out + c * ld + 9 * j + a;
            *o = accumulate ? Ar<T>::add(*o, s) : s;
        }
    }
}

// out[r][9j + a] = sum over c <= r of A[r][c] V[c][9j + a] - [r = 9 idx_j + a]
// (the lower triangle of a symmetric matrix times the camera's columns, minus
// the unit columns; idx null: no unit columns).  Grid (N / 8, k), a warp per row.
template <class T, class In>
__global__ void __launch_bounds__(256)
lt_row_kernel(int64_t N, int64_t Np, const In* __restrict__ A, float scale, const T* __restrict__ V, int k,
              const int* __restrict__ idx, T* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.y, ld = 9 * k;
    const int64_t r = blockIdx.x * 8 + warp;
    if (r >= Np) return;
    T acc[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) acc[a] = Ar<T>::zero();
    if (r < N) {
        for (int64_t c = lane; c <= r; c += 32) {
            const T x = Ar<T>::load(A + r * Np + c, scale);
            const T* v = V + c * ld + 9 * j;
#pragma unroll
            for (int a = 0; a < 9; ++a) acc[a] = Ar<T>::fma(acc[a], x, v[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 9; ++a)
        for (int o = 16; o > 0; o >>= 1) acc[a] = Ar<T>::add(acc[a], Ar<T>::shfl_xor(acc[a], o));
    if (lane < 9) {
        T s = acc[0];
#pragma unroll
        for (int a = 1; a < 9; ++a)
            if (lane == a) s = acc[a];
        if (idx && r == 9 * (int64_t)idx[j] + lane) s = Ar<T>::add(s, Ar<T>::from_double(-1.0));
        out[r * ld + 9 * j + lane] = s;
    }
}

// dS_j[a][b] = sum_r Y[r][9j + a] R[r][9j + b]: one CTA per sampled camera,
// 324 threads = 81 entries x 4 interleaved row subsets, summed in order.
template <class T>
__global__ void __launch_bounds__(324)
est_dot_kernel(int64_t N, const T* __restrict__ Y, const T* __restrict__ R, int k, double* __restrict__ dS) {
    __shared__ T part[4][81];
    const int j = blockIdx.x, ld = 9 * k;
    const int e = threadIdx.x % 81, q = threadIdx.x / 81, a = e / 9, b = e % 9;
    T acc = Ar<T>::zero();
    for (int64_t r = q; r < N; r += 4) acc = Ar<T>::fma(acc, Y[r * ld + 9 * j + a], R[r * ld + 9 * j + b]);
    part[q][e] = acc;
    __syncthreads();
    if (q == 0) {
        T s = Ar<T>::add(Ar<T>::add(part[0][e], part[1][e]), Ar<T>::add(part[2][e], part[3][e]));
        dS[81 * j + e] = Ar<T>::to_double(s);
    }
}

// For sampled camera j (one thread each): the unscaled error estimate
// D_i dS_j D_i (symmetrised) against the returned block Sigma_i:
//   out[3j]     = ||D dS D||_F / ||Sigma_i||_F            (relative Frobenius)
//   out[3j + 1] = the same after the scaling diag(Sigma_i)^-1/2
//   out[3j + 2] = camera index i
__global__ void est_final_kernel(int k, const int* __restrict__ idx, const double* __restrict__ dS,
                                 const double* __restrict__ D, const double* __restrict__ Sig,
                                 double* __restrict__ out, int* flag) {
    const int j = threadIdx.x;
    if (j >= k) return;
    const int64_t cam = idx[j];
    const double* s = Sig + 81 * cam;
    const double* d = D + 9 * cam;
    double num = 0.0, den = 0.0, nnum = 0.0, nden = 0.0;
    for (int a = 0; a < 9; ++a)
        for (int b = 0; b < 9; ++b) {
            const double e = 0.5 * (dS[81 * j + 9 * a + b] + dS[81 * j + 9 * b + a]) * d[a] * d[b];
            const double w = 1.0 / sqrt(fabs(s[10 * a]) * fabs(s[10 * b]));
            num += e * e;
            den += s[9 * a + b] * s[9 * a + b];
            nnum += e * e * w * w;
            nden += s[9 * a + b] * s[9 * a + b] * w * w;
        }
    const double rel = sqrt(num / den), nrel = sqrt(nnum / nden);
    if (!(rel == rel) || !(nrel == nrel)) est_flag(flag, DEV_RANGE, (int)cam);
    out[3 * j] = rel;
    out[3 * j + 1] = nrel;
    out[3 * j + 2] = (double)cam;
}

template <class T, class XIn, class ZIn>
void launch_est(Ctx& c, const XIn* X, float sx, const ZIn* Zs, float sz) {
    const int k = c.est_k;
    T* W = static_cast<T*>(c.d_estW);
    T* Y = static_cast<T*>(c.d_estY);
    T* R = static_cast<T*>(c.d_estR);
    const int64_t N = c.N, Np = c.Np;
    est_select_kernel<<<1, 1024, 0, c.stream>>>(c.n, c.d_Sig, k, c.d_est_idx);
    est_gather_kernel<T, XIn><<<(unsigned)((Np + 255) / 256), 256, 0, c.stream>>>(N, Np, X, sx, c.d_est_idx, k, W);
    const dim3 gt((unsigned)((Np + 31) / 32), (unsigned)k), gr((unsigned)((Np + 7) / 8), (unsigned)k);
    // y = X^T (X E)
    lt_t_kernel<T, XIn><<<gt, 256, 0, c.stream>>>(N, Np, X, sx, 0, W, k, Y, 0);
    // R = Z_s y - E: lower triangle by rows, then the strict upper part as the
    // transpose of the strict lower triangle
    lt_row_kernel<T, ZIn><<<gr, 256, 0, c.stream>>>(N, Np, Zs, sz, Y, k, c.d_est_idx, R);
    lt_t_kernel<T, ZIn><<<gt, 256, 0, c.stream>>>(N, Np, Zs, sz, 1, Y, k, R, 1);
    est_dot_kernel<T><<<k, 324, 0, c.stream>>>(N, Y, R, k, c.d_est_dS);
    c.launches += 6;
}

template <class T>
__global__ void to_arith_kernel(int64_t count, const double* __restrict__ in, T* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) out[e] = Ar<T>::from_double(in[e]);
}

template <class T>
__global__ void from_arith_kernel(int64_t count, const T* __restrict__ in, double* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) out[e] = Ar<T>::to_double(in[e]);
}

// Y = X^T (X V) for g groups of nine columns (V, Y: Np x 9g FP64, device),
// X the lower-triangular inverse factor of the last step (d); W, Y2 scratch
// of the same size.  The arithmetic is the estimate's.
template <class T, class XIn>
void xtxv(Ctx& c, const XIn* X, float sx, int g, const double* V, double* Y, void* s0, void* s1, void* s2) {
    const int64_t N = c.N, Np = c.Np, cnt = Np * 9 * (int64_t)g;
    T* v = static_cast<T*>(s0);
    T* w = static_cast<T*>(s1);
    T* y = static_cast<T*>(s2);
    const unsigned b = (unsigned)((cnt + 255) / 256);
    to_arith_kernel<T><<<b, 256, 0, c.stream>>>(cnt, V, v);
    const dim3 gt((unsigned)((Np + 31) / 32), (unsigned)g), gr((unsigned)((Np + 7) / 8), (unsigned)g);
    lt_row_kernel<T, XIn><<<gr, 256, 0, c.stream>>>(N, Np, X, sx, v, g, nullptr, w);
    lt_t_kernel<T, XIn><<<gt, 256, 0, c.stream>>>(N, Np, X, sx, 0, w, g, y, 0);
    from_arith_kernel<T><<<b, 256, 0, c.stream>>>(cnt, y, Y);
    c.launches += 4;
}

}  // namespace

void est_xtxv(Ctx& c, int g, const double* V, double* Y, void* s0, void* s1, void* s2) {
    if (c.opt.precision == CCOV_PREC_FP64)
        xtxv<double, double>(c, c.d_R, 1.f, g, V, Y, s0, s1, s2);
    else
        xtxv<dsf, long long>(c, mixed_inverse_factor(c), 2.2737367544323206e-13f /* 2^-42 */, g, V, Y, s0, s1, s2);
}

cudaError_t est_alloc(Ctx& c, int k) {
    if (c.d_Zkeep && c.est_cap >= k) return cudaSuccess;
    if (c.d_estW) { cudaFree(c.d_estW); cudaFree(c.d_estY); cudaFree(c.d_estR); c.d_estW = c.d_estY = c.d_estR = nullptr; }
    cudaError_t e;
    if (!c.d_Zkeep) {
        if ((e = cudaMalloc(&c.d_Zkeep, sizeof(double) * c.Np * c.Np)) != cudaSuccess) return e;
        c.bytes += (int64_t)(sizeof(double) * c.Np * c.Np);
    }
    const size_t thin = sizeof(double) * (size_t)c.Np * 9 * kEstMaxCams;
    if ((e = cudaMalloc(&c.d_estW, thin)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c.d_estY, thin)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&c.d_estR, thin)) != cudaSuccess) return e;
    if (!c.d_est_idx && (e = cudaMalloc(&c.d_est_idx, sizeof(int) * kEstMaxCams)) != cudaSuccess) return e;
    if (!c.d_est_dS && (e = cudaMalloc(&c.d_est_dS, sizeof(double) * 81 * kEstMaxCams)) != cudaSuccess) return e;
    if (!c.d_est_out && (e = cudaMalloc(&c.d_est_out, sizeof(double) * 3 * kEstMaxCams)) != cudaSuccess) return e;
    c.est_cap = kEstMaxCams;
    c.bytes += (int64_t)(3 * thin);
    return cudaSuccess;
}

void est_free(Ctx& c) {
    void* p[] = {c.d_Zkeep, c.d_estW, c.d_estY, c.d_estR, c.d_est_idx, c.d_est_dS, c.d_est_out};
    for (void* q : p)
        if (q) cudaFree(q);
}

void est_keep_fp64(Ctx& c) {
    // the FP64 path scales Z in place; keep the matrix that is factorised
    cudaMemcpyAsync(c.d_Zkeep, c.d_Z, sizeof(double) * c.Np * c.Np, cudaMemcpyDeviceToDevice, c.stream);
}

void est_launch(Ctx& c, const long long* Xq) {
    if (c.opt.precision == CCOV_PREC_FP64)
        launch_est<double, double, double>(c, c.d_R, 1.f, static_cast<const double*>(c.d_Zkeep), 1.f);
    else
        launch_est<dsf, long long, long long>(c, Xq, 2.2737367544323206e-13f /* 2^-42 */,
                                              static_cast<const long long*>(c.d_Zkeep),
                                              8.673617379884035e-19f /* 2^-60 */);
}

void est_launch_final(Ctx& c) {
    est_final_kernel<<<1, 32, 0, c.stream>>>(c.est_k, c.d_est_idx, c.d_est_dS, c.d_D, c.d_Sig, c.d_est_out,
                                             c.d_flag);
    c.launches++;
}

}  // namespace ccov

// Steps (a)-(c): reprojection Jacobians and information blocks, Schur
// elimination of the point blocks into the dense reduced camera matrix, and
// the camera rows of the similarity nullspace.  All FP64.
//
// Sec. 3 (Eq. normal-equation-system) defines M = J^T Sigma_u^-1 J; Sec. 4.2
// (Eq. block-inversion-Qp, schur-complement-inversion) eliminates the point
// block A_p; Sec. 4.1 (Eq. transformation-conditions, rotation-nullspace-
// equation) gives the nullspace H.  Layout: observations sorted by point
// (CSR by point, pt_ptr) plus a permutation grouping them by camera.
#include <type_traits>

#include "ccov_internal.cuh"
#include "ds_arith.cuh"

namespace ccov {
namespace {

constexpr int kWarps = 4;  // warps per CTA of the warp-per-item kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of the mixed form's sparse steps in double-single arithmetic (about
// 44 bits, above the 39 of the digits step (d) takes of Z); the FP64 form
// keeps FP64 with the same expressions as before.
template <class T>
struct SpAr;

template <>
struct SpAr<double> {
    typedef double V;
    static __device__ __forceinline__ double from(double x) { return x; }
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double value(double a) { return a; }
    static __device__ __forceinline__ double sum(double v) { return warp_sum(v); }
};

template <>
struct SpAr<dsf> {
    typedef dsf V;
    static __device__ __forceinline__ dsf from(double x) { return ds_from_double(x); }
    static __device__ __forceinline__ dsf zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ dsf add(dsf a, dsf b) { return ds_add(a, b); }
    static __device__ __forceinline__ double value(dsf a) { return (double)a.h + (double)a.l; }
    static __device__ __forceinline__ dsf sum(dsf v) {   // the same butterfly as warp_sum
        for (int o = 16; o > 0; o >>= 1)
            v = ds_add(v, {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
        return v;
    }
};


__device__ __forceinline__ void set_flag(int* flag, int code, int detail) {
    if (atomicMax(flag, code) < code) flag[1] = detail;
}

// R(r), t, f, k1, k2 and the left Jacobian J_l(r) of SO(3):
// R = I + a [r]x + b [r]x^2, a = sin(th)/th, b = (1 - cos th)/th^2,
// J_l = I + b [r]x + c [r]x^2, c = (th - sin th)/th^3, so that
// d(R X)/dr = -[R X]x J_l.  The centre camera {r, C, c, k} (slots 3-5: C)
// is stored as t = -R C, f = c, k1 = k, k2 = 0, with prep[24] = 1.
__global__ void cam_prep_kernel(int64_t n, const double* __restrict__ cams,
                                double* __restrict__ prep, int centre) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* c = cams + 9 * i;
    double r0 = c[0], r1 = c[1], r2 = c[2];
    double th2 = r0 * r0 + r1 * r1 + r2 * r2;
    double th = sqrt(th2);
    double a, b, cc;
    if (th < 0.05) {
        double t4 = th2 * th2;
        a = 1.0 - th2 / 6.0 + t4 / 120.0 - t4 * th2 / 5040.0;
        b = 0.5 - th2 / 24.0 + t4 / 720.0 - t4 * th2 / 40320.0;
        cc = 1.0 / 6.0 - th2 / 120.0 + t4 / 5040.0 - t4 * th2 / 362880.0;
    } else {
        double s = sin(th), h = sin(0.5 * th);
        a = s / th;
        b = 2.0 * h * h / th2;
        cc = (th - s) / (th2 * th);
    }
    // K = [r]x, K2 = K K
    double K[9] = {0, -r2, r1, r2, 0, -r0, -r1, r0, 0};
    double K2[9];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            K2[3 * p + q] = K[3 * p] * K[q] + K[3 * p + 1] * K[3 + q] + K[3 * p + 2] * K[6 + q];
    double* o = prep + kCamPrep * i;
    for (int e = 0; e < 9; ++e) {
        double I = (e % 4 == 0) ? 1.0 : 0.0;
        o[e] = I + a * K[e] + b * K2[e];
        o[15 + e] = I + b * K[e] + cc * K2[e];
    }
    if (centre) {
        for (int p = 0; p < 3; ++p) o[9 + p] = -(o[3 * p] * c[3] + o[3 * p + 1] * c[4] + o[3 * p + 2] * c[5]);
        o[12] = c[6]; o[13] = c[7]; o[14] = 0.0;
    } else {
        o[9] = c[3]; o[10] = c[4]; o[11] = c[5];
        o[12] = c[6]; o[13] = c[7]; o[14] = c[8];
    }
    o[24] = centre ? 1.0 : 0.0;
}

// Analytic Jacobians of one observation (Sec. 4.1 projection with the
// 9-parameter camera).  Jc: 2x9 row-major, Jp: 2x3.  Returns the depth.
// Centre camera: p = R (X - C), so dp/dr = -[p]x J_l, dp/dC = -R, and slot
// 8 (no parameter) has a zero column.
__device__ __forceinline__ double obs_jacobian(const double* __restrict__ cp, double X0, double X1,
                                               double X2, double* Jc, double* Jp) {
    const double* R = cp;
    double RX0 = R[0] * X0 + R[1] * X1 + R[2] * X2;
    double RX1 = R[3] * X0 + R[4] * X1 + R[5] * X2;
    double RX2 = R[6] * X0 + R[7] * X1 + R[8] * X2;
    double p0 = RX0 + cp[9], p1 = RX1 + cp[10], p2 = RX2 + cp[11];
    double f = cp[12], k1 = cp[13], k2 = cp[14];
    double s = 1.0 / p2;
    double x = p0 * s, y = p1 * s;
    double r2 = x * x + y * y;
    double g = 1.0 + r2 * (k1 + k2 * r2);
    double dg = 2.0 * k1 + 4.0 * k2 * r2;
    // d u / d(x, y) = f (g I + dg [x y]^T [x y])
    double a00 = f * (g + dg * x * x), a01 = f * dg * x * y, a11 = f * (g + dg * y * y);
    // D = (d u / d(x,y)) (d(x,y) / d p), d(x,y)/dp = s [1 0 -x; 0 1 -y]
    double D[6];
    D[0] = s * a00; D[1] = s * a01; D[2] = -s * (a00 * x + a01 * y);
    D[3] = s * a01; D[4] = s * a11; D[5] = -s * (a01 * x + a11 * y);
    // Q = -[RX]x J_l  (d p / d r); centre camera: -[p]x J_l
    const double* Jl = cp + 15;
    const bool centre = cp[24] != 0.0;
    const double q0 = centre ? p0 : RX0, q1 = centre ? p1 : RX1, q2 = centre ? p2 : RX2;
    double S[9] = {0, q2, -q1, -q2, 0, q0, q1, -q0, 0};        // -[q]x
    double Q[9];
#pragma unroll
    for (int pq = 0; pq < 9; ++pq) {
        int p = pq / 3, q = pq % 3;
        Q[pq] = S[3 * p] * Jl[q] + S[3 * p + 1] * Jl[3 + q] + S[3 * p + 2] * Jl[6 + q];
    }
#pragma unroll
    for (int row = 0; row < 2; ++row) {
        const double* d = D + 3 * row;
        double* jc = Jc + 9 * row;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            jc[q] = d[0] * Q[q] + d[1] * Q[3 + q] + d[2] * Q[6 + q];
            Jp[3 * row + q] = d[0] * R[q] + d[1] * R[3 + q] + d[2] * R[6 + q];
            jc[3 + q] = centre ? -Jp[3 * row + q] : d[q];
        }
    }
    Jc[6] = g * x;          Jc[15] = g * y;
    Jc[7] = f * r2 * x;     Jc[16] = f * r2 * y;
    Jc[8] = centre ? 0.0 : f * r2 * r2 * x;
    Jc[17] = centre ? 0.0 : f * r2 * r2 * y;
    return p2;
}

// Left-multiply the two Jacobian rows by Sigma_u^-1/2 (C^-1 with Sigma_u = C C^T).
__device__ __forceinline__ void whiten(double* Jc, double* Jp, double sigma,
                                       const double* __restrict__ cov) {
    if (cov == nullptr) {
        double w = 1.0 / sigma;
#pragma unroll
        for (int e = 0; e < 18; ++e) Jc[e] *= w;
#pragma unroll
        for (int e = 0; e < 6; ++e) Jp[e] *= w;
        return;
    }
    double c00 = sqrt(cov[0]);
    double c10 = cov[2] / c00;
    double c11 = sqrt(cov[3] - c10 * c10);
    double i00 = 1.0 / c00, i11 = 1.0 / c11, i10 = -c10 * i00 * i11;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        double a = Jc[q], b = Jc[9 + q];
        Jc[q] = i00 * a;
        Jc[9 + q] = i10 * a + i11 * b;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double a = Jp[q], b = Jp[3 + q];
        Jp[q] = i00 * a;
        Jp[3 + q] = i10 * a + i11 * b;
    }
}

// Step (a), point part in two passes (a warp per point leaves most lanes
// idle on tracks of a few observations): a thread per observation computes
// the Jacobian, keeps it unwhitened in J (Jc 2 x 9, then Jp 2 x 3: 24 values,
// read again by the camera blocks and the nullspace), whitens it and writes
// W_ij = Jc^T Jp and the observation's share Jp^T Jp of A_j (six values into
// `share`); a thread per point then sums the shares of its observations in
// order and inverts A_j.
__global__ void __launch_bounds__(128)
obs_info_kernel(int64_t t, const ccov_obs* __restrict__ obs, const double* __restrict__ pts,
                const double* __restrict__ prep, double sigma, const double* __restrict__ cov,
                double* __restrict__ W, double* __restrict__ share, double* __restrict__ J, int* flag) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= t) return;
    const int i = obs[o].cam;
    const int64_t j = obs[o].pt;
    double Jc[18], Jp[6];
    const double depth = obs_jacobian(prep + (int64_t)kCamPrep * i, pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], Jc, Jp);
    if (!(depth > 0.0)) set_flag(flag, DEV_BEHIND, (int)o);
    double* jo = J + 24 * o;
#pragma unroll
    for (int e = 0; e < 18; ++e) jo[e] = Jc[e];
#pragma unroll
    for (int e = 0; e < 6; ++e) jo[18 + e] = Jp[e];
    whiten(Jc, Jp, sigma, cov ? cov + 4 * o : nullptr);
    double* a = share + 6 * o;
    a[0] = Jp[0] * Jp[0] + Jp[3] * Jp[3];
    a[1] = Jp[0] * Jp[1] + Jp[3] * Jp[4];
    a[2] = Jp[0] * Jp[2] + Jp[3] * Jp[5];
    a[3] = Jp[1] * Jp[1] + Jp[4] * Jp[4];
    a[4] = Jp[1] * Jp[2] + Jp[4] * Jp[5];
    a[5] = Jp[2] * Jp[2] + Jp[5] * Jp[5];
    double* w = W + 27 * o;
#pragma unroll
    for (int p = 0; p < 9; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) w[3 * p + q] = Jc[p] * Jp[q] + Jc[9 + p] * Jp[3 + q];
}

__global__ void __launch_bounds__(128)
point_ainv_kernel(int64_t m, const int* __restrict__ pt_ptr, const double* __restrict__ share,
                  double* __restrict__ Ainv, int* flag) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= m) return;
    double a[6] = {0, 0, 0, 0, 0, 0};
    for (int o = pt_ptr[j]; o < pt_ptr[j + 1]; ++o)
#pragma unroll
        for (int e = 0; e < 6; ++e) a[e] += share[6 * (int64_t)o + e];
    // inverse of the symmetric 3x3 block by cofactors
    const double c00 = a[3] * a[5] - a[4] * a[4];
    const double c01 = a[2] * a[4] - a[1] * a[5];
    const double c02 = a[1] * a[4] - a[2] * a[3];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double scale = a[0] * a[3] * a[5];
    if (!(det > 1e-14 * scale) || !(a[0] > 0.0)) set_flag(flag, DEV_SINGULAR_A, (int)j);
    const double id = 1.0 / det;
    double* ai = Ainv + 6 * j;
    ai[0] = c00 * id;
    ai[1] = c01 * id;
    ai[2] = c02 * id;
    ai[3] = (a[0] * a[5] - a[2] * a[2]) * id;
    ai[4] = (a[1] * a[2] - a[0] * a[4]) * id;
    ai[5] = (a[0] * a[3] - a[1] * a[1]) * id;
}

// Step (a), camera part: warp per camera, U_i = sum Jc^T Jc (lower, 45),
// from the Jacobians that obs_info_kernel kept (J, unwhitened).
template <class T>
__global__ void __launch_bounds__(32 * kWarps)
cam_info_kernel(int64_t n, const int* __restrict__ cam_ptr, const int* __restrict__ cam_perm,
                const double* __restrict__ J, const double* __restrict__ prep, double sigma,
                const double* __restrict__ cov, double* __restrict__ U) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    typedef SpAr<T> Ar;
    for (int64_t i = warp; i < n; i += nwarp) {
        typename Ar::V u[45];
#pragma unroll
        for (int e = 0; e < 45; ++e) u[e] = Ar::zero();
        const double* cp = prep + (int64_t)kCamPrep * i;
        for (int k = cam_ptr[i] + lane; k < cam_ptr[i + 1]; k += 32) {
            const int o = cam_perm[k];
            const double* jo = J + 24 * (int64_t)o;
            double Jc[18], Jp[6];
#pragma unroll
            for (int e = 0; e < 18; ++e) Jc[e] = jo[e];
#pragma unroll
            for (int e = 0; e < 6; ++e) Jp[e] = jo[18 + e];
            whiten(Jc, Jp, sigma, cov ? cov + 4 * (int64_t)o : nullptr);
            int e = 0;
            if constexpr (std::is_same<T, double>::value) {
#pragma unroll
                for (int p = 0; p < 9; ++p)
#pragma unroll
                    for (int q = 0; q <= p; ++q, ++e) u[e] += Jc[p] * Jc[q] + Jc[9 + p] * Jc[9 + q];
            } else {
                dsf jc[18];
#pragma unroll
                for (int c = 0; c < 18; ++c) jc[c] = ds_from_double(Jc[c]);
#pragma unroll
                for (int p = 0; p < 9; ++p)
#pragma unroll
                    for (int q = 0; q <= p; ++q, ++e) u[e] = ds_fma(ds_fma(u[e], jc[p], jc[q]), jc[9 + p], jc[9 + q]);
            }
        }
#pragma unroll
        for (int e = 0; e < 45; ++e) {
            double v = Ar::value(Ar::sum(u[e]));
            // centre camera: a unit prior on the value that no observation sees (slot 8)
            if (e == 44 && cp[24] != 0.0) v += 1.0;
            if (lane == 0) U[45 * i + e] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Step (b): Z = blockdiag(U) - sum_j sum_{a,b in track j} V_a W_b^T with
// V_a = W_a A_j^-1 (Eq. schur-complement-inversion), and
// W7 = sum_j H_Xj^T A_j^-1 H_Xj.  Deterministic: every 9x9 block of Z is
// summed by one warp over a fixed list of observation pairs and written once,
// and the 7x7 sums are reduced in a fixed order, so that repeated runs give
// identical bits.

__device__ __forceinline__ void hx_row(double X0, double X1, double X2, int k, double* h) {
    // row k of H_X = [I, -[X]x, X]
    h[0] = (k == 0); h[1] = (k == 1); h[2] = (k == 2);
    if (k == 0) { h[3] = 0.0; h[4] = X2; h[5] = -X1; h[6] = X0; }
    else if (k == 1) { h[3] = -X2; h[4] = 0.0; h[5] = X0; h[6] = X1; }
    else { h[3] = X1; h[4] = -X0; h[5] = 0.0; h[6] = X2; }
}

// V_o = W_o A_j^-1 for every observation o of point j (thread per observation).
template <class T>
__global__ void vmat_kernel(int64_t t, const ccov_obs* __restrict__ obs, const double* __restrict__ W,
                            const double* __restrict__ Ainv, double* __restrict__ V) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= t) return;
    const double* ai = Ainv + 6 * (int64_t)obs[o].pt;
    const double A00 = ai[0], A01 = ai[1], A02 = ai[2], A11 = ai[3], A12 = ai[4], A22 = ai[5];
    const double* w = W + 27 * o;
    double* v = V + 27 * o;
    if constexpr (std::is_same<T, double>::value) {
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const double w0 = w[3 * p], w1 = w[3 * p + 1], w2 = w[3 * p + 2];
            v[3 * p] = w0 * A00 + w1 * A01 + w2 * A02;
            v[3 * p + 1] = w0 * A01 + w1 * A11 + w2 * A12;
            v[3 * p + 2] = w0 * A02 + w1 * A12 + w2 * A22;
        }
    } else {
        const dsf a[9] = {ds_from_double(A00), ds_from_double(A01), ds_from_double(A02),
                          ds_from_double(A01), ds_from_double(A11), ds_from_double(A12),
                          ds_from_double(A02), ds_from_double(A12), ds_from_double(A22)};
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const dsf w0 = ds_from_double(w[3 * p]), w1 = ds_from_double(w[3 * p + 1]),
                      w2 = ds_from_double(w[3 * p + 2]);
#pragma unroll
            for (int q = 0; q < 3; ++q)
                v[3 * p + q] = SpAr<dsf>::value(ds_fma(ds_fma(ds_mul(w0, a[q]), w1, a[3 + q]), w2, a[6 + q]));
        }
    }
}

// Warp per block Z_ik (i >= k) that has at least one shared point.  desc =
// (i, k, first entry, entries); an entry is the observation pair (o_i, o_k)
// of one shared point (o_i = o_k on the diagonal), listed in point order.
// Lane l owns the entries e = l, l + 32, l + 64 < 81 of the block; the
// observations' V and W rows are staged in the warp's shared memory.
// Several scenes at once (cam_scene not null): camera i belongs to scene
// cam_scene[i], whose matrix starts at Z + scene_zo[s] with leading
// dimension scene_ld[s] and whose first camera is scene_co[s].
// The sums run in FP64 (the FP64 form) or in double-single arithmetic on the
// FP32 pipes (the mixed form, whose digits keep 39 bits of Z anyway; GB300
// issues FP64 FMAs at a small fraction of the FP32 rate).
template <class T>
struct SchurAr;

template <>
struct SchurAr<double> {
    typedef double V;
    static __device__ __forceinline__ double load(double x) { return x; }
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double dot3(double acc, const double* v, const double* w) {
        return acc + (v[0] * w[0] + v[1] * w[1] + v[2] * w[2]);
    }
    static __device__ __forceinline__ double value(double a) { return a; }
};

template <>
struct SchurAr<dsf> {
    typedef dsf V;
    static __device__ __forceinline__ dsf load(double x) { return ds_from_double(x); }
    static __device__ __forceinline__ dsf zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ dsf dot3(dsf acc, const dsf* v, const dsf* w) {
        acc = ds_fma(acc, v[0], w[0]);
        acc = ds_fma(acc, v[1], w[1]);
        return ds_fma(acc, v[2], w[2]);
    }
    static __device__ __forceinline__ double value(dsf a) { return (double)a.h + (double)a.l; }
};

template <class T>
__global__ void __launch_bounds__(32 * kWarps)
schur_pairs_kernel(int64_t npairs, const int4* __restrict__ desc, const int2* __restrict__ ent,
                   const double* __restrict__ V, const double* __restrict__ W, const double* __restrict__ U,
                   double* __restrict__ Z, int64_t ldz, const int* __restrict__ cam_scene,
                   const int64_t* __restrict__ scene_zo, const int64_t* __restrict__ scene_ld,
                   const int* __restrict__ scene_co) {
    typedef SchurAr<T> Ar;
    typedef typename Ar::V E;
    // four entries (observation pairs) staged at a time, so that each lane has
    // eight loads in flight; the sums still run over the entries in order
    constexpr int kU = 4;
    __shared__ E sv[kWarps][kU][2][28];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int e0 = lane, e1 = lane + 32, e2 = lane + 64;
    const int r0 = e0 / 9, c0 = e0 % 9, r1 = e1 / 9, c1 = e1 % 9, r2 = e2 / 9, c2 = e2 % 9;
    for (int64_t p = warp; p < npairs; p += nwarp) {
        const int4 d = desc[p];
        E a0 = Ar::zero(), a1 = Ar::zero(), a2 = Ar::zero();
        const int qend = d.z + d.w;
        for (int q = d.z; q < qend; q += kU) {
            const int nq = qend - q < kU ? qend - q : kU;
            double rv[kU], rw[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                rv[u] = 0.0;
                rw[u] = 0.0;
                if (u < nq && lane < 27) {
                    const int2 oo = ent[q + u];
                    rv[u] = V[27 * (int64_t)oo.x + lane];
                    rw[u] = W[27 * (int64_t)oo.y + lane];
                }
            }
            __syncwarp();
            if (lane < 27)
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    sv[wi][u][0][lane] = Ar::load(rv[u]);
                    sv[wi][u][1][lane] = Ar::load(rw[u]);
                }
            __syncwarp();
            for (int u = 0; u < nq; ++u) {
                const E* vs = sv[wi][u][0];
                const E* ws = sv[wi][u][1];
                a0 = Ar::dot3(a0, vs + 3 * r0, ws + 3 * c0);
                a1 = Ar::dot3(a1, vs + 3 * r1, ws + 3 * c1);
                if (e2 < 81) a2 = Ar::dot3(a2, vs + 3 * r2, ws + 3 * c2);
            }
        }
        const bool diag = d.x == d.y;
        double* zs = Z;
        int64_t ld = ldz, li = d.x, lk = d.y;
        if (cam_scene) {
            const int sc = cam_scene[d.x];
            zs = Z + scene_zo[sc];
            ld = scene_ld[sc];
            li -= scene_co[sc];
            lk -= scene_co[sc];
        }
        double* zb = zs + 9 * li * ld + 9 * lk;
        const double* u = U + 45 * (int64_t)d.x;
        // a diagonal block keeps its lower triangle, plus U_i (lower, row by row)
        const double s0 = Ar::value(a0), s1 = Ar::value(a1), s2 = Ar::value(a2);
        if (!diag || c0 <= r0) zb[r0 * ld + c0] = (diag ? u[r0 * (r0 + 1) / 2 + c0] : 0.0) - s0;
        if (!diag || c1 <= r1) zb[r1 * ld + c1] = (diag ? u[r1 * (r1 + 1) / 2 + c1] : 0.0) - s1;
        if (e2 < 81 && (!diag || c2 <= r2)) zb[r2 * ld + c2] = (diag ? u[r2 * (r2 + 1) / 2 + c2] : 0.0) - s2;
    }
}

// W7 = sum_j H_Xj^T A_j^-1 H_Xj and sum_j H_Xj^T H_Xj (for H^T H of the gauge
// term), per scene: the scene's wps warps (w7_warps_for(its point count), so
// that a scene's sums run in the same order alone and in a batch); warp q of
// scene s takes the points po[s] + q + wps (32 u + l) on its lane l, each lane
// forming all 28 upper entries of both sums for its points (a column B_q =
// A_j^-1 H_Xj e_q at a time, H_X = [I, -[X]x, X]); the warp then sums its
// lanes by a fixed butterfly.  Warps of all scenes are numbered one after the
// other (wpo: prefix of the scenes' warp counts; null for one scene of m points
// and wps1 warps).  Partial sums part[w][56]: W7 entries (p, q), p <= q, row
// by row, then those of H_X^T H_X.
__device__ __forceinline__ constexpr int upper_index(int p, int q) { return p * 7 - p * (p - 1) / 2 + (q - p); }

constexpr int kW7MaxWarps = 2048;

__global__ void __launch_bounds__(32 * kWarps)
w7_partial_kernel(int64_t m, const double* __restrict__ Ainv, const double* __restrict__ pts,
                  double* __restrict__ part, const int* __restrict__ po, const int64_t* __restrict__ wpo,
                  int nscenes, int wps1, int64_t total) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (warp >= total) return;
    const int sc = wpo ? find_group(wpo, nscenes, warp) : 0;
    const int64_t q0 = wpo ? warp - wpo[sc] : warp;
    const int64_t wps = wpo ? wpo[sc + 1] - wpo[sc] : wps1;
    const int64_t j0 = po ? po[sc] : 0, j1 = po ? po[sc + 1] : m;
    double w7[28], hh[28];
#pragma unroll
    for (int e = 0; e < 28; ++e) { w7[e] = 0.0; hh[e] = 0.0; }
    for (int64_t j = j0 + q0 + (int64_t)wps * lane; j < j1; j += (int64_t)wps * 32) {
        const double* ai = Ainv + 6 * j;
        const double A00 = ai[0], A01 = ai[1], A02 = ai[2], A11 = ai[3], A12 = ai[4], A22 = ai[5];
        const double X0 = pts[3 * j], X1 = pts[3 * j + 1], X2 = pts[3 * j + 2];
        double H[3][7];
#pragma unroll
        for (int k = 0; k < 3; ++k) hx_row(X0, X1, X2, k, H[k]);
#pragma unroll
        for (int q = 0; q < 7; ++q) {
            const double b0 = A00 * H[0][q] + A01 * H[1][q] + A02 * H[2][q];
            const double b1 = A01 * H[0][q] + A11 * H[1][q] + A12 * H[2][q];
            const double b2 = A02 * H[0][q] + A12 * H[1][q] + A22 * H[2][q];
#pragma unroll
            for (int p = 0; p <= q; ++p) {
                const int e = upper_index(p, q);
                w7[e] += H[0][p] * b0 + H[1][p] * b1 + H[2][p] * b2;
                hh[e] += H[0][p] * H[0][q] + H[1][p] * H[1][q] + H[2][p] * H[2][q];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 28; ++e) {
        w7[e] = warp_sum(w7[e]);
        hh[e] = warp_sum(hh[e]);
    }
    if (lane == 0) {
        double* pw = part + 56 * warp;
#pragma unroll
        for (int e = 0; e < 28; ++e) { pw[e] = w7[e]; pw[28 + e] = hh[e]; }
    }
}

// The partial sums of scene s (block s) in warp order: W7 (upper, row-major
// 7x7) at W7[128 s, 128 s + 49), H_X^T H_X at W7[128 s + 49, 128 s + 98).
// One thread per entry.
__global__ void w7_reduce_kernel(const double* __restrict__ part, double* __restrict__ W7,
                                 const int64_t* __restrict__ wpo, int wps1) {
    const int lane = threadIdx.x;
    if (lane >= 56) return;
    const int64_t w0 = wpo ? wpo[blockIdx.x] : 0, wps = wpo ? wpo[blockIdx.x + 1] - w0 : wps1;
    part += 56 * w0;
    W7 += 128 * (int64_t)blockIdx.x;
    const int e0 = lane % 28;
    int e = e0, p = 0;
    while (p < 7 && e >= 7 - p) { e -= 7 - p; ++p; }
    const int q = p + e;
    double s = 0.0;
    for (int w = 0; w < wps; ++w) s += part[56 * w + lane];
    W7[(lane < 28 ? 0 : 49) + 7 * p + q] = s;
}

// Step (b), camera part: warp per camera.  G_i = -sum_j V_ij H_Xj (the border
// column block of Z_p without H_P), summed in a fixed lane order.
template <class T>
__global__ void __launch_bounds__(32 * kWarps)
cam_schur_kernel(int64_t n, const int* __restrict__ cam_ptr, const int* __restrict__ cam_perm,
                 const ccov_obs* __restrict__ obs, const double* __restrict__ pts,
                 const double* __restrict__ V, double* __restrict__ Gp) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    typedef SpAr<T> Ar;
    typedef typename Ar::V E;
    for (int64_t i = warp; i < n; i += nwarp) {
        // G_i = -[sum V, -sum V [X]x, sum V X]
        E sV[27], sVX[9], sVK[27];
#pragma unroll
        for (int e = 0; e < 27; ++e) { sV[e] = Ar::zero(); sVK[e] = Ar::zero(); }
#pragma unroll
        for (int e = 0; e < 9; ++e) sVX[e] = Ar::zero();
        for (int k = cam_ptr[i] + lane; k < cam_ptr[i + 1]; k += 32) {
            int o = cam_perm[k];
            int j = obs[o].pt;
            const double* vo = V + 27 * (int64_t)o;   // V = W A^-1 of this observation (vmat_kernel)
            if constexpr (std::is_same<T, double>::value) {
                double X0 = pts[3 * j], X1 = pts[3 * j + 1], X2 = pts[3 * j + 2];
#pragma unroll
                for (int p = 0; p < 9; ++p) {
                    const double v0 = vo[3 * p], v1 = vo[3 * p + 1], v2 = vo[3 * p + 2];
                    sV[3 * p] += v0; sV[3 * p + 1] += v1; sV[3 * p + 2] += v2;
                    sVX[p] += v0 * X0 + v1 * X1 + v2 * X2;
                    // V [X]x, [X]x = [[0,-X2,X1],[X2,0,-X0],[-X1,X0,0]]
                    sVK[3 * p] += v1 * X2 - v2 * X1;
                    sVK[3 * p + 1] += -v0 * X2 + v2 * X0;
                    sVK[3 * p + 2] += v0 * X1 - v1 * X0;
                }
            } else {
                const dsf X0 = ds_from_double(pts[3 * j]), X1 = ds_from_double(pts[3 * j + 1]),
                          X2 = ds_from_double(pts[3 * j + 2]);
                const dsf nX0 = ds_neg(X0), nX1 = ds_neg(X1), nX2 = ds_neg(X2);
#pragma unroll
                for (int p = 0; p < 9; ++p) {
                    const dsf v0 = ds_from_double(vo[3 * p]), v1 = ds_from_double(vo[3 * p + 1]),
                              v2 = ds_from_double(vo[3 * p + 2]);
                    sV[3 * p] = ds_add(sV[3 * p], v0);
                    sV[3 * p + 1] = ds_add(sV[3 * p + 1], v1);
                    sV[3 * p + 2] = ds_add(sV[3 * p + 2], v2);
                    sVX[p] = ds_fma(ds_fma(ds_fma(sVX[p], v0, X0), v1, X1), v2, X2);
                    sVK[3 * p] = ds_fma(ds_fma(sVK[3 * p], v1, X2), v2, nX1);
                    sVK[3 * p + 1] = ds_fma(ds_fma(sVK[3 * p + 1], v0, nX2), v2, X0);
                    sVK[3 * p + 2] = ds_fma(ds_fma(sVK[3 * p + 2], v0, X1), v1, nX0);
                }
            }
        }
        double* g = Gp + 63 * i;
#pragma unroll
        for (int p = 0; p < 9; ++p) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                double a = Ar::value(Ar::sum(sV[3 * p + q]));
                double b = Ar::value(Ar::sum(sVK[3 * p + q]));
                if (lane == 0) { g[7 * p + q] = -a; g[7 * p + 3 + q] = b; }
            }
            double c = Ar::value(Ar::sum(sVX[p]));
            if (lane == 0) g[7 * p + 6] = -c;
        }
    }
}

// ---------------------------------------------------------------------------
// Step (c): H_P per camera.  Paper route: accumulate J_r^T J_r and J_r^T B over
// the camera's observations, B = -(J_t H_t + J_X H_X), and solve (3x3 SPD).
// Position rows: H_t = [-R, 0, t] (translation form), H_C = [I, -[C]x, C]
// (centre camera, C in slots 3-5 of the camera).
__global__ void __launch_bounds__(32 * kWarps)
nullspace_kernel(int64_t n, const int* __restrict__ cam_ptr, const int* __restrict__ cam_perm,
                 const ccov_obs* __restrict__ obs, const double* __restrict__ pts,
                 const double* __restrict__ cams, const double* __restrict__ prep, int route,
                 const double* __restrict__ J, double* __restrict__ HP, int* flag) {
    const int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarp) {
        const double* cp = prep + (int64_t)kCamPrep * i;
        const double* R = cp;
        const bool centre = cp[24] != 0.0;
        // position values: t (translation form) or C (centre camera)
        const double t0 = centre ? cams[9 * i + 3] : cp[9], t1 = centre ? cams[9 * i + 4] : cp[10],
                     t2 = centre ? cams[9 * i + 5] : cp[11];
        // rows of H for the position values, 3 x 7
        double Hpos[21];
        for (int p = 0; p < 3; ++p) {
            for (int q = 0; q < 3; ++q) Hpos[7 * p + q] = centre ? (p == q ? 1.0 : 0.0) : -R[3 * p + q];
            Hpos[7 * p + 6] = p == 0 ? t0 : (p == 1 ? t1 : t2);
        }
        // -[C]x for the centre camera, 0 for the translation form
        Hpos[3] = 0.0;                 Hpos[4] = centre ? t2 : 0.0;  Hpos[5] = centre ? -t1 : 0.0;
        Hpos[10] = centre ? -t2 : 0.0; Hpos[11] = 0.0;               Hpos[12] = centre ? t0 : 0.0;
        Hpos[17] = centre ? t1 : 0.0;  Hpos[18] = centre ? -t0 : 0.0; Hpos[19] = 0.0;
        double Hr[21];
        if (route == CCOV_NULL_CLOSED) {
            // H_r = [0, -J_r^-1(r), 0], J_r^-1 = I + 1/2 K + c K^2
            const double* rv = cams + 9 * i;
            double th2 = rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2], th = sqrt(th2);
            double c = th < 1e-3 ? 1.0 / 12.0 + th2 / 720.0
                                 : 1.0 / th2 - (1.0 + cos(th)) / (2.0 * th * sin(th));
            double K[9] = {0, -rv[2], rv[1], rv[2], 0, -rv[0], -rv[1], rv[0], 0};
            for (int p = 0; p < 3; ++p)
                for (int q = 0; q < 3; ++q) {
                    double k2 = K[3 * p] * K[q] + K[3 * p + 1] * K[3 + q] + K[3 * p + 2] * K[6 + q];
                    Hr[7 * p + 3 + q] = -((p == q) + 0.5 * K[3 * p + q] + c * k2);
                    Hr[7 * p + q] = 0.0;
                }
            for (int p = 0; p < 3; ++p) Hr[7 * p + 6] = 0.0;
        } else {
            double jj[6] = {0, 0, 0, 0, 0, 0};
            double jb[21];
#pragma unroll
            for (int e = 0; e < 21; ++e) jb[e] = 0.0;
            for (int k = cam_ptr[i] + lane; k < cam_ptr[i + 1]; k += 32) {
                int o = cam_perm[k];
                int j = obs[o].pt;
                double X0 = pts[3 * j], X1 = pts[3 * j + 1], X2 = pts[3 * j + 2];
                double Jc[18], Jp[6];
                if (J) {   // kept by step (a) (unwhitened)
                    const double* jo = J + 24 * (int64_t)o;
#pragma unroll
                    for (int e = 0; e < 18; ++e) Jc[e] = jo[e];
#pragma unroll
                    for (int e = 0; e < 6; ++e) Jp[e] = jo[18 + e];
                } else {
                    obs_jacobian(cp, X0, X1, X2, Jc, Jp);
                }
#pragma unroll
                for (int row = 0; row < 2; ++row) {
                    const double* jr = Jc + 9 * row;       // d/dr (3)
                    const double* jt = Jc + 9 * row + 3;   // d/dt (3)
                    const double* jx = Jp + 3 * row;
                    // B row = -(J_pos H_pos + J_X H_X), H_X = [I, -[X]x, X]
                    double b[7];
                    for (int q = 0; q < 7; ++q) b[q] = -(jt[0] * Hpos[q] + jt[1] * Hpos[7 + q] + jt[2] * Hpos[14 + q]);
                    for (int q = 0; q < 3; ++q) b[q] -= jx[q];
                    // J_X (-[X]x): columns of -[X]x = [[0,X2,-X1],[-X2,0,X0],[X1,-X0,0]]
                    b[3] -= jx[1] * (-X2) + jx[2] * X1;
                    b[4] -= jx[0] * X2 + jx[2] * (-X0);
                    b[5] -= jx[0] * (-X1) + jx[1] * X0;
                    b[6] -= jx[0] * X0 + jx[1] * X1 + jx[2] * X2;
                    jj[0] += jr[0] * jr[0]; jj[1] += jr[0] * jr[1]; jj[2] += jr[0] * jr[2];
                    jj[3] += jr[1] * jr[1]; jj[4] += jr[1] * jr[2]; jj[5] += jr[2] * jr[2];
#pragma unroll
                    for (int p = 0; p < 3; ++p)
#pragma unroll
                        for (int q = 0; q < 7; ++q) jb[7 * p + q] += jr[p] * b[q];
                }
            }
#pragma unroll
            for (int e = 0; e < 6; ++e) jj[e] = warp_sum(jj[e]);
#pragma unroll
            for (int e = 0; e < 21; ++e) jb[e] = warp_sum(jb[e]);
            // Cholesky of J_r^T J_r, then two triangular solves per column
            double l00 = sqrt(jj[0]);
            double l10 = jj[1] / l00, l20 = jj[2] / l00;
            double d11 = jj[3] - l10 * l10;
            double l11 = sqrt(d11);
            double l21 = (jj[4] - l20 * l10) / l11;
            double d22 = jj[5] - l20 * l20 - l21 * l21;
            double l22 = sqrt(d22);
            if (!(d11 > 0.0) || !(d22 > 0.0)) {
                if (lane == 0) set_flag(flag, DEV_SINGULAR_JR, (int)i);
            }
            for (int q = 0; q < 7; ++q) {
                double y0 = jb[q] / l00;
                double y1 = (jb[7 + q] - l10 * y0) / l11;
                double y2 = (jb[14 + q] - l20 * y0 - l21 * y1) / l22;
                double x2 = y2 / l22;
                double x1 = (y1 - l21 * x2) / l11;
                double x0 = (y0 - l10 * x1 - l20 * x2) / l00;
                Hr[q] = x0; Hr[7 + q] = x1; Hr[14 + q] = x2;
            }
        }
        if (lane == 0) {
            double* h = HP + 63 * i;
            for (int e = 0; e < 21; ++e) h[e] = Hr[e];
            for (int e = 0; e < 21; ++e) h[21 + e] = Hpos[e];
            for (int e = 42; e < 63; ++e) h[e] = 0.0;
        }
    }
}

int grid_for(int64_t items, int per_cta) {
    int64_t g = (items + per_cta - 1) / per_cta;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

// Added observations (the Woodbury update of Sec. 5), thread per added
// observation o of point j by camera i: the whitened Jacobian rows at the
// current parameters, Jc (2 x 9) and Jp (2 x 3), JA = Jp A_j^-1 (2 x 3),
// Psi = JA H_X,j (2 x 7), and the columns 2o, 2o + 1 of Phi = K Psi^T
// (7 rows of leading dimension ldphi), K = (Lambda^-1 + W7)^-1.
__global__ void upd_obs_kernel(int64_t k, const ccov_obs* __restrict__ add, const double* __restrict__ add_cov,
                               double sigma, const double* __restrict__ prep, const double* __restrict__ pts,
                               const double* __restrict__ Ainv, const double* __restrict__ K, int64_t ldphi,
                               double* __restrict__ Jc, double* __restrict__ Jp, double* __restrict__ JA,
                               double* __restrict__ Psi, double* __restrict__ Phi, int* flag) {
    const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (o >= k) return;
    const int i = add[o].cam, j = add[o].pt;
    const double X0 = pts[3 * (int64_t)j], X1 = pts[3 * (int64_t)j + 1], X2 = pts[3 * (int64_t)j + 2];
    double jc[18], jp[6];
    const double depth = obs_jacobian(prep + (int64_t)kCamPrep * i, X0, X1, X2, jc, jp);
    if (!(depth > 0.0)) set_flag(flag, DEV_BEHIND, (int)o);
    whiten(jc, jp, sigma, add_cov ? add_cov + 4 * o : nullptr);
    const double* ai = Ainv + 6 * (int64_t)j;
    const double Am[9] = {ai[0], ai[1], ai[2], ai[1], ai[3], ai[4], ai[2], ai[4], ai[5]};
    double ja[6], psi[14];
#pragma unroll
    for (int row = 0; row < 2; ++row)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            ja[3 * row + q] = jp[3 * row] * Am[q] + jp[3 * row + 1] * Am[3 + q] + jp[3 * row + 2] * Am[6 + q];
    for (int e = 0; e < 14; ++e) psi[e] = 0.0;
    for (int l = 0; l < 3; ++l) {
        double h[7];
        hx_row(X0, X1, X2, l, h);
#pragma unroll
        for (int row = 0; row < 2; ++row)
#pragma unroll
            for (int p = 0; p < 7; ++p) psi[7 * row + p] += ja[3 * row + l] * h[p];
    }
    for (int e = 0; e < 18; ++e) Jc[18 * o + e] = jc[e];
    for (int e = 0; e < 6; ++e) { Jp[6 * o + e] = jp[e]; JA[6 * o + e] = ja[e]; }
    for (int e = 0; e < 14; ++e) Psi[14 * o + e] = psi[e];
    for (int row = 0; row < 2; ++row)
        for (int q = 0; q < 7; ++q) {
            double v = 0.0;
            for (int p = 0; p < 7; ++p) v += K[7 * q + p] * psi[7 * row + p];
            Phi[q * ldphi + 2 * o + row] = v;
        }
}

}  // namespace

void launch_cam_prep(Ctx& c) {
    cam_prep_kernel<<<(int)((c.n + 127) / 128), 128, 0, c.stream>>>(c.n, c.d_cams, c.d_camprep,
                                                                  c.opt.camera_model == CCOV_CAMERA_CENTRE8);
    CCOV_LAUNCH_CHECK(c);
}

void launch_point_info(Ctx& c) {
    // the observations' shares of A go into V (t x 27), which step (b) fills later
    obs_info_kernel<<<(unsigned)((c.t + 127) / 128), 128, 0, c.stream>>>(c.t, c.d_obs, c.d_pts, c.d_camprep,
                                                                         c.sigma, c.d_obscov, c.d_W, c.d_V,
                                                                         c.d_J, c.d_flag);
    CCOV_LAUNCH_CHECK(c);
    point_ainv_kernel<<<(unsigned)((c.m + 127) / 128), 128, 0, c.stream>>>(c.m, c.d_pt_ptr, c.d_V, c.d_Ainv,
                                                                           c.d_flag);
    CCOV_LAUNCH_CHECK(c);
}

void launch_cam_info(Ctx& c) {
    if (c.opt.precision == CCOV_PREC_MIXED)
        cam_info_kernel<dsf><<<grid_for(c.n, kWarps), 32 * kWarps, 0, c.stream>>>(
            c.n, c.d_cam_ptr, c.d_cam_perm, c.d_J, c.d_camprep, c.sigma, c.d_obscov, c.d_U);
    else
        cam_info_kernel<double><<<grid_for(c.n, kWarps), 32 * kWarps, 0, c.stream>>>(
            c.n, c.d_cam_ptr, c.d_cam_perm, c.d_J, c.d_camprep, c.sigma, c.d_obscov, c.d_U);
    CCOV_LAUNCH_CHECK(c);
}

void launch_schur(Ctx& c) {
    if (c.opt.precision == CCOV_PREC_MIXED)
        vmat_kernel<dsf><<<(int)((c.t + 255) / 256), 256, 0, c.stream>>>(c.t, c.d_obs, c.d_W, c.d_Ainv, c.d_V);
    else
        vmat_kernel<double><<<(int)((c.t + 255) / 256), 256, 0, c.stream>>>(c.t, c.d_obs, c.d_W, c.d_Ainv, c.d_V);
    CCOV_LAUNCH_CHECK(c);
    if (c.opt.precision == CCOV_PREC_MIXED)
        schur_pairs_kernel<dsf><<<grid_for(c.npairs, kWarps), 32 * kWarps, 0, c.stream>>>(
            c.npairs, c.d_pair_desc, c.d_pair_ent, c.d_V, c.d_W, c.d_U, c.d_Z, c.Np, c.d_cam_scene, c.d_scene_zo,
            c.d_scene_ld, c.d_scene_co);
    else
        schur_pairs_kernel<double><<<grid_for(c.npairs, kWarps), 32 * kWarps, 0, c.stream>>>(
            c.npairs, c.d_pair_desc, c.d_pair_ent, c.d_V, c.d_W, c.d_U, c.d_Z, c.Np, c.d_cam_scene, c.d_scene_zo,
            c.d_scene_ld, c.d_scene_co);
    CCOV_LAUNCH_CHECK(c);
    const int64_t total = c.d_scene_wpo ? c.w7_total : c.w7_wps;
    w7_partial_kernel<<<(unsigned)((total + kWarps - 1) / kWarps), 32 * kWarps, 0, c.stream>>>(
        c.m, c.d_Ainv, c.d_pts, c.d_w7part, c.d_scene_po, c.d_scene_wpo, c.nscenes, c.w7_wps, total);
    CCOV_LAUNCH_CHECK(c);
    w7_reduce_kernel<<<c.nscenes, 64, 0, c.stream>>>(c.d_w7part, c.d_W7, c.d_scene_wpo, c.w7_wps);
    CCOV_LAUNCH_CHECK(c);
    if (c.opt.precision == CCOV_PREC_MIXED)
        cam_schur_kernel<dsf><<<grid_for(c.n, kWarps), 32 * kWarps, 0, c.stream>>>(
            c.n, c.d_cam_ptr, c.d_cam_perm, c.d_obs, c.d_pts, c.d_V, c.d_Gp);
    else
        cam_schur_kernel<double><<<grid_for(c.n, kWarps), 32 * kWarps, 0, c.stream>>>(
            c.n, c.d_cam_ptr, c.d_cam_perm, c.d_obs, c.d_pts, c.d_V, c.d_Gp);
    CCOV_LAUNCH_CHECK(c);
}

int w7_warps_for(int64_t m) {
    const int64_t w = (m + 511) / 512;   // about 16 points per lane
    return (int)(w < 1 ? 1 : (w > kW7MaxWarps ? kW7MaxWarps : w));
}

void launch_nullspace(Ctx& c, bool kept_jacobians) {
    nullspace_kernel<<<grid_for(c.n, kWarps), 32 * kWarps, 0, c.stream>>>(
        c.n, c.d_cam_ptr, c.d_cam_perm, c.d_obs, c.d_pts, c.d_cams, c.d_camprep,
        c.opt.nullspace_route, kept_jacobians ? c.d_J : nullptr, c.d_HP, c.d_flag);
    CCOV_LAUNCH_CHECK(c);
}

void launch_upd_obs(Ctx& c, int64_t k, const ccov_obs* add, const double* add_cov, int64_t ldphi, double* Jc,
                    double* Jp, double* JA, double* Psi, double* Phi) {
    upd_obs_kernel<<<(unsigned)((k + 127) / 128), 128, 0, c.stream>>>(
        k, add, add_cov, c.sigma, c.d_camprep, c.d_pts, c.d_Ainv, c.d_small, ldphi, Jc, Jp, JA, Psi, Phi, c.d_flag);
    CCOV_LAUNCH_CHECK(c);
}

}  // namespace ccov

// Learned covariance surrogate (include/ccov_surrogate.h): per-camera
// features read from the reduced camera matrix, training targets from exact
// covariance blocks, and a 64-256-256-256-45 ReLU network whose forward and
// backward products run on the tensor cores (tcgen05, bf16 operands, fp32
// accumulation in TMEM, operands moved by bulk copies).
//
// Operand layout.  Every bf16 matrix [R x K] that feeds the tensor cores is
// stored in the order a no-swizzle K-major operand is read: per 16-wide
// slice of K, all R rows in groups of 8, each group two 8 x 8 core matrices
// (16-byte rows) along K.  A 64-wide K chunk of a 128-row tile is then four
// contiguous 4 KB pieces, and a chunk of a whole matrix one piece.  Each
// producer writes both a matrix and its transpose in this layout, so that the
// two backward products read plain K-major operands as well:
//   forward   z_l   = a_{l-1} W_l^T          A = a_{l-1} [B x in],  B = W_l   [out x in]
//   dW        dW_l  = g_l^T a_{l-1}          A = g_l^T   [out x B], B = a^T   [in x B]
//   dX        g_l-1 = (g_l W_l) * [a > 0]    A = g_l     [B x out], B = W_l^T [in x out]
// Widths are padded to 128 (input 64 -> 128, output 45 -> 128) with zero
// weights, which receive zero gradients and stay zero under Adam.
//
// The paper has no counterpart; Sec. 1 names the uses of camera covariances
// that such a screen serves.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ccov_internal.cuh"
#include "tc_ptx.cuh"
#include "../../include/ccov_surrogate.h"

namespace ccov {
namespace surr {

using namespace ptx;
typedef __nv_bfloat16 bf16;

constexpr int kIn = CCOV_SURR_FEATURES, kHid = CCOV_SURR_HIDDEN, kOut = CCOV_SURR_OUTPUTS;
constexpr int kInP = 128, kOutP = 128;            // padded operand widths
constexpr int kChunk = 64;                        // K per pipeline stage
constexpr int kStages = 4;
constexpr int kABytes = 128 * kChunk * 2;         // 16 KB
constexpr int kBBytesMax = 256 * kChunk * 2;      // 32 KB
constexpr int kStageBytes = kABytes + kBBytesMax;
constexpr int kGemmThreads = 192;                 // producer, MMA, 4 epilogue warps
constexpr size_t kGemmSmem = 1024 + (size_t)kStages * kStageBytes + 8 * (2 * kStages + 1) + 16;
constexpr int kNorm = CCOV_SURR_NORM;

// master parameter segments (padded): W1 b1 W2 b2 W3 b3 W4 b4
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + 256 * kInP;
constexpr int64_t kOffW2 = kOffB1 + 256, kOffB2 = kOffW2 + 256 * 256;
constexpr int64_t kOffW3 = kOffB2 + 256, kOffB3 = kOffW3 + 256 * 256;
constexpr int64_t kOffW4 = kOffB3 + 256, kOffB4 = kOffW4 + kOutP * 256;
constexpr int64_t kPadParams = kOffB4 + kOutP;
static_assert(CCOV_SURR_PARAMS == kIn * kHid + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut, "parameter count");
static_assert(kHid == 256, "hidden width is fixed by the tile shapes below");

__host__ __device__ __forceinline__ int64_t kb_off(int64_t r, int64_t k, int64_t R) {
    return (((k >> 4) * R) << 4) + ((r >> 3) << 7) + (((k >> 3) & 1) << 6) + ((r & 7) << 3) + (k & 7);
}

enum Epi : int { EPI_RELU = 0, EPI_OUT = 1, EPI_DX = 2, EPI_DW = 3 };

struct GemmP {
    const bf16* A;        // [a_rows x K], this CTA's 128 rows from 128 * blockIdx.x
    int64_t a_rows;
    const bf16* B;        // [N x K], all N rows
    int N;                // 128 or 256
    int K;                // multiple of kChunk
    int chunks_per_split; // K chunks of one blockIdx.y
    int epi;
    const float* bias;    // RELU, OUT
    bf16* out_n;          // RELU, DX: [a_rows x N]
    bf16* out_t;          // RELU, DX: [N x a_rows]
    const bf16* mask;     // DX: [a_rows x N], the activation the gradient passes through
    float* out_f;         // OUT: row-major, ld N; DW: this split's partial [a_rows x N] at
                          // out_f + blockIdx.y a_rows N (summed in order afterwards)
    float* db;            // DX: partial column sums of the output, row 4 blockIdx.x + quarter
                          // of a [tiles 4 x N] array (summed in order afterwards)
    int* flag;
};

__device__ __forceinline__ uint4 pack8(const float* x) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
    return *reinterpret_cast<uint4*>(h);
}

__device__ __forceinline__ void unpack8(uint4 u, float* x) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 f = __bfloat1622float2(h[j]);
        x[2 * j] = f.x;
        x[2 * j + 1] = f.y;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One 128 x N output tile per CTA over K chunks [y * cps, (y + 1) * cps).
// Warp 0 lane 0 issues the bulk copies, warp 1 allocates TMEM and lane 0
// issues the MMAs, warps 2..5 drain TMEM (warp w reads lanes 32 (w % 4)).
__global__ void __launch_bounds__(kGemmThreads, 1) mlp_gemm_kernel(GemmP g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(base + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* accf = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(accf + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = 128 * (int64_t)blockIdx.x;
    const int total = g.K / kChunk;
    const int c_begin = blockIdx.y * g.chunks_per_split;
    const int c_end = min(c_begin + g.chunks_per_split, total);
    const int nchunks = c_end - c_begin;
    const uint32_t b_bytes = (uint32_t)g.N * kChunk * 2;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        mbar_init(accf, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            for (int c = 0; c < nchunks; ++c) {
                if (!mbar_wait(empty + stage, phase ^ 1, g.flag, 21)) break;
                unsigned char* st = base + stage * kStageBytes;
                mbar_expect_tx(full + stage, (uint32_t)kABytes + b_bytes);
                const int64_t k0 = (int64_t)(c_begin + c) * kChunk;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    bulk_load(st + s * 4096, g.A + kb_off(m0, k0 + 16 * s, g.a_rows), 4096, full + stage);
                bulk_load(st + kABytes, g.B + kb_off(0, k0, g.N), b_bytes, full + stage);
                if (++stage == kStages) { stage = 0; phase ^= 1; }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            const uint32_t idesc = idesc_bf16(128, g.N);
            for (int c = 0; c < nchunks; ++c) {
                if (!mbar_wait(full + stage, phase, g.flag, 22)) break;
                tc_fence_after();
                const uint32_t sa = smem_u32(base + stage * kStageBytes), sb = sa + kABytes;
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    mma_bf16(tmem, smem_desc_kmajor(sa + 4096 * s), smem_desc_kmajor(sb + (uint32_t)(g.N * 32 * s)),
                             idesc, (c | s) ? 1 : 0);
                mma_commit(empty + stage);
                if (++stage == kStages) { stage = 0; phase ^= 1; }
            }
            mma_commit(accf);  // completes once every MMA issued above has
        }
    } else {
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;
        const int64_t grow = m0 + r;
        bool ok = mbar_wait(accf, 0, g.flag, 23);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        if (ok && nchunks > 0) {
            const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
            for (int c0 = 0; c0 < g.N; c0 += 8) {
                float v[8];
                tmem_ld8(trow + (uint32_t)c0, v);
                tmem_wait_ld();
                tmem_regs_after_wait<8>(v);
                if (g.epi == EPI_RELU || g.epi == EPI_DX) {
                    if (g.epi == EPI_RELU) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) v[j] = fmaxf(v[j] + g.bias[c0 + j], 0.f);
                    } else {
                        float a[8];
                        unpack8(*reinterpret_cast<const uint4*>(g.mask + kb_off(grow, c0, g.a_rows)), a);
#pragma unroll
                        for (int j = 0; j < 8; ++j) v[j] = a[j] > 0.f ? v[j] : 0.f;
                    }
                    const uint4 h = pack8(v);
                    *reinterpret_cast<uint4*>(g.out_n + kb_off(grow, c0, g.a_rows)) = h;
                    const bf16* hb = reinterpret_cast<const bf16*>(&h);
#pragma unroll
                    for (int j = 0; j < 8; ++j) g.out_t[kb_off(c0 + j, grow, g.N)] = hb[j];
                    if (g.epi == EPI_DX) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float s = warp_sum(v[j]);
                            if (lane == 0) g.db[(4 * (int64_t)blockIdx.x + quarter) * g.N + c0 + j] = s;
                        }
                    }
                } else if (g.epi == EPI_OUT) {
                    float4* o = reinterpret_cast<float4*>(g.out_f + grow * g.N + c0);
                    o[0] = make_float4(v[0] + g.bias[c0], v[1] + g.bias[c0 + 1], v[2] + g.bias[c0 + 2],
                                       v[3] + g.bias[c0 + 3]);
                    o[1] = make_float4(v[4] + g.bias[c0 + 4], v[5] + g.bias[c0 + 5], v[6] + g.bias[c0 + 6],
                                       v[7] + g.bias[c0 + 7]);
                } else {
                    float* o = g.out_f + (int64_t)blockIdx.y * g.a_rows * g.N + grow * g.N + c0;
#pragma unroll
                    for (int j = 0; j < 8; ++j) o[j] = v[j];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.N));
    }
}

// Size scale of the output head: feature 48 (10 / sqrt(n)) when positive,
// else 1.  The network learns target / s, and its output is multiplied by s:
// around the base with the gauge term the remainder shrinks about as
// n^-1/2, so the scaled target keeps its size from scene to scene.  Feature
// 48 is not a network input (its column of the input operand is zero), so
// that no input leaves the training range on larger scenes.
constexpr int kSizeFeature = 48;
__device__ __forceinline__ float head_scale(const float* feat_row) {
    const float v = feat_row[kSizeFeature];
    return v > 0.f ? v : 1.f;
}

// Gather rows idx[b] of the raw features and targets, standardise (targets
// after the division by the head's size scale), and write the input operand
// (and its transpose) as bf16; rows b >= B are zero.  The row offset into idx
// is ctr[1] * B (the step within a training call).
__global__ void pack_kernel(const float* __restrict__ feat, const float* __restrict__ targ,
                            const int* __restrict__ idx, int64_t n, const int* __restrict__ ctr, int B, int Bp,
                            const float* __restrict__ norm, bf16* __restrict__ A0n, bf16* __restrict__ A0t,
                            float* __restrict__ T, int* flag) {
    const int b = blockIdx.x, k = threadIdx.x;  // 128 threads
    int64_t src = -1;  // -1: a padding row (zero)
    if (b < B) {
        src = idx ? idx[(int64_t)(ctr ? ctr[1] : 0) * B + b] : b;
        if (src < 0 || src >= n) {  // out of range: flagged, row left zero
            if (k == 0) set_flag(flag, DEV_BAD_INDEX, b);
            src = -1;
        }
    }
    float x = 0.f;  // feature 48 sets only the head's size scale: its input column stays zero
    if (src >= 0 && k < kIn && k != kSizeFeature) x = (feat[(int64_t)src * kIn + k] - norm[k]) / norm[kIn + k];
    const bf16 h = __float2bfloat16_rn(x);
    A0n[kb_off(b, k, Bp)] = h;
    A0t[kb_off(k, b, kInP)] = h;
    if (T && k < kOut) {
        float t = 0.f;
        if (src >= 0)
            t = (targ[(int64_t)src * kOut + k] / head_scale(feat + src * kIn) - norm[2 * kIn + k]) /
                norm[2 * kIn + kOut + k];
        T[(int64_t)b * kOut + k] = t;
    }
}

// Output gradient of the mean squared error: g = 2 (y - t) / (B * 45) for the
// 45 outputs of real rows, zero elsewhere, as bf16 operands (and transpose);
// db4 and the loss accumulate in fp32.  64 rows per block, thread = column.
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ T, int B, int Bp,
                            bf16* __restrict__ Gn, bf16* __restrict__ Gt, float* __restrict__ part) {
    const int o = threadIdx.x;  // 128 threads
    const float inv = 2.f / ((float)B * (float)kOut);
    float acc_db = 0.f, acc_l = 0.f;
    for (int rr = 0; rr < 64; ++rr) {
        const int b = blockIdx.x * 64 + rr;
        float gv = 0.f;
        if (b < B && o < kOut) {
            const float res = Y[(int64_t)b * kOutP + o] - T[(int64_t)b * kOut + o];
            gv = inv * res;
            acc_l += res * res;
        }
        const bf16 h = __float2bfloat16_rn(gv);
        Gn[kb_off(b, o, Bp)] = h;
        Gt[kb_off(o, b, kOutP)] = h;
        acc_db += gv;
    }
    // this block's share: db4 partials [0, 128), the loss at 128
    part[(int64_t)blockIdx.x * 129 + o] = o < kOut ? acc_db : 0.f;
    __shared__ float red[4];
    acc_l = warp_sum(acc_l);
    if ((o & 31) == 0) red[o >> 5] = acc_l;
    __syncthreads();
    if (o == 0) part[(int64_t)blockIdx.x * 129 + 128] = (red[0] + red[1] + red[2] + red[3]) / ((float)B * (float)kOut);
}

// out[e] = sum over z < nz, in order, of part[z * stride + e] (e < count).
__global__ void sum_parts_kernel(const float* __restrict__ part, int nz, int64_t stride, int64_t count,
                                 float* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    float v = 0.f;
    for (int z = 0; z < nz; ++z) v += part[(int64_t)z * stride + e];
    out[e] = v;
}

// The loss of the step (block shares summed in order) into losses[ctr[1]].
__global__ void loss_sum_kernel(const float* __restrict__ part, int nb, float* __restrict__ losses,
                                const int* __restrict__ ctr) {
    if (threadIdx.x != 0) return;
    float v = 0.f;
    for (int b = 0; b < nb; ++b) v += part[(int64_t)b * 129 + 128];
    losses[ctr ? ctr[1] : 0] = v;
}

struct Seg {
    int64_t off, rows, cols;  // rows = outputs, cols = inputs (cols = 0: bias)
};

struct Segs {
    Seg s[8];
    bf16* wb[4];   // [out_p x in_p] operand of the forward product
    bf16* wt[4];   // [in_p x out_p] operand of the input-gradient product (layer 1: unused)
};

__device__ __forceinline__ void write_bf16(const Segs& S, int seg, int64_t e, float v) {
    if (seg & 1) return;  // biases stay fp32
    const int l = seg >> 1;
    const int64_t o = e / S.s[seg].cols, i = e - o * S.s[seg].cols;
    const bf16 h = __float2bfloat16_rn(v);
    S.wb[l][kb_off(o, i, S.s[seg].rows)] = h;
    if (S.wt[l]) S.wt[l][kb_off(i, o, S.s[seg].cols)] = h;
}

__device__ __forceinline__ int seg_of(const Segs& S, int64_t e) {
    int seg = 0;
#pragma unroll
    for (int k = 1; k < 8; ++k)
        if (e >= S.s[k].off) seg = k;
    return seg;
}

// Adam on every (padded) parameter; the step count t = ctr[0] + 1.  The last
// block to finish advances ctr[0] (and the in-call step ctr[1]).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int64_t P, float lr, Segs S, int* ctr,
                            unsigned* __restrict__ done) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int t = ctr[0] + 1;
    if (e < P) {
        const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
        const float gr = grad[e];
        const float mm = 0.9f * m[e] + 0.1f * gr;
        const float vv = 0.999f * v[e] + 0.001f * gr * gr;
        m[e] = mm;
        v[e] = vv;
        const float val = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
        p[e] = val;
        const int seg = seg_of(S, e);
        write_bf16(S, seg, e - S.s[seg].off, val);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned k = atomicAdd(done, 1u);
        if (k == gridDim.x - 1) {
            ctr[0] = t;
            ctr[1] += 1;
            *done = 0u;
            __threadfence();
        }
    }
}

// bf16 operand copies of the master parameters.
__global__ void cast_kernel(const float* __restrict__ p, int64_t P, Segs S) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= P) return;
    const int seg = seg_of(S, e);
    write_bf16(S, seg, e - S.s[seg].off, p[e]);
}

// Column mean and population deviation of x (n x w), each row divided by the
// head's size scale of feat's row when feat is given, into mu[w], sd[w] (a
// deviation below 1e-6 becomes 1); one block per column, fp64 sums.
__device__ __forceinline__ double norm_value(const float* x, const float* feat, int64_t r, int w, int col) {
    const double v = x[r * w + col];
    return feat ? v / head_scale(feat + r * kIn) : v;
}

__global__ void norm_kernel(const float* __restrict__ x, const float* __restrict__ feat, int64_t n, int w,
                            float* __restrict__ mu, float* __restrict__ sd) {
    const int col = blockIdx.x;
    __shared__ double red[2][8];
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += norm_value(x, feat, r, w, col);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = s;
    __syncthreads();
    double mean = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) mean += red[0][k];
    mean /= (double)n;
    double q = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double d = norm_value(x, feat, r, w, col) - mean;
        q += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0) red[1][threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double var = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) var += red[1][k];
        const double dev = sqrt(var / (double)n);
        mu[col] = (float)mean;
        sd[col] = dev < 1e-6 ? 1.f : (float)dev;
    }
}

// ---- features (warp per camera) ----
__device__ __forceinline__ void camera_centre(const double* cp, double* c) {
    // c = -R^T t
    for (int a = 0; a < 3; ++a) c[a] = -(cp[a] * cp[9] + cp[3 + a] * cp[10] + cp[6 + a] * cp[11]);
}

// Z_ii = U_i - sum over the camera's observations of W_ij A_j^-1 W_ij^T,
// accumulated from the information blocks (no dense Z needed): lanes take
// the observations, the 45 lower-triangle entries are reduced over the warp.
constexpr int kFeatWarps = 8;

__global__ void __launch_bounds__(32 * kFeatWarps)
features_kernel(int64_t n, const double* __restrict__ U, const double* __restrict__ W,
                const double* __restrict__ Ainv, const int* __restrict__ cam_ptr, const int* __restrict__ cam_perm,
                const ccov_obs* __restrict__ obs, const int* __restrict__ pt_ptr,
                const double* __restrict__ camprep, double* __restrict__ csum, float* __restrict__ feat,
                double* __restrict__ scale, int* flag) {
    __shared__ double zsh[kFeatWarps][45];
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double* zs = zsh[threadIdx.x >> 5];  // Z_ii, lower triangle row by row
    const int o0 = cam_ptr[i], o1 = cam_ptr[i + 1];
    {
        double acc[45];
#pragma unroll
        for (int e = 0; e < 45; ++e) acc[e] = 0.0;
        for (int q = o0 + lane; q < o1; q += 32) {
            const int o = cam_perm[q];
            const int j = obs[o].pt;
            const double* w = W + 27 * (int64_t)o;
            const double* a = Ainv + 6 * (int64_t)j;
            const double Am[9] = {a[0], a[1], a[2], a[1], a[3], a[4], a[2], a[4], a[5]};
            double V[27];  // W A^-1
#pragma unroll
            for (int r = 0; r < 9; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    V[3 * r + k] = w[3 * r] * Am[k] + w[3 * r + 1] * Am[3 + k] + w[3 * r + 2] * Am[6 + k];
            int e = 0;
#pragma unroll
            for (int r = 0; r < 9; ++r)
#pragma unroll
                for (int c = 0; c <= r; ++c, ++e)
                    acc[e] += V[3 * r] * w[3 * c] + V[3 * r + 1] * w[3 * c + 1] + V[3 * r + 2] * w[3 * c + 2];
        }
#pragma unroll
        for (int e = 0; e < 45; ++e) {
            double v = acc[e];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) zs[e] = U[45 * i + e] - v;
        }
    }
    __syncwarp();
    double d = 1.0;
    if (lane < 9) {
        const double zz = zs[lane * (lane + 1) / 2 + lane];
        if (!(zz > 0.0)) set_flag(flag, DEV_NOT_SPD, (int)(9 * i + lane));
        d = zz > 0.0 ? sqrt(zz) : 1.0;
        feat[i * kIn + 36 + lane] = (float)log(d);
    }
    if (lane == 0) {
        // L_z: Cholesky factor of Z_ii, written as a full 9 x 9 row-major block
        double L[45];
        bool spd = true;
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c <= r; ++c) {
                double v = zs[r * (r + 1) / 2 + c];
                for (int k = 0; k < c; ++k) v -= L[r * (r + 1) / 2 + k] * L[c * (c + 1) / 2 + k];
                if (r == c) {
                    if (!(v > 0.0)) { spd = false; v = 1.0; }
                    L[r * (r + 1) / 2 + r] = sqrt(v);
                } else {
                    L[r * (r + 1) / 2 + c] = v / L[c * (c + 1) / 2 + c];
                }
            }
        if (!spd) set_flag(flag, DEV_NOT_SPD, (int)(9 * i));
        double* o = scale + 81 * i;
        for (int r = 0; r < 9; ++r)
            for (int c = 0; c < 9; ++c) o[9 * r + c] = c <= r ? L[r * (r + 1) / 2 + c] : 0.0;
    }
    double dall[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) dall[k] = __shfl_sync(0xffffffffu, d, k);
    // C_kl, k < l, row by row: pair p -> (k, l); Z_kl = Z_lk from the lower triangle
    for (int p = lane; p < 36; p += 32) {
        int k = 0, rem = p;
        while (rem >= 8 - k) { rem -= 8 - k; ++k; }
        const int l = k + 1 + rem;
        feat[i * kIn + p] = (float)(zs[l * (l + 1) / 2 + k] / (dall[k] * dall[l]));
    }
    double slog = 0.0, two = 0.0;
    for (int q = o0 + lane; q < o1; q += 32) {
        const int j = obs[cam_perm[q]].pt;
        const int L = pt_ptr[j + 1] - pt_ptr[j];
        slog += log((double)L);
        two += (L == 2) ? 1.0 : 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        slog += __shfl_xor_sync(0xffffffffu, slog, o);
        two += __shfl_xor_sync(0xffffffffu, two, o);
    }
    if (lane == 0) {
        const double cnt = (double)(o1 - o0);
        float* f = feat + i * kIn;
        f[45] = (float)log(cnt);
        f[46] = (float)(slog / cnt);
        f[47] = (float)(two / cnt);
        f[48] = (float)(10.0 / sqrt((double)n));
    }
    if (lane >= 17) feat[i * kIn + 32 + lane] = 0.f;  // [49, 64); 49 is written by centre_feature_kernel
}

// The mean camera centre (csum[0..2], as sums) and the sum of squared
// distances from it (csum[3]): one block of 1024 threads, each a strided
// share of the cameras, reduced by a fixed tree, so that the features are the
// same bits on every run.
__global__ void __launch_bounds__(1024) centre_stats_kernel(int64_t n, const double* __restrict__ camprep,
                                                           double* __restrict__ csum) {
    __shared__ double red[4][32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t i = tid; i < n; i += 1024) {
        double c[3];
        camera_centre(camprep + kCamPrep * i, c);
        for (int a = 0; a < 3; ++a) s[a] += c[a];
    }
    for (int a = 0; a < 3; ++a) {
        const double v = warp_sum_d(s[a]);
        if (lane == 0) red[a][w] = v;
    }
    __syncthreads();
    if (tid < 3) {
        double v = 0.0;
        for (int k = 0; k < 32; ++k) v += red[tid][k];
        csum[tid] = v;
    }
    __syncthreads();
    const double m0 = csum[0] / (double)n, m1 = csum[1] / (double)n, m2 = csum[2] / (double)n;
    double q = 0.0;
    for (int64_t i = tid; i < n; i += 1024) {
        double c[3];
        camera_centre(camprep + kCamPrep * i, c);
        q += (c[0] - m0) * (c[0] - m0) + (c[1] - m1) * (c[1] - m1) + (c[2] - m2) * (c[2] - m2);
    }
    q = warp_sum_d(q);
    if (lane == 0) red[3][w] = q;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int k = 0; k < 32; ++k) v += red[3][k];
        csum[3] = v;
    }
}

__global__ void centre_feature_kernel(int64_t n, const double* __restrict__ camprep, const double* __restrict__ csum,
                                      float* __restrict__ feat) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double c[3];
    camera_centre(camprep + kCamPrep * i, c);
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double dv = c[a] - csum[a] / (double)n;
        s += dv * dv;
    }
    const double rms = sqrt(csum[3] / (double)n);
    feat[i * kIn + 49] = (float)(rms > 0.0 ? sqrt(s) / rms : 0.0);
}

// ---- targets and predictions (thread per camera, fp64) ----
__global__ void targets_kernel(int64_t n, const double* __restrict__ scale, const double* __restrict__ sigma,
                               float* __restrict__ targ, int* flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* s = sigma + 81 * i;
    const double* Lz = scale + 81 * i;
    // S = L_z^T Sigma L_z (lower triangle), via Y = Sigma L_z
    double Y[81];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            double v = 0.0;
            for (int k = c; k < 9; ++k) v += s[9 * r + k] * Lz[9 * k + c];
            Y[9 * r + c] = v;
        }
    double L[45];  // Cholesky factor of S, lower triangle row by row
    for (int r = 0; r < 9; ++r) {
        for (int c = 0; c <= r; ++c) {
            double v = 0.0;
            for (int k = r; k < 9; ++k) v += Lz[9 * k + r] * Y[9 * k + c];  // S_rc = (L_z^T Y)_rc
            for (int k = 0; k < c; ++k) v -= L[r * (r + 1) / 2 + k] * L[c * (c + 1) / 2 + k];
            if (r == c) {
                if (!(v > 0.0)) { set_flag(flag, DEV_NOT_SPD, (int)i); v = 1.0; }
                L[r * (r + 1) / 2 + r] = sqrt(v);
            } else {
                L[r * (r + 1) / 2 + c] = v / L[c * (c + 1) / 2 + c];
            }
        }
    }
    float* t = targ + kOut * i;
    int q = 9;
    for (int r = 0; r < 9; ++r) {
        t[r] = (float)log(L[r * (r + 1) / 2 + r]);
        for (int c = 0; c < r; ++c) t[q++] = (float)L[r * (r + 1) / 2 + c];
    }
}

// Target form t = s (y sd + mu) (s the head's size scale), then
// Sigma_hat = L_z^-T L L^T L_z^-1 = X X^T with L_z^T X = L (back substitution).
__global__ void predict_out_kernel(int64_t n, const float* __restrict__ Y, const float* __restrict__ norm,
                                   const float* __restrict__ feat, const double* __restrict__ scale,
                                   double* __restrict__ sigma) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* y = Y + kOutP * i;
    const float* mu = norm + 2 * kIn;
    const float* sd = mu + kOut;
    const double hs = head_scale(feat + i * kIn);
    double X[9][9];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) X[r][c] = 0.0;
    int q = 9;
    for (int r = 0; r < 9; ++r) {
        X[r][r] = exp(hs * ((double)y[r] * sd[r] + mu[r]));
        for (int c = 0; c < r; ++c, ++q) X[r][c] = hs * ((double)y[q] * sd[q] + mu[q]);
    }
    const double* Lz = scale + 81 * i;
    for (int c = 0; c < 9; ++c)
        for (int r = 8; r >= 0; --r) {
            double v = X[r][c];
            for (int k = r + 1; k < 9; ++k) v -= Lz[9 * k + r] * X[k][c];
            X[r][c] = v / Lz[9 * r + r];
        }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            double v = 0.0;
            for (int k = 0; k < 9; ++k) v += X[r][k] * X[c][k];
            sigma[81 * i + 9 * r + c] = v;
        }
}

// ---- gauge term of the base covariance (fp64, small dense blocks) ----
// Z_ii^-1 holds every other camera fixed and so pins the datum as well; in
// the similarity gauge (Sec. 4.1) the camera moves with the datum too, along
// its own nullspace rows H_i.  The base B_i = Z_ii^-1 + Q_i M Q_i^T adds that
// motion: Q_i = H_i L_c, L_c the Cholesky factor of (sum_i H_i^T Z_ii H_i)^-1,
// and M a learned symmetric 7 x 7 matrix.  Targets and predictions are then
// whitened by T_i = chol(B_i^-1) in place of L_z (T_i = L_z when M = 0).

// Cholesky factor (lower, row-major, zero above) of a K x K SPD matrix;
// false when a pivot is not above `tiny`.
template <int K>
__device__ bool chol_k(const double* a, double* l, double tiny = 0.0) {
    for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c) l[K * r + c] = 0.0;
    for (int r = 0; r < K; ++r)
        for (int c = 0; c <= r; ++c) {
            double v = a[K * r + c];
            for (int k = 0; k < c; ++k) v -= l[K * r + k] * l[K * c + k];
            if (r == c) {
                if (!(v > tiny)) return false;
                l[K * r + r] = sqrt(v);
            } else {
                l[K * r + c] = v / l[K * c + c];
            }
        }
    return true;
}

// x = l^-1 for a lower-triangular l (forward substitution column by column).
template <int K>
__device__ void tri_inv_k(const double* l, double* x) {
    for (int c = 0; c < K; ++c)
        for (int r = 0; r < K; ++r) {
            if (r < c) {
                x[K * r + c] = 0.0;
                continue;
            }
            double v = r == c ? 1.0 : 0.0;
            for (int k = c; k < r; ++k) v -= l[K * r + k] * x[K * k + c];
            x[K * r + c] = v / l[K * r + r];
        }
}

// a^-1 = x^T x with x = chol(a)^-1; false when a is not positive definite.
template <int K>
__device__ bool spd_inv_k(const double* a, double* ainv) {
    double l[K * K], x[K * K];
    if (!chol_k<K>(a, l)) return false;
    tri_inv_k<K>(l, x);
    for (int r = 0; r < K; ++r)
        for (int c = 0; c < K; ++c) {
            double v = 0.0;
            for (int k = r > c ? r : c; k < K; ++k) v += x[K * k + r] * x[K * k + c];
            ainv[K * r + c] = v;
        }
    return true;
}

// AH = sum_i P_i^T P_i with P_i = L_z^T H_i (9 x 7), over a scene's cameras:
// block b sums the cameras [b chunk, (b + 1) chunk) (its threads strided, the
// 28 entries k <= l reduced by fixed trees), and one block then adds the
// blocks' sums in order (the same bits on every run), forms
// L_c = chol(AH^-1), and a camera-parallel kernel writes Q_i = H_i L_c.
constexpr int kGaugeThreads = 256;

__global__ void __launch_bounds__(kGaugeThreads)
gauge_sum_kernel(int64_t n, const double* __restrict__ Lz, const double* __restrict__ HP,
                 double* __restrict__ part) {
    __shared__ double red[28][kGaugeThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t chunk = (n + kSurrGaugeBlocks - 1) / kSurrGaugeBlocks;
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double acc[28];
#pragma unroll
    for (int e = 0; e < 28; ++e) acc[e] = 0.0;
    for (int64_t i = i0 + tid; i < i1; i += kGaugeThreads) {
        const double* L = Lz + 81 * i;
        const double* H = HP + 63 * i;
        double P[63];
        for (int a = 0; a < 9; ++a)
            for (int k = 0; k < 7; ++k) {
                double v = 0.0;
                for (int b = a; b < 9; ++b) v += L[9 * b + a] * H[7 * b + k];
                P[7 * a + k] = v;
            }
        int e = 0;
        for (int k = 0; k < 7; ++k)
            for (int l = k; l < 7; ++l, ++e) {
                double v = 0.0;
                for (int a = 0; a < 9; ++a) v += P[7 * a + k] * P[7 * a + l];
                acc[e] += v;
            }
    }
#pragma unroll
    for (int e = 0; e < 28; ++e) {
        const double v = warp_sum_d(acc[e]);
        if (lane == 0) red[e][w] = v;
    }
    __syncthreads();
    if (tid < 28) {
        double v = 0.0;
        for (int q = 0; q < kGaugeThreads / 32; ++q) v += red[tid][q];
        part[28 * (int64_t)blockIdx.x + tid] = v;
    }
}

// One warp: the blocks' sums in order, then L_c (49 values after the partials).
__global__ void gauge_factor_kernel(double* __restrict__ part, int* flag) {
    __shared__ double AH[49];
    const int tid = threadIdx.x;
    if (tid < 28) {
        int k = 0, rem = tid;
        while (rem >= 7 - k) { rem -= 7 - k; ++k; }
        const int l = k + rem;
        double v = 0.0;
        for (int b = 0; b < kSurrGaugeBlocks; ++b) v += part[28 * b + tid];
        AH[7 * k + l] = AH[7 * l + k] = v;
    }
    __syncwarp();
    if (tid != 0) return;
    double AHi[49], L7[49];
    const bool ok = spd_inv_k<7>(AH, AHi) && chol_k<7>(AHi, L7);
    if (!ok) set_flag(flag, DEV_NOT_SPD, 0);
    double* Lc = part + 28 * kSurrGaugeBlocks;
    for (int k = 0; k < 49; ++k) Lc[k] = ok ? L7[k] : 0.0;
}

__global__ void gauge_q_kernel(int64_t n, const double* __restrict__ HP, const double* __restrict__ Lcg,
                               double* __restrict__ Q) {
    __shared__ double Lc[49];
    if (threadIdx.x < 49) Lc[threadIdx.x] = Lcg[threadIdx.x];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* H = HP + 63 * i;
    double* q = Q + 63 * i;
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 7; ++c) {
            double v = 0.0;
            for (int k = c; k < 7; ++k) v += H[7 * r + k] * Lc[7 * k + c];
            q[7 * r + c] = v;
        }
}

// Least squares for M over the training cameras.  Per camera:
// Qt = L_z^T Q_i (9 x 7), E = L_z^T Sigma_i L_z - I, G = Qt^T Qt and
// R = Qt^T E Qt.  With the 28 symmetric basis matrices E_p (p = (k, l),
// k <= l, ones at (k, l) and (l, k)) the normal equations are
//   sum_q N_pq m_q = r_p,  N_pq = sum_i tr(E_p G E_q G),  r_p = sum_i tr(R E_p).
// The 406 entries p <= q of N and the 28 of r are summed per block (fixed
// camera ranges, warp trees, warps in order) and the blocks in order.
constexpr int kFitBlocks = 256, kFitThreads = 256, kFitN = 406, kFitEntries = kFitN + 28;

__constant__ unsigned char c_sym_k[28], c_sym_l[28];
__constant__ unsigned char c_pair_p[kFitN], c_pair_q[kFitN];

__global__ void __launch_bounds__(kFitThreads)
gauge_fit_partial_kernel(int64_t n, const double* __restrict__ Lz, const double* __restrict__ Qg,
                         const double* __restrict__ sigma, double* __restrict__ part) {
    __shared__ double wacc[kFitThreads / 32][kFitEntries];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int e = lane; e < kFitEntries; e += 32) wacc[w][e] = 0.0;
    const int64_t chunk = (n + kFitBlocks - 1) / kFitBlocks;
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int64_t base = i0; base < i1; base += kFitThreads) {
        const int64_t i = base + tid;
        double G[49], R[49];
        if (i < i1) {
            const double* L = Lz + 81 * i;
            const double* q = Qg + 63 * i;
            const double* S = sigma + 81 * i;
            double Qt[63], Y[81], E[81];
            for (int a = 0; a < 9; ++a)
                for (int k = 0; k < 7; ++k) {
                    double v = 0.0;
                    for (int b = a; b < 9; ++b) v += L[9 * b + a] * q[7 * b + k];
                    Qt[7 * a + k] = v;
                }
            for (int r = 0; r < 9; ++r)  // Y = Sigma L_z
                for (int c = 0; c < 9; ++c) {
                    double v = 0.0;
                    for (int k = c; k < 9; ++k) v += S[9 * r + k] * L[9 * k + c];
                    Y[9 * r + c] = v;
                }
            for (int r = 0; r < 9; ++r)  // E = L_z^T Y - I
                for (int c = 0; c < 9; ++c) {
                    double v = 0.0;
                    for (int k = r; k < 9; ++k) v += L[9 * k + r] * Y[9 * k + c];
                    E[9 * r + c] = v - (r == c ? 1.0 : 0.0);
                }
            for (int k = 0; k < 7; ++k)
                for (int l = 0; l < 7; ++l) {
                    double g = 0.0, rr = 0.0;
                    for (int a = 0; a < 9; ++a) {
                        g += Qt[7 * a + k] * Qt[7 * a + l];
                        double t = 0.0;
                        for (int b = 0; b < 9; ++b) t += E[9 * a + b] * Qt[7 * b + l];
                        rr += Qt[7 * a + k] * t;
                    }
                    G[7 * k + l] = g;
                    R[7 * k + l] = rr;
                }
        } else {
            for (int k = 0; k < 49; ++k) G[k] = R[k] = 0.0;
        }
        for (int e = 0; e < kFitEntries; ++e) {
            double v;
            if (e < kFitN) {
                const int p = c_pair_p[e], q = c_pair_q[e];
                const int k = c_sym_k[p], l = c_sym_l[p], a = c_sym_k[q], b = c_sym_l[q];
                // tr(E_p G E_q G): sum over the unit terms e_x e_y^T of E_p and e_u e_v^T of E_q
                v = G[7 * b + k] * G[7 * l + a];
                if (a != b) v += G[7 * a + k] * G[7 * l + b];
                if (k != l) {
                    v += G[7 * b + l] * G[7 * k + a];
                    if (a != b) v += G[7 * a + l] * G[7 * k + b];
                }
            } else {
                const int p = e - kFitN, k = c_sym_k[p], l = c_sym_l[p];
                v = k == l ? R[7 * k + k] : R[7 * k + l] + R[7 * l + k];
            }
            v = warp_sum_d(v);
            if (lane == 0) wacc[w][e] += v;
        }
    }
    __syncthreads();
    for (int e = tid; e < kFitEntries; e += kFitThreads) {
        double v = 0.0;
        for (int q = 0; q < kFitThreads / 32; ++q) v += wacc[q][e];
        part[(int64_t)blockIdx.x * kFitEntries + e] = v;
    }
}

// Blocks' partial sums in order, then N m = r by Cholesky (one thread).
__global__ void __launch_bounds__(512) gauge_fit_solve_kernel(const double* __restrict__ part,
                                                             double* __restrict__ M, int* flag) {
    __shared__ double tot[kFitEntries];
    __shared__ double N[28 * 28], L[28 * 28];  // shared, not per-thread: one thread factors them
    for (int e = threadIdx.x; e < kFitEntries; e += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < kFitBlocks; ++b) v += part[(int64_t)b * kFitEntries + e];
        tot[e] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double m[28], dmax = 0.0;
    for (int e = 0; e < kFitN; ++e) {
        const int p = c_pair_p[e], q = c_pair_q[e];
        N[28 * p + q] = N[28 * q + p] = tot[e];
        if (p == q) dmax = fmax(dmax, tot[e]);
    }
    // a pivot below 1e-9 of the largest diagonal entry: the cameras do not
    // determine M (one camera's rows have rank 6, so it fixes 21 of the 28
    // entries; the normal matrices of real scenes have eigenvalue ratios near 0.4)
    if (!(dmax > 0.0) || !chol_k<28>(N, L, 1e-9 * dmax)) {
        set_flag(flag, DEV_NOT_SPD, 0);
        return;
    }
    for (int p = 0; p < 28; ++p) {  // L y = r
        double v = tot[kFitN + p];
        for (int k = 0; k < p; ++k) v -= L[28 * p + k] * m[k];
        m[p] = v / L[28 * p + p];
    }
    for (int p = 27; p >= 0; --p) {  // L^T m = y
        double v = m[p];
        for (int k = p + 1; k < 28; ++k) v -= L[28 * k + p] * m[k];
        m[p] = v / L[28 * p + p];
    }
    for (int p = 0; p < 28; ++p) {
        const int k = c_sym_k[p], l = c_sym_l[p];
        M[7 * k + l] = M[7 * l + k] = m[p];
    }
}

// T_i = chol(B_i^-1), B_i = Z_ii^-1 + Q_i M Q_i^T, Z_ii^-1 = X^T X with X = L_z^-1.
__global__ void gauge_apply_kernel(int64_t n, const double* __restrict__ Lz, const double* __restrict__ Qg,
                                   const double* __restrict__ Mg, double* __restrict__ T, int* flag) {
    __shared__ double Ms[49];
    if (threadIdx.x < 49) Ms[threadIdx.x] = Mg[threadIdx.x];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* q = Qg + 63 * i;
    double X[81], B[81], QM[63], Bi[81], Tl[81];
    tri_inv_k<9>(Lz + 81 * i, X);
    for (int a = 0; a < 9; ++a)  // (Q M)^T, 7 x 9
        for (int l = 0; l < 7; ++l) {
            double v = 0.0;
            for (int k = 0; k < 7; ++k) v += q[7 * a + k] * Ms[7 * k + l];
            QM[9 * l + a] = v;
        }
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            double v = 0.0;
            for (int k = r > c ? r : c; k < 9; ++k) v += X[9 * k + r] * X[9 * k + c];
            for (int l = 0; l < 7; ++l) v += QM[9 * l + r] * q[7 * c + l];
            B[9 * r + c] = v;
        }
    for (int r = 0; r < 9; ++r)  // symmetric to the last bit before the factorisations
        for (int c = 0; c < r; ++c) B[9 * c + r] = B[9 * r + c] = 0.5 * (B[9 * r + c] + B[9 * c + r]);
    const bool ok = spd_inv_k<9>(B, Bi) && chol_k<9>(Bi, Tl);
    if (!ok) set_flag(flag, DEV_NOT_SPD, (int)i);
    for (int k = 0; k < 81; ++k) T[81 * i + k] = ok ? Tl[k] : 0.0;
}

}  // namespace surr

void surr_launch_features(Ctx& c, float* feat, double* scale) {
    using namespace surr;
    double* csum = c.d_small + 100;  // 4 slots that nothing else uses
    features_kernel<<<(unsigned)((c.n + kFeatWarps - 1) / kFeatWarps), 32 * kFeatWarps, 0, c.stream>>>(
        c.n, c.d_U, c.d_W, c.d_Ainv, c.d_cam_ptr, c.d_cam_perm, c.d_obs, c.d_pt_ptr, c.d_camprep, csum, feat, scale,
        c.d_flag);
    centre_stats_kernel<<<1, 1024, 0, c.stream>>>(c.n, c.d_camprep, csum);
    centre_feature_kernel<<<(unsigned)((c.n + 127) / 128), 128, 0, c.stream>>>(c.n, c.d_camprep, csum, feat);
    c.launches += 3;
}

void surr_launch_gauge_rows(Ctx& c, const double* scale, double* q) {
    surr::gauge_sum_kernel<<<kSurrGaugeBlocks, surr::kGaugeThreads, 0, c.stream>>>(c.n, scale, c.d_HP, c.d_sgauge);
    surr::gauge_factor_kernel<<<1, 32, 0, c.stream>>>(c.d_sgauge, c.d_flag);
    surr::gauge_q_kernel<<<(unsigned)((c.n + 127) / 128), 128, 0, c.stream>>>(
        c.n, c.d_HP, c.d_sgauge + 28 * kSurrGaugeBlocks, q);
    c.launches += 3;
}

}  // namespace ccov

// ---------------------------------------------------------------------------
// Host side of the model.
using namespace ccov::surr;

struct ccov_surrogate {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t max_batch = 0, Bp = 0;
    std::string err;
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;  // padded master, kPadParams
    float* norm = nullptr;                                             // kNorm
    bf16* wb[4] = {};
    bf16* wt[4] = {};
    bf16 *a_n[4] = {}, *a_t[4] = {};   // activations a0..a3 and transposes
    bf16 *g_n[5] = {}, *g_t[5] = {};   // gradients g1..g4 (index = layer)
    float *Y = nullptr, *T = nullptr;
    float* losses = nullptr;           // device, per in-call step
    float* part = nullptr;             // partial sums of a step, summed in order (kPartFloats)
    int64_t losses_cap = 0;
    int* ctr = nullptr;                // [0] Adam steps, [1] in-call step
    unsigned* done = nullptr;
    int* flag = nullptr;
    double* gauge = nullptr;           // M, 7 x 7 row-major (zero until fitted or set)
    double* gpart = nullptr;           // partial sums of the gauge fit, kFitBlocks x kFitEntries
    std::vector<void*> allocs;
};

namespace {

ccov_status sfail(ccov_surrogate* s, ccov_status st, const char* fmt, ...) {
    if (s) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        s->err = buf;
    }
    return st;
}

#define SCK(expr, where)                                                                   \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return sfail(s, _e == cudaErrorMemoryAllocation ? CCOV_ERR_OOM : CCOV_ERR_CUDA, \
                         "%s: %s", where, cudaGetErrorString(_e));                         \
    } while (0)

template <class T>
cudaError_t salloc(ccov_surrogate* s, T** ptr, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
    if (e == cudaSuccess) s->allocs.push_back(*ptr);
    return e;
}

Segs segs(const ccov_surrogate* s) {
    Segs S;
    const int64_t offs[8] = {kOffW1, kOffB1, kOffW2, kOffB2, kOffW3, kOffB3, kOffW4, kOffB4};
    const int64_t rows[8] = {256, 256, 256, 256, 256, 256, kOutP, kOutP};
    const int64_t cols[8] = {kInP, 0, 256, 0, 256, 0, 256, 0};
    for (int k = 0; k < 8; ++k) S.s[k] = Seg{offs[k], rows[k], cols[k]};
    for (int l = 0; l < 4; ++l) {
        S.wb[l] = s->wb[l];
        S.wt[l] = s->wt[l];
    }
    return S;
}

// logical (host) parameter order <-> padded master
void to_padded(const float* in, std::vector<float>& out) {
    out.assign(kPadParams, 0.f);
    const float* q = in;
    for (int o = 0; o < 256; ++o)
        for (int i = 0; i < kIn; ++i) out[kOffW1 + o * kInP + i] = *q++;
    for (int o = 0; o < 256; ++o) out[kOffB1 + o] = *q++;
    for (int k = 0; k < 65536; ++k) out[kOffW2 + k] = *q++;
    for (int o = 0; o < 256; ++o) out[kOffB2 + o] = *q++;
    for (int k = 0; k < 65536; ++k) out[kOffW3 + k] = *q++;
    for (int o = 0; o < 256; ++o) out[kOffB3 + o] = *q++;
    for (int o = 0; o < kOut; ++o)
        for (int i = 0; i < 256; ++i) out[kOffW4 + o * 256 + i] = *q++;
    for (int o = 0; o < kOut; ++o) out[kOffB4 + o] = *q++;
}

void from_padded(const std::vector<float>& in, float* out) {
    float* q = out;
    for (int o = 0; o < 256; ++o)
        for (int i = 0; i < kIn; ++i) *q++ = in[kOffW1 + o * kInP + i];
    for (int o = 0; o < 256; ++o) *q++ = in[kOffB1 + o];
    for (int k = 0; k < 65536; ++k) *q++ = in[kOffW2 + k];
    for (int o = 0; o < 256; ++o) *q++ = in[kOffB2 + o];
    for (int k = 0; k < 65536; ++k) *q++ = in[kOffW3 + k];
    for (int o = 0; o < 256; ++o) *q++ = in[kOffB3 + o];
    for (int o = 0; o < kOut; ++o)
        for (int i = 0; i < 256; ++i) *q++ = in[kOffW4 + o * 256 + i];
    for (int o = 0; o < kOut; ++o) *q++ = in[kOffB4 + o];
}

ccov_status check_flag(ccov_surrogate* s, const char* where) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return sfail(s, CCOV_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    int f[2] = {0, 0};
    e = cudaMemcpy(f, s->flag, sizeof f, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return sfail(s, CCOV_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
    if (f[0] == ccov::DEV_TIMEOUT) return sfail(s, CCOV_ERR_TIMEOUT, "%s: device wait gave up (site %d)", where, f[1]);
    if (f[0] == ccov::DEV_BAD_INDEX)
        return sfail(s, CCOV_ERR_INVALID_ARG, "%s: sample index of batch row %d outside the training set", where, f[1]);
    if (f[0] == ccov::DEV_NOT_SPD)
        return sfail(s, CCOV_ERR_DEGENERATE, "%s: a matrix is not positive definite (row %d)", where, f[1]);
    if (f[0] != 0) return sfail(s, CCOV_ERR_CUDA, "%s: device error %d", where, f[0]);
    return CCOV_OK;
}

void gemm(ccov_surrogate* s, const bf16* A, int64_t a_rows, const bf16* B, int N, int K, int epi,
          const float* bias, bf16* out_n, bf16* out_t, const bf16* mask, float* out_f, float* db) {
    GemmP g;
    g.A = A; g.a_rows = a_rows; g.B = B; g.N = N; g.K = K; g.epi = epi;
    g.bias = bias; g.out_n = out_n; g.out_t = out_t; g.mask = mask; g.out_f = out_f; g.db = db;
    g.flag = s->flag;
    const int chunks = K / kChunk;
    const int tiles = (int)(a_rows / 128);
    int splits = 1;
    if (epi == EPI_DW) {  // long K (the batch): split it so that the grid fills the GPU
        splits = 64 / tiles;
        if (splits > chunks) splits = chunks;
        if (splits < 1) splits = 1;
    }
    g.chunks_per_split = (chunks + splits - 1) / splits;
    splits = (chunks + g.chunks_per_split - 1) / g.chunks_per_split;
    // gradient sums go through partials in s->part, summed in a fixed order
    // below (bit-for-bit repeatable training), not through atomics
    if (epi == EPI_DW) g.out_f = s->part;
    if (epi == EPI_DX) g.db = s->part;
    mlp_gemm_kernel<<<dim3((unsigned)tiles, (unsigned)splits), kGemmThreads, kGemmSmem, s->stream>>>(g);
    if (epi == EPI_DW) {
        const int64_t count = a_rows * N;
        sum_parts_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s->stream>>>(s->part, splits, count, count,
                                                                                 out_f);
    } else if (epi == EPI_DX) {
        sum_parts_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s->stream>>>(s->part, 4 * tiles, N, N, db);
    }
}

// One training step's launches (no host synchronisation): pack, forward,
// loss gradient, backward products and (if lr >= 0) Adam.
void enqueue_step(ccov_surrogate* s, const float* feat, const float* targ, int64_t n, const int* idx, int B,
                  float lr, bool adam) {
    const int64_t Bp = (B + 127) / 128 * 128;
    cudaMemsetAsync(s->grad, 0, sizeof(float) * kPadParams, s->stream);
    pack_kernel<<<(unsigned)Bp, 128, 0, s->stream>>>(feat, targ, idx, n, s->ctr, B, (int)Bp, s->norm, s->a_n[0],
                                                     s->a_t[0], s->T, s->flag);
    // forward
    gemm(s, s->a_n[0], Bp, s->wb[0], 256, kInP, EPI_RELU, s->p + kOffB1, s->a_n[1], s->a_t[1], nullptr, nullptr, nullptr);
    gemm(s, s->a_n[1], Bp, s->wb[1], 256, 256, EPI_RELU, s->p + kOffB2, s->a_n[2], s->a_t[2], nullptr, nullptr, nullptr);
    gemm(s, s->a_n[2], Bp, s->wb[2], 256, 256, EPI_RELU, s->p + kOffB3, s->a_n[3], s->a_t[3], nullptr, nullptr, nullptr);
    gemm(s, s->a_n[3], Bp, s->wb[3], kOutP, 256, EPI_OUT, s->p + kOffB4, nullptr, nullptr, nullptr, s->Y, nullptr);
    loss_kernel<<<(unsigned)(Bp / 64), 128, 0, s->stream>>>(s->Y, s->T, B, (int)Bp, s->g_n[4], s->g_t[4], s->part);
    sum_parts_kernel<<<1, 128, 0, s->stream>>>(s->part, (int)(Bp / 64), 129, kOut, s->grad + kOffB4);
    loss_sum_kernel<<<1, 32, 0, s->stream>>>(s->part, (int)(Bp / 64), s->losses, s->ctr);
    // backward: dW_l = g_l^T a_{l-1}; g_{l-1} = (g_l W_l) * [a_{l-1} > 0]
    gemm(s, s->g_t[4], kOutP, s->a_t[3], 256, (int)Bp, EPI_DW, nullptr, nullptr, nullptr, nullptr, s->grad + kOffW4, nullptr);
    gemm(s, s->g_n[4], Bp, s->wt[3], 256, kOutP, EPI_DX, nullptr, s->g_n[3], s->g_t[3], s->a_n[3], nullptr, s->grad + kOffB3);
    gemm(s, s->g_t[3], 256, s->a_t[2], 256, (int)Bp, EPI_DW, nullptr, nullptr, nullptr, nullptr, s->grad + kOffW3, nullptr);
    gemm(s, s->g_n[3], Bp, s->wt[2], 256, 256, EPI_DX, nullptr, s->g_n[2], s->g_t[2], s->a_n[2], nullptr, s->grad + kOffB2);
    gemm(s, s->g_t[2], 256, s->a_t[1], 256, (int)Bp, EPI_DW, nullptr, nullptr, nullptr, nullptr, s->grad + kOffW2, nullptr);
    gemm(s, s->g_n[2], Bp, s->wt[1], 256, 256, EPI_DX, nullptr, s->g_n[1], s->g_t[1], s->a_n[1], nullptr, s->grad + kOffB1);
    gemm(s, s->g_t[1], 256, s->a_t[0], kInP, (int)Bp, EPI_DW, nullptr, nullptr, nullptr, nullptr, s->grad + kOffW1, nullptr);
    if (adam) {
        const unsigned blocks = (unsigned)((kPadParams + 255) / 256);
        adam_kernel<<<blocks, 256, 0, s->stream>>>(s->p, s->grad, s->m, s->v, kPadParams, lr, segs(s), s->ctr,
                                                   s->done);
    }
}

ccov_status ensure_losses(ccov_surrogate* s, int64_t k) {
    if (s->losses_cap >= k) return CCOV_OK;
    if (s->losses) cudaFree(s->losses);
    s->losses = nullptr;
    s->losses_cap = 0;
    SCK(cudaMalloc(&s->losses, sizeof(float) * k), "alloc losses");
    s->losses_cap = k;
    return CCOV_OK;
}

ccov_status validate_batch(ccov_surrogate* s, const float* feat, const float* targ, int64_t n, const int32_t* idx,
                           int64_t batch) {
    if (!feat || !targ || !idx) return sfail(s, CCOV_ERR_INVALID_ARG, "null array");
    if (n < 1 || n > INT32_MAX) return sfail(s, CCOV_ERR_INVALID_ARG, "training set size %lld", (long long)n);
    if (batch < 1 || batch > s->max_batch)
        return sfail(s, CCOV_ERR_INVALID_ARG, "batch %lld outside [1, %lld]", (long long)batch, (long long)s->max_batch);
    return CCOV_OK;
}

}  // namespace

extern "C" {

ccov_status ccov_surrogate_targets(int64_t n, const double* scale, const double* sigma, float* targets,
                                   void* stream) {
    if (n < 1 || !scale || !sigma || !targets) return CCOV_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* flag = nullptr;
    if (cudaMalloc(&flag, 2 * sizeof(int)) != cudaSuccess) return CCOV_ERR_OOM;
    cudaMemsetAsync(flag, 0, 2 * sizeof(int), st);
    targets_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, scale, sigma, targets, flag);
    int f[2] = {0, 0};
    ccov_status res = CCOV_OK;
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(f, flag, sizeof f, cudaMemcpyDeviceToHost) != cudaSuccess)
        res = CCOV_ERR_CUDA;
    else if (f[0] == ccov::DEV_NOT_SPD)
        res = CCOV_ERR_DEGENERATE;
    cudaFree(flag);
    return res;
}

ccov_status ccov_surrogate_create(const float* params, int64_t max_batch, void* stream, ccov_surrogate** out) {
    if (!out) return CCOV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || max_batch < 1 || max_batch > 65536) return CCOV_ERR_INVALID_ARG;
    ccov_surrogate* s = new (std::nothrow) ccov_surrogate();
    if (!s) return CCOV_ERR_OOM;
    *out = s;
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        SCK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "stream");
        s->own_stream = true;
    }
    SCK(cudaFuncSetAttribute(mlp_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem),
        "kernel attribute");
    s->max_batch = max_batch;
    const int64_t Bp = (max_batch + 127) / 128 * 128;
    s->Bp = Bp;
    SCK(salloc(s, &s->p, kPadParams), "alloc");
    SCK(salloc(s, &s->grad, kPadParams), "alloc");
    SCK(salloc(s, &s->m, kPadParams), "alloc");
    SCK(salloc(s, &s->v, kPadParams), "alloc");
    SCK(salloc(s, &s->norm, kNorm), "alloc");
    const int64_t wrows[4] = {256, 256, 256, kOutP}, wcols[4] = {kInP, 256, 256, 256};
    for (int l = 0; l < 4; ++l) {
        SCK(salloc(s, &s->wb[l], wrows[l] * wcols[l]), "alloc");
        if (l > 0) SCK(salloc(s, &s->wt[l], wrows[l] * wcols[l]), "alloc");
    }
    const int64_t width[5] = {kInP, 256, 256, 256, kOutP};
    for (int l = 0; l < 4; ++l) {
        SCK(salloc(s, &s->a_n[l], Bp * width[l]), "alloc");
        SCK(salloc(s, &s->a_t[l], Bp * width[l]), "alloc");
    }
    for (int l = 1; l <= 4; ++l) {
        SCK(salloc(s, &s->g_n[l], Bp * width[l]), "alloc");
        SCK(salloc(s, &s->g_t[l], Bp * width[l]), "alloc");
    }
    SCK(salloc(s, &s->Y, Bp * kOutP), "alloc");
    {
        // the largest set of partial sums of a step: the weight gradients'
        // splits (at most 64 x 128 x 256 or 32 x 256 x 256), the bias
        // gradients' row quarters, the loss blocks
        int64_t np = (int64_t)1 << 21;
        np = std::max<int64_t>(np, Bp / 128 * 4 * 256);
        np = std::max<int64_t>(np, Bp / 64 * 129);
        SCK(salloc(s, &s->part, np), "alloc");
    }
    SCK(salloc(s, &s->T, Bp * kOut), "alloc");
    SCK(salloc(s, &s->ctr, 2), "alloc");
    SCK(salloc(s, &s->done, 1), "alloc");
    SCK(salloc(s, &s->flag, 2), "alloc");
    SCK(salloc(s, &s->gauge, 49), "alloc");
    SCK(salloc(s, &s->gpart, (size_t)kFitBlocks * kFitEntries), "alloc");
    SCK(cudaMemsetAsync(s->gauge, 0, 49 * sizeof(double), s->stream), "memset");
    {
        unsigned char sk[28], sl[28], pp[kFitN], pq[kFitN];
        int p = 0;
        for (int k = 0; k < 7; ++k)
            for (int l = k; l < 7; ++l, ++p) sk[p] = (unsigned char)k, sl[p] = (unsigned char)l;
        int e = 0;
        for (int a = 0; a < 28; ++a)
            for (int b = a; b < 28; ++b, ++e) pp[e] = (unsigned char)a, pq[e] = (unsigned char)b;
        SCK(cudaMemcpyToSymbol(c_sym_k, sk, sizeof sk), "constants");
        SCK(cudaMemcpyToSymbol(c_sym_l, sl, sizeof sl), "constants");
        SCK(cudaMemcpyToSymbol(c_pair_p, pp, sizeof pp), "constants");
        SCK(cudaMemcpyToSymbol(c_pair_q, pq, sizeof pq), "constants");
    }
    ccov_status st = ensure_losses(s, 1);
    if (st != CCOV_OK) return st;
    SCK(cudaMemsetAsync(s->m, 0, sizeof(float) * kPadParams, s->stream), "memset");
    SCK(cudaMemsetAsync(s->v, 0, sizeof(float) * kPadParams, s->stream), "memset");
    SCK(cudaMemsetAsync(s->ctr, 0, 2 * sizeof(int), s->stream), "memset");
    SCK(cudaMemsetAsync(s->done, 0, sizeof(unsigned), s->stream), "memset");
    SCK(cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream), "memset");
    for (int l = 0; l < 4; ++l) {  // padding of the operand copies stays zero
        SCK(cudaMemsetAsync(s->wb[l], 0, sizeof(bf16) * wrows[l] * wcols[l], s->stream), "memset");
        if (s->wt[l]) SCK(cudaMemsetAsync(s->wt[l], 0, sizeof(bf16) * wrows[l] * wcols[l], s->stream), "memset");
    }
    std::vector<float> unit(kNorm, 0.f);
    for (int k = 0; k < kIn; ++k) unit[kIn + k] = 1.f;
    for (int k = 0; k < kOut; ++k) unit[2 * kIn + kOut + k] = 1.f;
    st = ccov_surrogate_set_normalization(s, unit.data());
    if (st != CCOV_OK) return st;
    return ccov_surrogate_set_params(s, params);
}

ccov_status ccov_surrogate_set_params(ccov_surrogate* s, const float* params) {
    if (!s || !params) return CCOV_ERR_INVALID_ARG;
    std::vector<float> pad;
    to_padded(params, pad);
    SCK(cudaMemcpyAsync(s->p, pad.data(), sizeof(float) * kPadParams, cudaMemcpyHostToDevice, s->stream), "copy");
    cast_kernel<<<(unsigned)((kPadParams + 255) / 256), 256, 0, s->stream>>>(s->p, kPadParams, segs(s));
    SCK(cudaGetLastError(), "cast");
    return check_flag(s, "ccov_surrogate_set_params");
}

ccov_status ccov_surrogate_get_params(const ccov_surrogate* cs, float* params) {
    ccov_surrogate* s = const_cast<ccov_surrogate*>(cs);
    if (!s || !params) return CCOV_ERR_INVALID_ARG;
    std::vector<float> pad(kPadParams);
    SCK(cudaStreamSynchronize(s->stream), "sync");
    SCK(cudaMemcpy(pad.data(), s->p, sizeof(float) * kPadParams, cudaMemcpyDeviceToHost), "copy");
    from_padded(pad, params);
    return CCOV_OK;
}

ccov_status ccov_surrogate_get_grads(const ccov_surrogate* cs, float* grads) {
    ccov_surrogate* s = const_cast<ccov_surrogate*>(cs);
    if (!s || !grads) return CCOV_ERR_INVALID_ARG;
    std::vector<float> pad(kPadParams);
    SCK(cudaStreamSynchronize(s->stream), "sync");
    SCK(cudaMemcpy(pad.data(), s->grad, sizeof(float) * kPadParams, cudaMemcpyDeviceToHost), "copy");
    from_padded(pad, grads);
    return CCOV_OK;
}

ccov_status ccov_surrogate_set_normalization(ccov_surrogate* s, const float* norm) {
    if (!s || !norm) return CCOV_ERR_INVALID_ARG;
    for (int k = 0; k < kIn; ++k)
        if (!(norm[kIn + k] > 0.f)) return sfail(s, CCOV_ERR_INVALID_ARG, "feature deviation %d not positive", k);
    for (int k = 0; k < kOut; ++k)
        if (!(norm[2 * kIn + kOut + k] > 0.f)) return sfail(s, CCOV_ERR_INVALID_ARG, "target deviation %d not positive", k);
    SCK(cudaMemcpyAsync(s->norm, norm, sizeof(float) * kNorm, cudaMemcpyHostToDevice, s->stream), "copy");
    SCK(cudaStreamSynchronize(s->stream), "sync");
    return CCOV_OK;
}

ccov_status ccov_surrogate_get_normalization(const ccov_surrogate* cs, float* norm) {
    ccov_surrogate* s = const_cast<ccov_surrogate*>(cs);
    if (!s || !norm) return CCOV_ERR_INVALID_ARG;
    SCK(cudaStreamSynchronize(s->stream), "sync");
    SCK(cudaMemcpy(norm, s->norm, sizeof(float) * kNorm, cudaMemcpyDeviceToHost), "copy");
    return CCOV_OK;
}

ccov_status ccov_surrogate_fit_normalization(ccov_surrogate* s, const float* features, const float* targets,
                                             int64_t n) {
    if (!s || !features || !targets || n < 1) return CCOV_ERR_INVALID_ARG;
    norm_kernel<<<kIn, 256, 0, s->stream>>>(features, nullptr, n, kIn, s->norm, s->norm + kIn);
    norm_kernel<<<kOut, 256, 0, s->stream>>>(targets, features, n, kOut, s->norm + 2 * kIn,
                                             s->norm + 2 * kIn + kOut);
    SCK(cudaGetLastError(), "normalisation");
    return check_flag(s, "ccov_surrogate_fit_normalization");
}

ccov_status ccov_surrogate_backward(ccov_surrogate* s, const float* features, const float* targets, int64_t n,
                                    const int32_t* idx, int64_t batch, float* loss) {
    if (!s) return CCOV_ERR_INVALID_ARG;
    ccov_status st = validate_batch(s, features, targets, n, idx, batch);
    if (st != CCOV_OK) return st;
    SCK(cudaMemsetAsync(s->ctr + 1, 0, sizeof(int), s->stream), "memset");
    SCK(cudaMemsetAsync(s->losses, 0, sizeof(float), s->stream), "memset");
    SCK(cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream), "memset");
    enqueue_step(s, features, targets, n, idx, (int)batch, 0.f, false);
    SCK(cudaGetLastError(), "ccov_surrogate_backward launch");
    st = check_flag(s, "ccov_surrogate_backward");
    if (st != CCOV_OK) return st;
    if (loss) SCK(cudaMemcpy(loss, s->losses, sizeof(float), cudaMemcpyDeviceToHost), "copy loss");
    return CCOV_OK;
}

ccov_status ccov_surrogate_adam(ccov_surrogate* s, float lr) {
    if (!s || !(lr >= 0.f)) return CCOV_ERR_INVALID_ARG;
    const unsigned blocks = (unsigned)((kPadParams + 255) / 256);
    adam_kernel<<<blocks, 256, 0, s->stream>>>(s->p, s->grad, s->m, s->v, kPadParams, lr, segs(s), s->ctr, s->done);
    SCK(cudaGetLastError(), "adam");
    return check_flag(s, "ccov_surrogate_adam");
}

ccov_status ccov_surrogate_train(ccov_surrogate* s, const float* features, const float* targets, int64_t n,
                                 const int32_t* idx, int64_t batch, int steps, float lr, float* losses) {
    if (!s || steps < 1 || !(lr >= 0.f)) return CCOV_ERR_INVALID_ARG;
    ccov_status st = validate_batch(s, features, targets, n, idx, batch);
    if (st != CCOV_OK) return st;
    st = ensure_losses(s, steps);
    if (st != CCOV_OK) return st;
    SCK(cudaMemsetAsync(s->ctr + 1, 0, sizeof(int), s->stream), "memset");
    SCK(cudaMemsetAsync(s->losses, 0, sizeof(float) * steps, s->stream), "memset");
    // record one step (its idx offset and loss slot come from the device
    // counter that Adam advances) and replay it `steps` times
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SCK(cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream), "memset");
    SCK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal), "capture");
    enqueue_step(s, features, targets, n, idx, (int)batch, lr, true);
    cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (int k = 0; e == cudaSuccess && k < steps; ++k) e = cudaGraphLaunch(exec, s->stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    SCK(e, "ccov_surrogate_train graph");
    st = check_flag(s, "ccov_surrogate_train");
    if (st != CCOV_OK) return st;
    if (losses) SCK(cudaMemcpy(losses, s->losses, sizeof(float) * steps, cudaMemcpyDeviceToHost), "copy losses");
    return CCOV_OK;
}

ccov_status ccov_surrogate_predict(ccov_surrogate* s, const float* features, const double* scale, int64_t n,
                                   double* sigma) {
    if (!s || !features || !scale || !sigma || n < 1) return CCOV_ERR_INVALID_ARG;
    SCK(cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream), "memset");
    for (int64_t r0 = 0; r0 < n; r0 += s->max_batch) {
        const int B = (int)((n - r0) < s->max_batch ? (n - r0) : s->max_batch);
        const int64_t Bp = (B + 127) / 128 * 128;
        pack_kernel<<<(unsigned)Bp, 128, 0, s->stream>>>(features + r0 * kIn, nullptr, nullptr, (int64_t)B, nullptr,
                                                         B, (int)Bp, s->norm, s->a_n[0], s->a_t[0], nullptr, s->flag);
        gemm(s, s->a_n[0], Bp, s->wb[0], 256, kInP, EPI_RELU, s->p + kOffB1, s->a_n[1], s->a_t[1], nullptr, nullptr, nullptr);
        gemm(s, s->a_n[1], Bp, s->wb[1], 256, 256, EPI_RELU, s->p + kOffB2, s->a_n[2], s->a_t[2], nullptr, nullptr, nullptr);
        gemm(s, s->a_n[2], Bp, s->wb[2], 256, 256, EPI_RELU, s->p + kOffB3, s->a_n[3], s->a_t[3], nullptr, nullptr, nullptr);
        gemm(s, s->a_n[3], Bp, s->wb[3], kOutP, 256, EPI_OUT, s->p + kOffB4, nullptr, nullptr, nullptr, s->Y, nullptr);
        predict_out_kernel<<<(unsigned)((B + 127) / 128), 128, 0, s->stream>>>(B, s->Y, s->norm, features + r0 * kIn,
                                                                               scale + 81 * r0,
                                                                               sigma + 81 * r0);
        SCK(cudaGetLastError(), "ccov_surrogate_predict launch");
    }
    return check_flag(s, "ccov_surrogate_predict");
}

ccov_status ccov_surrogate_set_gauge(ccov_surrogate* s, const double* M) {
    if (!s || !M) return CCOV_ERR_INVALID_ARG;
    for (int k = 0; k < 7; ++k)
        for (int l = 0; l < 7; ++l)
            if (!std::isfinite(M[7 * k + l]) || M[7 * k + l] != M[7 * l + k])
                return sfail(s, CCOV_ERR_INVALID_ARG, "gauge matrix not finite and symmetric at (%d, %d)", k, l);
    SCK(cudaMemcpyAsync(s->gauge, M, 49 * sizeof(double), cudaMemcpyHostToDevice, s->stream), "copy");
    SCK(cudaStreamSynchronize(s->stream), "sync");
    return CCOV_OK;
}

ccov_status ccov_surrogate_get_gauge(const ccov_surrogate* cs, double* M) {
    ccov_surrogate* s = const_cast<ccov_surrogate*>(cs);
    if (!s || !M) return CCOV_ERR_INVALID_ARG;
    SCK(cudaStreamSynchronize(s->stream), "sync");
    SCK(cudaMemcpy(M, s->gauge, 49 * sizeof(double), cudaMemcpyDeviceToHost), "copy");
    return CCOV_OK;
}

ccov_status ccov_surrogate_fit_gauge(ccov_surrogate* s, const double* scale, const double* q, const double* sigma,
                                     int64_t n) {
    if (!s || !scale || !q || !sigma || n < 1) return CCOV_ERR_INVALID_ARG;
    SCK(cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream), "memset");
    gauge_fit_partial_kernel<<<kFitBlocks, kFitThreads, 0, s->stream>>>(n, scale, q, sigma, s->gpart);
    gauge_fit_solve_kernel<<<1, 512, 0, s->stream>>>(s->gpart, s->gauge, s->flag);
    SCK(cudaGetLastError(), "ccov_surrogate_fit_gauge launch");
    return check_flag(s, "ccov_surrogate_fit_gauge");
}

ccov_status ccov_surrogate_apply_gauge(ccov_surrogate* s, const double* scale, const double* q, int64_t n,
                                       double* base) {
    if (!s || !scale || !q || !base || n < 1) return CCOV_ERR_INVALID_ARG;
    SCK(cudaMemsetAsync(s->flag, 0, 2 * sizeof(int), s->stream), "memset");
    gauge_apply_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s->stream>>>(n, scale, q, s->gauge, base, s->flag);
    SCK(cudaGetLastError(), "ccov_surrogate_apply_gauge launch");
    return check_flag(s, "ccov_surrogate_apply_gauge");
}

void ccov_surrogate_destroy(ccov_surrogate* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (void* p : s->allocs) cudaFree(p);
    if (s->losses) cudaFree(s->losses);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char* ccov_surrogate_last_error(const ccov_surrogate* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"

// Mixed-precision step (d): the Cholesky factorisation and triangular inverse
// of the Jacobi-scaled reduced camera matrix with every O(N^3) trailing
// update on the 5th-generation tensor cores (tcgen05, bf16 operands, fp32
// accumulation in TMEM, operands staged by TMA).
//
// Accuracy is kept by an error-free split of the operands into 8-bit digits
// (after Ozaki et al., "Error-free transformations of matrix multiplication
// by using fast routines of matrix multiplication and its applications",
// 2012): a row with exponent e holds v = 2^e sum_a d_a 2^-(7 + 8(a-1)),
// d_a integers in [-128, 128] that bf16 represents exactly.  A product of two
// digits has at most 14 bits, a sum of K = 128 of them at most 21, and the
// products of one digit order g = a + b (at most s of them) stay below 2^24,
// so each order accumulates exactly in one fp32 TMEM accumulator.  Orders
// above s - 1 are dropped (relative truncation ~2^-(8 s)).  The working
// matrices are held in int64 fixed point (Q60 for the factor, whose entries
// are bounded by 1 after Jacobi scaling; Q42 for the inverse), where every
// exact partial product is added by integer shifts: no FP64 arithmetic in the
// O(N^3) part at all.  The residual rounding is that of the digit split.
//
// Paper counterpart: the dense inversion of Z_p (Sec. 4.2); the paper runs it
// in double precision with LAPACK on a CPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "ccov_internal.cuh"
#include "../../include/ccov_testing.h"

namespace ccov {

constexpr int kBM = 128, kBN = 64, kBK = 32, kChunks = kNB / kBK;  // K = 128 per update
constexpr int kAPlane = kBM * kBK * 2;                              // 8 KB per digit plane
constexpr int kBPlane = kBN * kBK * 2;                              // 4 KB
constexpr int kFX = 42;                                             // fixed point of X = L^-1
constexpr int kFL = 60;                                             // fixed point of Z_s and L
constexpr unsigned long long kWaitNs = 1000000000ull;               // 1 s per barrier wait

struct MixedState {
    int s = 5;
    int stages = 3;
    __nv_bfloat16* digP = nullptr;   // [s][Np][128] first-operand digits
    __nv_bfloat16* digQ = nullptr;   // [s][Np][128] second-operand digits
    int* expP = nullptr;             // Np
    int* expQ = nullptr;             // Np
    long long* R = nullptr;          // Np x Np, Q42
    CUtensorMap mapP128, mapP64, mapQ128, mapQ64;
    int64_t tiles_done = 0;
};

namespace {

__device__ __forceinline__ void set_flag(int* flag, int code, int detail) {
    if (atomicMax(flag, code) < code) flag[1] = detail;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after kWaitNs, records DEV_TIMEOUT with the site.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* flag, int site) {
    if (mbar_try(bar, parity)) return true;
    unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) {
            set_flag(flag, DEV_TIMEOUT, site);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// K-major operand tile in shared memory written by TMA with 64-byte swizzle:
// rows of 64 bytes (32 bf16 along K), 8-row atoms of 512 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused with swizzle)
    d |= (uint64_t)(512 >> 4) << 32;           // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)4 << 61;                    // 64-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: bf16 x bf16 -> f32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tile schedule: M tiles of 128 rows x N tiles of 64 columns; `lower` keeps
// only tiles that reach the diagonal of a square region (tj*64 <= ti*128+127).
__device__ __forceinline__ void tile_coords(int64_t t, int tiles_n, int lower, int& ti, int& tj) {
    if (!lower) {
        ti = (int)(t / tiles_n);
        tj = (int)(t - (int64_t)ti * tiles_n);
        return;
    }
    // rows ti < T0 hold 2 ti + 2 tiles (cumulative ti^2 + ti); later rows tiles_n
    int T0 = tiles_n / 2;
    int64_t tri = (int64_t)T0 * T0 + T0;
    if (t < tri) {
        int r = (int)((sqrt(4.0 * (double)t + 1.0) - 1.0) * 0.5);
        while ((int64_t)(r + 1) * (r + 2) <= t) ++r;
        while ((int64_t)r * (r + 1) > t) --r;
        ti = r;
        tj = (int)(t - (int64_t)r * (r + 1));
    } else {
        int64_t u = t - tri;
        ti = T0 + (int)(u / tiles_n);
        tj = (int)(u - (int64_t)(ti - T0) * tiles_n);
    }
}

struct GemmArgs {
    int M, N;             // rows of A and of B (multiples of 128 and 64)
    int s;                // digit planes
    int plane_rows;       // rows per digit plane in the buffers (Np)
    int a_row0, b_row0;   // first row of the operands inside their planes
    int lower;            // keep only tiles touching the lower triangle
    int sub;              // 1: C -= A B^T, 0: C = A B^T
    int shift0;           // F_C - 14
    const int* expA;      // per row of A (nullptr = 0)
    const int* expB;      // per row of B (nullptr = 0)
    long long* C;         // int64 fixed point
    int64_t ldc;
    int stages;
    int* flag;
};

// Persistent warp-specialised kernel.  Warp 0 lane 0: TMA producer.  Warp 1:
// TMEM allocation, lane 0 issues tcgen05.mma.  Warps 2-5: epilogue (warp w
// reads TMEM lanes 32 (w % 4) .. +31).  s accumulators of 128 x 64 fp32.
template <int S>
__global__ void __launch_bounds__(192, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tile area
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = S * (kAPlane + kBPlane);
    unsigned char* tiles = base;
    uint64_t* bars = (uint64_t*)(base + g.stages * stage_bytes);
    uint64_t* full = bars;                 // [stages]
    uint64_t* empty = bars + g.stages;     // [stages]
    uint64_t* accf = bars + 2 * g.stages;
    uint64_t* acce = accf + 1;
    uint64_t* drain = acce + 1;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = g.M / kBM, tiles_n = g.N / kBN;
    int64_t ntiles;
    if (g.lower) {
        int T0 = tiles_n / 2;
        int64_t tri = (int64_t)T0 * T0 + T0;
        ntiles = tiles_m <= T0 ? (int64_t)tiles_m * tiles_m + tiles_m : tri + (int64_t)(tiles_m - T0) * tiles_n;
    } else {
        ntiles = (int64_t)tiles_m * tiles_n;
    }

    if (threadIdx.x == 0) {
        for (int i = 0; i < g.stages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        mbar_init(accf, 1);
        mbar_init(acce, 128);
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
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
            bool ok = true;
            const uint32_t tx = (uint32_t)stage_bytes;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int ti, tj;
                tile_coords(t, tiles_n, g.lower, ti, tj);
                for (int c = 0; c < kChunks && ok; ++c) {
                    if (!mbar_wait(empty + stage, phase ^ 1, g.flag, 1)) { ok = false; break; }
                    unsigned char* st = tiles + stage * stage_bytes;
                    mbar_expect_tx(full + stage, tx);
                    for (int p = 0; p < S; ++p) {
                        tma_load_2d(st + p * kAPlane, &mapA, full + stage, c * kBK,
                                    p * g.plane_rows + g.a_row0 + ti * kBM);
                        tma_load_2d(st + S * kAPlane + p * kBPlane, &mapB, full + stage, c * kBK,
                                    p * g.plane_rows + g.b_row0 + tj * kBN);
                    }
                    if (++stage == g.stages) { stage = 0; phase ^= 1; }
                }
            }
            // Every stage armed here is waited on by the MMA issuer before it
            // finishes (normal path), so no copy is in flight at exit; after a
            // timeout the copies issued earlier have long landed.
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true;
            const uint32_t idesc = idesc_bf16(kBM, kBN);
            bool issued = false;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                if (!mbar_wait(acce, acc_phase ^ 1, g.flag, 2)) { ok = false; break; }
                tc_fence_after();
                for (int c = 0; c < kChunks && ok; ++c) {
                    if (!mbar_wait(full + stage, phase, g.flag, 3)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + stage * stage_bytes);
                    const uint32_t sb = sa + S * kAPlane;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
                        for (int gi = 0; gi < S; ++gi) {
                            // orders g = a + b <= S - 1 only
                            const int a0 = 0;
                            const int a1 = gi;
                            for (int a = a0; a <= a1; ++a) {
                                const int b = gi - a;
                                const uint64_t da = smem_desc_sw64(sa + a * kAPlane + kk * 32);
                                const uint64_t db = smem_desc_sw64(sb + b * kBPlane + kk * 32);
                                const int acc = (c == 0 && kk == 0 && a == a0) ? 0 : 1;
                                mma_bf16(tmem + (uint32_t)(gi * kBN), da, db, idesc, acc);
                                issued = true;
                            }
                        }
                    }
                    mma_commit(empty + stage);
                    if (++stage == g.stages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                mma_commit(accf);
                acc_phase ^= 1;
            }
            if (issued) {
                // all issued MMAs complete before TMEM can be released
                mma_commit(drain);
                mbar_wait(drain, 0, g.flag, 4);
            }
        }
    } else {
        // epilogue: warps 2..5
        const int sub = warp & 3;
        const int row_in_tile = 32 * sub + lane;
        uint32_t acc_phase = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int ti, tj;
            tile_coords(t, tiles_n, g.lower, ti, tj);
            if (!mbar_wait(accf, acc_phase, g.flag, 5)) break;
            tc_fence_after();
            const int i = ti * kBM + row_in_tile;
            const int eA = g.expA ? g.expA[g.a_row0 + i] : 0;
            long long* crow = g.C + (int64_t)i * g.ldc + (int64_t)tj * kBN;
            const uint32_t trow = tmem + ((uint32_t)(32 * sub) << 16);
            for (int cc = 0; cc < kBN / 16; ++cc) {
                float v[S][16];
#pragma unroll
                for (int gi = 0; gi < S; ++gi) tmem_ld16(trow + (uint32_t)(gi * kBN + cc * 16), v[gi]);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = tj * kBN + cc * 16 + j;
                    const int eB = g.expB ? g.expB[g.b_row0 + col] : 0;
                    const int sh0 = eA + eB + g.shift0;
                    long long acc = 0;
#pragma unroll
                    for (int gi = 0; gi < S; ++gi) {
                        const long long p = (long long)__float2int_rn(v[gi][j]);
                        const int sh = sh0 - 8 * gi;
                        if (sh >= 0) {
                            acc += (long long)((unsigned long long)p << (sh > 62 ? 62 : sh));
                        } else if (sh > -62) {
                            acc += (p + (1ll << (-sh - 1))) >> (-sh);
                        }
                    }
                    long long* cp = crow + cc * 16 + j;
                    if (g.sub) *cp -= acc;
                    else *cp = acc;
                }
            }
            tc_fence_before();
            mbar_arrive(acce);
            acc_phase ^= 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ---------------------------------------------------------------------------
// Digit split of int64 fixed-point rows (Q(F)), K = 128 values per row, one
// warp per row.  exp_mode 0: the row exponent is `fixed_exp`; 1: the smallest
// e with |v| < 2^e (from the row maximum).  Writes s bf16 planes and expo[].
__device__ __forceinline__ void split_digits(long long w, int s, float* d) {
    // balanced base-256 digits from the least significant; top digit in [-128, 128]
    for (int a = s - 1; a > 0; --a) {
        long long lo = ((w + 128) & 255) - 128;
        d[a] = (float)lo;
        w = (w - lo) >> 8;
    }
    d[0] = (float)w;
}

__device__ __forceinline__ long long round_shift(long long v, int sh) {
    if (sh >= 0) return (long long)((unsigned long long)v << sh);
    if (sh <= -63) return 0;
    return (v + (1ll << (-sh - 1))) >> (-sh);
}

__global__ void slice_rows_kernel(int rows, const long long* __restrict__ src, int64_t ld, int F, int exp_mode,
                                  int fixed_exp, int s, int plane_rows, __nv_bfloat16* __restrict__ dst,
                                  int* __restrict__ expo) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    long long v[4];
    unsigned long long mx = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = src[(int64_t)r * ld + lane + 32 * q];
        unsigned long long a = (unsigned long long)(v[q] < 0 ? -v[q] : v[q]);
        mx = a > mx ? a : mx;
    }
    int e = fixed_exp;
    if (exp_mode == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = t > mx ? t : mx;
        }
        e = mx == 0 ? 0 : (64 - __clzll((long long)mx)) - F;
    }
    if (lane == 0) expo[r] = e;
    const int T = 7 + 8 * (s - 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float d[7];
        split_digits(round_shift(v[q], T - e - F), s, d);
        for (int a = 0; a < s; ++a)
            dst[((int64_t)a * plane_rows + r) * kNB + lane + 32 * q] = __float2bfloat16_rn(d[a]);
    }
}

// Column split: a 128-row block of an int64 Q(F) matrix, columns [0, ncols),
// transposed into digit rows (row = column of the source, K = source row),
// per-column exponent from the column maximum.  One warp per column.
__global__ void slice_cols_kernel(int ncols, const long long* __restrict__ src, int64_t ld, int F, int s,
                                  int plane_rows, __nv_bfloat16* __restrict__ dst, int* __restrict__ expo) {
    __shared__ long long tile[kNB][33];
    const int c0 = blockIdx.x * 32;
    const int tid = threadIdx.x;  // 256 threads
    for (int e = tid; e < kNB * 32; e += 256) {
        int r = e >> 5, c = e & 31;
        tile[r][c] = (c0 + c < ncols) ? src[(int64_t)r * ld + c0 + c] : 0;
    }
    __syncthreads();
    const int lane = tid & 31, w = tid >> 5;
    for (int c = w; c < 32; c += 8) {
        const int col = c0 + c;
        if (col >= ncols) break;
        long long v[4];
        unsigned long long mx = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = tile[lane + 32 * q][c];
            unsigned long long a = (unsigned long long)(v[q] < 0 ? -v[q] : v[q]);
            mx = a > mx ? a : mx;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = t > mx ? t : mx;
        }
        const int e = mx == 0 ? 0 : (64 - __clzll((long long)mx)) - F;
        if (lane == 0) expo[col] = e;
        const int T = 7 + 8 * (s - 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float d[7];
            split_digits(round_shift(v[q], T - e - F), s, d);
            for (int a = 0; a < s; ++a)
                dst[((int64_t)a * plane_rows + col) * kNB + lane + 32 * q] = __float2bfloat16_rn(d[a]);
        }
    }
}

// Rows of a 128 x 128 FP64 matrix (the inverse of a diagonal block), per-row
// exponent; w = round(v 2^(T - e)) is exact in double (|w| <= 2^T <= 2^55).
__global__ void slice_f64_kernel(const double* __restrict__ src, int s, int plane_rows,
                                 __nv_bfloat16* __restrict__ dst, int* __restrict__ expo) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= kNB) return;
    double v[4];
    double mx = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = src[r * kNB + lane + 32 * q];
        mx = fmax(mx, fabs(v[q]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) {
        frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): mx < 2^e
    }
    if (lane == 0) expo[r] = e;
    const int T = 7 + 8 * (s - 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float d[7];
        long long w = llrint(ldexp(v[q], T - e));
        split_digits(w, s, d);
        for (int a = 0; a < s; ++a)
            dst[((int64_t)a * plane_rows + r) * kNB + lane + 32 * q] = __float2bfloat16_rn(d[a]);
    }
}

// Lower triangle of Z_s = D (Z + F G^T) D written as Q60 int64 in place
// (padded rows/columns: identity).
__global__ void zscale_q_kernel(int64_t N, int64_t Np, double* __restrict__ Z, const double* __restrict__ F,
                                const double* __restrict__ G, const double* __restrict__ D) {
    int64_t bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    int64_t i = bi * 32 + threadIdx.y, j = bj * 32 + threadIdx.x;
    if (i >= Np || j > i) return;
    double* z = Z + i * Np + j;
    long long* q = reinterpret_cast<long long*>(z);
    if (i >= N || j >= N) { *q = (i == j) ? (1ll << kFL) : 0; return; }
    double v = *z;
    const double* fi = F + 7 * i;
    const double* gj = G + 7 * j;
#pragma unroll
    for (int k = 0; k < 7; ++k) v += fi[k] * gj[k];
    *q = llrint(ldexp(D[i] * v * D[j], kFL));
}

// Cholesky of the 128 x 128 diagonal block from Q60, in FP64 shared memory;
// writes L back as Q60 and its inverse (FP64) to Linv.
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void __launch_bounds__(512)
potrf_diag_q_kernel(long long* __restrict__ Z, int64_t ld, int64_t k0, double* __restrict__ Linv, int* flag) {
    extern __shared__ __align__(16) double sh[];
    double* S = sh;
    double* Xs = sh + kNB * (kNB + 1) / 2;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const double sc = ldexp(1.0, -kFL);
    for (int e = tid; e < kNB * kNB; e += nt) {
        int i = e / kNB, j = e % kNB;
        if (j <= i) S[pk(i, j)] = (double)Z[(k0 + i) * ld + k0 + j] * sc;
    }
    __syncthreads();
    for (int j = 0; j < kNB; ++j) {
        if (tid == 0) {
            double d = S[pk(j, j)];
            if (!(d > 0.0)) { set_flag(flag, DEV_NOT_SPD, (int)(k0 + j)); d = 1.0; }
            S[pk(j, j)] = sqrt(d);
        }
        __syncthreads();
        double inv = 1.0 / S[pk(j, j)];
        for (int i = j + 1 + tid; i < kNB; i += nt) S[pk(i, j)] *= inv;
        __syncthreads();
        for (int i = j + 1 + warp; i < kNB; i += nw) {
            double lij = S[pk(i, j)];
            for (int l = j + 1 + lane; l <= i; l += 32) S[pk(i, l)] -= lij * S[pk(l, j)];
        }
        __syncthreads();
    }
    for (int e = tid; e < kNB * kNB; e += nt) {
        int i = e / kNB, j = e % kNB;
        if (j <= i) Z[(k0 + i) * ld + k0 + j] = llrint(ldexp(S[pk(i, j)], kFL));
    }
    if (tid < kNB) {
        const int c = tid;
        Xs[pk(c, c)] = 1.0 / S[pk(c, c)];
        for (int i = c + 1; i < kNB; ++i) {
            double s = 0.0;
            for (int k = c; k < i; ++k) s += S[pk(i, k)] * Xs[pk(k, c)];
            Xs[pk(i, c)] = -s / S[pk(i, i)];
        }
    }
    __syncthreads();
    for (int e = tid; e < kNB * kNB; e += nt) {
        int i = e / kNB, j = e % kNB;
        Linv[e] = (j <= i) ? Xs[pk(i, j)] : 0.0;
    }
}

// Camera Gram blocks Sig_c += X[k, c]^T X[k, c] from the finished Q42 row
// block k of X (128 rows), 4 cameras (36 columns) per CTA.
constexpr int kGW = 36;
__global__ void __launch_bounds__(128)
gram_q_kernel(int64_t n, int64_t Np, int64_t k0, int64_t ncols, const long long* __restrict__ R,
              double* __restrict__ Sig) {
    __shared__ double T[kNB][kGW + 1];
    const int tid = threadIdx.x;
    const int64_t c0 = blockIdx.x * (int64_t)kGW;
    const double sc = ldexp(1.0, -kFX);
    for (int e = tid; e < kNB * kGW; e += 128) {
        int r = e / kGW, c = e % kGW;
        int64_t gc = c0 + c;
        T[r][c] = (gc < ncols) ? (double)R[(k0 + r) * Np + gc] * sc : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < 4 * 81; e += 128) {
        int g = e / 81, ab = e % 81, a = ab / 9, b = ab % 9;
        int64_t cam = (c0 / 9) + g;
        if (cam >= n || c0 + 9 * g >= ncols) continue;
        double v = 0.0;
        for (int r = 0; r < kNB; ++r) v += T[r][9 * g + a] * T[r][9 * g + b];
        Sig[81 * cam + ab] += v;
    }
}

__global__ void identity_q_kernel(int64_t Np, long long* X) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < Np) X[i * Np + i] = 1ll << kFX;
}

// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* map, __nv_bfloat16* buf, int s, int64_t plane_rows, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kNB, (cuuint64_t)(s * plane_rows)};
    cuuint64_t strides[1] = {(cuuint64_t)kNB * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, buf, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t gemm_smem(int s, int stages) {
    return 1024 + (size_t)stages * s * (kAPlane + kBPlane) + 8 * (2 * stages + 3) + 16;
}

int g_num_sms = 0;

template <int S>
void set_gemm_attr(size_t smem) {
    cudaFuncSetAttribute(ozaki_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void launch_ozaki(Ctx& c, const CUtensorMap& mA, const CUtensorMap& mB, int M, int N, int a_row0, int b_row0,
                  int lower, int sub, int Fc, const int* expA, const int* expB, long long* C, int64_t ldc) {
    MixedState& st = *c.mixed;
    GemmArgs g;
    g.M = M; g.N = N; g.s = st.s; g.plane_rows = (int)c.Np; g.a_row0 = a_row0; g.b_row0 = b_row0;
    g.lower = lower; g.sub = sub; g.shift0 = Fc - 14; g.expA = expA; g.expB = expB; g.C = C; g.ldc = ldc;
    g.stages = st.stages; g.flag = c.d_flag;
    const int tiles_m = M / kBM, tiles_n = N / kBN;
    int64_t ntiles;
    if (lower) {
        int T0 = tiles_n / 2;
        ntiles = tiles_m <= T0 ? (int64_t)tiles_m * tiles_m + tiles_m
                               : (int64_t)T0 * T0 + T0 + (int64_t)(tiles_m - T0) * tiles_n;
    } else {
        ntiles = (int64_t)tiles_m * tiles_n;
    }
    int grid = (int)(ntiles < g_num_sms ? ntiles : g_num_sms);
    if (grid < 1) return;
    // executed tensor-core work: every kept tile, every digit product
    const double flops = (double)ntiles * 2.0 * kBM * kBN * kNB * (st.s * (st.s + 1) / 2);
    const size_t smem = gemm_smem(st.s, st.stages);
    prof_begin(c);
    switch (st.s) {
        case 4: ozaki_gemm_kernel<4><<<grid, 192, smem, c.stream>>>(mA, mB, g); break;
        case 5: ozaki_gemm_kernel<5><<<grid, 192, smem, c.stream>>>(mA, mB, g); break;
        case 6: ozaki_gemm_kernel<6><<<grid, 192, smem, c.stream>>>(mA, mB, g); break;
        default: ozaki_gemm_kernel<7><<<grid, 192, smem, c.stream>>>(mA, mB, g); break;
    }
    prof_end(c, flops);
    c.launches++;
    st.tiles_done += ntiles;
}

}  // namespace

cudaError_t mixed_alloc(Ctx& c) {
    c.mixed = new MixedState();
    MixedState& st = *c.mixed;
    st.s = c.opt.mixed_slices;
    const int64_t Np = c.Np;
    size_t plane = (size_t)st.s * Np * kNB;
    cudaError_t e;
    if ((e = cudaMalloc(&st.digP, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.digQ, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expP, Np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expQ, Np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.R, Np * Np * sizeof(long long))) != cudaSuccess) return e;
    c.bytes += (int64_t)(plane * 4 + Np * 8 + Np * Np * 8);
    if ((e = cudaMemset(st.digP, 0, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMemset(st.digQ, 0, plane * 2)) != cudaSuccess) return e;
    if (!make_map(&st.mapP128, st.digP, st.s, Np, kBM) || !make_map(&st.mapP64, st.digP, st.s, Np, kBN) ||
        !make_map(&st.mapQ128, st.digQ, st.s, Np, kBM) || !make_map(&st.mapQ64, st.digQ, st.s, Np, kBN))
        return cudaErrorInvalidValue;
    size_t budget = 227 * 1024;
    st.stages = 4;
    while (st.stages > 2 && gemm_smem(st.s, st.stages) > budget) --st.stages;
    if (gemm_smem(st.s, st.stages) > budget) return cudaErrorInvalidConfiguration;
    set_gemm_attr<4>(gemm_smem(st.s, st.stages));
    set_gemm_attr<5>(gemm_smem(st.s, st.stages));
    set_gemm_attr<6>(gemm_smem(st.s, st.stages));
    set_gemm_attr<7>(gemm_smem(st.s, st.stages));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(potrf_diag_q_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(double) * kNB * (kNB + 1)))) != cudaSuccess)
        return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    return cudaSuccess;
}

void mixed_free(Ctx& c) {
    if (!c.mixed) return;
    MixedState& st = *c.mixed;
    void* ptrs[] = {st.digP, st.digQ, st.expP, st.expQ, st.R};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete c.mixed;
    c.mixed = nullptr;
}

// Z_s (lower triangle, FP64 from the shared preparation) -> Q60, then the
// blocked Cholesky and the blocked triangular inverse on the tensor cores.
cudaError_t mixed_factor_inverse(Ctx& c) {
    MixedState& st = *c.mixed;
    const int64_t Np = c.Np, nb = Np / kNB;
    const int s = st.s;
    long long* Zq = reinterpret_cast<long long*>(c.d_Z);
    {
        int64_t nt = (Np + 31) / 32;
        zscale_q_kernel<<<dim3((unsigned)nt, (unsigned)nt), dim3(32, 32), 0, c.stream>>>(c.N, Np, c.d_Z, c.d_F,
                                                                                       c.d_G, c.d_D);
        c.launches++;
    }
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB;
        double* Linv = c.d_Linv + kb * kNB * kNB;
        potrf_diag_q_kernel<<<1, 512, sizeof(double) * kNB * (kNB + 1), c.stream>>>(Zq, Np, k0, Linv, c.d_flag);
        c.launches++;
        if (rem <= 0) continue;
        // panel: L21 = A21 L_kk^-T (A21 bounded by 1: exponent 0)
        slice_rows_kernel<<<(int)((rem + 7) / 8), 256, 0, c.stream>>>(
            (int)rem, Zq + (k0 + kNB) * Np + k0, Np, kFL, 0, 0, s, (int)Np, st.digP, st.expP);
        slice_f64_kernel<<<kNB / 8, 256, 0, c.stream>>>(Linv, s, (int)Np, st.digQ, st.expQ);
        c.launches += 2;
        launch_ozaki(c, st.mapP128, st.mapQ64, (int)rem, kNB, 0, 0, 0, 0, kFL, nullptr, st.expQ,
                     Zq + (k0 + kNB) * Np + k0, Np);
        // trailing update A22 -= L21 L21^T on lower tiles
        slice_rows_kernel<<<(int)((rem + 7) / 8), 256, 0, c.stream>>>(
            (int)rem, Zq + (k0 + kNB) * Np + k0, Np, kFL, 0, 0, s, (int)Np, st.digP, st.expP);
        c.launches++;
        launch_ozaki(c, st.mapP128, st.mapP64, (int)rem, (int)rem, 0, 0, 1, 1, kFL, nullptr, nullptr,
                     Zq + (k0 + kNB) * Np + k0 + kNB, Np);
    }
    cudaEventRecord(c.ev[3], c.stream);
    // triangular inverse X = L^-1 in Q42, row block by row block
    cudaError_t e = cudaMemsetAsync(st.R, 0, sizeof(long long) * Np * Np, c.stream);
    if (e != cudaSuccess) return e;
    identity_q_kernel<<<(int)((Np + 255) / 256), 256, 0, c.stream>>>(Np, st.R);
    c.launches++;
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB, nc = k0 + kNB;
        const double* Linv = c.d_Linv + kb * kNB * kNB;
        // X[k, :nc] = L_kk^-1 R[k, :nc]
        slice_cols_kernel<<<(int)((nc + 31) / 32), 256, 0, c.stream>>>((int)nc, st.R + k0 * Np, Np, kFX, s,
                                                                        (int)Np, st.digQ, st.expQ);
        slice_f64_kernel<<<kNB / 8, 256, 0, c.stream>>>(Linv, s, (int)Np, st.digP, st.expP);
        c.launches += 2;
        launch_ozaki(c, st.mapP128, st.mapQ64, kNB, (int)nc, 0, 0, 0, 0, kFX, st.expP, st.expQ, st.R + k0 * Np, Np);
        gram_q_kernel<<<(int)((nc + kGW - 1) / kGW), 128, 0, c.stream>>>(c.n, Np, k0, nc, st.R, c.d_Sig);
        c.launches++;
        if (rem <= 0) continue;
        // R[k+1:, :nc] -= L[k+1:, k] X[k, :nc]
        slice_cols_kernel<<<(int)((nc + 31) / 32), 256, 0, c.stream>>>((int)nc, st.R + k0 * Np, Np, kFX, s,
                                                                        (int)Np, st.digQ, st.expQ);
        slice_rows_kernel<<<(int)((rem + 7) / 8), 256, 0, c.stream>>>(
            (int)rem, Zq + (k0 + kNB) * Np + k0, Np, kFL, 0, 0, s, (int)Np, st.digP, st.expP);
        c.launches += 2;
        launch_ozaki(c, st.mapP128, st.mapQ64, (int)rem, (int)nc, 0, 0, 0, 1, kFX, nullptr, st.expQ,
                     st.R + (k0 + kNB) * Np, Np);
    }
    return cudaGetLastError();
}

}  // namespace ccov

// Test hook (include/ccov_testing.h): one call of the digit-split tensor-core
// GEMM on caller data, with its own temporary workspace.
extern "C" CCOV_API ccov_status ccov_test_ozaki_gemm(int s, int M, int N, const uint16_t* digA, const int* expA,
                                                    const uint16_t* digB, const int* expB, int Fc, int sub,
                                                    int lower, long long* C) {
    using namespace ccov;
    if (s < 4 || s > 7 || M <= 0 || N <= 0 || M % kBM || N % kBN || !digA || !digB || !C)
        return CCOV_ERR_INVALID_ARG;
    if (lower && N != M) return CCOV_ERR_INVALID_ARG;
    Ctx c;
    c.opt.mixed_slices = s;
    c.opt.precision = CCOV_PREC_MIXED;
    c.Np = M > N ? M : N;
    c.N = c.Np;
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) return CCOV_ERR_CUDA;
    ccov_status st = CCOV_OK;
    long long* dC = nullptr;
    int* dEA = nullptr;
    int* dEB = nullptr;
    do {
        if (mixed_alloc(c) != cudaSuccess) { st = CCOV_ERR_CUDA; break; }
        MixedState& ms = *c.mixed;
        if (cudaMalloc(&c.d_flag, 2 * sizeof(int)) != cudaSuccess) { st = CCOV_ERR_OOM; break; }
        cudaMemset(c.d_flag, 0, 2 * sizeof(int));
        for (int a = 0; a < s; ++a) {
            cudaMemcpy(ms.digP + (size_t)a * c.Np * kNB, digA + (size_t)a * M * kNB, (size_t)M * kNB * 2,
                       cudaMemcpyHostToDevice);
            cudaMemcpy(ms.digQ + (size_t)a * c.Np * kNB, digB + (size_t)a * N * kNB, (size_t)N * kNB * 2,
                       cudaMemcpyHostToDevice);
        }
        if (expA) { cudaMalloc(&dEA, M * sizeof(int)); cudaMemcpy(dEA, expA, M * sizeof(int), cudaMemcpyHostToDevice); }
        if (expB) { cudaMalloc(&dEB, N * sizeof(int)); cudaMemcpy(dEB, expB, N * sizeof(int), cudaMemcpyHostToDevice); }
        if (cudaMalloc(&dC, (size_t)M * N * 8) != cudaSuccess) { st = CCOV_ERR_OOM; break; }
        cudaMemcpy(dC, C, (size_t)M * N * 8, cudaMemcpyHostToDevice);
        launch_ozaki(c, ms.mapP128, ms.mapQ64, M, N, 0, 0, lower, sub, Fc, dEA, dEB, dC, N);
        if (cudaStreamSynchronize(c.stream) != cudaSuccess) { st = CCOV_ERR_CUDA; break; }
        int flag[2];
        cudaMemcpy(flag, c.d_flag, sizeof flag, cudaMemcpyDeviceToHost);
        if (flag[0] == DEV_TIMEOUT) { st = CCOV_ERR_TIMEOUT; break; }
        cudaMemcpy(C, dC, (size_t)M * N * 8, cudaMemcpyDeviceToHost);
    } while (0);
    if (dC) cudaFree(dC);
    if (dEA) cudaFree(dEA);
    if (dEB) cudaFree(dEB);
    if (c.d_flag) cudaFree(c.d_flag);
    mixed_free(c);
    cudaStreamDestroy(c.stream);
    return st;
}

// Mixed-precision step (d): the Cholesky factorisation and triangular inverse
// of the Jacobi-scaled reduced camera matrix with every O(N^3) trailing
// update on the 5th-generation tensor cores (tcgen05, bf16 operands, fp32
// accumulation in TMEM, operands and result tiles moved by TMA).
//
// Accuracy is kept by an error-free split of the operands into 8-bit digits
// (after Ozaki et al., "Error-free transformations of matrix multiplication
// by using fast routines of matrix multiplication and its applications",
// 2012): a row with exponent e holds v = 2^e sum_a d_a 2^-(7 + 8(a-1)),
// d_a integers in [-128, 128] that bf16 represents exactly.  A product of two
// digits has at most 14 bits and a sum of K of them at most 14 + log2 K, so
// 1024 / K digit products of one order g = a + b sum exactly in one fp32
// TMEM accumulator (below 2^24); an order with more products gets a second
// accumulator.  Orders above s - 1 are dropped (relative truncation about
// 2^-(8 s)).  The working matrices are held in int64 fixed point (Q60 for
// the factor, whose entries are bounded by 1 after Jacobi scaling; Q42 for
// the inverse), where the exact partial products are added by integer
// shifts: no FP64 arithmetic in the O(N^3) part.
//
// Blocking: 128-column sub-panels factored and inverted one at a time, with
// the big trailing updates applied for four sub-panels at once (K = 512; two,
// K = 256, for scenes under 64 sub-panels and for s = 6).  The
// diagonal blocks are factored and inverted by one CTA in double-single
// arithmetic.  The triangular inverse runs on a second stream, each pair of
// row blocks as soon as the Cholesky has finished the same pair of columns,
// so that its GEMMs fill the GPU while the Cholesky's serial steps run.
//
// Paper counterpart: the dense inversion of Z_p (Sec. 4.2); the paper runs it
// in double precision with LAPACK on a CPU.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "ccov_internal.cuh"
#include "ds_arith.cuh"
#include "group.cuh"
#include "tc_ptx.cuh"
#include "../../include/ccov_testing.h"

namespace ccov {

constexpr int kBM = 128, kBN = 64, kKS = 16;              // tile M x N, K per pipeline stage
constexpr int kAPl = kBM * kKS * 2;                        // 4 KB: one digit plane of A per stage
constexpr int kBPl = kBN * kKS * 2;                        // 2 KB
constexpr int kCBox = kBM * 16 * 8;                        // 16 KB: 16 int64 columns x 128 rows
constexpr int kCTile = kCBox;                              // 16 KB: a quarter of the result tile, staged for TMA
constexpr int kFX = 42;                                    // fixed point of X = L^-1
constexpr int kFL = 60;                                    // fixed point of Z_s and L
constexpr int kKMax = 512;                                 // digit columns of the per-scene buffers
constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;              // producer, MMA, epilogue warps
constexpr int kEpiCols = kBN / (kEpiWarps / 4);            // tile columns per epilogue thread

struct MixedState {
    int s = 5;
    __nv_bfloat16* digP = nullptr;   // s digit planes of Np rows x kKMax, layout of blk_off
    __nv_bfloat16* digQ = nullptr;
    int* expP = nullptr;             // Np
    int* expQ = nullptr;             // Np
    long long* R = nullptr;          // Np x Np, Q42
    CUtensorMap mapZ, mapR;          // int64 result maps
    CUtensorMap mapBP, mapBQ;        // B-operand views of digP and digQ
    __nv_bfloat16* digL = nullptr;   // digits of the inverses of the diagonal blocks (row block b: L_bb^-1)
    int* expL = nullptr;             // their row exponents
    CUtensorMap mapBL;
    // the triangular inverse runs on a second stream with a second set of
    // digit buffers, behind the Cholesky one group of sub-panels at a time
    __nv_bfloat16 *digP2 = nullptr, *digQ2 = nullptr;
    int *expP2 = nullptr, *expQ2 = nullptr;
    CUtensorMap mapBP2, mapBQ2;
    unsigned long long wait_ns = ptx::kWaitNs;  // limit of the GEMM's barrier waits
    long long skip_fill = -1;        // test hook: a pipeline fill the GEMM producer leaves out
    cudaStream_t side = nullptr;     // triangular inverse, lowest priority
    cudaStream_t hi = nullptr;       // Cholesky (the critical path), highest priority
    std::vector<cudaEvent_t> ev;     // [0] fork, [1] inverse done, [2] Cholesky done, [3 + p] group at p final

    void swap_sets() {
        std::swap(digP, digP2);
        std::swap(digQ, digQ2);
        std::swap(expP, expP2);
        std::swap(expQ, expQ2);
        std::swap(mapBP, mapBP2);
        std::swap(mapBQ, mapBQ2);
    }
};

namespace {

using namespace ptx;

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory"); }

// Digit planes are stored in the order the tensor cores read K-major
// operands without swizzle: per 16-wide slice of K, per block of 128 rows
// and per plane, one contiguous 4 KB block of 16 groups of 8 rows, each
// group two 8 x 8 core matrices (8 rows x 16 bytes) along K.  The S planes
// of one row block and K slice are adjacent, so a pipeline stage takes the
// A tile of all planes as one bulk copy and the 64-row B tile of all planes
// (every other 2 KB half block) as one tensor copy.
__host__ __device__ __forceinline__ int64_t blk_off(int plane, int r, int k, int plane_rows, int S) {
    const int64_t rb = plane_rows / 128;
    return (((((int64_t)(k >> 4) * rb + (r >> 7)) * S + plane) << 11) + (((r & 127) >> 3) << 7) +
           (((k & 15) >> 3) << 6) + ((r & 7) << 3) + (k & 7));
}

// Accumulators of the digit orders.  Order g = a + b collects the products
// A_a B_b^T; at most cap = 1024 / K of them sum exactly in one fp32
// accumulator.  Products of A planes a < cap go to the main accumulator of
// their order (TMEM columns 64 g), those of planes a >= cap to a second one
// (columns 64 (S + g - cap)).  With the B planes side by side in shared
// memory, plane a then meets all B planes in one MMA of N = 64 (S - a)
// (split at N = 256), whose output columns land on the orders a .. S-1.
// With S = 2 cap + 1 (S = 5, K = 512) the second accumulator of the lowest
// kept order, g = S - 1, takes cap + 1 products: its sum (below 1.5 2^24)
// may round, by at most a few units of that order per K-step.  Its weight
// is 2^-8(S-1) of the leading order's, so over K = 512 the rounding stays
// near 2^-49 of the largest result, against the 2^-39 of the orders that
// the split drops; every other accumulator stays exact.
template <int S, int K>
struct Slots {
    static constexpr int cap = 1024 / K;
    static constexpr int extra = S > cap ? S - cap : 0;
    static constexpr int total = S + extra;
    static_assert(total * kBN <= 512, "TMEM columns");
    static_assert(S <= 2 * cap + (K == 512 ? 1 : 0), "two accumulator levels at most");
    // digit products summed in accumulator sl (main accumulators of the
    // orders 0..S-1, then the second ones of the orders cap..S-1)
    __host__ __device__ static constexpr int products(int sl) {
        return sl < S ? (sl < cap - 1 ? sl : cap - 1) - (sl > S - 1 ? sl - (S - 1) : 0) + 1
                      : (sl - S + cap) - cap + 1;
    }
    // |P| <= products * K * 2^14 <= 2^22: the biased pattern is exact unchecked
    __host__ __device__ static constexpr bool small(int sl) { return products(sl) * K <= 256; }
};

// Tile schedule: M tiles of 128 rows x N tiles of 64 columns; `lower` keeps
// only tiles that reach the diagonal of a square region (tj*64 <= ti*128+127).
__host__ __device__ __forceinline__ int64_t tile_count(int tiles_m, int tiles_n, int lower) {
    if (!lower) return (int64_t)tiles_m * tiles_n;
    int T0 = tiles_n / 2;
    return tiles_m <= T0 ? (int64_t)tiles_m * tiles_m + tiles_m
                         : (int64_t)T0 * T0 + T0 + (int64_t)(tiles_m - T0) * tiles_n;
}

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

// Combining the accumulators of one element into T = sum_g P_g 2^(8 (S-1-g)).
// Every accumulator holds an integer P with |P| <= 2^24.  combine_converted
// converts each with a float-to-int instruction.  When -2^22 <= P < 2^22,
// P + 1.5 * 2^23 is exact and lies in [2^23, 2^24), so its bit pattern is
// 0x4B400000 + P (sign 0, exponent field 150, checked on the pattern itself);
// combine_biased sums those patterns with the weights of the orders and
// removes the constants' share at the end, modulo 2^64, which is exact because
// the true T fits in 63 bits.
constexpr float kMagic = 12582912.f;   // 1.5 * 2^23, bit pattern 0x4B400000
constexpr unsigned kMagicTop = 0x96;   // sign and exponent field of [2^23, 2^24)

template <int S, int K>
__device__ __forceinline__ long long combine_converted(const float (&v)[Slots<S, K>::total][8], int j) {
    using SL = Slots<S, K>;
    long long T = 0;
#pragma unroll
    for (int gi = 0; gi < S; ++gi) {
        int p = __float2int_rn(v[gi][j]);
        if (gi >= SL::cap) p += __float2int_rn(v[S + gi - SL::cap][j]);
        T = (long long)((unsigned long long)T << 8) + p;
    }
    return T;
}

template <int S, int K>
__host__ __device__ constexpr unsigned long long magic_share() {
    unsigned long long t = 0;
    for (int gi = 0; gi < S; ++gi) t = (t << 8) + 0x4B400000ull * (gi >= Slots<S, K>::cap ? 2u : 1u);
    return t;
}

template <int S, int K>
__device__ __forceinline__ long long combine_biased(const unsigned (&u)[Slots<S, K>::total][8], int j) {
    using SL = Slots<S, K>;
    unsigned long long T = 0;
#pragma unroll
    for (int gi = 0; gi < S; ++gi) {
        unsigned c = u[gi][j];
        if (gi >= SL::cap) c += u[S + gi - SL::cap][j];   // two patterns < 2^31 each
        T += (unsigned long long)c << (8 * (S - 1 - gi));
    }
    return (long long)(T - magic_share<S, K>());
}

struct TileRef {
    const GemmArgs* a;
    const CUtensorMap* mB;
    const CUtensorMap* mC;
    int ti, tj;
};

// The problem and tile of global tile pair pr for CTA `rank` of its pair.
template <bool Grouped>
__device__ __forceinline__ TileRef locate_tile(int64_t pr, uint32_t rank, const GemmArgs* g, const CUtensorMap* mB,
                                              const CUtensorMap* mC, const GemmProblem* probs, int nprobs) {
    TileRef r;
    int64_t lp = pr;
    if (Grouped) {
        int lo = 0, hi = nprobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].pair0 <= pr) lo = mid;
            else hi = mid - 1;
        }
        r.a = &probs[lo].g;
        r.mB = &probs[lo].mapB;
        r.mC = &probs[lo].mapC;
        lp = pr - probs[lo].pair0;
    } else {
        r.a = g;
        r.mB = mB;
        r.mC = mC;
    }
    tile_coords(2 * lp + rank, r.a->N / kBN, r.a->lower, r.ti, r.tj);
    return r;
}

__device__ __forceinline__ long long shift_round(long long p, int sh) {
    if (sh >= 0) return (long long)((unsigned long long)p << (sh > 62 ? 62 : sh));
    if (sh <= -62) return 0;
    return (p + (1ll << (-sh - 1))) >> (-sh);
}

// Persistent warp-specialised kernel.  CTAs 2P and 2P + 1 work on the two
// halves (adjacent 64-column tiles) of one 128 x 128 block at about the same
// time, so the A tile that both read is fetched from DRAM once and served to
// the second from L2; each CTA copies every operand it uses into its own
// shared memory.  Warp 0 lane 0: producer of the digit tiles.
// Warp 1: TMEM allocation; lane 0 issues tcgen05.mma.  Warps 2..17:
// epilogue; warp w reads TMEM lanes 32 (w % 4) .. +31 and one quarter of the
// 64 columns.  The result tile leaves through shared memory with TMA, a
// quarter at a time: C -= A B^T as a reduce-add of -A B^T into C (the
// addition happens in L2, so C is never read into the SM), C = A B^T as a
// plain store.  Grouped: the tile pairs of `nprobs` problems are numbered
// one after the other and every CTA finds the problem of each of its pairs.
template <int S, int K, bool Grouped>
// 18 warps: two of the SM's four register files host five warps each, which
// caps a thread at 96 registers
__global__ void __launch_bounds__(kThreads, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mapC, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ GemmArgs g, const GemmProblem* __restrict__ probs, int nprobs) {
    using SL = Slots<S, K>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the 128-byte-swizzled staging buffer needs a 1024-byte aligned start;
    // the launch reserves no padding for it (the space holds a pipeline
    // stage), so a misaligned window is reported instead of used
    if (smem_u32(smem_raw) & 1023u) {
        if (threadIdx.x == 0) set_flag(g.flag, DEV_SMEM_ALIGN, 0);
        return;
    }
    unsigned char* base = smem_raw;
    constexpr int stage_bytes = S * (kAPl + kBPl);
    unsigned char* ctile = base;
    unsigned char* tiles = base + kCTile;
    uint64_t* bars = (uint64_t*)(tiles + g.stages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + g.stages;
    uint64_t* accf = bars + 2 * g.stages;
    uint64_t* acce = accf + 1;
    uint64_t* drain = acce + 1;
    uint32_t* tmem_slot = (uint32_t*)(drain + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles come in pairs (2P, 2P + 1) in one row of tiles; CTA 2c + rank
    // takes tile 2P + rank of every pair P of CTA pair c (the grid is even)
    const uint32_t rank = blockIdx.x & 1;
    const int64_t npairs = Grouped ? g.total_pairs : tile_count(g.M / kBM, g.N / kBN, g.lower) / 2;
    const int64_t pair0 = blockIdx.x >> 1, pair_step = gridDim.x >> 1;
    const unsigned long long wlim = g.wait_ns;

    if (threadIdx.x == 0) {
        for (int i = 0; i < g.stages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);  // released by this CTA's MMAs
        }
        mbar_init(accf, 1);
        mbar_init(acce, kEpiWarps);
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
            long long fill = 0;
            for (int64_t pr = pair0; pr < npairs && ok; pr += pair_step) {
                const TileRef tr = locate_tile<Grouped>(pr, rank, &g, &mapB, &mapC, probs, nprobs);
                const GemmArgs& a = *tr.a;
                for (int ks = 0; ks < K / kKS; ++ks, ++fill) {
                    if (!mbar_wait(empty + stage, phase ^ 1, g.flag, 1, wlim)) { ok = false; break; }
                    if (fill != g.skip_fill) {
                        unsigned char* st = tiles + stage * stage_bytes;
                        mbar_expect_tx(full + stage, (uint32_t)stage_bytes);
                        // A: all digit planes of the 128-row tile, adjacent in memory
                        bulk_load(st, a.digA + blk_off(0, a.a_row0 + tr.ti * kBM, ks * kKS, a.plane_rows, S),
                                  (uint32_t)(S * kAPl), full + stage);
                        // B: this CTA's 64 rows of every plane, one tensor copy
                        const int br = a.b_row0 + tr.tj * kBN;
                        tma_load_5d(st + S * kAPl, tr.mB, full + stage, 0, 0, (br >> 6) & 1, 0,
                                    ks * (a.plane_rows >> 7) + (br >> 7));
                    }
                    if (++stage == g.stages) { stage = 0; phase ^= 1; }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, acc_phase = 0;
            bool ok = true, issued = false;

            for (int64_t pr = pair0; pr < npairs && ok; pr += pair_step) {
                if (!mbar_wait(acce, acc_phase ^ 1, g.flag, 2, wlim)) break;
                tc_fence_after();
                for (int ks = 0; ks < K / kKS; ++ks) {
                    if (!mbar_wait(full + stage, phase, g.flag, 3, wlim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(tiles + stage * stage_bytes);
                    const uint32_t sb = sa + S * kAPl;
                    const uint64_t dA0 = smem_desc_kmajor(sa), dB0 = smem_desc_kmajor(sb);
#pragma unroll
                    for (int a = 0; a < S; ++a) {
                        const bool second = a >= SL::cap;
                        const int slot0 = second ? S + a - SL::cap : a;  // accumulator of order a
                        const int first_a = second ? SL::cap : 0;
#pragma unroll
                        for (int c = 0; 4 * c < S - a; ++c) {
                            const int nb = (S - a - 4 * c) < 4 ? (S - a - 4 * c) : 4;  // B planes in this MMA
                            mma_bf16(tmem + (uint32_t)((slot0 + 4 * c) * kBN), dA0 + (uint64_t)(a * (kAPl >> 4)),
                                     dB0 + (uint64_t)(4 * c * (kBPl >> 4)), idesc_bf16(kBM, kBN * nb),
                                     (ks == 0 && a == first_a) ? 0 : 1);
                            issued = true;
                        }
                    }
                    mma_commit(empty + stage);  // the stage is free once these MMAs have read it
                    if (++stage == g.stages) { stage = 0; phase ^= 1; }
                }
                if (!ok) break;
                mma_commit(accf);
                acc_phase ^= 1;
            }
            if (issued) {
                // every issued MMA completes before TMEM is released
                mma_commit(drain);
                mbar_wait(drain, 0, g.flag, 4, wlim);
            }
        }
    } else {
        const int quarter = warp & 3;
        const int part = (warp - 2) >> 2;   // which kEpiCols columns
        const int r = 32 * quarter + lane;  // row in the tile = TMEM lane
        const bool leader = (warp == 2 && lane == 0);
        uint32_t acc_phase = 0;
        for (int64_t pr = pair0; pr < npairs; pr += pair_step) {
            const TileRef tr = locate_tile<Grouped>(pr, rank, &g, &mapB, &mapC, probs, nprobs);
            const GemmArgs& a = *tr.a;
            const int ti = tr.ti, tj = tr.tj;
            const int cx = a.c_x0 + tj * kBN, cy = a.c_y0 + ti * kBM;
            if (leader) bulk_wait_read0();  // the previous tile's copy-out has left shared memory
            epi_bar();
            // warp-uniform: the vote, the re-read and the arrival below are per warp
            if (!__all_sync(0xffffffffu, mbar_wait(accf, acc_phase, g.flag, 5, wlim))) break;
            tc_fence_after();
            // phase 1: drain the accumulators into exact int64 sums (registers),
            // then release TMEM so that the next tile's MMAs start at once;
            // everything else waits until after the release
            const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
            long long res[kEpiCols];
#pragma unroll
            for (int cc = 0; cc < kEpiCols / 8; ++cc) {
                const int col0 = kEpiCols * part + 8 * cc;  // column within the tile
                float v[SL::total][8];
#pragma unroll
                for (int sl = 0; sl < SL::total; ++sl) tmem_ld8(trow + (uint32_t)(sl * kBN + col0), v[sl]);
                tmem_wait_ld();
#pragma unroll
                for (int sl = 0; sl < SL::total; ++sl) tmem_regs_after_wait<8>(v[sl]);
                // T = sum_g P_g 2^(8 (S-1-g)) exactly (|T| < 2^63); the usual
                // case takes the biased bit patterns, the rare one (some
                // |P| > 2^22 in the warp) reads the chunk again and converts
                unsigned u[SL::total][8];
                unsigned all_and = 0x4B400000u, all_or = 0x4B400000u;   // the pattern of 0
#pragma unroll
                for (int sl = 0; sl < SL::total; ++sl)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        u[sl][j] = __float_as_uint(__fadd_rn(v[sl][j], kMagic));
                        if (!SL::small(sl)) {   // accumulators of one product need no check
                            all_and &= u[sl][j];
                            all_or |= u[sl][j];
                        }
                    }
                if (__all_sync(0xffffffffu, (all_and >> 23) == kMagicTop && (all_or >> 23) == kMagicTop)) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) res[8 * cc + j] = combine_biased<S, K>(u, j);
                } else {
#pragma unroll
                    for (int sl = 0; sl < SL::total; ++sl) tmem_ld8(trow + (uint32_t)(sl * kBN + col0), v[sl]);
                    tmem_wait_ld();
#pragma unroll
                    for (int sl = 0; sl < SL::total; ++sl) tmem_regs_after_wait<8>(v[sl]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) res[8 * cc + j] = combine_converted<S, K>(v, j);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce);   // one arrival per warp, after all its TMEM reads
            acc_phase ^= 1;
            // one rounding shift of each sum to the fixed point of C
            {
                const int sh = (a.expA ? a.expA[a.a_row0 + ti * kBM + r] : 0) + a.shift0 - 8 * (S - 1);
                const int* eBp = a.expB ? a.expB + a.b_row0 + tj * kBN + kEpiCols * part : nullptr;
#pragma unroll
                for (int q = 0; q < kEpiCols; ++q) res[q] = shift_round(res[q], sh + (eBp ? eBp[q] : 0));
            }
            // phase 2: stage -A B^T (or A B^T) for the copy-out, 16 columns (one
            // part's warps) at a time through a 16 KB buffer, so that the
            // space of the rest of the tile holds two more pipeline stages; two
            // columns (one 16-byte chunk) per access; with the 128-byte swizzle
            // (chunk index XOR row % 8) the 32 rows of a warp spread over all banks
            for (int rd = 0; rd < kBN / kEpiCols; ++rd) {
                if (rd > 0) {
                    if (leader) bulk_wait_read0();   // the previous columns have left shared memory
                    epi_bar();
                }
                if (part == rd) {
#pragma unroll
                    for (int q = 0; q < kEpiCols; q += 2) {
                        longlong2* cp = (longlong2*)(ctile + r * 128 + ((((q >> 1)) ^ (r & 7)) << 4));
                        *cp = a.sub ? make_longlong2(-res[q], -res[q + 1]) : make_longlong2(res[q], res[q + 1]);
                    }
                }
                fence_proxy_async();
                epi_bar();
                if (leader) {
                    if (a.sub) tma_reduce_add_2d(tr.mC, ctile, cx + kEpiCols * rd, cy);
                    else tma_store_2d(tr.mC, ctile, cx + kEpiCols * rd, cy);
                    bulk_commit();
                }
            }
        }
        if (leader) bulk_wait0();
    }
    // after a timeout: every copy this CTA issued was issued before the wait
    // that gave up began (the producer only issues after a stage is freed),
    // so it has landed long before the limit ran out
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ---------------------------------------------------------------------------

__device__ __forceinline__ long long round_shift(long long v, int sh) {
    if (sh >= 0) return (long long)((unsigned long long)v << sh);
    if (sh <= -63) return 0;
    return (v + (1ll << (-sh - 1))) >> (-sh);
}

// Two small integers (|d| <= 256) as a bf16 pair, element 0 in the low half:
// 1.5 * 2^23 + d is exact with bit pattern 0x4B400000 + d, subtracting
// 1.5 * 2^23 leaves d as a float, and the upper half of a float that holds
// such an integer is its exact bf16 encoding.
__device__ __forceinline__ unsigned bf16x2_small(int d0, int d1) {
    const float a = __int_as_float(0x4B400000 + d0) - 12582912.f;
    const float b = __int_as_float(0x4B400000 + d1) - 12582912.f;
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// Digits of eight values consecutive along K (w already in units of the
// last digit, |w| <= 2^(7 + 8 (s-1)) + 1), plane by plane from the least
// significant one: digit = ((w + 128) mod 256) - 128, w <- (w + 128) >> 8.
// The lowest s - 3 digits are taken in 64-bit arithmetic, after which |w| <
// 2^31 and the rest in 32-bit.  Each plane's eight digits (a core-matrix
// row) go out as one 16-byte store.
__device__ __forceinline__ void split_store8(long long* w, int s, __nv_bfloat16* dst0, int64_t plane_stride) {
    int d[8], wi[8];
    for (int a = s - 1; a >= 0; --a) {
        if (a >= 3) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const long long t = w[j] + 128;
                d[j] = (int)(t & 255) - 128;
                w[j] = t >> 8;
                wi[j] = (int)w[j];
            }
        } else if (a > 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int t = wi[j] + 128;
                d[j] = (t & 255) - 128;
                wi[j] = t >> 8;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) d[j] = wi[j];
        }
        uint4 out;
        out.x = bf16x2_small(d[0], d[1]);
        out.y = bf16x2_small(d[2], d[3]);
        out.z = bf16x2_small(d[4], d[5]);
        out.w = bf16x2_small(d[6], d[7]);
        *reinterpret_cast<uint4*>(dst0 + a * plane_stride) = out;
    }
}

// Lane of a warp that covers 16 digit rows x one 16-wide K slice: rows
// (lane & 7) + 8 (lane >> 4), K half (lane >> 3) & 1.  Its 16-byte stores of
// one plane then fill 512 contiguous bytes of the digit layout (two 8-row
// groups of one K slice).
__device__ __forceinline__ int tile16_row(int lane) { return (lane & 7) + 8 * (lane >> 4); }
__device__ __forceinline__ int tile16_khalf(int lane) { return (lane >> 3) & 1; }

// Rows of an int64 Q(F) matrix, K = 128 or 256 values per row, exponent 0
// (entries of the scaled factor are bounded by 1).  A thread takes eight
// consecutive values of a row (64 bytes, read as four 16-byte loads) and
// writes each digit plane with one 16-byte store; a warp covers 16 rows of
// one K slice.  rows is a multiple of 16.
template <int K>
__device__ __forceinline__ void slice_rows_body(int rows, const long long* __restrict__ src, int64_t ld, int F, int s,
                                                int plane_rows, __nv_bfloat16* __restrict__ dst,
                                                int* __restrict__ expo, int* flag, int64_t bid) {
    constexpr int KS = K / 16;
    const int lane = threadIdx.x & 31;
    const int64_t wt = (bid * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int r = (int)(wt / KS) * 16 + tile16_row(lane);
    const int k0 = 16 * (int)(wt % KS) + 8 * tile16_khalf(lane);
    if (r >= rows) return;
    if (k0 == 0) expo[r] = 0;
    const int T = 7 + 8 * (s - 1);
    const longlong2* p = reinterpret_cast<const longlong2*>(src + (int64_t)r * ld + k0);
    long long w[8];
    bool out_of_range = false;
    // entries of the scaled factor are bounded by 1 (2^F): beyond 2^(F+1)
    // the value has left the fixed-point range (or wrapped)
    const long long lim = 1ll << (F + 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const longlong2 v = p[j];
        out_of_range |= v.x > lim || v.x < -lim || v.y > lim || v.y < -lim;
        w[2 * j] = round_shift(v.x, T - F);
        w[2 * j + 1] = round_shift(v.y, T - F);
    }
    if (out_of_range) ptx::set_flag(flag, DEV_RANGE, r);
    split_store8(w, s, dst + blk_off(0, r, k0, plane_rows, s), blk_off(1, 0, 0, plane_rows, s));
}

template <int K>
__global__ void __launch_bounds__(256)
slice_rows_kernel(int rows, const long long* __restrict__ src, int64_t ld, int F, int s, int plane_rows,
                  __nv_bfloat16* __restrict__ dst, int* __restrict__ expo, int* flag) {
    slice_rows_body<K>(rows, src, ld, F, s, plane_rows, dst, expo, flag, blockIdx.x);
}

// Column split: a K-row block (K = 128 or 256) of an int64 Q(F) matrix,
// columns [0, ncols), transposed into digit rows (row = source column,
// K = source rows), per-column exponent from the column maximum.  The block
// stages 32 columns in shared memory; a warp finds each column's exponent,
// then a thread splits eight consecutive source rows of a column and writes
// each digit plane with one 16-byte store (a warp: 16 columns of one K
// slice, so that its stores are contiguous).
template <int K>
__device__ __forceinline__ void slice_cols_body(int ncols, const long long* __restrict__ src, int64_t ld, int F, int s,
                                                int plane_rows, __nv_bfloat16* __restrict__ dst,
                                                int* __restrict__ expo, int* flag, int64_t bid) {
    extern __shared__ __align__(16) long long tile[];   // [K][33]
    __shared__ int cexp[32];
    const int c0 = (int)bid * 32;
    const int tid = threadIdx.x;
    for (int e = tid; e < K * 32; e += 256) {
        int rr = e >> 5, c = e & 31;
        tile[rr * 33 + c] = (c0 + c < ncols) ? src[(int64_t)rr * ld + c0 + c] : 0;
    }
    __syncthreads();
    const int lane = tid & 31, w = tid >> 5;
    for (int c = w; c < 32; c += 8) {
        unsigned long long mx = 0;
#pragma unroll
        for (int q = 0; q < K / 32; ++q) {
            const long long v = tile[(lane + 32 * q) * 33 + c];
            const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
            mx = a > mx ? a : mx;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = t > mx ? t : mx;
        }
        if (lane == 0) {
            const int e = mx == 0 ? 0 : (64 - __clzll((long long)mx)) - F;
            cexp[c] = e;
            if (c0 + c < ncols) expo[c0 + c] = e;
            // an entry of X = L^-1 at 2^19 or beyond: two bits short of the
            // int64 range of its fixed point (a larger one may have wrapped)
            if (mx >= (1ull << 61)) ptx::set_flag(flag, DEV_RANGE, c0 + c);
        }
    }
    __syncthreads();
    const int T = 7 + 8 * (s - 1);
    // warp tiles: 2 halves of the 32 columns x K / 16 slices
    for (int wt = w; wt < 2 * (K / 16); wt += 8) {
        const int c = 16 * (wt & 1) + tile16_row(lane);
        const int k0 = 16 * (wt >> 1) + 8 * tile16_khalf(lane);
        const int col = c0 + c;
        if (col >= ncols) continue;
        const int e = cexp[c];
        long long wv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) wv[j] = round_shift(tile[(k0 + j) * 33 + c], T - e - F);
        split_store8(wv, s, dst + blk_off(0, col, k0, plane_rows, s), blk_off(1, 0, 0, plane_rows, s));
    }
}

template <int K>
__global__ void __launch_bounds__(256)
slice_cols_kernel(int ncols, const long long* __restrict__ src, int64_t ld, int F, int s, int plane_rows,
                  __nv_bfloat16* __restrict__ dst, int* __restrict__ expo, int* flag) {
    slice_cols_body<K>(ncols, src, ld, F, s, plane_rows, dst, expo, flag, blockIdx.x);
}

// Row and column of entry t of a lower triangle stored row by row.
__device__ __forceinline__ void tri_index(int t, int& i, int& l) {
    i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    l = t - i * (i + 1) / 2;
}

// Q60 fixed point <-> double-single (see ds_from_fixed).
__device__ __forceinline__ dsf ds_from_q60(long long v) {
    return ds_from_fixed(v, 8.673617379884035e-19f);  // 2^-60
}

__device__ __forceinline__ long long ds_to_q60(dsf a) {
    constexpr float kU = 1.152921504606847e18f;  // 2^60
    return __float2ll_rn(__fmul_rn(a.h, kU)) + __float2ll_rn(__fmul_rn(a.l, kU));
}


// sqrt(d), 1 / sqrt(d) and 1 / d: one Newton step on the float estimate of
// 1 / sqrt(d) doubles its 22 correct bits.
__device__ __forceinline__ void ds_sqrt_inv(dsf d, dsf& l, dsf& inv, dsf& inv2) {
    const float y0 = rsqrtf(d.h);
    const dsf y = {y0, 0.f};
    const dsf e = ds_fma({1.f, 0.f}, ds_neg(d), ds_mul(y, y));  // 1 - d y0^2
    inv = ds_fma(y, {0.5f * y0, 0.f}, e);                      // y0 + y0 (1 - d y0^2) / 2
    l = ds_mul(d, inv);
    inv2 = ds_mul(inv, inv);
}


// Lower triangle of Z_s = D (Z + F G^T) D written as Q60 int64 in place
// (padded rows/columns: identity), in double-single arithmetic (Z_s is split
// into digits of 39 bits afterwards).  A block covers 32 x 32 entries, a
// thread four consecutive columns of one row; the block's rows of F and D
// (with the 2^60 folded into D_i) and columns of G and D are converted once
// into shared memory.
__device__ __forceinline__ void zscale_q_body(int64_t N, int64_t Np, double* __restrict__ Z,
                                              const double* __restrict__ F, const double* __restrict__ G,
                                              const double* __restrict__ D, long long* __restrict__ Zkeep, int* flag,
                                              int64_t bi, int64_t bj) {
    if (bj > bi) return;
    __shared__ dsf Fs[32][7], Gs[32][7], Dr[32], Dc[32];
    const int tid = threadIdx.y * 8 + threadIdx.x;
    for (int e = tid; e < 2 * 32 * 7 + 64; e += 256) {
        if (e < 224) {
            const int64_t i = bi * 32 + e / 7;
            Fs[e / 7][e % 7] = i < N ? ds_from_double(F[7 * i + e % 7]) : dsf{0.f, 0.f};
        } else if (e < 448) {
            const int q = e - 224;
            const int64_t j = bj * 32 + q / 7;
            Gs[q / 7][q % 7] = j < N ? ds_from_double(G[7 * j + q % 7]) : dsf{0.f, 0.f};
        } else if (e < 480) {
            const int64_t i = bi * 32 + (e - 448);
            Dr[e - 448] = i < N ? ds_from_double(D[i] * 0x1p60) : dsf{0.f, 0.f};
        } else {
            const int64_t j = bj * 32 + (e - 480);
            Dc[e - 480] = j < N ? ds_from_double(D[j]) : dsf{0.f, 0.f};
        }
    }
    __syncthreads();
    const int y = threadIdx.y;
    const int64_t i = bi * 32 + y;
    const int64_t j0 = bj * 32 + 4 * threadIdx.x;   // 8 x 32 threads
    if (i >= Np || j0 > i) return;
    const bool row_in = i < N;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int64_t j = j0 + c;
        if (j > i) break;
        double* z = Z + i * Np + j;
        long long* q = reinterpret_cast<long long*>(z);
        if (!row_in || j >= N) {
            const long long e = (i == j) ? (1ll << kFL) : 0;
            *q = e;
            if (Zkeep) Zkeep[i * Np + j] = e;
            continue;
        }
        const int jc = (int)(j - bj * 32);
        dsf v = ds_from_double(*z);
#pragma unroll
        for (int k = 0; k < 7; ++k) v = ds_fma(v, Fs[y][k], Gs[jc][k]);
        v = ds_mul(ds_mul(Dr[y], v), Dc[jc]);
        // |Z_s| <= 1 for a positive definite scaled matrix (2^60 in Q60)
        if (!(fabsf(v.h) <= 2.3058430e18f)) ptx::set_flag(flag, DEV_RANGE, (int)i);   // 2^61
        const long long e = __float2ll_rn(v.h) + __float2ll_rn(v.l);
        *q = e;
        if (Zkeep) Zkeep[i * Np + j] = e;
    }
}

__global__ void __launch_bounds__(256)
zscale_q_kernel(int64_t N, int64_t Np, double* __restrict__ Z, const double* __restrict__ F,
                const double* __restrict__ G, const double* __restrict__ D, long long* __restrict__ Zkeep,
                int* flag) {
    zscale_q_body(N, Np, Z, F, G, D, Zkeep, flag, blockIdx.y, blockIdx.x);
}

// Cholesky of the 128 x 128 diagonal block from Q60 (L in the lower
// triangle, its inverse X = L^-1 transposed in the upper one, both in
// double-single shared memory), L written back as Q60, X as digit planes
// with row exponents.  Blocked by 32-column panels: all threads factor the
// panel's diagonal block column by column, invert it by blocks (8 x 8 column
// sweeps, then X21 = -X22 L21 X11 twice), solve the rows below with that
// inverse and update the trailing block; the off-diagonal blocks of X then
// follow by block rows, X_ij = -X_ii sum_k L_ik X_kj.
constexpr int kLD = kNB + 1;
constexpr int kPW = 32;                                   // panel width
constexpr size_t kDiagSmem = sizeof(dsf) * (kNB * kLD + kNB + 3 * kPW * kPW);
__device__ __forceinline__ void potrf_diag_q_body(long long* __restrict__ Z, int64_t ld, int64_t k0,
                                                  __nv_bfloat16* __restrict__ digL, int* __restrict__ expL, int s,
                                                  int* flag) {
    extern __shared__ __align__(16) dsf S[];      // 128 x 129
    dsf* invd = S + kNB * kLD;                    // 1 / L_jj
    dsf* T = invd + kNB;                          // 3 x 32 x 32: one block row of sum_k L_ik X_kj
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < kNB * kNB; e += 512) {
        int i = e >> 7, j = e & 127;
        if (j <= i) S[i * kLD + j] = ds_from_q60(Z[(k0 + i) * ld + k0 + j]);
    }
    // update pair of this thread inside a 32 x 32 diagonal block: the
    // tid-th (row, column) of a lower triangle, row by row
    int tr = (int)((sqrtf(8.f * (float)tid + 1.f) - 1.f) * 0.5f);
    while ((tr + 1) * (tr + 2) / 2 <= tid) ++tr;
    while (tr * (tr + 1) / 2 > tid) --tr;
    const int tk = tid - tr * (tr + 1) / 2;
    __syncthreads();
    for (int p = 0; p < kNB / kPW; ++p) {
        const int b0 = kPW * p;
        // diagonal block, right-looking over its 32 columns with all threads:
        // column jj is used unscaled (with 1 / L_jj^2) and scaled one step later
        for (int jj = 0; jj < kPW; ++jj) {
            const int j = b0 + jj;
            if (tid == 0) {
                dsf d = S[j * kLD + j];
                if (!(d.h > 0.f)) { set_flag(flag, DEV_NOT_SPD, (int)(k0 + j)); d = {1.f, 0.f}; }
                dsf l, inv, inv2;
                ds_sqrt_inv(d, l, inv, inv2);
                S[j * kLD + j] = l;
                invd[j] = inv;
                T[jj] = inv2;
            } else if (jj > 0 && warp == 1 && lane > jj - 1) {
                S[(b0 + lane) * kLD + j - 1] = ds_mul(S[(b0 + lane) * kLD + j - 1], invd[j - 1]);
            }
            __syncthreads();
            const int m = kPW - 1 - jj;  // rows (and columns) below jj
            if (tid < m * (m + 1) / 2) {
                const int r = b0 + jj + 1 + tr, k = b0 + jj + 1 + tk;
                const dsf t = ds_mul(S[k * kLD + j], T[jj]);
                S[r * kLD + k] = ds_fma(S[r * kLD + k], ds_neg(S[r * kLD + j]), t);
            }
            __syncthreads();
        }
        // X_pp = L_pp^-1 by blocks: the four 8 x 8 diagonal blocks by column
        // sweeps (one warp each: row j of X is scaled by 1 / L_jj, then removed
        // from the rows below), then X21 = -X22 L21 X11 for the two 16 x 16
        // blocks and for the whole 32 x 32 block (T holds L21 X11); X[r][c]
        // (r > c) lives at S[c][r]
        if (warp < 4) {
            const int o = b0 + 8 * warp;
            int r = 0, c = 0;                       // lane -> entry (r, c), c < r < 8
            if (lane < 28) {
                r = 1;
                while ((r + 1) * r / 2 <= lane) ++r;
                c = lane - r * (r - 1) / 2;
            }
            for (int j = 0; j < 8; ++j) {
                if (lane < 28 && r == j) S[(o + c) * kLD + o + j] = ds_mul(S[(o + c) * kLD + o + j], invd[o + j]);
                __syncwarp();
                if (lane < 28 && r > j && c <= j) {
                    const dsf m = ds_neg(S[(o + r) * kLD + o + j]);
                    const dsf xjc = c == j ? invd[o + j] : S[(o + c) * kLD + o + j];
                    dsf* xr = &S[(o + c) * kLD + o + r];
                    *xr = ds_fma(c == j ? dsf{0.f, 0.f} : *xr, m, xjc);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int w = 8; w < kPW; w *= 2) {          // blocks of 2w rows: X21 (w x w) from X11, X22
            const int nb = kPW / (2 * w);           // such blocks in the panel
            if (tid < nb * w * w) {
                const int h = tid / (w * w), i = (tid / w) % w, j = tid % w, o = b0 + 2 * w * h;
                dsf v = {0.f, 0.f};
                for (int k = j; k < w; ++k) {
                    const dsf x = k == j ? invd[o + j] : S[(o + j) * kLD + o + k];
                    v = ds_fma(v, S[(o + w + i) * kLD + o + k], x);
                }
                T[tid] = v;
            }
            __syncthreads();
            if (tid < nb * w * w) {
                const int h = tid / (w * w), i = (tid / w) % w, j = tid % w, o = b0 + 2 * w * h;
                dsf v = {0.f, 0.f};
                for (int k = 0; k <= i; ++k) {
                    const dsf x = k == i ? invd[o + w + i] : S[(o + w + k) * kLD + o + w + i];
                    v = ds_fma(v, x, T[h * w * w + k * w + j]);
                }
                S[(o + j) * kLD + o + w + i] = ds_neg(v);
            }
            __syncthreads();
        }
        if (b0 + kPW == kNB) break;
        // rows below: L[i][b0 + c] = sum_{k <= c} A[i][b0 + k] X_pp[c][k].
        // Warp w takes columns w and 31 - w (sums of 32 terms together), its
        // lanes 32 rows at a time, so that no lane of a warp idles
        const int rows = kNB - b0 - kPW;
        {
            const int c0 = warp, c1 = kPW - 1 - warp;
            for (int ri = lane; ri < rows; ri += 32) {
                const dsf* ai = S + (b0 + kPW + ri) * kLD + b0;
                dsf v0 = ds_mul(ai[c0], invd[b0 + c0]);
                dsf v1 = ds_mul(ai[c1], invd[b0 + c1]);
                int k = 0;
                for (; k < c0; ++k) {
                    const dsf aik = ai[k];
                    v0 = ds_fma(v0, aik, S[(b0 + k) * kLD + b0 + c0]);
                    v1 = ds_fma(v1, aik, S[(b0 + k) * kLD + b0 + c1]);
                }
                for (; k < c1; ++k) v1 = ds_fma(v1, ai[k], S[(b0 + k) * kLD + b0 + c1]);
                T[ri * kPW + c0] = v0;
                T[ri * kPW + c1] = v1;
            }
        }
        __syncthreads();
        for (int e = tid; e < rows * kPW; e += 512) S[(b0 + kPW + e / kPW) * kLD + b0 + e % kPW] = T[e];
        __syncthreads();
        // trailing update of the lower triangle below and right of the panel;
        // entries t and t + 512 of the triangle (row by row) share a thread,
        // two independent chains for the FP32 pipes
        const int t0 = b0 + kPW, w = kNB - t0, nt = w * (w + 1) / 2;
        for (int t = tid; t < nt; t += 1024) {
            int i0, l0, i1 = 0, l1 = 0;
            tri_index(t, i0, l0);
            const bool two = t + 512 < nt;
            if (two) tri_index(t + 512, i1, l1);
            i0 += t0; l0 += t0; i1 += t0; l1 += t0;
            dsf v0 = S[i0 * kLD + l0], v1 = two ? S[i1 * kLD + l1] : dsf{0.f, 0.f};
            for (int k = 0; k < kPW; ++k) {
                v0 = ds_fma(v0, ds_neg(S[i0 * kLD + b0 + k]), S[l0 * kLD + b0 + k]);
                if (two) v1 = ds_fma(v1, ds_neg(S[i1 * kLD + b0 + k]), S[l1 * kLD + b0 + k]);
            }
            S[i0 * kLD + l0] = v0;
            if (two) S[i1 * kLD + l1] = v1;
        }
        __syncthreads();
    }
    // off-diagonal blocks of X by block rows; X[r][c] (r > c) lives at S[c][r]
    for (int bi = 1; bi < kNB / kPW; ++bi) {
        const int r0 = kPW * bi;
        // warp w takes columns w and 31 - w (sums of equal total length),
        // its lanes the 32 rows
        for (int bj = 0; bj < bi; ++bj) {
            const int r = lane, cc = warp;
            const int col0 = kPW * bj + cc, col1 = kPW * bj + kPW - 1 - cc;
            const dsf* ra = S + (r0 + r) * kLD;
            dsf v0 = ds_mul(ra[col0], invd[col0]), v1 = ds_mul(ra[col1], invd[col1]);
            int k = col0 + 1;
            for (; k <= col1; ++k) v0 = ds_fma(v0, ra[k], S[col0 * kLD + k]);
            for (; k < r0; ++k) {
                const dsf a = ra[k];
                v0 = ds_fma(v0, a, S[col0 * kLD + k]);
                v1 = ds_fma(v1, a, S[col1 * kLD + k]);
            }
            T[bj * kPW * kPW + r * kPW + cc] = v0;
            T[bj * kPW * kPW + r * kPW + kPW - 1 - cc] = v1;
        }
        __syncthreads();
        for (int bj = 0; bj < bi; ++bj) {
            const int r = tid / kPW, cc = tid % kPW, col = kPW * bj + cc;   // rows r and r + 16
            const dsf* Tb = T + bj * kPW * kPW;
            const int r1 = r + 16;
            dsf v0 = ds_mul(invd[r0 + r], Tb[r * kPW + cc]);
            dsf v1 = ds_mul(invd[r0 + r1], Tb[r1 * kPW + cc]);
            for (int k = 0; k < r; ++k) {
                const dsf t = Tb[k * kPW + cc];
                v0 = ds_fma(v0, S[(r0 + k) * kLD + r0 + r], t);
                v1 = ds_fma(v1, S[(r0 + k) * kLD + r0 + r1], t);
            }
            for (int k = r; k < r1; ++k) v1 = ds_fma(v1, S[(r0 + k) * kLD + r0 + r1], Tb[k * kPW + cc]);
            S[col * kLD + r0 + r] = ds_neg(v0);
            S[col * kLD + r0 + r1] = ds_neg(v1);
        }
        __syncthreads();
    }
    for (int e = tid; e < kNB * kNB; e += 512) {
        int i = e >> 7, j = e & 127;
        if (j <= i) Z[(k0 + i) * ld + k0 + j] = ds_to_q60(S[i * kLD + j]);
    }
    // X = L^-1 as digit planes (row block k0 / 128 of the inverses' buffer):
    // per row the exponent e of its largest entry (|x| < 2^e), then
    // w = round(x 2^(T - e)) from both halves of the double-single value
    int* rexp = reinterpret_cast<int*>(T);          // 128 row exponents (T is free again)
    auto xval = [&](int r, int k) -> dsf {          // X[r][k]
        return k < r ? S[k * kLD + r] : (k == r ? invd[r] : dsf{0.f, 0.f});
    };
    for (int r = warp; r < kNB; r += 16) {
        float mx = 0.f;
        for (int k = lane; k <= r; k += 32) mx = fmaxf(mx, fabsf(xval(r, k).h));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int ex = 0;
        if (mx > 0.f) frexpf(mx * 1.00001f, &ex);   // margin for the low half: |x| < 2^ex
        if (lane == 0) {
            rexp[r] = ex;
            expL[k0 + r] = ex;
            // X = L^-1 is held in Q42 (|x| < 2^21); stop two bits short
            if (ex > 19) ptx::set_flag(flag, DEV_RANGE, (int)(k0 + r));
        }
    }
    __syncthreads();
    const int Tb = 7 + 8 * (s - 1);
    const int64_t pstride = blk_off(1, 0, 0, (int)ld, s) - blk_off(0, 0, 0, (int)ld, s);
    // lanes take consecutive rows of one group of eight columns: X[r][k]
    // lives at S[k][r], so a warp's reads of one k are contiguous
    for (int item = tid; item < kNB * (kNB / 8); item += 512) {
        const int r = item & (kNB - 1), g8 = item >> 7;
        const int sh = Tb - rexp[r];
        const float scale = __int_as_float((127 + sh) << 23);   // 2^sh (ex >= 1: the diagonal 1 / L_rr >= 1)
        long long w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const dsf x = xval(r, 8 * g8 + j);
            const float hs = __fmul_rn(x.h, scale), ls = __fmul_rn(x.l, scale);
            const long long wh = __float2ll_rn(hs);
            w[j] = wh + __float2ll_rn(__fadd_rn(__fsub_rn(hs, __ll2float_rn(wh)), ls));
        }
        split_store8(w, s, digL + blk_off(0, (int)k0 + r, 8 * g8, (int)ld, s), pstride);
    }
}

__global__ void __launch_bounds__(512)
potrf_diag_q_kernel(long long* __restrict__ Z, int64_t ld, int64_t k0, __nv_bfloat16* __restrict__ digL,
                    int* __restrict__ expL, int s, int* flag) {
    potrf_diag_q_body(Z, ld, k0, digL, expL, s, flag);
}

// Camera Gram blocks Sig_c += X[k, c]^T X[k, c] from the finished Q42 row
// block k of X (128 rows), 4 cameras (36 columns) per CTA, summed in
// double-single arithmetic and added to the FP64 blocks once.  A thread
// takes entries (a, b), a <= b, of the symmetric blocks (45 per camera) and
// sums the 128 rows in four interleaved chains.
constexpr int kGW = 36;
constexpr int kGT = 192;                    // threads: one per entry (4 cameras x 45 = 180)
__device__ __forceinline__ void gram_q_body(int64_t n, int64_t Np, int64_t k0, int64_t ncols,
                                            const long long* __restrict__ R, double* __restrict__ Sig, int64_t bid) {
    __shared__ dsf T[kNB][kGW + 1];
    const int tid = threadIdx.x;
    const int64_t c0 = bid * (int64_t)kGW;
    constexpr float kS = 2.2737367544323206e-13f;  // 2^-42
    // every load issued before any is used: the row block comes from L2 or
    // DRAM, and one load at a time would pay that latency kNB kGW / kGT times
    constexpr int kPer = kNB * kGW / kGT;
    long long vals[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = tid + kGT * u, r = e / kGW, c = e % kGW;
        const int64_t gc = c0 + c;
        vals[u] = gc < ncols ? R[(k0 + r) * Np + gc] : 0;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = tid + kGT * u, r = e / kGW, c = e % kGW;
        T[r][c] = ds_from_fixed(vals[u], kS);
    }
    __syncthreads();
    if (tid >= 4 * 45) return;
    const int g = tid / 45;
    int q = tid % 45, a = 0;                   // q -> (a, b) of the upper triangle, row by row
    while (q >= 9 - a) { q -= 9 - a; ++a; }
    const int b = a + q;
    const int64_t cam = (c0 / 9) + g;
    if (cam >= n || c0 + 9 * g >= ncols) return;
    const int ca = 9 * g + a, cb = 9 * g + b;
    dsf v0 = {0.f, 0.f}, v1 = v0, v2 = v0, v3 = v0;
    for (int r = 0; r < kNB; r += 4) {
        v0 = ds_fma(v0, T[r][ca], T[r][cb]);
        v1 = ds_fma(v1, T[r + 1][ca], T[r + 1][cb]);
        v2 = ds_fma(v2, T[r + 2][ca], T[r + 2][cb]);
        v3 = ds_fma(v3, T[r + 3][ca], T[r + 3][cb]);
    }
    const dsf v = ds_add(ds_add(v0, v1), ds_add(v2, v3));
    const double sum = (double)v.h + (double)v.l;
    Sig[81 * cam + 9 * a + b] += sum;
    if (a != b) Sig[81 * cam + 9 * b + a] += sum;
}

__global__ void __launch_bounds__(kGT)
gram_q_kernel(int64_t n, int64_t Np, int64_t k0, int64_t ncols, const long long* __restrict__ R,
              double* __restrict__ Sig) {
    gram_q_body(n, Np, k0, ncols, R, Sig, blockIdx.x);
}

__global__ void identity_q_kernel(int64_t Np, long long* X) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < Np) X[i * Np + i] = 1ll << kFX;
}

// ---- grouped forms: one launch for the same step of many scenes ----
template <int K>
__global__ void __launch_bounds__(256)
slice_rows_grouped(const SliceRowsP* __restrict__ P, const int64_t* __restrict__ pre, int k, int* flag) {
    const int q = find_group(pre, k, blockIdx.x);
    const SliceRowsP& a = P[q];
    slice_rows_body<K>(a.rows, a.src, a.ld, a.F, a.s, a.plane_rows, a.dst, a.expo, flag, blockIdx.x - pre[q]);
}

template <int K>
__global__ void __launch_bounds__(256)
slice_cols_grouped(const SliceColsP* __restrict__ P, const int64_t* __restrict__ pre, int k, int* flag) {
    const int q = find_group(pre, k, blockIdx.x);
    const SliceColsP& a = P[q];
    slice_cols_body<K>(a.ncols, a.src, a.ld, a.F, a.s, a.plane_rows, a.dst, a.expo, flag, blockIdx.x - pre[q]);
}

__global__ void __launch_bounds__(512) potrf_diag_q_grouped(const PotrfP* __restrict__ P, int* flag) {
    const PotrfP& a = P[blockIdx.x];
    potrf_diag_q_body(a.Z, a.ld, a.k0, a.digL, a.expL, a.s, flag);
}

__global__ void __launch_bounds__(kGT)
gram_q_grouped(const GramP* __restrict__ P, const int64_t* __restrict__ pre, int k) {
    const int q = find_group(pre, k, blockIdx.x);
    const GramP& a = P[q];
    gram_q_body(a.n, a.Np, a.k0, a.ncols, a.R, a.Sig, blockIdx.x - pre[q]);
}

__global__ void __launch_bounds__(256)
zscale_q_grouped(const ZscaleP* __restrict__ P, const int64_t* __restrict__ pre, int k, int* flag) {
    const int q = find_group(pre, k, blockIdx.x);
    const ZscaleP& a = P[q];
    const int64_t b = blockIdx.x - pre[q];
    zscale_q_body(a.N, a.Np, a.Z, a.F, a.G, a.D, nullptr, flag, b / a.nt, b % a.nt);
}

__global__ void identity_q_grouped(const IdentP* __restrict__ P, const int64_t* __restrict__ pre, int k) {
    const int q = find_group(pre, k, blockIdx.x);
    const IdentP& a = P[q];
    const int64_t i = (blockIdx.x - pre[q]) * (int64_t)blockDim.x + threadIdx.x;
    if (i < a.Np) a.X[i * a.Np + i] = 1ll << kFX;
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

// int64 result matrix rows x cols (row stride ld elements), box 16 x 128, 128-byte swizzle.
bool make_c_map(CUtensorMap* map, long long* buf, int64_t rows, int64_t cols, int64_t ld) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
    cuuint32_t box[2] = {16, (cuuint32_t)kBM};
    cuuint32_t estr[2] = {1, 1};
    // unsigned: the reduce-add of the epilogue adds 64-bit words modulo 2^64,
    // which is two's-complement addition of the signed fixed-point values
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The B-operand view of a digit buffer: (128 elements of an 8-row group,
// 8 groups, 2 halves of a 128-row block, s planes, K slice x row block).
bool make_b_map(CUtensorMap* map, __nv_bfloat16* buf, int s, int64_t Np, int kmax) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[5] = {128, 8, 2, (cuuint64_t)s, (cuuint64_t)(kmax / 16) * (cuuint64_t)(Np / 128)};
    cuuint64_t strides[4] = {256, 2048, 4096, (cuuint64_t)s * 4096};
    cuuint32_t box[5] = {128, 8, 1, (cuuint32_t)s, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t gemm_smem(int s, int stages) {
    return (size_t)kCTile + (size_t)stages * s * (kAPl + kBPl) + 8 * (2 * stages + 4) + 16;
}

int pick_stages(int s) {
    int st = 8;
    while (st > 2 && gemm_smem(s, st) > 227 * 1024) --st;
    return st;
}

int g_num_sms = 0;

template <int S, int K>
cudaError_t set_attr() {
    cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel<S, K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_smem(S, pick_stages(S)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ozaki_gemm_kernel<S, K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gemm_smem(S, pick_stages(S)));
}

enum Buf { BUF_P = 0, BUF_Q = 1, BUF_L = 2 };

__nv_bfloat16* buf_ptr(const MixedState& st, Buf b) {
    return b == BUF_P ? st.digP : (b == BUF_Q ? st.digQ : st.digL);
}

// C op= A B^T with A = rows [a_row0, a_row0 + M) of digit buffer `ba`, B =
// rows [b_row0, b_row0 + N) of buffer `bb`, both with K digits per row.
void launch_ozaki(Ctx& c, int K, Buf ba, int a_row0, int M, Buf bb, int b_row0, int N, const CUtensorMap& mapC,
                  int c_x0, int c_y0, int lower, int sub, int Fc, const int* expA, const int* expB) {
    MixedState& st = *c.mixed;
    GemmArgs g;
    g.M = M; g.N = N; g.plane_rows = (int)c.Np; g.a_row0 = a_row0; g.b_row0 = b_row0;
    g.c_x0 = c_x0; g.c_y0 = c_y0; g.lower = lower; g.sub = sub; g.shift0 = Fc - 14;
    g.expA = expA; g.expB = expB; g.stages = pick_stages(st.s); g.flag = c.d_flag;
    g.wait_ns = st.wait_ns; g.skip_fill = st.skip_fill;
    g.digA = buf_ptr(st, ba);
    g.digB = buf_ptr(st, bb);
    const int64_t ntiles = tile_count(M / kBM, N / kBN, lower);  // even: pairs of tiles
    if ((ntiles & 1) || (N % (2 * kBN))) {
        c.mixed_bad_launch = true;  // cannot happen with N a multiple of 128
        return;
    }
    const int64_t npairs = ntiles / 2;
    const int grid = 2 * (int)(npairs < g_num_sms / 2 ? npairs : g_num_sms / 2);
    if (grid < 2) return;
    // executed tensor-core work: every kept tile, every digit product
    const double flops = (double)ntiles * 2.0 * kBM * kBN * K * (st.s * (st.s + 1) / 2);
    const size_t smem = gemm_smem(st.s, g.stages);
    prof_begin(c);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    const CUtensorMap& mapB = bb == BUF_P ? st.mapBP : (bb == BUF_Q ? st.mapBQ : st.mapBL);
    const GemmProblem* no_probs = nullptr;
    int no_n = 0;
#define CCOV_OZ(S_, K_) cudaLaunchKernelEx(&cfg, ozaki_gemm_kernel<S_, K_, false>, mapC, mapB, g, no_probs, no_n)
    if (K == 512) {
        switch (st.s) {
            case 4: CCOV_OZ(4, 512); break;
            case 5: CCOV_OZ(5, 512); break;
            default: c.mixed_bad_launch = true; break;   // six digits: eight accumulators do not suffice
        }
    } else if (K == 256) {
        switch (st.s) {
            case 4: CCOV_OZ(4, 256); break;
            case 5: CCOV_OZ(5, 256); break;
            default: CCOV_OZ(6, 256); break;
        }
    } else {
        switch (st.s) {
            case 4: CCOV_OZ(4, 128); break;
            case 5: CCOV_OZ(5, 128); break;
            default: CCOV_OZ(6, 128); break;
        }
    }
#undef CCOV_OZ
    prof_end(c, flops);
    c.launches++;
}

void slice_rows(Ctx& c, int K, int rows, const long long* src, Buf b) {
    MixedState& st = *c.mixed;
    __nv_bfloat16* dst = b == BUF_P ? st.digP : st.digQ;
    int* ex = b == BUF_P ? st.expP : st.expQ;
    // one warp per 16 rows x 16 values
    const int grid = (int)(((int64_t)rows / 16 * (K / 16) * 32 + 255) / 256);
    if (rows % 16) { c.mixed_bad_launch = true; return; }
    if (K == 512)
        slice_rows_kernel<512><<<grid, 256, 0, c.stream>>>(rows, src, c.Np, kFL, st.s, (int)c.Np, dst, ex,
                                                           c.d_flag);
    else if (K == 256)
        slice_rows_kernel<256><<<grid, 256, 0, c.stream>>>(rows, src, c.Np, kFL, st.s, (int)c.Np, dst, ex,
                                                           c.d_flag);
    else
        slice_rows_kernel<128><<<grid, 256, 0, c.stream>>>(rows, src, c.Np, kFL, st.s, (int)c.Np, dst, ex,
                                                           c.d_flag);
    c.launches++;
}

void slice_cols(Ctx& c, int K, int ncols, const long long* src, Buf b) {
    MixedState& st = *c.mixed;
    __nv_bfloat16* dst = b == BUF_P ? st.digP : st.digQ;
    int* ex = b == BUF_P ? st.expP : st.expQ;
    const int grid = (ncols + 31) / 32;
    const size_t smem = (size_t)K * 33 * 8;
    if (K == 512)
        slice_cols_kernel<512><<<grid, 256, smem, c.stream>>>(ncols, src, c.Np, kFX, st.s, (int)c.Np, dst, ex,
                                                              c.d_flag);
    else if (K == 256)
        slice_cols_kernel<256><<<grid, 256, smem, c.stream>>>(ncols, src, c.Np, kFX, st.s, (int)c.Np, dst, ex,
                                                              c.d_flag);
    else
        slice_cols_kernel<128><<<grid, 256, smem, c.stream>>>(ncols, src, c.Np, kFX, st.s, (int)c.Np, dst, ex,
                                                              c.d_flag);
    c.launches++;
}

void potrf_block(Ctx& c, int64_t blk) {
    MixedState& st = *c.mixed;
    long long* Zq = reinterpret_cast<long long*>(c.d_Z);
    potrf_diag_q_kernel<<<1, 512, kDiagSmem, c.stream>>>(Zq, c.Np, blk * kNB, st.digL, st.expL, st.s, c.d_flag);
    c.launches++;
}

}  // namespace

// ---- grouped launchers (the batched form) ----
int64_t grp_slice_rows_blocks(int K, int rows) { return ((int64_t)rows / 16 * (K / 16) * 32 + 255) / 256; }
int64_t grp_slice_cols_blocks(int ncols) { return (ncols + 31) / 32; }
int64_t grp_gram_blocks(int64_t ncols) { return (ncols + kGW - 1) / kGW; }

void grp_slice_rows(cudaStream_t st, int K, const SliceRowsP* P, const int64_t* pre, int k, int64_t blocks,
                    int* flag) {
    if (K == 512) slice_rows_grouped<512><<<(unsigned)blocks, 256, 0, st>>>(P, pre, k, flag);
    else if (K == 256) slice_rows_grouped<256><<<(unsigned)blocks, 256, 0, st>>>(P, pre, k, flag);
    else slice_rows_grouped<128><<<(unsigned)blocks, 256, 0, st>>>(P, pre, k, flag);
}

void grp_slice_cols(cudaStream_t st, int K, const SliceColsP* P, const int64_t* pre, int k, int64_t blocks,
                    int* flag) {
    const size_t smem = (size_t)K * 33 * 8;
    if (K == 512) slice_cols_grouped<512><<<(unsigned)blocks, 256, smem, st>>>(P, pre, k, flag);
    else if (K == 256) slice_cols_grouped<256><<<(unsigned)blocks, 256, smem, st>>>(P, pre, k, flag);
    else slice_cols_grouped<128><<<(unsigned)blocks, 256, smem, st>>>(P, pre, k, flag);
}

void grp_potrf(cudaStream_t st, const PotrfP* P, int k, int* flag) {
    potrf_diag_q_grouped<<<k, 512, kDiagSmem, st>>>(P, flag);
}

void grp_gram(cudaStream_t st, const GramP* P, const int64_t* pre, int k, int64_t blocks) {
    gram_q_grouped<<<(unsigned)blocks, kGT, 0, st>>>(P, pre, k);
}

void grp_zscale(cudaStream_t st, const ZscaleP* P, const int64_t* pre, int k, int64_t blocks, int* flag) {
    zscale_q_grouped<<<(unsigned)blocks, dim3(8, 32), 0, st>>>(P, pre, k, flag);
}

void grp_identity(cudaStream_t st, const IdentP* P, const int64_t* pre, int k, int64_t blocks) {
    identity_q_grouped<<<(unsigned)blocks, 256, 0, st>>>(P, pre, k);
}

// The persistent GEMM over the tile pairs of `nprobs` problems (device
// array, each with its own maps), at most max_ctas CTAs.
cudaError_t grp_gemm(cudaStream_t st, int s, int K, const GemmProblem* probs, int nprobs, int64_t total_pairs,
                     int* flag, int max_ctas, int stages) {
    if (total_pairs <= 0) return cudaSuccess;
    GemmArgs g = {};
    g.stages = stages > 0 && gemm_smem(s, stages) <= gemm_smem(s, pick_stages(s)) ? stages : pick_stages(s);
    g.flag = flag;
    g.wait_ns = ptx::kWaitNs;
    g.skip_fill = -1;
    g.total_pairs = total_pairs;
    const int cap = (max_ctas < g_num_sms ? max_ctas : g_num_sms) / 2;
    const int grid = 2 * (int)(total_pairs < cap ? total_pairs : cap);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = gemm_smem(s, g.stages);
    cfg.stream = st;
    CUtensorMap none;
    std::memset(&none, 0, sizeof none);
#define CCOV_OZG(S_, K_) cudaLaunchKernelEx(&cfg, ozaki_gemm_kernel<S_, K_, true>, none, none, g, probs, nprobs)
    cudaError_t e;
    if (K == 512) {
        switch (s) {
            case 4: e = CCOV_OZG(4, 512); break;
            case 5: e = CCOV_OZG(5, 512); break;
            default: e = cudaErrorInvalidValue; break;   // six digits group by pairs (K <= 256)
        }
    } else if (K == 256) {
        switch (s) {
            case 4: e = CCOV_OZG(4, 256); break;
            case 5: e = CCOV_OZG(5, 256); break;
            default: e = CCOV_OZG(6, 256); break;
        }
    } else {
        switch (s) {
            case 4: e = CCOV_OZG(4, 128); break;
            case 5: e = CCOV_OZG(5, 128); break;
            default: e = CCOV_OZG(6, 128); break;
        }
    }
#undef CCOV_OZG
    return e;
}

// Kernel attributes of the mixed path (shared memory sizes) and the SM count.
cudaError_t mixed_setup() {
    cudaError_t a[8] = {set_attr<4, 128>(), set_attr<5, 128>(), set_attr<6, 128>(), set_attr<4, 256>(),
                        set_attr<5, 256>(), set_attr<6, 256>(), set_attr<4, 512>(), set_attr<5, 512>()};
    for (cudaError_t x : a)
        if (x != cudaSuccess) return x;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(potrf_diag_q_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kDiagSmem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(potrf_diag_q_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kDiagSmem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(slice_cols_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  256 * 33 * 8)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(slice_cols_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  512 * 33 * 8)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(slice_cols_grouped<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  256 * 33 * 8)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(slice_cols_grouped<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  512 * 33 * 8)) != cudaSuccess)
        return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    return cudaSuccess;
}

bool mixed_make_c_map(CUtensorMap* map, long long* buf, int64_t rows, int64_t cols, int64_t ld) {
    return make_c_map(map, buf, rows, cols, ld);
}

bool mixed_make_b_map(CUtensorMap* map, __nv_bfloat16* buf, int s, int64_t Np) {
    return make_b_map(map, buf, s, Np, kGroupDigitK);
}

int mixed_stages(int s) { return pick_stages(s); }

int64_t mixed_tile_pairs(int M, int N, int lower) { return tile_count(M / kBM, N / kBN, lower) / 2; }

cudaError_t mixed_alloc(Ctx& c) {
    c.mixed = new MixedState();
    MixedState& st = *c.mixed;
    st.s = c.opt.mixed_slices;
    if (st.s > 6) return cudaErrorInvalidValue;
    const int64_t Np = c.Np;
    const size_t plane = (size_t)st.s * Np * kKMax;
    cudaError_t e;
    if ((e = cudaMalloc(&st.digP, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.digQ, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expP, Np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expQ, Np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.R, Np * Np * sizeof(long long))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.digL, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expL, Np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.digP2, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.digQ2, plane * 2)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expP2, Np * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&st.expQ2, Np * sizeof(int))) != cudaSuccess) return e;
    c.bytes += (int64_t)(plane * 10 + Np * 20 + Np * Np * 8);
    // on the context's stream (it need not synchronise with the legacy stream)
    if ((e = cudaMemsetAsync(st.digP, 0, plane * 2, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(st.digQ, 0, plane * 2, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(st.digP2, 0, plane * 2, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(st.digQ2, 0, plane * 2, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(st.digL, 0, plane * 2, c.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
    int prio_lo = 0, prio_hi = 0;
    if ((e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithPriority(&st.side, cudaStreamNonBlocking, prio_lo)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithPriority(&st.hi, cudaStreamNonBlocking, prio_hi)) != cudaSuccess) return e;
    st.ev.assign(3 + (size_t)(Np / kNB), nullptr);
    for (auto& ev : st.ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    if (c.d_Z && !make_c_map(&st.mapZ, reinterpret_cast<long long*>(c.d_Z), Np, Np, Np)) return cudaErrorInvalidValue;
    if (!make_c_map(&st.mapR, st.R, Np, Np, Np)) return cudaErrorInvalidValue;
    if (!make_b_map(&st.mapBP, st.digP, st.s, Np, kKMax) || !make_b_map(&st.mapBQ, st.digQ, st.s, Np, kKMax) ||
        !make_b_map(&st.mapBP2, st.digP2, st.s, Np, kKMax) || !make_b_map(&st.mapBQ2, st.digQ2, st.s, Np, kKMax) ||
        !make_b_map(&st.mapBL, st.digL, st.s, Np, kKMax))
        return cudaErrorInvalidValue;
    return mixed_setup();
}

const long long* mixed_inverse_factor(const Ctx& c) { return c.mixed ? c.mixed->R : nullptr; }

// ---- Y = X^T X V on the tensor cores (the covariance update after added
// observations): the two triangular products with the inverse factor X =
// L^-1 (Q42) of the last step (d), each as a sequence of digit-split GEMMs
// over 256-wide panels of X, accumulated in int64 fixed point by the GEMM's
// reduce-add.  W = X V by column panels of X (rows of X split with a
// per-row exponent), then Y = X^T W by row panels (columns of X split with
// a per-column exponent, as in the triangular inverse).  The columns of V
// enter scaled to |v| < 1 (per-column exponent, folded back at the end); the
// fixed points of W and Y come from |W| <= ||X||_inf and |Y| <= ||X||_1
// ||X||_inf, measured on X first. ----
namespace {

// Sum over the row of |X[r][c]| (c <= r), warp per row, in units of X.
__global__ void __launch_bounds__(256) xnorm_rows_kernel(int64_t Np, const long long* __restrict__ X,
                                                         double* __restrict__ rs) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= Np) return;
    double acc = 0.0;
    for (int64_t col = lane; col <= r; col += 32) acc += fabs((double)X[r * Np + col]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rs[r] = acc * 0x1p-42;
}

// Sum over the column of |X[r][c]| (r >= c): a CTA per 32 columns (one per
// lane), its eight warps over the rows, summed in a fixed order.
__global__ void __launch_bounds__(256) xnorm_cols_kernel(int64_t Np, const long long* __restrict__ X,
                                                         double* __restrict__ cs) {
    __shared__ double part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t col = blockIdx.x * 32 + lane;
    double acc = 0.0;
    for (int64_t r = blockIdx.x * 32 + warp; r < Np; r += 8)
        if (col <= r) acc += fabs((double)X[r * Np + col]);
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && col < Np) {
        double v = part[0][lane];
        for (int w = 1; w < 8; ++w) v += part[w][lane];
        cs[col] = v * 0x1p-42;
    }
}

// out[0] = max of a, out[1] = max of b (n entries each); one CTA.
__global__ void __launch_bounds__(1024) max2_kernel(int64_t n, const double* __restrict__ a,
                                                    const double* __restrict__ b, double* __restrict__ out) {
    __shared__ double ma[32], mb[32];
    double x = 0.0, y = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) { x = fmax(x, a[i]); y = fmax(y, b[i]); }
    for (int o = 16; o > 0; o >>= 1) {
        x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        y = fmax(y, __shfl_xor_sync(0xffffffffu, y, o));
    }
    if ((threadIdx.x & 31) == 0) { ma[threadIdx.x >> 5] = x; mb[threadIdx.x >> 5] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 32; ++w) { x = fmax(x, ma[w]); y = fmax(y, mb[w]); }
        out[0] = fmax(x, ma[0]);
        out[1] = fmax(y, mb[0]);
    }
}

__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Column maxima of |V| (j < ncols) as the bit patterns of non-negative
// doubles, whose integer order is their order: a CTA per 32 columns and row
// chunk, eight row phases, one atomicMax per column (cmax starts at 0).
__global__ void __launch_bounds__(256) colmax_kernel(int64_t rows, int64_t ld, int64_t ncols, int64_t chunk,
                                                     const double* __restrict__ V,
                                                     unsigned long long* __restrict__ cmax) {
    __shared__ double part[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j = blockIdx.x * 32 + tx, r0 = blockIdx.y * chunk, r1 = r0 + chunk < rows ? r0 + chunk : rows;
    double mx = 0.0;
    if (j < ncols)
        for (int64_t r = r0 + ty; r < r1; r += 8) mx = fmax(mx, fabs(V[r * ld + j]));
    part[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && j < ncols) {
        for (int w = 1; w < 8; ++w) mx = fmax(mx, part[w][tx]);
        atomicMax(cmax + j, (unsigned long long)__double_as_longlong(mx));
    }
}

// e_j with |V[:, j]| < 2^e_j (0 for a zero column, or one below 2^-900 that
// rounds to zero in Q60 anyway).
__device__ __forceinline__ int col_exponent(unsigned long long bits) {
    const double mx = __longlong_as_double((long long)bits);
    int e = 0;
    if (mx > 0x1p-900) frexp(mx, &e);
    return e;
}

// Vq[r][j] = V[r][j] 2^(60 - e_j) as int64 (Q60 of the scaled column), zero
// beyond ncols; row 0 also writes e_j.
__global__ void tofixed_kernel(int64_t rows, int64_t ld, int64_t ncols, int64_t ldq, const double* __restrict__ V,
                               const unsigned long long* __restrict__ cmax, int* __restrict__ ecol,
                               long long* __restrict__ Vq, int* flag) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * ldq) return;
    const int64_t r = e / ldq, j = e % ldq;
    long long q = 0;
    if (j < ncols) {
        const unsigned long long b = cmax[j];
        if (!(__longlong_as_double((long long)b) < 0x1p1000)) {   // not finite or far too large
            if (r == 0) { ptx::set_flag(flag, DEV_RANGE, (int)j); ecol[j] = 0; }
        } else {
            const int ej = col_exponent(b);
            if (r == 0) ecol[j] = ej;
            q = __double2ll_rn(V[r * ld + j] * pow2(60 - ej));
        }
    }
    Vq[e] = q;
}

// Y[r][j] = Yq[r][j] 2^(e_j - F).
__global__ void fromfixed_kernel(int64_t rows, int64_t ld, int64_t ncols, int64_t ldq,
                                 const long long* __restrict__ Yq, const int* __restrict__ ecol, int F,
                                 double* __restrict__ Y) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * ncols) return;
    const int64_t r = e / ncols, j = e % ncols;
    Y[r * ld + j] = (double)Yq[r * ldq + j] * pow2(ecol[j] - F);
}

// emax[0] = the largest e_j (j < ncols); one warp.
__global__ void emax_kernel(int64_t ncols, const int* __restrict__ ecol, int* __restrict__ emax) {
    int m = -100000;
    for (int64_t j = threadIdx.x; j < ncols; j += 32) m = max(m, ecol[j]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) emax[0] = m;
}

// XSq[a][j] = X_S[a][j] 2^(e_j - emax + 60) for j < ncols (|X_S| <= 1: S >= I),
// zero beyond; ldq x ldq, X_S with leading dimension ldq.
__global__ void xs_tofixed_kernel(int64_t ldq, int64_t ncols, const double* __restrict__ XS,
                                  const int* __restrict__ ecol, const int* __restrict__ emax,
                                  long long* __restrict__ XSq) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= ldq * ldq) return;
    const int64_t j = e % ldq;
    XSq[e] = j < ncols ? __double2ll_rn(ldexp(XS[e], ecol[j] - emax[0] + 60)) : 0;
}

// P[i][a] = -Pq[i][a] 2^(emax - F) for a < ncols (P: rows x ld FP64).
__global__ void p_fromfixed_kernel(int64_t rows, int64_t ncols, int64_t ld, int64_t ldq,
                                   const long long* __restrict__ Pq, const int* __restrict__ emax, int F,
                                   double* __restrict__ P) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * ncols) return;
    const int64_t i = e / ncols, a = e % ncols;
    P[i * ld + a] = -ldexp((double)Pq[i * ldq + a], emax[0] - F);
}

// Rows of an int64 Q(F) matrix, K = 128 or 256 values per row (a column
// panel), each row with its own exponent e (|v| < 2^(e + F) over the
// panel), as digit planes.  A CTA takes 16 rows, 16 threads per row with K /
// 16 consecutive values each; the row maximum is reduced over the 16 lanes.
template <int K>
__global__ void __launch_bounds__(256)
slice_rows_exp_kernel(int rows, const long long* __restrict__ src, int64_t ld, int F, int s, int plane_rows,
                      __nv_bfloat16* __restrict__ dst, int* __restrict__ expo, int* flag) {
    constexpr int PER = K / 16;
    const int q = threadIdx.x & 15;
    const int r = blockIdx.x * 16 + (threadIdx.x >> 4);
    const bool active = r < rows;
    long long v[PER];
    unsigned long long mx = 0;
    const longlong2* p = reinterpret_cast<const longlong2*>(src + (int64_t)(active ? r : 0) * ld + q * PER);
#pragma unroll
    for (int j = 0; j < PER / 2; ++j) {
        const longlong2 t = active ? p[j] : make_longlong2(0, 0);
        v[2 * j] = t.x;
        v[2 * j + 1] = t.y;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const unsigned long long a = (unsigned long long)(v[j] < 0 ? -v[j] : v[j]);
        mx = a > mx ? a : mx;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if (!active) return;
    const int e = mx == 0 ? 0 : (64 - __clzll((long long)mx)) - F;
    if (q == 0) expo[r] = e;
    if (mx >= (1ull << 61)) ptx::set_flag(flag, DEV_RANGE, r);
    const int T = 7 + 8 * (s - 1);
#pragma unroll
    for (int h = 0; h < PER / 8; ++h) {
        long long w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) w[j] = round_shift(v[8 * h + j], T - e - F);
        split_store8(w, s, dst + blk_off(0, r, q * PER + 8 * h, plane_rows, s), blk_off(1, 0, 0, plane_rows, s));
    }
}

void slice_rows_exp(Ctx& c, int K, int rows, const long long* src, int64_t ld, int F, Buf b) {
    MixedState& st = *c.mixed;
    __nv_bfloat16* dst = b == BUF_P ? st.digP : st.digQ;
    int* ex = b == BUF_P ? st.expP : st.expQ;
    const unsigned grid = (unsigned)((rows + 15) / 16);
    if (K == 256)
        slice_rows_exp_kernel<256><<<grid, 256, 0, c.stream>>>(rows, src, ld, F, st.s, (int)c.Np, dst, ex, c.d_flag);
    else
        slice_rows_exp_kernel<128><<<grid, 256, 0, c.stream>>>(rows, src, ld, F, st.s, (int)c.Np, dst, ex, c.d_flag);
    c.launches++;
}

void slice_cols_f(Ctx& c, int K, int ncols, const long long* src, int64_t ld, int F, Buf b) {
    MixedState& st = *c.mixed;
    __nv_bfloat16* dst = b == BUF_P ? st.digP : st.digQ;
    int* ex = b == BUF_P ? st.expP : st.expQ;
    const int grid = (ncols + 31) / 32;
    const size_t smem = (size_t)K * 33 * 8;
    if (K == 256)
        slice_cols_kernel<256><<<grid, 256, smem, c.stream>>>(ncols, src, ld, F, st.s, (int)c.Np, dst, ex, c.d_flag);
    else
        slice_cols_kernel<128><<<grid, 256, smem, c.stream>>>(ncols, src, ld, F, st.s, (int)c.Np, dst, ex, c.d_flag);
    c.launches++;
}

int fixed_point_for(double bound) {
    // the largest F with bound * 2^F below 2^61 (at most 60)
    int e = 0;
    if (bound > 0.0) frexp(bound, &e);   // bound < 2^e
    const int F = 61 - e;
    return F > 60 ? 60 : F;
}

}  // namespace

int64_t mixed_xtxv_ld(int64_t ncols) { return (ncols + 127) / 128 * 128; }

cudaError_t mixed_xtxv(Ctx& c, int64_t ncols, const double* V, int64_t ld, double* Y, long long* Vq, long long* Wq,
                       long long* Yq, long long* Sq, int* ecol, unsigned long long* cmax, double* norms, int* FS) {
    if (!c.mixed) return cudaErrorInvalidValue;
    MixedState& st = *c.mixed;
    const int64_t Np = c.Np, nb = Np / kNB, ldq = mixed_xtxv_ld(ncols);
    if (ldq > Np) return cudaErrorInvalidValue;   // the operand buffers hold Np rows
    cudaError_t e;
    // norms of X, once per factorisation: |W| <= ||X||_inf, |Y| <= ||X||_1
    // ||X||_inf for columns scaled to |v| < 1
    if (!c.upd_norm_ok) {
        double* rs = norms + 2;
        double* cs = norms + 2 + Np;
        xnorm_rows_kernel<<<(unsigned)((Np * 32 + 255) / 256), 256, 0, c.stream>>>(Np, st.R, rs);
        xnorm_cols_kernel<<<(unsigned)((Np + 31) / 32), 256, 0, c.stream>>>(Np, st.R, cs);
        max2_kernel<<<1, 1024, 0, c.stream>>>(Np, rs, cs, norms);
        c.launches += 3;
        double nrm[2] = {0.0, 0.0};
        if ((e = cudaMemcpyAsync(nrm, norms, sizeof nrm, cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
        if (!(nrm[0] < 0x1p40) || !(nrm[1] < 0x1p40)) return cudaErrorInvalidValue;   // not a usable factor
        c.upd_norm[0] = nrm[0];
        c.upd_norm[1] = nrm[1];
        c.upd_norm_ok = true;
    }
    const double ninf = c.upd_norm[0], n1 = c.upd_norm[1];
    const int FW = fixed_point_for(ninf);
    const int FY = fixed_point_for(ninf * n1);
    *FS = fixed_point_for((double)c.N * ninf * ninf);
    // columns scaled to |v| < 1, as Q60
    if ((e = cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * ldq, c.stream)) != cudaSuccess) return e;
    {
        const int64_t cb = (ncols + 31) / 32;
        const int64_t nch = std::max<int64_t>(1, std::min<int64_t>(64, (4 * 152 + cb - 1) / cb));
        const int64_t chunk = (Np + nch - 1) / nch;
        colmax_kernel<<<dim3((unsigned)cb, (unsigned)nch), 256, 0, c.stream>>>(Np, ld, ncols, chunk, V, cmax);
    }
    tofixed_kernel<<<(unsigned)((Np * ldq + 255) / 256), 256, 0, c.stream>>>(Np, ld, ncols, ldq, V, cmax, ecol, Vq,
                                                                             c.d_flag);
    c.launches += 2;
    if ((e = cudaMemsetAsync(Wq, 0, sizeof(long long) * Np * ldq, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Yq, 0, sizeof(long long) * Np * ldq, c.stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Sq, 0, sizeof(long long) * ldq * ldq, c.stream)) != cudaSuccess) return e;
    CUtensorMap mapW, mapY, mapS;
    if (!make_c_map(&mapW, Wq, Np, ldq, ldq) || !make_c_map(&mapY, Yq, Np, ldq, ldq) ||
        !make_c_map(&mapS, Sq, ldq, ldq, ldq))
        return cudaErrorInvalidValue;
    // W = -X V: column panels of X (rows kp.. of the panel), rows kp.. of V
    for (int64_t kb = 0; kb < nb; kb += 2) {
        const int K = kb + 1 < nb ? 256 : 128;
        const int64_t kp = kb * kNB;
        const int rows = (int)(Np - kp);
        slice_rows_exp(c, K, rows, st.R + kp * Np + kp, Np, kFX, BUF_P);
        slice_cols_f(c, K, (int)ldq, Vq + kp * ldq, ldq, 60, BUF_Q);
        launch_ozaki(c, K, BUF_P, 0, rows, BUF_Q, 0, (int)ldq, mapW, 0, (int)kp, 0, 1, FW, st.expP, st.expQ);
    }
    // Y = -X^T (-X V) by row panels of X (columns up to the panel's end) and
    // rows of W; with the same digits of W, S = -W^T W (= -V^T X^T X V)
    for (int64_t kb = 0; kb < nb; kb += 2) {
        const int K = kb + 1 < nb ? 256 : 128;
        const int64_t kp = kb * kNB;
        slice_cols_f(c, K, (int)(kp + K), st.R + kp * Np, Np, kFX, BUF_P);
        slice_cols_f(c, K, (int)ldq, Wq + kp * ldq, ldq, FW, BUF_Q);
        launch_ozaki(c, K, BUF_P, 0, (int)(kp + K), BUF_Q, 0, (int)ldq, mapY, 0, 0, 0, 1, FY, st.expP, st.expQ);
        launch_ozaki(c, K, BUF_Q, 0, (int)ldq, BUF_Q, 0, (int)ldq, mapS, 0, 0, 0, 1, *FS, st.expQ, st.expQ);
    }
    fromfixed_kernel<<<(unsigned)((Np * ncols + 255) / 256), 256, 0, c.stream>>>(Np, ld, ncols, ldq, Yq, ecol, FY, Y);
    c.launches++;
    if (c.mixed_bad_launch) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// P = Y_s X_S^T for the covariance update, on the tensor cores: Y_s from the
// normalised fixed-point Yq of mixed_xtxv (Y_s = Y' 2^e_j by column), X_S =
// L_S^-1 (FP64, ldq x ldq, |X_S| <= 1) with its columns scaled by 2^(e_j -
// emax) into Q60; P = Y' (X_S E)^T over 256-wide panels of the ncols
// columns.  XSq ldq x ldq and Pq Np x ldq int64 workspaces; P rows x ld FP64.
cudaError_t mixed_update_p(Ctx& c, int64_t ncols, const long long* Yq, const double* XS, const int* ecol,
                           int* emax, long long* XSq, long long* Pq, double* P, int64_t ld) {
    MixedState& st = *c.mixed;
    const int64_t Np = c.Np, ldq = mixed_xtxv_ld(ncols);
    const double ninf = c.upd_norm[0], n1 = c.upd_norm[1];
    const int FY = fixed_point_for(ninf * n1);
    const int FP = fixed_point_for((double)ldq * ninf * n1);
    cudaError_t e;
    emax_kernel<<<1, 32, 0, c.stream>>>(ncols, ecol, emax);
    xs_tofixed_kernel<<<(unsigned)((ldq * ldq + 255) / 256), 256, 0, c.stream>>>(ldq, ncols, XS, ecol, emax, XSq);
    c.launches += 2;
    if ((e = cudaMemsetAsync(Pq, 0, sizeof(long long) * Np * ldq, c.stream)) != cudaSuccess) return e;
    CUtensorMap mapP;
    if (!make_c_map(&mapP, Pq, Np, ldq, ldq)) return cudaErrorInvalidValue;
    for (int64_t kp = 0; kp < ldq; kp += 256) {
        const int K = kp + 256 <= ldq ? 256 : 128;
        slice_rows_exp(c, K, (int)Np, Yq + kp, ldq, FY, BUF_P);
        slice_rows_exp(c, K, (int)ldq, XSq + kp, ldq, 60, BUF_Q);
        launch_ozaki(c, K, BUF_P, 0, (int)Np, BUF_Q, 0, (int)ldq, mapP, 0, 0, 0, 1, FP, st.expP, st.expQ);
    }
    p_fromfixed_kernel<<<(unsigned)((c.N * ncols + 255) / 256), 256, 0, c.stream>>>(c.N, ncols, ld, ldq, Pq, emax,
                                                                                    FP, P);
    c.launches++;
    if (c.mixed_bad_launch) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

void mixed_free(Ctx& c) {
    if (!c.mixed) return;
    MixedState& st = *c.mixed;
    if (st.side) cudaStreamSynchronize(st.side);
    if (st.hi) cudaStreamSynchronize(st.hi);
    void* ptrs[] = {st.digP, st.digQ, st.expP, st.expQ, st.R, st.digP2, st.digQ2, st.expP2, st.expQ2, st.digL, st.expL};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto ev : st.ev)
        if (ev) cudaEventDestroy(ev);
    if (st.side) cudaStreamDestroy(st.side);
    if (st.hi) cudaStreamDestroy(st.hi);
    delete c.mixed;
    c.mixed = nullptr;
}

// Z_s -> Q60, blocked Cholesky, blocked triangular inverse (both with the big
// trailing updates for groups of four 128-column sub-panels, K = 512) and
// the camera Gram blocks of the inverse.
cudaError_t mixed_factor_inverse(Ctx& c) {
    MixedState& st = *c.mixed;
    const int64_t Np = c.Np, nb = Np / kNB;
    long long* Zq = reinterpret_cast<long long*>(c.d_Z);
    cudaError_t e;
    // both phases start after what the context stream holds
    if ((e = cudaEventRecord(st.ev[0], c.stream)) != cudaSuccess) return e;
    cudaStream_t main_stream = c.stream;
    if ((e = cudaStreamWaitEvent(st.hi, st.ev[0], 0)) != cudaSuccess) return e;
    c.stream = st.hi;
    {
        int64_t nt = (Np + 31) / 32;
        zscale_q_kernel<<<dim3((unsigned)nt, (unsigned)nt), dim3(8, 32), 0, c.stream>>>(
            c.N, Np, c.d_Z, c.d_F, c.d_G, c.d_D, c.est_on ? static_cast<long long*>(c.d_Zkeep) : nullptr,
            c.d_flag);
        c.launches++;
    }
    auto Zat = [&](int64_t row, int64_t col) { return Zq + row * Np + col; };
    auto Rat = [&](int64_t row, int64_t col) { return st.R + row * Np + col; };
    // Sub-panels in groups of m = mixed_group_max (4, or 2 for small scenes
    // and for six digits, whose eight accumulators hold K = 256 at most;
    // fewer at the end): inside a group, each sub-panel's update of the
    // group's later columns (K = 128); after it, one trailing update with all
    // m sub-panels (K = 128 m).
    const int64_t gmax = mixed_group_max(st.s, nb);
    auto group_len = [&](int64_t p) {
        const int64_t left = nb - p;
        return left >= gmax ? gmax : (left >= 2 ? 2 : 1);
    };
    // ---- Cholesky (context stream); event 3 + p once the group at p is final ----
    auto group_done = [&](int64_t p) { return cudaEventRecord(st.ev[3 + p], c.stream); };
    for (int64_t p = 0; p < nb;) {
        const int64_t m = group_len(p);
        bool last = false;
        for (int64_t j = p; j < p + m; ++j) {
            const int64_t kj = j * kNB, remJ = Np - kj - kNB;
            potrf_block(c, j);
            if (remJ <= 0) { last = true; break; }
            // L[rows > j, j] = A[rows > j, j] L_jj^-T
            slice_rows(c, 128, (int)remJ, Zat(kj + kNB, kj), BUF_P);
            launch_ozaki(c, 128, BUF_P, 0, (int)remJ, BUF_L, (int)kj, kNB, st.mapZ, (int)kj, (int)(kj + kNB), 0, 0,
                         kFL, nullptr, st.expL);
            // the group's later columns: A[rows > j, j+1 .. p+m-1] -= L[rows > j, j] L[j+1 .. p+m-1, j]^T
            const int64_t w = p + m - 1 - j;
            if (w > 0) {
                slice_rows(c, 128, (int)remJ, Zat(kj + kNB, kj), BUF_P);
                launch_ozaki(c, 128, BUF_P, 0, (int)remJ, BUF_P, 0, (int)(w * kNB), st.mapZ, (int)(kj + kNB),
                             (int)(kj + kNB), 1, 1, kFL, nullptr, nullptr);
            }
        }
        const int64_t kg = (p + m) * kNB, remG = Np - kg;
        if (last || remG <= 0) { group_done(p); break; }
        // trailing update with the group's sub-panels: A22 -= L[:, group] L[:, group]^T (lower tiles)
        slice_rows(c, (int)(m * kNB), (int)remG, Zat(kg, p * kNB), BUF_P);
        // the group's columns of L are final once the trailing update is
        // issued: it only writes columns beyond the group
        group_done(p);
        launch_ozaki(c, (int)(m * kNB), BUF_P, 0, (int)remG, BUF_P, 0, (int)remG, st.mapZ, (int)kg, (int)kg, 1, 1,
                     kFL, nullptr, nullptr);
        p += m;
    }
    if (!c.capturing) cudaEventRecord(c.ev[3], c.stream);
    if ((e = cudaEventRecord(st.ev[2], c.stream)) != cudaSuccess) { c.stream = main_stream; return e; }
    // ---- triangular inverse X = L^-1 (Q42), row blocks of 128 in the same
    // groups, on a low-priority stream with the second digit buffers: the
    // group at p waits only for the Cholesky's group at p, so its GEMMs fill
    // the GPU while the Cholesky (high priority) runs its serial diagonal
    // blocks ----
    if ((e = cudaStreamWaitEvent(st.side, st.ev[0], 0)) != cudaSuccess) { c.stream = main_stream; return e; }
    c.stream = st.side;
    st.swap_sets();
    e = cudaMemsetAsync(st.R, 0, sizeof(long long) * Np * Np, c.stream);
    if (e != cudaSuccess) { st.swap_sets(); c.stream = main_stream; return e; }
    identity_q_kernel<<<(int)((Np + 255) / 256), 256, 0, c.stream>>>(Np, st.R);
    c.launches++;
    auto finalize = [&](int64_t blk) {
        const int64_t k0 = blk * kNB, nc = k0 + kNB;
        // X[blk, :nc] = L_blk^-1 R[blk, :nc]
        slice_cols(c, 128, (int)nc, Rat(k0, 0), BUF_Q);
        launch_ozaki(c, 128, BUF_L, (int)k0, kNB, BUF_Q, 0, (int)nc, st.mapR, 0, (int)k0, 0, 0, kFX, st.expL, st.expQ);
        gram_q_kernel<<<(int)((nc + kGW - 1) / kGW), kGT, 0, c.stream>>>(c.n, Np, k0, nc, st.R, c.d_Sig);
        c.launches++;
    };
    for (int64_t p = 0; p < nb;) {
        const int64_t m = group_len(p);
        cudaStreamWaitEvent(c.stream, st.ev[3 + p], 0);
        for (int64_t j = p; j < p + m; ++j) {
            const int64_t kj = j * kNB, ncj = kj + kNB;
            finalize(j);
            // the group's later rows: R[j+1 .. p+m-1, :ncj] -= L[j+1 .. p+m-1, j] X[j, :ncj]
            const int64_t w = p + m - 1 - j;
            if (w > 0) {
                slice_cols(c, 128, (int)ncj, Rat(kj, 0), BUF_Q);
                slice_rows(c, 128, (int)(w * kNB), Zat(kj + kNB, kj), BUF_P);
                launch_ozaki(c, 128, BUF_P, 0, (int)(w * kNB), BUF_Q, 0, (int)ncj, st.mapR, 0, (int)(kj + kNB), 0, 1,
                             kFX, nullptr, st.expQ);
            }
        }
        const int64_t kg = (p + m) * kNB, remG = Np - kg;
        if (remG <= 0) break;
        // R[rows >= kg, :kg] -= L[rows >= kg, group] X[group, :kg]  (K = 128 m)
        slice_cols(c, (int)(m * kNB), (int)kg, Rat(p * kNB, 0), BUF_Q);
        slice_rows(c, (int)(m * kNB), (int)remG, Zat(kg, p * kNB), BUF_P);
        launch_ozaki(c, (int)(m * kNB), BUF_P, 0, (int)remG, BUF_Q, 0, (int)kg, st.mapR, 0, (int)kg, 0, 1, kFX,
                     nullptr, st.expQ);
        p += m;
    }
    st.swap_sets();
    c.stream = main_stream;
    // join: the rest of the step (extraction of the blocks) follows both streams
    if ((e = cudaEventRecord(st.ev[1], st.side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream, st.ev[1], 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c.stream, st.ev[2], 0)) != cudaSuccess) return e;
    if (c.mixed_bad_launch) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace ccov

// Test hooks (include/ccov_testing.h): one call of the digit-split
// tensor-core GEMM on caller data, with its own temporary workspace.
static ccov_status test_gemm(int s, int K, int M, int N, const uint16_t* digA, const int* expA,
                             const uint16_t* digB, const int* expB, int Fc, int sub, int lower, long long* C,
                             long long skip_fill, unsigned long long wait_ns) {
    using namespace ccov;
    if (s < 4 || s > 6 || (K != 128 && K != 256 && K != 512) || (K == 512 && s > 5) || M <= 0 || N <= 0 ||
        M % kBM || N % (2 * kBN) || !digA ||
        !digB || !C || wait_ns < 100000ull || wait_ns > 10000000000ull)
        return CCOV_ERR_INVALID_ARG;
    if (lower && N != M) return CCOV_ERR_INVALID_ARG;
    Ctx c;
    c.opt.mixed_slices = s;
    c.opt.precision = CCOV_PREC_MIXED;
    c.Np = ((M > N ? M : N) + 127) / 128 * 128;
    c.N = c.Np;
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) return CCOV_ERR_CUDA;
    ccov_status st = CCOV_OK;
    long long* dC = nullptr;
    int* dEA = nullptr;
    int* dEB = nullptr;
    do {
        if (mixed_alloc(c) != cudaSuccess) { st = CCOV_ERR_CUDA; break; }
        MixedState& ms = *c.mixed;
        ms.wait_ns = wait_ns;
        ms.skip_fill = skip_fill;
        if (cudaMalloc(&c.d_flag, 2 * sizeof(int)) != cudaSuccess) { st = CCOV_ERR_OOM; break; }
        cudaMemset(c.d_flag, 0, 2 * sizeof(int));
        {
            // row-major planes from the caller -> the tensor-core block layout
            std::vector<uint16_t> ha((size_t)s * c.Np * K, 0), hb((size_t)s * c.Np * K, 0);
            for (int a = 0; a < s; ++a)
                for (int r = 0; r < c.Np; ++r)
                    for (int k = 0; k < K; ++k) {
                        const int64_t o = blk_off(a, r, k, (int)c.Np, s);
                        if (r < M) ha[o] = digA[((size_t)a * M + r) * K + k];
                        if (r < N) hb[o] = digB[((size_t)a * N + r) * K + k];
                    }
            cudaMemcpy(ms.digP, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice);
            cudaMemcpy(ms.digQ, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice);
        }
        if (expA) { cudaMalloc(&dEA, M * sizeof(int)); cudaMemcpy(dEA, expA, M * sizeof(int), cudaMemcpyHostToDevice); }
        if (expB) { cudaMalloc(&dEB, N * sizeof(int)); cudaMemcpy(dEB, expB, N * sizeof(int), cudaMemcpyHostToDevice); }
        if (cudaMalloc(&dC, (size_t)M * N * 8) != cudaSuccess) { st = CCOV_ERR_OOM; break; }
        cudaMemcpy(dC, C, (size_t)M * N * 8, cudaMemcpyHostToDevice);
        CUtensorMap mapC;
        if (!make_c_map(&mapC, dC, M, N, N)) { st = CCOV_ERR_CUDA; break; }
        // the copies above ran on the legacy stream; the kernel's stream does not
        // wait for them by itself
        if (cudaDeviceSynchronize() != cudaSuccess) { st = CCOV_ERR_CUDA; break; }
        launch_ozaki(c, K, BUF_P, 0, M, BUF_Q, 0, N, mapC, 0, 0, lower, sub, Fc, dEA, dEB);
        if (c.mixed_bad_launch) { st = CCOV_ERR_INVALID_ARG; break; }
        if (cudaGetLastError() != cudaSuccess) { st = CCOV_ERR_CUDA; break; }
        if (cudaStreamSynchronize(c.stream) != cudaSuccess) { st = CCOV_ERR_CUDA; break; }
        int flag[2];
        cudaMemcpy(flag, c.d_flag, sizeof flag, cudaMemcpyDeviceToHost);
        if (flag[0] == DEV_TIMEOUT) { st = CCOV_ERR_TIMEOUT; break; }
        if (flag[0] != DEV_OK) { st = CCOV_ERR_CUDA; break; }
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

extern "C" CCOV_API ccov_status ccov_test_ozaki_gemm(int s, int K, int M, int N, const uint16_t* digA,
                                                    const int* expA, const uint16_t* digB, const int* expB,
                                                    int Fc, int sub, int lower, long long* C) {
    return test_gemm(s, K, M, N, digA, expA, digB, expB, Fc, sub, lower, C, -1, ccov::ptx::kWaitNs);
}

extern "C" CCOV_API ccov_status ccov_test_ozaki_gemm_wait(int s, int K, int M, int N, const uint16_t* digA,
                                                         const int* expA, const uint16_t* digB, const int* expB,
                                                         int Fc, int sub, int lower, long long* C,
                                                         long long skip_fill, unsigned long long wait_ns) {
    return test_gemm(s, K, M, N, digA, expA, digB, expB, Fc, sub, lower, C, skip_fill, wait_ns);
}

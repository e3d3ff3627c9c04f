// Parameter records of the grouped launches of the batched form (many
// scenes, Sec. 5 sub-reconstructions): one record per scene, and per launch
// a prefix array of the scenes' block counts, so that block b of the launch
// works on scene q with pre[q] <= b < pre[q + 1], as block b - pre[q] of that
// scene's own launch.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ccov {

struct GemmArgs {
    const __nv_bfloat16* digA;  // digit planes of A and B (layout of blk_off)
    const __nv_bfloat16* digB;
    int M, N;             // rows of A and of B (multiples of 128 and 64)
    int plane_rows;       // rows per digit plane in the operand buffers (Np)
    int a_row0, b_row0;   // first row of the operands inside their planes
    int c_x0, c_y0;       // origin of C in its map (column, row)
    int lower;            // keep only tiles touching the lower triangle
    int sub;              // 1: C -= A B^T, 0: C = A B^T
    int shift0;           // F_C - 14
    const int* expA;      // per row of A (nullptr = 0)
    const int* expB;      // per row of B (nullptr = 0)
    int stages;
    int* flag;
    unsigned long long wait_ns;  // limit of every barrier wait
    long long skip_fill;         // test hook: the producer leaves out this pipeline fill (-1: none)
    int64_t total_pairs;         // grouped launches: tile pairs of all problems
};

// One problem of a grouped launch (many independent GEMMs of the same s and K
// in one persistent kernel, e.g. the same trailing update of many scenes):
// its own operands, result map and tile range.  The maps live in global
// memory, written by the host before any launch that reads them.
struct alignas(128) GemmProblem {
    CUtensorMap mapC;
    CUtensorMap mapB;
    GemmArgs g;
    int64_t pair0;               // first tile pair of this problem in the launch
};

struct SliceRowsP {
    const long long* src;
    int64_t ld;
    int rows, F, s, plane_rows;
    __nv_bfloat16* dst;
    int* expo;
};

struct SliceColsP {
    const long long* src;
    int64_t ld;
    int ncols, F, s, plane_rows;
    __nv_bfloat16* dst;
    int* expo;
};

struct PotrfP {
    long long* Z;
    int64_t ld, k0;
    __nv_bfloat16* digL;
    int* expL;
    int s;
};

struct GramP {
    int64_t n, Np, k0, ncols;
    const long long* R;
    double* Sig;
};

struct ZscaleP {
    int64_t N, Np, nt;
    double* Z;
    const double* F;
    const double* G;
    const double* D;
};

struct IdentP {
    int64_t Np;
    long long* X;
};

struct GaugeP {
    int64_t N, ldz;
    const double* G;
    const double* HP;
    const double* Z;
    const double* W7s;
    double* small;
};

struct FdP {
    int64_t N, Np;
    const double* K;
    const double* Z;
    const double* G;
    double* F;
    double* D;
};

struct ExtractP {
    int64_t n;
    const double* D;
    const double* HP;
    const double* Cg;
    double* Sig;
};

// Scene q of block b: the largest q with pre[q] <= b (pre has k + 1 entries).
__device__ __forceinline__ int find_group(const int64_t* __restrict__ pre, int k, int64_t b) {
    int lo = 0, hi = k - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace ccov

// Allocation-free variant of the FP64 factor-and-invert routine of step (d).
//
// Some callers cannot call cudaMalloc: a real-time loop that must not
// allocate, or code inside a process whose device memory is owned by another
// allocator (a framework's caching allocator that has reserved it), where a
// cudaMalloc may fail or stall the whole device.  For
// them, ccov_spd_inverse_blocks_noalloc returns the 9x9 diagonal blocks of the
// inverse of a caller-provided SPD matrix with every piece of workspace held
// in one file-scope device array of fixed size (below).  The caller passes the
// input matrix and the output buffer; nothing is allocated by this call.
//
// Set-up: the first call on a device (with that device current) takes the
// array's device address with cudaGetSymbolAddress and sets the kernels'
// shared-memory attributes.
// Every call shares the array and starts by clearing what must start at zero
// (so a call that failed half-way leaves nothing that the next call reads);
// calls that overlap on the GPU (other streams, other threads) race on it.
// Every call waits for its stream to finish before it returns.
#include <mutex>

#include "ccov_internal.cuh"

namespace ccov {
namespace {

constexpr int64_t kNAMaxN = 576;                      // 64 cameras
constexpr int64_t kNAMaxNp = 640;                     // padded to the 128 block size
constexpr int64_t kOffZ = 0;                          // working copy, then the factor
constexpr int64_t kOffR = kOffZ + kNAMaxNp * kNAMaxNp;   // triangular inverse
constexpr int64_t kOffP = kOffR + kNAMaxNp * kNAMaxNp;   // panel copy
constexpr int64_t kOffLinv = kOffP + kNAMaxNp * kNB;     // diagonal-block inverses
constexpr int64_t kOffD = kOffLinv + kNAMaxNp * kNB;     // Jacobi scale
constexpr int64_t kOffSig = kOffD + kNAMaxNp;            // scaled blocks
constexpr int64_t kOffFlag = kOffSig + (kNAMaxN / 9) * 81;
constexpr int64_t kTotal = kOffFlag + 2;              // doubles: 7.9 MB
}  // namespace
}  // namespace ccov

// The workspace: one array per device, held until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[ccov::kTotal];

namespace ccov {
namespace {

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

__device__ __forceinline__ void na_flag(int* flag, int code, int detail) {
    if (atomicMax(flag, code) < code) flag[1] = detail;
}

// D_i = A_ii^-1/2 (rows of the padding: 1).
__global__ void na_scale_kernel(const double* __restrict__ A, int64_t lda, int64_t N, int64_t Np,
                                double* __restrict__ D, int* flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= Np) return;
    if (i >= N) { D[i] = 1.0; return; }
    double d = A[i * lda + i];
    if (!(d > 0.0)) { na_flag(flag, DEV_NOT_SPD, (int)i); d = 1.0; }
    D[i] = 1.0 / sqrt(d);
}

// Lower triangle of the working matrix D A D, identity on the padding.
__global__ void na_copy_kernel(const double* __restrict__ A, int64_t lda, int64_t N, int64_t Np,
                               const double* __restrict__ D, double* __restrict__ Z) {
    int64_t i = blockIdx.y * 32 + threadIdx.y, j = blockIdx.x * 32 + threadIdx.x;
    if (i >= Np || j > i) return;
    Z[i * Np + j] = (i < N && j < N) ? D[i] * A[i * lda + j] * D[j] : (i == j ? 1.0 : 0.0);
}

__global__ void na_unscale_kernel(int64_t n, const double* __restrict__ D, const double* __restrict__ Sig,
                                  double* __restrict__ out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * 81) return;
    int64_t cam = e / 81;
    int ab = (int)(e % 81), a = ab / 9, b = ab % 9;
    out[e] = Sig[e] * D[9 * cam + a] * D[9 * cam + b];
}

// Address of the array on the current device, taken once per device.
ccov_status scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CCOV_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CCOV_ERR_CUDA;
        if (setup_dense64() != cudaSuccess) return CCOV_ERR_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return CCOV_OK;
}

}  // namespace
}  // namespace ccov

extern "C" CCOV_API ccov_status ccov_spd_inverse_blocks_noalloc(const double* A, int64_t lda, int64_t N,
                                                               double* blocks, void* stream) {
    using namespace ccov;
    if (!A || !blocks || N <= 0 || N % 9 != 0 || lda < N) return CCOV_ERR_INVALID_ARG;
    if (N > kNAMaxN) return CCOV_ERR_INVALID_ARG;  // beyond the fixed workspace
    double* base = nullptr;
    ccov_status st = scratch_for_current_device(&base);
    if (st != CCOV_OK) return st;
    Ctx c;  // views into the static array only
    c.n = N / 9;
    c.N = N;
    c.Np = (N + kNB - 1) / kNB * kNB;
    c.stream = static_cast<cudaStream_t>(stream);
    c.d_Z = base + kOffZ;
    c.d_R = base + kOffR;
    c.d_P = base + kOffP;
    c.d_Linv = base + kOffLinv;
    c.d_D = base + kOffD;
    c.d_Sig = base + kOffSig;
    c.d_flag = reinterpret_cast<int*>(base + kOffFlag);
    const int64_t Np = c.Np, nb = Np / kNB;
    // what must start at zero: the error flag, the Gram blocks, the inverse workspace
    if (cudaMemsetAsync(c.d_flag, 0, 2 * sizeof(int), c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.d_Sig, 0, sizeof(double) * 81 * c.n, c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.d_R, 0, sizeof(double) * Np * Np, c.stream) != cudaSuccess)
        return CCOV_ERR_CUDA;
    na_scale_kernel<<<(int)((Np + 255) / 256), 256, 0, c.stream>>>(A, lda, N, Np, c.d_D, c.d_flag);
    {
        const unsigned nt = (unsigned)((Np + 31) / 32);
        na_copy_kernel<<<dim3(nt, nt), dim3(32, 32), 0, c.stream>>>(A, lda, N, Np, c.d_D, c.d_Z);
    }
    // blocked Cholesky: diagonal block, panel L21 = A21 L_kk^-T, trailing update
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
    // triangular inverse row block by row block, with the 9x9 Gram blocks
    launch_init_identity(c, c.d_R, Np);
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB;
        launch_trtri_row(c, k0);
        if (rem > 0)
            launch_gemm64(c, false, false, rem, k0 + kNB, kNB, -1.0, c.d_Z + (k0 + kNB) * Np + k0, Np,
                          c.d_R + k0 * Np, Np, 1.0, c.d_R + (k0 + kNB) * Np, Np, 0, 0);
    }
    na_unscale_kernel<<<(int)((c.n * 81 + 255) / 256), 256, 0, c.stream>>>(c.n, c.d_D, c.d_Sig, blocks);
    if (cudaGetLastError() != cudaSuccess) return CCOV_ERR_CUDA;
    int flag[2] = {0, 0};
    if (cudaMemcpyAsync(flag, c.d_flag, sizeof flag, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess)
        return CCOV_ERR_CUDA;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return CCOV_ERR_CUDA;
    if (flag[0] == DEV_NOT_SPD) return CCOV_ERR_DEGENERATE;
    if (flag[0] != DEV_OK) return CCOV_ERR_CUDA;
    return CCOV_OK;
}

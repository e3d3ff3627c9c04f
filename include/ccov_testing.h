/*
 * Test hooks of libccov (not part of the covariance API).
 */
#ifndef CCOV_TESTING_H
#define CCOV_TESTING_H

#include "ccov.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One call of the digit-split tensor-core GEMM used by the mixed path of step
 * (d) (the trailing updates of the blocked factorisation and inverse).
 *   s     digit planes, 4..6;  K  digits per row, 128 or 256
 *   digA  host, s planes of M x K bf16 bit patterns (plane-major), integer
 *         digits in [-128, 128]; row i of A = 2^expA[i] sum_a d_a 2^-(7+8a)
 *   digB  host, s planes of N x K, the same for the rows of B
 *   expA, expB  host int arrays (M, N) or NULL for all zero
 *   C     host int64 M x N row-major fixed point Q(Fc), updated in place:
 *         sub = 1: C -= A B^T, sub = 0: C = A B^T; products of digit orders
 *         a + b > s - 1 are left out
 *   lower 1: only tiles of 128 x 64 that reach the diagonal (M == N)
 * M and N must be multiples of 128 (tiles of 128 x 64 are worked on in pairs
 * by adjacent CTAs).  Returns TIMEOUT if a bounded device wait gave up. */
CCOV_API ccov_status ccov_test_ozaki_gemm(int s, int K, int M, int N, const uint16_t* digA, const int* expA,
                                          const uint16_t* digB, const int* expB, int Fc, int sub, int lower,
                                          long long* C);

/* The same GEMM with its barrier waits limited to wait_ns nanoseconds and, if
 * skip_fill >= 0, the producer of every CTA leaving out its pipeline fill
 * number skip_fill (counted from 0 over the CTA's tiles and K slices): the
 * MMA issuer then waits for data that never comes, gives up after wait_ns,
 * and the call returns CCOV_ERR_TIMEOUT with C unchanged on the host.  This
 * exercises the timeout exit of the kernel (producer, MMA issuer and
 * epilogue leave their loops, the issued MMAs are drained, TMEM is freed)
 * without hanging the device.  wait_ns: 1e5 .. 1e10. */
CCOV_API ccov_status ccov_test_ozaki_gemm_wait(int s, int K, int M, int N, const uint16_t* digA, const int* expA,
                                               const uint16_t* digB, const int* expB, int Fc, int sub, int lower,
                                               long long* C, long long skip_fill, unsigned long long wait_ns);

#ifdef __cplusplus
}
#endif

#endif /* CCOV_TESTING_H */

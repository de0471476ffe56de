// Dense split-precision strategy: workspace layout and launchers.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace be {

// A (M x K) of one row, element (m, k) at alpha * A[m * lda + k * ska] + beta
struct DenseA {
  const double *A;
  int64_t M, lda, ska;
  double alpha = 1.0, beta = 0.0;
};

// B (K x N), element (k, n) at alpha * B[k * ldb + n * snb] + beta; M_max
// sizes the workspace
struct DenseB {
  const double *B;
  int64_t K, N, ldb, snb, M_max;
  double alpha = 1.0, beta = 0.0;
};

// workspace carve-up: split operands (three BF16 parts each, K-major,
// zero-padded to the tile grid), power-of-two scales, and the per-column
// maxima of B
struct DenseWs {
  __nv_bfloat16 *a[3], *b[3];   // parts 1..3 of A (Mp x Kp) and of B^T (Np x Kp)
  int *sa, *sb;
  unsigned long long *bmax;
};

size_t dense_workspace_bytes(int64_t M_max, int64_t N, int64_t K);
DenseWs dense_ws_layout(void *ws, int64_t M_max, int64_t N, int64_t K);
// split the shared operand B into the workspace
cudaError_t dense_split_b(const DenseB &b, void *ws, cudaStream_t s);
// split A (one row of the batch) into the workspace
cudaError_t dense_split_a(const DenseA &a, int64_t K, int64_t M_max, int64_t N, void *ws, cudaStream_t s);
// tensor-core GEMM of the split operands into C (M x N, row stride ldc)
// lolo adds the next level's products x2*y3 and x3*y2 (tighter bound, two
// more MMAs per K-step); hdrain: k-blocks of 64 between drains of the
// leading-product accumulator;
// wait_limit: SM cycles before a pipeline wait gives up and records
// BE_ETIMEOUT in *status (0: about one second)
cudaError_t dense_split_gemm(const DenseA &a, int64_t N, int64_t K, int64_t M_max, double *C, int64_t ldc,
                             void *ws, bool lolo, int hdrain, int *status, long long wait_limit, cudaStream_t s);

}  // namespace be

// be_gemm_split_noalloc: the split-precision tensor-core GEMM with every
// byte of its scratch in a fixed array compiled into this library, so a call
// allocates no device memory at all.
//
// Who needs it: applications that route every device allocation through their
// own pool or budget and cannot let a library call cudaMalloc / cudaFree
// behind their back -- those calls can fail under a tight budget, take time,
// and cudaFree can synchronize the device, stalling the caller's other
// streams.  They pass their own inputs and outputs; the library's scratch
// comes from the array below.
//
// The array (NOALLOC_SCRATCH_BYTES + a status word) is held by every GPU where
// this library's device code is loaded until the process exits; with lazy
// module loading the driver reserves it on a device when the first call
// there looks up the array's device address (with that device current: the
// array's host-side name is only a stand-in and must never reach a kernel).
// Make that first call early, before the caller sets up its memory pool and
// before any stream capture.  A kernel whose bounded wait ran out leaves
// BE_ETIMEOUT in the status word until be_gemm_split_noalloc_status reads it.  All calls share the one array and
// it keeps the previous call's contents, so calls whose work overlaps on the
// GPU race with each other; run them in order on one stream.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/be.h"
#include "dense.hpp"

namespace be {
void set_last_error(const std::string &msg);   // abi.cpp
}

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;   // 64 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

// split operands, scales and column maxima; then one status word
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES + 256];

std::mutex g_mu;
void *g_dev_ptr[NOALLOC_MAX_DEVICES] = {};

// failures are reported through be_last_error() like every other call
int noalloc_fail(int code, const std::string &m) {
  be::set_last_error(m);
  return code;
}

// device address of the scratch array on the current device (once per device)
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(BE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return noalloc_fail(BE_EUNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(BE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return BE_OK;
}

}  // namespace

extern "C" {

int be_gemm_split_noalloc(const double *A, int64_t lda, const double *B, int64_t ldb, double *C, int64_t ldc,
                          int64_t M, int64_t N, int64_t K, void *stream) {
  if (M < 0 || N < 0 || K < 0) return noalloc_fail(BE_EARG, "negative size");
  if (M == 0 || N == 0) return BE_OK;
  if (!C || (K > 0 && (!A || !B))) return noalloc_fail(BE_EARG, "NULL matrix");
  if (ldc < N || (K > 0 && (lda < K || ldb < N))) return noalloc_fail(BE_EARG, "row stride shorter than the row");
  const size_t need = be::dense_workspace_bytes(M, N, K);
  if (need > NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(BE_ETOOMANY, "needs " + std::to_string(need) + " bytes of scratch; the fixed array holds " +
                                         std::to_string(NOALLOC_SCRATCH_BYTES) +
                                         " (about (M + N) * K * 6 bytes after padding M, N to 128 and K to 64)");
  void *ws = nullptr;
  int st = scratch_address(&ws);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the status word is not cleared here: it keeps BE_ETIMEOUT from any call
  // until be_gemm_split_noalloc_status reads and clears it
  int *status = (int *)((unsigned char *)ws + NOALLOC_SCRATCH_BYTES);
  cudaError_t e = cudaSuccess;
  if (K == 0) {
    e = cudaMemset2DAsync(C, (size_t)ldc * sizeof(double), 0, (size_t)N * sizeof(double), (size_t)M, s);
  } else if (e == cudaSuccess) {
    // the split kernels overwrite every workspace entry they use (padding
    // included) and dense_split_b clears the column maxima it accumulates
    e = be::dense_split_b(be::DenseB{B, K, N, ldb, 1, M}, ws, s);
    if (e == cudaSuccess) e = be::dense_split_a(be::DenseA{A, M, lda, 1}, K, M, N, ws, s);
    if (e == cudaSuccess)
      e = be::dense_split_gemm(be::DenseA{A, M, lda, 1}, N, K, M, C, ldc, ws, false, 1, status, 0, s);
  }
  if (e != cudaSuccess) return noalloc_fail(BE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return BE_OK;
}

// the status word after the scratch bytes of the current device's array,
// read and cleared by two synchronous one-word copies (no allocation)
int be_gemm_split_noalloc_status(int32_t *status) {
  if (!status) return noalloc_fail(BE_EARG, "NULL status");
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_noalloc_scratch, sizeof(int), NOALLOC_SCRATCH_BYTES);
  if (e == cudaSuccess) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_noalloc_scratch, &zero, sizeof(int), NOALLOC_SCRATCH_BYTES);
  }
  if (e != cudaSuccess) return noalloc_fail(BE_ECUDA, std::string("status word: ") + cudaGetErrorString(e));
  *status = v;
  return BE_OK;
}

}  // extern "C"

// Peak-rate probes of the FP64 and FP32 pipes: every thread runs independent
// chains of fused multiply-adds on register values (no memory traffic), so
// the kernel time measures the pipe's throughput; the result is written out
// only to keep the arithmetic alive.  Used to state the rooflines of the
// FP64 and double-float evaluation paths against this device's measured
// rates rather than nominal ones.
#include <string>

#include <cuda_runtime.h>

#include "../../include/be.h"

namespace be {
void set_last_error(const std::string &msg);   // abi.cpp
}

namespace {

constexpr int PROBE_CHAINS = 8;     // independent chains per thread
constexpr int PROBE_ITERS = 4096;   // multiply-adds per chain

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T *out, T a, T b) {
  T v[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = (T)(threadIdx.x + c);
#pragma unroll 4
  for (int k = 0; k < PROBE_ITERS; ++k)
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = v[c] * a + b;
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += v[c];
  if (s == (T)1234.5) out[blockIdx.x] = s;   // never true for these inputs; keeps the chains alive
}

}  // namespace

extern "C" {

int be_peak_probe(int32_t kind, int32_t reps, double *tflops) {
  if (!tflops || (kind != 0 && kind != 1) || reps < 1) return (be::set_last_error("bad arguments"), BE_EARG);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 8, block = 256;
  void *out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = -1;
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // the first launch warms up
    cudaEventRecord(a);
    if (kind == 0) fma_probe_kernel<double><<<grid, block>>>((double *)out, 0.999999, 1e-7);
    else fma_probe_kernel<float><<<grid, block>>>((float *)out, 0.9999f, 1e-4f);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (r > 0 && (best < 0 || ms < best)) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (out) cudaFree(out);
  if (e != cudaSuccess) return (be::set_last_error(std::string("probe: ") + cudaGetErrorString(e)), BE_ECUDA);
  const double flops = 2.0 * grid * block * (double)PROBE_CHAINS * PROBE_ITERS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return BE_OK;
}

}  // extern "C"

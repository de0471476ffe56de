// Generic strategy: one thread per output element of one einsum, any
// notation.  Evaluates Eq. (1) directly -- the output indices come from the
// thread's element, the contracted indices run as an odometer -- and each
// operand value is either a strided load or the result of the operand's
// producer program (the lambda of a functional batched einsum, evaluated at
// the access, i.e. fused into the load).  Accumulates in the output's type.
#include "generic_eval.cuh"
#include "launch_rec.hpp"

namespace be {

namespace {

__global__ void __launch_bounds__(256, 3) generic_kernel(const __grid_constant__ GParams p) {
  __shared__ double red[256];
  __shared__ __align__(16) unsigned char gsm[gen::GEMM_SMEM];
  // outputs per CTA per step: a thread, a warp or the whole CTA per output,
  // or one GEMM tile
  const int64_t per = p.mode == 0 ? blockDim.x : (p.mode == 1 ? (blockDim.x >> 5) : 1);
  const int64_t total = p.mode == 3 ? p.gemm.tiles : p.total_out;
  for (int64_t start = (int64_t)blockIdx.x * per; start < total; start += (int64_t)gridDim.x * per)
    gen::eval_range(p, start, min(per, total - start), red, gsm);
}

}  // namespace

cudaError_t launch_generic(const GParams &p0, cudaStream_t s) {
  if (p0.total_out == 0) return cudaSuccess;
  const int block = 256;
  GParams p = p0;
  if (p.mode == 3) {
    // the largest tile that still gives every SM work (two tiles each for
    // FP64, whose pipe bounds the tile)
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = p.out_dtype == F64 ? 2 * sms : sms;
    for (int t = p.out_dtype == F64 ? 32 : 64; t >= 16; t /= 2) {
      set_gemm_tile(p.gemm, t);
      if (p.gemm.tiles >= want) break;
    }
  }
  const int64_t per = p.mode == 0 ? block : (p.mode == 1 ? block / 32 : 1);
  const int64_t blocks = p.mode == 3 ? p.gemm.tiles : (p.total_out + per - 1) / per;
  const int grid = (int)(blocks < 148 * 16 ? blocks : 148 * 16);
  return be_launch(generic_kernel, dim3(grid), dim3(block), 0, s, p);
}

}  // namespace be

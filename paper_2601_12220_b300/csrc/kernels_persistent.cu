// Persistent multi-instance executor: one launch evaluates many batched
// einsums of different notations, sizes and dtypes (a batch of batched
// einsums, Sec. "Batched Einstein Summation").  The host cuts every row of
// every instance into output tiles of roughly equal work and lists them,
// largest first; a grid of a few CTAs per SM pulls tile numbers from a
// global counter until the list is exhausted.  A CTA copies the row's
// descriptor (notation, strides, producer program) into shared memory when
// the row changes and evaluates each output of the tile with the same
// per-element code as the generic kernel -- so every output has one owner,
// no partial sums are combined across CTAs, and the bits do not depend on
// the schedule.  The counter is only ever incremented: no CTA waits on
// another.
#include "generic_eval.cuh"

namespace be {

namespace {

__global__ void __launch_bounds__(256, 4) persistent_kernel(const GParams *__restrict__ rows,
                                                         const PTile *__restrict__ tiles, int64_t n_tiles,
                                                         unsigned long long *__restrict__ counter) {
  __shared__ GParams sp;
  __shared__ double red[256];
  __shared__ __align__(16) unsigned char gsm[gen::GEMM_SMEM];
  __shared__ long long tile_id;
  __shared__ int cur_row;
  if (threadIdx.x == 0) cur_row = -1;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) tile_id = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long t = tile_id;
    if (t >= n_tiles) break;
    const PTile tl = tiles[t];
    if (tl.row != cur_row) {
      const int4 *src = (const int4 *)(rows + tl.row);
      int4 *dst = (int4 *)&sp;
      for (int k = threadIdx.x; k < (int)(sizeof(GParams) / sizeof(int4)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) cur_row = tl.row;
    gen::eval_range(sp, tl.start, tl.count, red, gsm);
    __syncthreads();   // tile consumed before tile_id and sp are rewritten
  }
}

static_assert(sizeof(GParams) % sizeof(int4) == 0, "descriptor copied as int4 words");

}  // namespace

cudaError_t launch_persistent(const GParams *rows, const PTile *tiles, int64_t n_tiles, unsigned long long *counter,
                              int grid, int block, cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  persistent_kernel<<<grid, block, 0, s>>>(rows, tiles, n_tiles, counter);
  return cudaGetLastError();
}

}  // namespace be

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
// the schedule.  The counter is only ever incremented.  A tile with a
// dependency (a factored step reading the intermediate of earlier steps)
// waits until every tile of the rows it reads has finished: a CTA counts a
// row's finished tiles after a release fence, the waiting thread reads the
// count with acquire semantics.  The list is ordered so that every tile a
// tile depends on comes before it, and a tile is only pulled by a running
// CTA, so every awaited tile is held by a running CTA whose own waits point
// further back: the waits cannot form a cycle.  Each wait is bounded
// (about one second of SM cycles, or the caller's limit); on expiry
// BE_ETIMEOUT goes to the status word, the tile is skipped and still
// counted, so that no later wait depends on it.
#include "generic_eval.cuh"

namespace be {

namespace {

__device__ __forceinline__ unsigned int load_acquire(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(256, 4) persistent_kernel(const GParams *__restrict__ rows,
                                                         const PTile *__restrict__ tiles, int64_t n_tiles,
                                                         unsigned long long *__restrict__ counter,
                                                         unsigned int *done, int *status, long long limit) {
  __shared__ GParams sp;
  __shared__ double red[256];
  __shared__ __align__(16) unsigned char gsm[gen::GEMM_SMEM];
  __shared__ long long tile_id;
  __shared__ int cur_row, skip;
  if (threadIdx.x == 0) cur_row = -1;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) tile_id = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long t = tile_id;
    if (t >= n_tiles) break;
    const PTile tl = tiles[t];
    if (threadIdx.x == 0) {
      skip = 0;
      for (int q = 0; q < 2; ++q) {
        if (tl.dep[q] < 0 || !done) continue;
        const long long t0 = clock64();
        while (load_acquire(done + tl.dep[q]) < (unsigned int)tl.need[q]) {
          if (clock64() - t0 > limit) {
            if (status) atomicExch(status, 9);   // BE_ETIMEOUT
            skip = 1;
            break;
          }
          __nanosleep(200);
        }
      }
    }
    if (tl.row != cur_row) {
      const int4 *src = (const int4 *)(rows + tl.row);
      int4 *dst = (int4 *)&sp;
      for (int k = threadIdx.x; k < (int)(sizeof(GParams) / sizeof(int4)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) cur_row = tl.row;
    if (!skip) gen::eval_range(sp, tl.start, tl.count, red, gsm);
    __syncthreads();   // tile consumed before tile_id and sp are rewritten
    if (threadIdx.x == 0 && done) {
      __threadfence();                       // the tile's outputs before its count
      atomicAdd(done + tl.row, 1u);
    }
  }
}

static_assert(sizeof(GParams) % sizeof(int4) == 0, "descriptor copied as int4 words");

}  // namespace

cudaError_t launch_persistent(const GParams *rows, const PTile *tiles, int64_t n_tiles, unsigned long long *counter,
                              unsigned int *done, int *status, long long wait_limit, int grid, int block,
                              cudaStream_t s) {
  if (n_tiles == 0) return cudaSuccess;
  persistent_kernel<<<grid, block, 0, s>>>(rows, tiles, n_tiles, counter, done, status,
                                           wait_limit > 0 ? wait_limit : 2000000000LL);
  return cudaGetLastError();
}

}  // namespace be

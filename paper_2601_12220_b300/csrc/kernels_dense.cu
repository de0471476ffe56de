// Dense split-precision strategy: an FP64 contraction that is a plain GEMM
// after flattening (e.g. the cluster-operator form 'abef,efij->abij' of the
// introduction, M = ab, K = ef, N = ij) evaluated on the tcgen05 tensor
// cores.
//
//  1. split_rows / split_cols: each FP64 operand (or its affine producer
//     alpha * x + beta, evaluated here) is scaled by a power of two per row
//     of A (per column of B) so that its largest entry lies in [2^13, 2^14),
//     rounded to a float x and written as three BF16 parts
//     x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2) (both
//     differences are exact in FP32; about 24 significant bits in all) into a
//     zero-padded K-major workspace.  BF16 keeps FP32's exponent range, so
//     entries far below their row's maximum (the exp-decaying cluster
//     amplitudes) keep their relative precision.
//  2. gemm_split_kernel: TMA streams 128 x 64 tiles of the six parts into
//     shared memory (128-byte swizzle, two stages); one thread issues
//     tcgen05.mma kind::f16 (BF16 inputs, FP32 accumulators in tensor
//     memory) per K-step of 16: the leading product x1*y1 into H and the
//     five products of the next two levels (x1*y2, x2*y1, x1*y3, x2*y2,
//     x3*y1; plus x2*y3, x3*y2 when requested) into L, each double-buffered
//     (4 x 128 columns).  Six BF16 products take the tensor pipe as long as
//     three TF32 ones and move 6 bytes of operand per element instead of 8.
//     The tensor core rounds its FP32 accumulator toward zero (about 2^-23
//     of the accumulator per MMA), so H is drained every hdrain k-blocks of
//     64 values (4 MMAs each) and L, which holds terms 2^-8 of H's size and
//     smaller, every 8 k-blocks; sixteen epilogue warps read them
//     (tcgen05.ld) and add H into an FP32 pair per output by Kahan's
//     compensated summation and L into its compensation term.  The result
//     is scaled back and stored in FP64.
//  Error per output, relative to S = sum |a||b|: rounding to float and the
//  three-part residual about 2^-23 per operand, dropped products
//  (x2*y3, x3*y2, x3*y3) about 2^-23, H truncation about 2^-23 per MMA
//  between drains (4 * 2^-23 at hdrain = 1, 8 * 2^-23 at hdrain = 2), L
//  truncation below 2^-22, the compensated sum of the drains about 2^-23.
// Every mbarrier wait is bounded (about one second of clock cycles); on
// expiry the CTA records BE_ETIMEOUT in a status word, stops issuing work,
// waits (bounded) for its own copies and frees its tensor memory.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dense.hpp"
#include "launch_attr.hpp"
#include "tc_common.cuh"

namespace be {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;           // BK: BF16 values per 128-byte row
constexpr int NPART = 3;                               // BF16 parts per operand
constexpr int STAGES = 2;
constexpr int L_CHUNK = 8;                             // k-blocks per drain of the small-term accumulator
constexpr int SPLIT_CTAS_PER_SM = 8;                   // rows in flight per SM in split_rows
constexpr int TILE_BYTES = BM * BK * 2;                // one BF16 128 x 64 tile
constexpr int STAGE_BYTES = 2 * NPART * TILE_BYTES;    // A1 A2 A3, B1 B2 B3
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int NTHREADS = 576;                          // warp 0 TMA, warp 1 MMA, warps 2-17 epilogue
constexpr int NEPI = 512;                              // epilogue threads
constexpr long long TIMEOUT_CYCLES = 2000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait (tc::mbar_wait: suspended between tries, the clock read
// every eighth try); false when it gave up (or another thread already did)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status,
                                          long long limit) {
  return tc::mbar_wait(bar, parity, abort_flag, status, limit);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = 128
constexpr uint32_t IDESC = tc::idesc_bf16(BM, BN);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 2^k as a double for k in [-1022, 1023]
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }
// v * 2^k without a library call (two steps keep each factor normal)
__device__ __forceinline__ double scale2(double v, int k) {
  const int k1 = k / 2, k2 = k - k1;
  return (v * pow2(k1)) * pow2(k2);
}

// Kahan-compensated accumulation of v into (hi, c), whose running sum is
// hi - c: the error of the sum of n drained values stays within
// 2u |sum of |v|| + O(n u^2) (Kahan's bound, u = 2^-24), four FP32
// operations per value instead of TwoSum's seven
__device__ __forceinline__ void kahan_acc(float &hi, float &c, float v) {
  const float y = v - c;
  const float t = hi + y;
  c = (t - hi) - y;
  hi = t;
}

// drain 32 accumulator columns at taddr: the leading-product accumulator H
// by Kahan's compensated sum into (hi, c); the small-term accumulator L
// (terms at most about 2^-7 of H's) straight into the compensation
template <bool LEAD>
__device__ __forceinline__ void drain32(uint32_t taddr, float *hi, float *c) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t r[8];
    tc::tmem_ld8(taddr + (uint32_t)(8 * q), r);
    tc::tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (LEAD) kahan_acc(hi[8 * q + j], c[8 * q + j], __uint_as_float(r[j]));
      else c[8 * q + j] -= __uint_as_float(r[j]);
    }
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_split_kernel(const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmA2,
                      const __grid_constant__ CUtensorMap tmA3, const __grid_constant__ CUtensorMap tmB1,
                      const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ CUtensorMap tmB3,
                      const int *__restrict__ sa, const int *__restrict__ sb, double *__restrict__ C, int64_t M,
                      int64_t N, int64_t ldc, int nkb, int lolo, int hdrain, int *status, long long limit) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES);
  uint64_t *full = bars, *empty = bars + STAGES;
  uint64_t *hf = bars + 2 * STAGES, *he = hf + 2, *lf = he + 2, *le = lf + 2, *fin = le + 2;
  uint32_t *tmem_slot = (uint32_t *)(fin + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&hf[b], 1);
      mbar_init(&he[b], NEPI);
      mbar_init(&lf[b], 1);
      mbar_init(&le[b], NEPI);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // tensor memory columns: H0 [0,128) H1 [128,256) L0 [256,384) L1 [384,512)

  if (warp == 0) {
    if (lane == 0) {
      int last_kb[STAGES];
      for (int s = 0; s < STAGES; ++s) last_kb[s] = -1;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, status, limit)) break;
        uint8_t *st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d(st, &tmA1, &full[s], kb * BK, m0);
        tma_load_2d(st + TILE_BYTES, &tmA2, &full[s], kb * BK, m0);
        tma_load_2d(st + 2 * TILE_BYTES, &tmA3, &full[s], kb * BK, m0);
        tma_load_2d(st + 3 * TILE_BYTES, &tmB1, &full[s], kb * BK, n0);
        tma_load_2d(st + 4 * TILE_BYTES, &tmB2, &full[s], kb * BK, n0);
        tma_load_2d(st + 5 * TILE_BYTES, &tmB3, &full[s], kb * BK, n0);
        last_kb[s] = kb;
      }
      // on an abort the MMA thread may not have consumed every stage: wait
      // (bounded by the full limit, not the caller's) until the last copies
      // issued into each stage have landed, so that none is outstanding when
      // the CTA leaves
      if (*abort_flag) {
        for (int s = 0; s < STAGES; ++s) {
          if (last_kb[s] < 0) continue;
          const uint32_t par = (uint32_t)(last_kb[s] / STAGES) & 1u;
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[s], par) && clock64() - t0 < TIMEOUT_CYCLES) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int hc = kb / hdrain, hb = hc & 1, lc = kb / L_CHUNK, lb = lc & 1;
        const bool hfirst = (kb % hdrain) == 0;
        const bool hlast = (kb % hdrain) == hdrain - 1 || kb == nkb - 1;
        const bool lfirst = (kb % L_CHUNK) == 0;
        const bool llast = (kb % L_CHUNK) == L_CHUNK - 1 || kb == nkb - 1;
        if (hfirst && !mbar_wait(&he[hb], ((uint32_t)(hc >> 1) & 1u) ^ 1u, abort_flag, status, limit)) break;
        if (lfirst && !mbar_wait(&le[lb], ((uint32_t)(lc >> 1) & 1u) ^ 1u, abort_flag, status, limit)) break;
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (uint32_t)(kb / STAGES) & 1u, abort_flag, status, limit)) break;
        tc_fence_after();
        const uint32_t dh = tmem + (uint32_t)(hb * BN), dl = tmem + (uint32_t)(2 * BN + lb * BN);
        const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
        // K-steps of 16 BF16 values (32 bytes of each 128-byte row)
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint64_t a1 = sdesc(base + ks * 32), a2 = sdesc(base + TILE_BYTES + ks * 32),
                         a3 = sdesc(base + 2 * TILE_BYTES + ks * 32);
          const uint64_t b1 = sdesc(base + 3 * TILE_BYTES + ks * 32), b2 = sdesc(base + 4 * TILE_BYTES + ks * 32),
                         b3 = sdesc(base + 5 * TILE_BYTES + ks * 32);
          mma_bf16(dh, a1, b1, (hfirst && ks == 0) ? 0u : 1u);
          mma_bf16(dl, a1, b2, (lfirst && ks == 0) ? 0u : 1u);
          mma_bf16(dl, a2, b1, 1u);
          mma_bf16(dl, a1, b3, 1u);
          mma_bf16(dl, a2, b2, 1u);
          mma_bf16(dl, a3, b1, 1u);
          if (lolo) {
            mma_bf16(dl, a2, b3, 1u);
            mma_bf16(dl, a3, b2, 1u);
          }
        }
        mma_commit(&empty[s]);   // frees the stage once these MMAs have read it
        if (hlast) mma_commit(&hf[hb]);
        if (llast) mma_commit(&lf[lb]);
      }
      // all MMAs issued by this thread have completed once fin fires
      mma_commit(fin);
      long long t0 = clock64();
      while (!mbar_try_wait(fin, 0) && clock64() - t0 < TIMEOUT_CYCLES) {
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32*(w%4)..; warps 2-5, 6-9, 10-13, 14-17 take column quarters 0..3
    const int sub = warp & 3, quarter = (warp - 2) >> 2;
    const int row = sub * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(quarter * 32);
    float hi[32], lo[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
    bool ok = true;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int hc = kb / hdrain, hb = hc & 1, lc = kb / L_CHUNK, lb = lc & 1;
      const bool hlast = (kb % hdrain) == hdrain - 1 || kb == nkb - 1;
      const bool llast = (kb % L_CHUNK) == L_CHUNK - 1 || kb == nkb - 1;
      if (hlast) {
        const bool got = mbar_wait(&hf[hb], (uint32_t)(hc >> 1) & 1u, abort_flag, status, limit);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }   // warp-uniform before tcgen05.ld
        tc_fence_after();
        drain32<true>(lane_base + (uint32_t)(hb * BN), hi, lo);
        tc_fence_before();
        mbar_arrive(&he[hb]);
      }
      if (llast) {
        const bool gl = mbar_wait(&lf[lb], (uint32_t)(lc >> 1) & 1u, abort_flag, status, limit);
        if (!__all_sync(0xffffffffu, gl)) { ok = false; break; }
        tc_fence_after();
        drain32<false>(lane_base + (uint32_t)(2 * BN + lb * BN), hi, lo);
        tc_fence_before();
        mbar_arrive(&le[lb]);
      }
    }
    const int64_t m = m0 + row;
    if (ok && m < M) {
      const int sm = sa[m];
      double *crow = C + m * ldc;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t n = n0 + quarter * 32 + j;
        if (n < N) crow[n] = scale2((double)hi[j] - (double)lo[j], -(sm + sb[n]));
      }
    }
  }

  // teardown: the copy thread has waited for its outstanding copies and the
  // MMA thread for its MMAs (fin) before the tensor memory is released
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();   // lane 0 ran the issue loop alone
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ---------------------------------------------------------------- split

__device__ __forceinline__ double block_max(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

__device__ __forceinline__ int scale_for(double mx) {
  if (!(mx > 0.0)) return 0;
  int e;
  frexp(mx, &e);          // mx = f * 2^e, f in [0.5, 1)
  return 14 - e;          // mx * 2^(14-e) in [2^13, 2^14)
}

// x * 2^s rounded to a float (half up) from the bits of x, integer operations
// only; results below FP32's normal range (2^-100 and more below the row's
// maximum, which scales to [2^13, 2^14)) become zero
__device__ __forceinline__ float scaled_float(double x, int s) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const uint32_t ax = hw & 0x7FFFFFFFu;
  const int fe = (int)(ax >> 20) - 1023 + 127 + s;             // biased exponent of the float
  if (fe <= 0) return 0.0f;
  const uint32_t mag = (((uint32_t)fe << 23) | ((ax & 0xFFFFFu) << 3) | (lw >> 29)) + ((lw >> 28) & 1u);
  return __uint_as_float(mag | (hw & 0x80000000u));
}

__device__ __forceinline__ float bf16_rn(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// three BF16 parts of a float x: p1 = bf16(x), p2 = bf16(x - p1),
// p3 = bf16(x - p1 - p2).  x - p1 and (x - p1) - p2 are exact in FP32 (each
// part takes the leading 8 significant bits of what is left), so
// |x - p1 - p2 - p3| <= 2^-9 |x - p1 - p2| <= 2^-25 |x| or so
struct Parts {
  float p1, p2, p3;
};
__device__ __forceinline__ Parts parts3(float x) {
  Parts r;
  r.p1 = bf16_rn(x);
  const float r1 = x - r.p1;
  r.p2 = bf16_rn(r1);
  r.p3 = bf16_rn(r1 - r.p2);
  return r;
}

// x * 2^s split into three BF16 parts; the float image from the bits when
// the scaled row stays in FP32's normal range (F32, a template parameter so
// that the FP64 form is not evaluated beside it), else through FP64
template <bool F32>
__device__ __forceinline__ Parts split_scaled(double x, int s) {
  return parts3(F32 ? scaled_float(x, s) : __double2float_rn(x * pow2(s)));
}

// the operand value of an affine producer, alpha * x + beta (AFF), else x
template <bool AFF>
__device__ __forceinline__ double affine(double x, double alpha, double beta) {
  return AFF ? fma(alpha, x, beta) : x;
}

// A (M x K): A[m*lda + k*ska] -> three BF16 parts [Mp x Kp], zero-padded;
// sa[m].  Rows with unit stride and 16-byte alignment are read as double2,
// four in flight per thread, and written as BF16 pairs.  AFF: the operand is
// alpha * A + beta (an affine producer fused into the split).
// one pass over row m: every entry (its affine producer's value) times 2^s
// split into three BF16 parts and written to the padded row; returns this
// thread's largest high word of |x| (the row maximum's exponent) when TRACK
template <bool AFF, bool TRACK, bool F32>
__device__ __forceinline__ uint32_t split_pass(const double *__restrict__ row, bool vec, int64_t K, int64_t ska,
                                               __nv_bfloat16 *__restrict__ r1, __nv_bfloat16 *__restrict__ r2p,
                                               __nv_bfloat16 *__restrict__ r3, int64_t Kp, int s,
                                               double alpha, double beta) {
  uint32_t bits = 0;
  if (vec) {
    const double2 *r2 = (const double2 *)row;
    __nv_bfloat162 *o1 = (__nv_bfloat162 *)r1, *o2 = (__nv_bfloat162 *)r2p, *o3 = (__nv_bfloat162 *)r3;
    const int64_t K2 = K >> 1, Kp2 = Kp >> 1;
    int64_t k = threadIdx.x;
    for (; k + 3 * blockDim.x < K2; k += 4 * blockDim.x) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = r2[k + u * blockDim.x];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double x = affine<AFF>(v[u].x, alpha, beta), y = affine<AFF>(v[u].y, alpha, beta);
        if (TRACK) {
          bits = max(bits, (uint32_t)__double2hiint(x) & 0x7fffffffu);
          bits = max(bits, (uint32_t)__double2hiint(y) & 0x7fffffffu);
        }
        const Parts a = split_scaled<F32>(x, s), b = split_scaled<F32>(y, s);
        o1[k + u * blockDim.x] = __floats2bfloat162_rn(a.p1, b.p1);
        o2[k + u * blockDim.x] = __floats2bfloat162_rn(a.p2, b.p2);
        o3[k + u * blockDim.x] = __floats2bfloat162_rn(a.p3, b.p3);
      }
    }
    for (; k < Kp2; k += blockDim.x) {
      Parts a{0.f, 0.f, 0.f}, b{0.f, 0.f, 0.f};
      if (k < K2) {
        const double2 v = r2[k];
        const double x = affine<AFF>(v.x, alpha, beta), y = affine<AFF>(v.y, alpha, beta);
        if (TRACK) {
          bits = max(bits, (uint32_t)__double2hiint(x) & 0x7fffffffu);
          bits = max(bits, (uint32_t)__double2hiint(y) & 0x7fffffffu);
        }
        a = split_scaled<F32>(x, s);
        b = split_scaled<F32>(y, s);
      }
      o1[k] = __floats2bfloat162_rn(a.p1, b.p1);
      o2[k] = __floats2bfloat162_rn(a.p2, b.p2);
      o3[k] = __floats2bfloat162_rn(a.p3, b.p3);
    }
    return bits;
  }
  for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) {
    Parts a{0.f, 0.f, 0.f};
    if (k < K) {
      const double x = affine<AFF>(row[k * ska], alpha, beta);
      if (TRACK) bits = max(bits, (uint32_t)__double2hiint(x) & 0x7fffffffu);
      a = split_scaled<F32>(x, s);
    }
    r1[k] = __float2bfloat16_rn(a.p1);
    r2p[k] = __float2bfloat16_rn(a.p2);
    r3[k] = __float2bfloat16_rn(a.p3);
  }
  return bits;
}

// Row m of A into its three parts and its scale sa[m].  BF16 parts keep
// FP32's exponent range, so one fixed scale S0 = 2^40 serves every row whose
// largest |x| lies in [2^-26, 2^40): scaled products with B's parts and their
// sums over K stay inside FP32's range, and what FP32 drops (scaled entries
// below 2^-126) is at least 2^-140 of the row maximum, as with a row's own
// scale.  One pass splits the row at S0 while it finds the maximum; a row
// outside the window is split again with the power-of-two scale that puts
// its maximum in [2^13, 2^14).  Padding rows (m >= M) are written as zeros.
constexpr int S0 = 40;
template <bool AFF>
__device__ __forceinline__ void split_row(int64_t m, const double *__restrict__ A, int64_t M, int64_t K, int64_t lda,
                                          int64_t ska, __nv_bfloat16 *__restrict__ p1, __nv_bfloat16 *__restrict__ p2,
                                          __nv_bfloat16 *__restrict__ p3, int64_t Kp, int *__restrict__ sa,
                                          double alpha, double beta, double *red) {
  const double *row = A + m * lda;
  __nv_bfloat16 *r1 = p1 + m * Kp, *r2 = p2 + m * Kp, *r3 = p3 + m * Kp;
  const bool vec = ska == 1 && ((uintptr_t)row & 15) == 0 && (K & 1) == 0 && (Kp & 1) == 0;
  // |x| compared as integers on the sign-cleared high word (32-bit: a 64-bit
  // integer max issues on the FP64 pipe); the scale needs only the largest
  // exponent, which the high word carries
  const uint32_t bits = m < M ? split_pass<AFF, true, true>(row, vec, K, ska, r1, r2, r3, Kp, S0, alpha, beta)
                              : split_pass<AFF, false, true>(row, vec, 0, ska, r1, r2, r3, Kp, S0, alpha, beta);
  const double mx = block_max(__hiloint2double((int)bits, 0), red);
  int s = S0;
  if (!(mx == 0.0 || (mx >= 0x1p-26 && mx < 0x1p+40))) {
    s = scale_for(mx);
    // the scaled row max is below 2^14; FP32 scaling is exact while |x| >= 2^-100 * max
    if (mx > 0x1p-26 && mx < 0x1p+100 && s > -120 && s < 120)
      split_pass<AFF, false, true>(row, vec, K, ska, r1, r2, r3, Kp, s, alpha, beta);
    else
      split_pass<AFF, false, false>(row, vec, K, ska, r1, r2, r3, Kp, s, alpha, beta);
  }
  if (threadIdx.x == 0 && m < M) sa[m] = s;
}

// one CTA per row at a time over a grid of a few CTAs per SM
template <bool AFF>
__global__ void __launch_bounds__(256) split_rows(const double *__restrict__ A, int64_t M, int64_t Mp, int64_t K,
                                                  int64_t lda, int64_t ska, __nv_bfloat16 *__restrict__ p1,
                                                  __nv_bfloat16 *__restrict__ p2, __nv_bfloat16 *__restrict__ p3,
                                                  int64_t Kp, int *__restrict__ sa, double alpha, double beta) {
  __shared__ double red[32];
  for (int64_t m = blockIdx.x; m < Mp; m += gridDim.x) {
    split_row<AFF>(m, A, M, K, lda, ska, p1, p2, p3, Kp, sa, alpha, beta, red);
    __syncthreads();   // red is reused by the next row's maximum
  }
}

// per-column max |B| of B (K x N), B[k*ldb + n*snb], rounded down to its high
// word (the scale needs only the exponent); K split over blockIdx.y,
// combined with an integer max on the (non-negative) double bit patterns
template <bool AFF>
__global__ void __launch_bounds__(256) col_max(const double *__restrict__ B, int64_t K, int64_t N, int64_t ldb,
                                               int64_t snb, unsigned long long *__restrict__ bmax, double alpha,
                                               double beta) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t kper = (K + gridDim.y - 1) / gridDim.y;
  const int64_t k0 = (int64_t)blockIdx.y * kper, k1 = min(K, k0 + kper);
  uint32_t bits = 0;
  for (int64_t k = k0; k < k1; ++k)
    bits = max(bits, (uint32_t)__double2hiint(affine<AFF>(B[k * ldb + n * snb], alpha, beta)) & 0x7fffffffu);
  atomicMax(&bmax[n], (unsigned long long)bits << 32);
}

// B (K x N) -> transposed BF16 parts [Np x Kp] (K-major), zero-padded;
// AFF: the operand is alpha * B + beta
template <bool AFF>
__global__ void __launch_bounds__(256) split_cols_t(const double *__restrict__ B, int64_t K, int64_t N, int64_t ldb,
                                                   int64_t snb, const unsigned long long *__restrict__ bmax,
                                                   int *__restrict__ sb, __nv_bfloat16 *__restrict__ p1,
                                                   __nv_bfloat16 *__restrict__ p2, __nv_bfloat16 *__restrict__ p3,
                                                   int64_t Kp, int64_t Np, double alpha, double beta) {
  __shared__ double tile[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32, nb = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int64_t nn = nb + tx;
  const int scl = nn < N ? scale_for(__longlong_as_double((long long)bmax[nn])) : 0;
  if (blockIdx.x == 0 && ty == 0 && nn < N) sb[nn] = scl;
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r;
    tile[r][tx] = (k < K && nn < N) ? scale2(affine<AFF>(B[k * ldb + nn * snb], alpha, beta), scl) : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t n = nb + r, k = k0 + tx;
    if (n < Np && k < Kp) {
      const Parts q = parts3(__double2float_rn(tile[tx][r]));   // scaled by 2^sb[n] already
      p1[n * Kp + k] = __float2bfloat16_rn(q.p1);
      p2[n * Kp + k] = __float2bfloat16_rn(q.p2);
      p3[n * Kp + k] = __float2bfloat16_rn(q.p3);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static bool make_map(CUtensorMap *map, const void *base, int64_t inner, int64_t outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  cuuint64_t strides[1] = {(cuuint64_t)(inner * 2)};
  cuuint32_t box[2] = {BK, BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t dense_workspace_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Mp = (M + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
  return (size_t)(Mp * Kp * 2 * NPART + Np * Kp * 2 * NPART) + (size_t)(Mp + Np) * 4 + (size_t)Np * 8 + 2048;
}

cudaError_t dense_split_b(const DenseB &b, void *ws, cudaStream_t s) {
  const int64_t Np = (b.N + BN - 1) / BN * BN, Kp = (b.K + BK - 1) / BK * BK;
  DenseWs w = dense_ws_layout(ws, b.M_max, b.N, b.K);
  cudaError_t e = cudaMemsetAsync(w.bmax, 0, sizeof(unsigned long long) * (size_t)b.N, s);
  if (e != cudaSuccess) return e;
  const bool aff = b.alpha != 1.0 || b.beta != 0.0;
  if (b.N > 0 && b.K > 0) {
    dim3 gm((unsigned)((b.N + 255) / 256), (unsigned)std::min<int64_t>(64, b.K));
    if (aff) col_max<true><<<gm, 256, 0, s>>>(b.B, b.K, b.N, b.ldb, b.snb, w.bmax, b.alpha, b.beta);
    else col_max<false><<<gm, 256, 0, s>>>(b.B, b.K, b.N, b.ldb, b.snb, w.bmax, 1.0, 0.0);
  }
  dim3 g((unsigned)(Kp / 32), (unsigned)(Np / 32));
  if (aff)
    split_cols_t<true><<<g, 256, 0, s>>>(b.B, b.K, b.N, b.ldb, b.snb, w.bmax, w.sb, w.b[0], w.b[1], w.b[2], Kp, Np,
                                         b.alpha, b.beta);
  else
    split_cols_t<false><<<g, 256, 0, s>>>(b.B, b.K, b.N, b.ldb, b.snb, w.bmax, w.sb, w.b[0], w.b[1], w.b[2], Kp, Np,
                                          1.0, 0.0);
  return cudaGetLastError();
}

cudaError_t dense_split_a(const DenseA &a, int64_t K, int64_t M_max, int64_t N, void *ws, cudaStream_t s) {
  const int64_t Mp = (a.M + BM - 1) / BM * BM, Kp = (K + BK - 1) / BK * BK;
  DenseWs w = dense_ws_layout(ws, M_max, N, K);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>(Mp, (int64_t)sms * SPLIT_CTAS_PER_SM);
  if (a.alpha != 1.0 || a.beta != 0.0)
    split_rows<true><<<grid, 256, 0, s>>>(a.A, a.M, Mp, K, a.lda, a.ska, w.a[0], w.a[1], w.a[2], Kp, w.sa, a.alpha,
                                          a.beta);
  else
    split_rows<false><<<grid, 256, 0, s>>>(a.A, a.M, Mp, K, a.lda, a.ska, w.a[0], w.a[1], w.a[2], Kp, w.sa, 1.0, 0.0);
  return cudaGetLastError();
}

cudaError_t dense_split_gemm(const DenseA &a, int64_t N, int64_t K, int64_t M_max, double *C, int64_t ldc, void *ws,
                             bool lolo, int hdrain, int *status, long long wait_limit, cudaStream_t s) {
  const int64_t Mp = (a.M + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
  DenseWs w = dense_ws_layout(ws, M_max, N, K);
  cudaError_t e = cudaSuccess;
  if (hdrain < 1) hdrain = 1;
  if (hdrain > L_CHUNK) hdrain = L_CHUNK;
  CUtensorMap ma[NPART], mb[NPART];
  for (int q = 0; q < NPART; ++q)
    if (!make_map(&ma[q], w.a[q], Kp, Mp) || !make_map(&mb[q], w.b[q], Kp, Np)) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr{0};
  e = smem_limit_once((const void *)gemm_split_kernel, SMEM_BYTES, attr);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(Np / BN), (unsigned)(Mp / BM));
  gemm_split_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], w.sa, w.sb, C, a.M,
                                                       N, ldc, (int)(Kp / BK), lolo ? 1 : 0, hdrain, status,
                                                       wait_limit > 0 ? wait_limit : TIMEOUT_CYCLES);
  return cudaGetLastError();
}

DenseWs dense_ws_layout(void *ws, int64_t M_max, int64_t N, int64_t K) {
  const int64_t Mp = (M_max + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
  uint8_t *p = (uint8_t *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  DenseWs w;
  for (int q = 0; q < NPART; ++q) {
    w.a[q] = (__nv_bfloat16 *)p;
    p += Mp * Kp * 2;
  }
  for (int q = 0; q < NPART; ++q) {
    w.b[q] = (__nv_bfloat16 *)p;
    p += Np * Kp * 2;
  }
  w.sa = (int *)p;
  p += Mp * 4;
  w.sb = (int *)p;
  p += Np * 4;
  p = (uint8_t *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  w.bmax = (unsigned long long *)p;
  return w;
}

}  // namespace be

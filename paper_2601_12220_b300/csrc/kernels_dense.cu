// Dense split-precision strategy: an FP64 contraction that is a plain GEMM
// after flattening (e.g. the cluster-operator form 'abef,efij->abij' of the
// introduction, M = ab, K = ef, N = ij) evaluated on the tcgen05 tensor
// cores.
//
//  1. split_rows / split_cols: each FP64 operand (or its affine producer
//     alpha * x + beta, evaluated here) is scaled by a power of two
//     per row of A (per column of B) so that its largest entry lies in
//     [2^13, 2^14), then written as two TF32 parts hi = tf32(x),
//     lo = tf32(x - hi) (11 significant bits each) into a zero-padded
//     K-major workspace.  TF32 keeps FP32's exponent range, so entries far
//     below their row's maximum (the exp-decaying cluster amplitudes) keep
//     their relative precision; FP16 parts would fall into subnormals.
//  2. gemm_split_kernel: TMA streams 128 x 32 tiles of A_hi, A_lo, B_hi,
//     B_lo into shared memory (128-byte swizzle); one thread issues
//     tcgen05.mma kind::tf32 into FP32 accumulators in tensor memory: the
//     large term hi*hi into H, the small terms hi*lo + lo*hi (+ lo*lo when
//     requested) into L, each double-buffered (4 x 128 columns).  The
//     tensor core rounds its FP32 accumulator toward zero (about 2^-23 of
//     the accumulator per MMA, measured), so H is drained every hdrain
//     k-blocks of 32 values (2 by default: 64 values, 8 MMAs) and L every
//     512 values; sixteen epilogue warps read them
//     (tcgen05.ld) and add them into an FP32 pair per output with an
//     error-free two-sum (about 48 bits).  The result is scaled back and
//     stored in FP64.
//  Error per output, relative to S = sum |a||b|: split residuals 3 * 2^-22
//  (2 * 2^-22 with lo*lo), H truncation about 2^-23 per MMA between drains
//  (8 * 2^-23 at the default drain), L truncation below 2^-26.
// Every mbarrier wait is bounded (about one second of clock cycles); on
// expiry the CTA records BE_ETIMEOUT in a status word, stops issuing work,
// waits (bounded) for its own copies and frees its tensor memory.
#include <algorithm>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dense.hpp"
#include "launch_attr.hpp"
#include "tc_common.cuh"

namespace be {

namespace {

constexpr int BM = 128, BN = 128, BK = 32;           // BK: TF32 values per 128-byte row
constexpr int STAGES = 3;
constexpr int L_CHUNK = 16;                            // k-blocks per drain of the small-term accumulator
constexpr int TILE_BYTES = BM * BK * 4;                // one TF32 128 x 32 tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;            // A_hi, A_lo, B_hi, B_lo
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

// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
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

// error-free accumulation of v into the pair (hi, lo)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
  float s = hi + v;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (v - bp);
  hi = s;
  lo += err;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// drain 32 accumulator columns at taddr into the pairs (hi, lo)
__device__ __forceinline__ void drain32(uint32_t taddr, float *hi, float *lo) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float v[16];
    tmem_ld16(taddr + (uint32_t)(16 * q), v);
#pragma unroll
    for (int j = 0; j < 16; ++j) two_sum_acc(hi[16 * q + j], lo[16 * q + j], v[j]);
  }
}

__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_split_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                      const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
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
        tma_load_2d(st, &tmAh, &full[s], kb * BK, m0);
        tma_load_2d(st + TILE_BYTES, &tmAl, &full[s], kb * BK, m0);
        tma_load_2d(st + 2 * TILE_BYTES, &tmBh, &full[s], kb * BK, n0);
        tma_load_2d(st + 3 * TILE_BYTES, &tmBl, &full[s], kb * BK, n0);
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
#pragma unroll
        for (int ks = 0; ks < BK / 8; ++ks) {
          const uint64_t ah = sdesc(base + ks * 32), al = sdesc(base + TILE_BYTES + ks * 32);
          const uint64_t bh = sdesc(base + 2 * TILE_BYTES + ks * 32), bl = sdesc(base + 3 * TILE_BYTES + ks * 32);
          mma_tf32(dh, ah, bh, (hfirst && ks == 0) ? 0u : 1u);
          mma_tf32(dl, ah, bl, (lfirst && ks == 0) ? 0u : 1u);
          mma_tf32(dl, al, bh, 1u);
          if (lolo) mma_tf32(dl, al, bl, 1u);
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
        drain32(lane_base + (uint32_t)(hb * BN), hi, lo);
        tc_fence_before();
        mbar_arrive(&he[hb]);
      }
      if (llast) {
        const bool gl = mbar_wait(&lf[lb], (uint32_t)(lc >> 1) & 1u, abort_flag, status, limit);
        if (!__all_sync(0xffffffffu, gl)) { ok = false; break; }
        tc_fence_after();
        drain32(lane_base + (uint32_t)(2 * BN + lb * BN), hi, lo);
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
        if (n < N) crow[n] = scale2((double)hi[j] + (double)lo[j], -(sm + sb[n]));
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

// round a float to TF32 (11 significant bits, low 13 mantissa bits zero), nearest
__device__ __forceinline__ float to_tf32(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  return __uint_as_float(u);
}

// x (already scaled) = hi + lo + r with hi, lo TF32 and |r| <= 1.25 * 2^-22 |x|:
// one FP64 -> FP32 conversion (|x - xf| <= 2^-24 |x|), then hi = tf32(xf)
// and lo = tf32(xf - hi) in FP32 (that difference is exact)
__device__ __forceinline__ void split_one(double x, float &h, float &l) {
  const float xf = __double2float_rn(x);
  h = to_tf32(xf);
  l = to_tf32(xf - h);
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

// x * 2^s split into TF32 hi + lo; in FP32 from the bits when the scaled row
// stays in FP32's normal range, else through FP64
__device__ __forceinline__ void split_scaled(double x, int s, bool fp32_ok, float &h, float &l) {
  if (fp32_ok) {
    const float xf = scaled_float(x, s);
    h = to_tf32(xf);
    l = to_tf32(xf - h);
  } else {
    split_one(x * pow2(s), h, l);
  }
}

// the operand value of an affine producer, alpha * x + beta (AFF), else x
template <bool AFF>
__device__ __forceinline__ double affine(double x, double alpha, double beta) {
  return AFF ? fma(alpha, x, beta) : x;
}

// A (M x K): A[m*lda + k*ska] -> TF32 hi/lo [Mp x Kp], zero-padded; sa[m].
// Rows with unit stride and 16-byte alignment are read as double2, four in
// flight per thread, and written as float2.  AFF: the operand is
// alpha * A + beta (an affine producer fused into the split).
template <bool AFF>
__global__ void __launch_bounds__(256) split_rows(const double *__restrict__ A, int64_t M, int64_t K, int64_t lda,
                                                  int64_t ska, float *__restrict__ hi, float *__restrict__ lo,
                                                  int64_t Kp, int *__restrict__ sa, double alpha, double beta) {
  __shared__ double red[32];
  const int64_t m = blockIdx.x;
  const double *row = A + m * lda;
  const bool vec = ska == 1 && ((uintptr_t)row & 15) == 0 && (K & 1) == 0 && (Kp & 1) == 0;
  // |x| compared as integers on the sign-cleared high word (32-bit: a 64-bit
  // integer max issues on the FP64 pipe); the scale needs only the largest
  // exponent, which the high word carries
  uint32_t bits = 0;
  if (m < M) {
    if (vec) {
      const double2 *r2 = (const double2 *)row;
      const int64_t K2 = K >> 1;
      int64_t k = threadIdx.x;
      for (; k + 3 * blockDim.x < K2; k += 4 * blockDim.x) {
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = r2[k + u * blockDim.x];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          bits = max(bits, (uint32_t)__double2hiint(affine<AFF>(v[u].x, alpha, beta)) & 0x7fffffffu);
          bits = max(bits, (uint32_t)__double2hiint(affine<AFF>(v[u].y, alpha, beta)) & 0x7fffffffu);
        }
      }
      for (; k < K2; k += blockDim.x) {
        const double2 v = r2[k];
        bits = max(bits, (uint32_t)__double2hiint(affine<AFF>(v.x, alpha, beta)) & 0x7fffffffu);
        bits = max(bits, (uint32_t)__double2hiint(affine<AFF>(v.y, alpha, beta)) & 0x7fffffffu);
      }
    } else {
      for (int64_t k = threadIdx.x; k < K; k += blockDim.x)
        bits = max(bits, (uint32_t)__double2hiint(affine<AFF>(row[k * ska], alpha, beta)) & 0x7fffffffu);
    }
  }
  // the row maximum rounded down to its high word (same exponent, hence the
  // same power-of-two scale)
  double mx = block_max(__hiloint2double((int)bits, 0), red);
  const int s = scale_for(mx);
  // the scaled row max is below 2^14; FP32 scaling is exact while |x| >= 2^-100 * max
  const bool fp32_ok = mx == 0.0 || (mx > 0x1p-26 && mx < 0x1p+100 && s > -120 && s < 120);
  if (threadIdx.x == 0 && m < M) sa[m] = s;
  float *hrow = hi + m * Kp, *lrow = lo + m * Kp;
  if (vec && m < M) {
    const double2 *r2 = (const double2 *)row;
    float2 *h2 = (float2 *)hrow, *l2 = (float2 *)lrow;
    const int64_t K2 = K >> 1, Kp2 = Kp >> 1;
    int64_t k = threadIdx.x;
    for (; k + 3 * blockDim.x < K2; k += 4 * blockDim.x) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = r2[k + u * blockDim.x];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float ha, la, hb, lb;
        split_scaled(affine<AFF>(v[u].x, alpha, beta), s, fp32_ok, ha, la);
        split_scaled(affine<AFF>(v[u].y, alpha, beta), s, fp32_ok, hb, lb);
        h2[k + u * blockDim.x] = make_float2(ha, hb);
        l2[k + u * blockDim.x] = make_float2(la, lb);
      }
    }
    for (; k < Kp2; k += blockDim.x) {
      float ha = 0.f, la = 0.f, hb = 0.f, lb = 0.f;
      if (k < K2) {
        const double2 v = r2[k];
        split_scaled(affine<AFF>(v.x, alpha, beta), s, fp32_ok, ha, la);
        split_scaled(affine<AFF>(v.y, alpha, beta), s, fp32_ok, hb, lb);
      }
      h2[k] = make_float2(ha, hb);
      l2[k] = make_float2(la, lb);
    }
    return;
  }
  for (int64_t k = threadIdx.x; k < Kp; k += blockDim.x) {
    float h = 0.f, l = 0.f;
    if (m < M && k < K) split_scaled(affine<AFF>(row[k * ska], alpha, beta), s, fp32_ok, h, l);
    hrow[k] = h;
    lrow[k] = l;
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

// B (K x N) -> transposed TF32 hi/lo [Np x Kp] (K-major), zero-padded;
// AFF: the operand is alpha * B + beta
template <bool AFF>
__global__ void __launch_bounds__(256) split_cols_t(const double *__restrict__ B, int64_t K, int64_t N, int64_t ldb,
                                                   int64_t snb, const unsigned long long *__restrict__ bmax,
                                                   int *__restrict__ sb, float *__restrict__ hi,
                                                   float *__restrict__ lo, int64_t Kp, int64_t Np, double alpha,
                                                   double beta) {
  __shared__ double tile[32][33];
  const int64_t k0 = (int64_t)blockIdx.x * 32, nb = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int64_t nn = nb + tx;
  const int scl = nn < N ? scale_for(__longlong_as_double((long long)bmax[nn])) : 0;
  if (blockIdx.x == 0 && ty == 0 && nn < N) sb[nn] = scl;
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r;
    tile[r][tx] = (k < K && nn < N) ? ldexp(affine<AFF>(B[k * ldb + nn * snb], alpha, beta), scl) : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t n = nb + r, k = k0 + tx;
    if (n < Np && k < Kp) {
      float h, l;
      split_one(tile[tx][r], h, l);   // scaled by 2^sb[n] already
      hi[n * Kp + k] = h;
      lo[n * Kp + k] = l;
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
  cuuint64_t strides[1] = {(cuuint64_t)(inner * 4)};
  cuuint32_t box[2] = {BK, BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t dense_workspace_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t Mp = (M + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
  return (size_t)(Mp * Kp * 8 + Np * Kp * 8) + (size_t)(Mp + Np) * 4 + (size_t)Np * 8 + 2048;
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
    split_cols_t<true><<<g, 256, 0, s>>>(b.B, b.K, b.N, b.ldb, b.snb, w.bmax, w.sb, w.bh, w.bl, Kp, Np, b.alpha, b.beta);
  else
    split_cols_t<false><<<g, 256, 0, s>>>(b.B, b.K, b.N, b.ldb, b.snb, w.bmax, w.sb, w.bh, w.bl, Kp, Np, 1.0, 0.0);
  return cudaGetLastError();
}

cudaError_t dense_split_a(const DenseA &a, int64_t K, int64_t M_max, int64_t N, void *ws, cudaStream_t s) {
  const int64_t Mp = (a.M + BM - 1) / BM * BM, Kp = (K + BK - 1) / BK * BK;
  DenseWs w = dense_ws_layout(ws, M_max, N, K);
  if (a.alpha != 1.0 || a.beta != 0.0)
    split_rows<true><<<(unsigned)Mp, 256, 0, s>>>(a.A, a.M, K, a.lda, a.ska, w.ah, w.al, Kp, w.sa, a.alpha, a.beta);
  else
    split_rows<false><<<(unsigned)Mp, 256, 0, s>>>(a.A, a.M, K, a.lda, a.ska, w.ah, w.al, Kp, w.sa, 1.0, 0.0);
  return cudaGetLastError();
}

cudaError_t dense_split_gemm(const DenseA &a, int64_t N, int64_t K, int64_t M_max, double *C, int64_t ldc, void *ws,
                             bool lolo, int hdrain, int *status, long long wait_limit, cudaStream_t s) {
  const int64_t Mp = (a.M + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
  DenseWs w = dense_ws_layout(ws, M_max, N, K);
  cudaError_t e = cudaSuccess;
  if (hdrain < 1) hdrain = 1;
  if (hdrain > L_CHUNK) hdrain = L_CHUNK;
  CUtensorMap mah, mal, mbh, mbl;
  if (!make_map(&mah, w.ah, Kp, Mp) || !make_map(&mal, w.al, Kp, Mp) || !make_map(&mbh, w.bh, Kp, Np) ||
      !make_map(&mbl, w.bl, Kp, Np))
    return cudaErrorInvalidValue;
  static std::atomic<uint64_t> attr{0};
  e = smem_limit_once((const void *)gemm_split_kernel, SMEM_BYTES, attr);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(Np / BN), (unsigned)(Mp / BM));
  gemm_split_kernel<<<grid, NTHREADS, SMEM_BYTES, s>>>(mah, mal, mbh, mbl, w.sa, w.sb, C, a.M, N, ldc,
                                                       (int)(Kp / BK), lolo ? 1 : 0, hdrain, status,
                                                       wait_limit > 0 ? wait_limit : TIMEOUT_CYCLES);
  return cudaGetLastError();
}

DenseWs dense_ws_layout(void *ws, int64_t M_max, int64_t N, int64_t K) {
  const int64_t Mp = (M_max + BM - 1) / BM * BM, Np = (N + BN - 1) / BN * BN, Kp = (K + BK - 1) / BK * BK;
  uint8_t *p = (uint8_t *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  DenseWs w;
  w.ah = (float *)p;
  p += Mp * Kp * 4;
  w.al = (float *)p;
  p += Mp * Kp * 4;
  w.bh = (float *)p;
  p += Np * Kp * 4;
  w.bl = (float *)p;
  p += Np * Kp * 4;
  w.sa = (int *)p;
  p += Mp * 4;
  w.sb = (int *)p;
  p += Np * 4;
  p = (uint8_t *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
  w.bmax = (unsigned long long *)p;
  return w;
}

}  // namespace be

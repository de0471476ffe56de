// Element strategy on the tensor cores: the same batched einsums as
// element_kernel (R_k[e,i] = sum_{r,j} D[r,i,j] g_k[e,r] u[e,j], D shared by
// all elements, Sec. "Batched einsums in DG-FEM Operators"), with the hoisted
// contraction t[e,r,i] = sum_j D[r,i,j] u[e,j] evaluated as a GEMM on
// tcgen05 (M = 128 elements, N = (i, r) pairs, K = j) to FP64 accuracy by
// an error-free split of both operands into small integer digits:
//
//  * u[e, :] (one element, produced by the fused producer in double-float)
//    is scaled by 2^-k_e so that every |v_j| <= 1 and written as six
//    balanced base-512 digits, v = sum_q d_q 2^(-8-9q) with |d_q| <= 256;
//    each d_q 2^(-8-9q) is exact in bf16.  Each row n = (r, i) of D gets its
//    own 2^-k_n and digits c_p (D 2^-k_n = 2^-8 sum_p c_p 2^-9p, c_p 2^-9p
//    stored), from the FP64 bits once per CTA.
//  * sum_j D[n,j] u[e,j] = 2^(k_e + k_n - 8) sum_{p,q} sum_j (c_p 2^-9p)(d_q 2^(-8-9q)).
//    The digit products are grouped by level L = p + q.  Levels 0..3 each
//    accumulate in their own FP32 tensor-memory accumulator: every partial
//    sum is an integer multiple of 2^(-8-9L) below 2^24 times that (at most 4 pairs
//    x 64 terms x 2^16), so the tensor core adds them exactly.  Levels 4 and
//    5 share a fifth accumulator (its truncation stays below 2^-49 of
//    NJ max|u| max|D|); levels 6 and up are dropped (below 2^-50 of the same).
//  * The epilogue adds the five accumulators of each column in double-float,
//    applies the scales, contracts with g_k[e, :] in double-float and stores
//    FP64.
// Bound per output: |err| <= 2^-48 NJ max_j|u_j| sum_r |g_r| max_j|D_rij|
// plus double-float rounding (about 2^-46 of the absolute contraction S).
// The bound is normwise (the digits share one exponent per row): on dense
// data of moderate dynamic range it is far below 1e-12 S (about 2e-15 S on
// the DG workload), but for rows whose entries span many orders of
// magnitude it can exceed 1e-12 S; element_df_kernel is the componentwise
// path for such data.
//
// Warp roles (512 threads, one CTA per SM, persistent over tiles of 128
// elements):
//  * warps 0-6 produce the digit planes of u (two buffers, so that tile t+1
//    is produced while the MMAs of tile t run) in the 32-byte-swizzle
//    K-major layout, reading a and b with coalesced loads and prefetching
//    the next tile's rows into L2;
//  * warp 7 issues the MMAs (one thread) into three tensor-memory slots of
//    5 accumulators x 32 columns, one column block (two 16-column halves of
//    16 / R values of i with their R terms) per slot.  Every accumulator
//    starts on a 32-column boundary: with accumulators at 48-column offsets,
//    MMAs issued back to back into neighbouring accumulators gave wrong sums
//    on B300 (correct when the issue was slowed down);
//  * warps 8-15 drain a slot (two warps per TMEM lane quarter, one per half
//    of the block) while the next blocks accumulate, and write the outputs.
// D's digit planes are built once per CTA with integer arithmetic on the
// FP64 bits (no FP64 instruction).  Every wait is bounded: on expiry the
// CTA records BE_ETIMEOUT, stops issuing and frees its tensor memory after
// its MMAs complete.
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>

#include "df_math.cuh"
#include "exec.hpp"
#include "tc_common.cuh"

namespace be {

namespace {

using dfm::df;

constexpr int TC_M = 128;                       // elements per tile
constexpr int TC_P = 6;                         // digits per operand
constexpr int TC_LEV = 5;                       // accumulators per column block
constexpr int TC_NCOL = 32;                     // accumulator columns per level (32-column aligned)
constexpr int TC_SLOT = TC_LEV * TC_NCOL;       // 160 columns per slot
constexpr int TC_NSLOT = 3;                     // 480 of the 512 tensor-memory columns
constexpr int TC_KU = 8;                        // buffers of per-element row scales
constexpr int NPROD = 224, NEPI = 256;
constexpr int MMA_WARP = NPROD / 32;            // 7
constexpr int TC_THREADS = NPROD + 32 + NEPI;   // producer warps 0-6, MMA warp 7, epilogue warps 8-15
constexpr int TC_MAXROWS = 4;                   // einsums (rows) per launch
constexpr int TC_MAXNB = 160;                   // B rows (all column blocks)

// the 21 digit products (level, digit of D, digit of u) with level <= 5, in
// accumulator order: levels 0..3 alone, levels 4 and 5 into accumulator 4
struct TcParams {
  EParams p;
  int *status;
  int ncb, IB, NBtot, KS, NG;                   // column blocks, i per block, B rows, K steps, j groups of 8
  int ncol[8], n0[8];                           // per block: MMA N and first B row
};

// scale exponent k with |x| < 2^k for the largest |x| of a row, clamped so
// that the scaled values stay in FP32's normal range
__device__ __forceinline__ int row_exp(double mx) {
  const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7FF);
  if (ex == 0) return -100;
  return min(100, max(-100, ex - 1023 + 1));
}
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }   // |k| <= 126

// six digits of v = h + l (a double-float value, |v| <= 1): digit q is the
// remainder rounded to a multiple of 2^(-8-9q), at most 256 such multiples
// in magnitude and hence exact in bf16; v = sum_q r_q up to 2^-54.  The
// rounding adds and subtracts 1.5 * 2^23 times the grid, taking the digit
// off is exact (both are multiples of the remainder's last place), and the
// low part is folded in by Fast2Sum after each of the first four digits
// (valid since the remainder is zero or a multiple of that last place, at
// least twice |l|), which keeps every later digit within its bound
__device__ __forceinline__ void digits_df(float h, float l, float *r) {
  const float M[TC_P] = {0x1.8p+15f, 0x1.8p+6f, 0x1.8p-3f, 0x1.8p-12f, 0x1.8p-21f, 0x1.8p-30f};
#pragma unroll
  for (int q = 0; q < TC_P; ++q) {
    const float d = __fadd_rn(__fadd_rn(h, M[q]), -M[q]);
    r[q] = d;
    if (q + 1 < TC_P) h = __fadd_rn(h, -d);
    if (q < 4) {
      const float s = __fadd_rn(h, l);
      l = __fadd_rn(l, -__fadd_rn(s, -h));
      h = s;
    }
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // lo at the lower address
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Operand planes are K-major in the 32-byte-swizzle layout: for each slice
// of 16 values of K (one MMA K-step) the rows are 32 bytes long and packed,
// 8-row groups 256 bytes apart, slices rows * 32 bytes apart; within an
// 8-row group the two 16-byte halves of a row swap places when the row's
// bit 2 is set.  One MMA K-step thus reads one contiguous block.
// Byte offset of the 16-byte chunk g (values 8g .. 8g+7 of K) of row m in a
// plane of `rows` rows (256-byte aligned):
__device__ __forceinline__ uint32_t sw32(int rows, int m, int g) {
  return (uint32_t)((g >> 1) * rows * 32 + (m >> 3) * 256 + (m & 7) * 32 + (((g & 1) ^ ((m >> 2) & 1)) << 4));
}

// high word of a bound on |u| for the row scale (|sin a| <= 1); for a
// nonnegative double the high word orders like the value and carries its
// exponent, so the row maximum is an integer maximum
__device__ __forceinline__ int bound_hw(const EProd &q, int64_t e, int j) {
  if (q.kind == 1) return __double2hiint(q.b.ptr[e * q.b.se + j * q.b.sk]) & 0x7FFFFFFF;
  const double a = q.a.ptr[e * q.a.se + j * q.a.sk];
  if (q.kind == 0) return __double2hiint(a) & 0x7FFFFFFF;
  return __double2hiint(fabs(a) * fabs(q.b.ptr[e * q.b.se + j * q.b.sk]));
}

// operands (a, b) at j and j + 1 of pair pi of a tile (row m = pi / JP,
// j = 2 (pi mod JP)), from the tile's row pointers with 32-bit offsets;
// zeros past the row's end or the tile's last pair
struct TileRows {
  const double *a, *b;
  int sea, ska, seb, skb;
};
__device__ __forceinline__ void load_pair(const TileRows &t, bool need_b, int pi, int np, int JP, uint32_t jinv, int NJ,
                                          double *v) {
  const int m = pi < np ? (int)(((uint32_t)pi * jinv) >> 20) : 0, j = 2 * (pi - m * JP);
  const bool ok0 = pi < np, ok1 = ok0 && j + 1 < NJ;
  const int oa = m * t.sea + j * t.ska, ob = m * t.seb + j * t.skb;
  v[0] = ok0 ? t.a[oa] : 0.0;
  v[1] = ok1 ? t.a[oa + t.ska] : 0.0;
  v[2] = (ok0 && need_b) ? t.b[ob] : 0.0;
  v[3] = (ok1 && need_b) ? t.b[ob + t.skb] : 0.0;
}

// L2 prefetch of rows e1 .. e1+te1-1 (j = 0..NJ-1) of a view whose rows are
// contiguous; the range is shrunk to 16-byte boundaries inside it
__device__ __forceinline__ void prefetch_rows(const EView &v, int64_t e1, int te1, int NJ) {
  if (v.sk != 1 || te1 <= 0) return;
  const uintptr_t lo = (uintptr_t)(v.ptr + e1 * v.se);
  const uintptr_t hi = (uintptr_t)(v.ptr + (e1 + te1 - 1) * v.se + NJ);
  const uintptr_t a = (lo + 15) & ~(uintptr_t)15, b = hi & ~(uintptr_t)15;
  if (b <= a) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a)) : "memory");
}

// six balanced base-512 digits of x * 2^-k (|x| < 2^k), each times 2^-9q,
// by integer arithmetic on the bits of x: X = round(x * 2^(53 - k)) is split
// from the bottom, d = ((X + 256) mod 512) - 256, X = (X - d) / 512
__device__ __forceinline__ void digits_bits(double x, int k, float *d) {
  const long long b = __double_as_longlong(x);
  int ex = (int)((b >> 52) & 0x7FF);
  long long m = b & 0xFFFFFFFFFFFFFll;
  if (ex == 0) ex = 1;
  else m |= 1ll << 52;
  const int sh = 1022 + k - ex;                          // >= 0 since |x| < 2^k
  long long X = sh >= 63 ? 0 : (sh == 0 ? m : ((m >> (sh - 1)) + 1) >> 1);
  if (b < 0) X = -X;
#pragma unroll
  for (int q = TC_P - 1; q > 0; --q) {
    const long long dq = ((X + 256) & 511) - 256;
    X = (X - dq) >> 9;
    d[q] = (float)(int)dq * pow2f(-9 * q);
  }
  d[0] = (float)(int)X;
}

// the fused producer's value in double-float: a, a * b or sin(a) * b (the
// conversions stay off the FP64 pipe, which the epilogue's output sums use)
__device__ __forceinline__ df produce(const EProd &q, double a, double b, const float2 *sin_tab) {
  if (q.kind == 0) return dfm::df_from_double(a);
  if (q.kind == 2) return dfm::df_mul(dfm::df_from_double(a), dfm::df_from_double(b));
  return dfm::df_mul(dfm::df_sin_tab2(a, sin_tab), dfm::df_from_double(b));
}

// the producer without range tests or out-of-line calls, for operands that
// produce_fast_ok accepted: a batch whose operands all pass runs as one
// straight-line block (the tested variant's rare-case branches and calls
// split the block and cost about a fifth of the kernel's time)
template <bool FAST>
__device__ __forceinline__ df produce_t(const EProd &q, double a, double b, const float2 *sin_tab) {
  if (!FAST) return produce(q, a, b, sin_tab);
  if (q.kind == 0) return dfm::df_from_double_fast(a);
  if (q.kind == 2) return dfm::df_mul(dfm::df_from_double_fast(a), dfm::df_from_double_fast(b));
  return dfm::df_mul(dfm::df_sin_tab2_fast(a, sin_tab), dfm::df_from_double_fast(b));
}
__device__ __forceinline__ bool produce_fast_ok(const EProd &q, double a, double b) {
  if (q.kind == 0) return dfm::df_fast_ok(a);
  if (q.kind == 2) return dfm::df_fast_ok(a) && dfm::df_fast_ok(b);
  return dfm::sin_fast_ok(a) && dfm::df_fast_ok(b);
}

// named barrier of the producer warps, and the same barrier returning
// the AND of a predicate over them (so that all of them leave together)
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, 224;" ::: "memory"); }
__device__ __forceinline__ bool prod_all(bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, 224, q;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(r)
               : "r"((uint32_t)v)
               : "memory");
  return r != 0;
}

// Columns of a block: two halves of 16, each holding H0 = 16 / R values of
// i with their R terms (column = il * R + r) and zero padding after them, so
// that an epilogue thread's half never splits an i.  B row n -> (i, r).
template <int R>
__device__ __forceinline__ bool brow(const TcParams &tp, int n, int &i, int &r) {
  constexpr int H0 = 16 / R;
  int cb = 0;
  while (cb + 1 < tp.ncb && n >= tp.n0[cb + 1]) ++cb;
  const int c = n - tp.n0[cb], h = c >> 4, cc = c & 15;
  r = cc % R;
  const int il = cc / R;
  i = cb * 2 * H0 + h * H0 + il;
  return il < H0 && i < tp.p.NI;
}

// ROWS: the number of einsums when specialized, 0 for any count up to 4
template <int R, int ROWS>
__global__ void __launch_bounds__(TC_THREADS, 1) element_tc_kernel(const __grid_constant__ TcParams tp) {
  constexpr int H0 = 16 / R;                    // i per 16-column half of a block
  constexpr int KR = ROWS ? ROWS : TC_MAXROWS;  // einsums held per thread
  constexpr int IB = 2 * H0;                    // i per column block
  const EParams &p = tp.p;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *Bp = smem;                                       // TC_P planes x NBtot rows x 128 B
  const int bplane = tp.KS * tp.NBtot * 32;                 // bytes per digit plane of D
  const int aplane = tp.KS * TC_M * 32;                     // bytes per digit plane of u
  uint8_t *Ap = Bp + TC_P * bplane;                         // 2 buffers x TC_P planes x KS slices x 128 rows x 32 B
  float2 *sin_tab = (float2 *)(Ap + 2 * TC_P * aplane);     // full-circle sine table
  int *kD = (int *)(sin_tab + dfm::SIN2_N);                 // [TC_MAXNB]
  float *kDs = (float *)(kD + TC_MAXNB);                    // [TC_MAXNB] 2^kD
  // Row scales of u for the last TC_KU tiles: the epilogue can trail the
  // producer by up to 2 + ceil(3 / ncb) tiles (two digit buffers ahead of
  // the MMAs, which run at most three column blocks ahead of the epilogue)
  int *kU = (int *)(kDs + TC_MAXNB);                        // [TC_KU][TC_M]
  int *mxw = kU + TC_KU * TC_M;                             // [TC_M] high words of the row bounds
  uint64_t *bars = (uint64_t *)(mxw + TC_M);
  uint64_t *a_full = bars, *a_empty = bars + 2, *s_full = bars + 4, *s_empty = bars + 4 + TC_NSLOT;
  uint64_t *fin = bars + 4 + 2 * TC_NSLOT;
  uint32_t *tmem_slot = (uint32_t *)(fin + 1);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NJ = p.NJ, NI = p.NI;

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&a_full[b], NPROD);
      tc::mbar_init(&a_empty[b], 1);
    }
    for (int b = 0; b < TC_NSLOT; ++b) {
      tc::mbar_init(&s_full[b], 1);
      tc::mbar_init(&s_empty[b], NEPI);
    }
    tc::mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(tc::smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // zero both operand regions (K padding and padding rows stay zero)
  {
    uint4 *z = (uint4 *)smem;
    const int n16 = (TC_P * bplane + 2 * TC_P * aplane) / 16;
    for (int k = tid; k < n16; k += TC_THREADS) z[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  dfm::sin2_table_fill(sin_tab);
  // B row n -> (i, r); scale exponent per real row
  for (int n = tid; n < tp.NBtot; n += TC_THREADS) {
    int i, r;
    int hw = 0;
    if (brow<R>(tp, n, i, r))
      for (int j = 0; j < NJ; ++j) hw = max(hw, __double2hiint(p.D[r * p.sr + i * p.si + j * p.sj]) & 0x7FFFFFFF);
    kD[n] = row_exp(__hiloint2double(hw, 0));
    kDs[n] = pow2f(kD[n]);
  }
  __syncthreads();
  // digit planes of D: item (row n, group g of 8 values of j)
  for (int item = tid; item < tp.NBtot * tp.NG; item += TC_THREADS) {
    const int n = item / tp.NG, g = item % tp.NG;
    int i, r;
    if (!brow<R>(tp, n, i, r)) continue;
    const int kn = kD[n];
    uint32_t w[TC_P][4];
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) {
      float d0[TC_P], d1[TC_P];
      const int j = g * 8 + 2 * jp;
      digits_bits(j < NJ ? p.D[r * p.sr + i * p.si + j * p.sj] : 0.0, kn, d0);
      digits_bits(j + 1 < NJ ? p.D[r * p.sr + i * p.si + (j + 1) * p.sj] : 0.0, kn, d1);
#pragma unroll
      for (int q = 0; q < TC_P; ++q) w[q][jp] = pack_bf16(d0[q], d1[q]);
    }
#pragma unroll
    for (int q = 0; q < TC_P; ++q)
      *(uint4 *)(Bp + q * bplane + sw32(tp.NBtot, n, g)) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n_tiles = (p.E + TC_M - 1) / TC_M;
  int *status = tp.status;

  if (warp < MMA_WARP) {
    // ------------------------------------------------------------ producer
    // Two buffers of digit planes: tile t+1 is produced while the MMAs of
    // tile t run.  Pass 1 takes the largest |u| bound per element (the row
    // scale, one warp per row, lanes over j); pass 2 evaluates u in
    // double-float over pairs (j, j + 1) and writes its digits.  The next
    // tile's rows are prefetched into L2.
    const EProd &q = p.groups[0];
    int t = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
      const int64_t e0 = tile * TC_M;
      const int te = (int)(p.E - e0 < TC_M ? p.E - e0 : TC_M);
      if (tid == 0 && tile + gridDim.x < n_tiles) {
        const int64_t e1 = e0 + (int64_t)gridDim.x * TC_M;
        const int te1 = (int)(p.E - e1 < TC_M ? p.E - e1 : TC_M);
        prefetch_rows(q.a, e1, te1, NJ);
        if (q.kind != 0) prefetch_rows(q.b, e1, te1, NJ);
      }
      if (tid < TC_M) mxw[tid] = 0;
      prod_sync();
      constexpr int NPW = NPROD / 32;
      for (int r0 = warp; r0 < te; r0 += NPW * 4) {
        int hw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int row = r0 + NPW * u;
          const bool okr = row < te;
          const int h0 = (okr && lane < NJ) ? bound_hw(q, e0 + row, lane) : 0;
          const int h1 = (okr && lane + 32 < NJ) ? bound_hw(q, e0 + row, lane + 32) : 0;
          hw[u] = max(h0, h1);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int h = __reduce_max_sync(0xffffffffu, hw[u]);
          if (lane == 0 && r0 + NPW * u < te) mxw[r0 + NPW * u] = h;
        }
      }
      const int ab = t & 1;
      const uint32_t use = (uint32_t)(t >> 1);
      if (!prod_all(tc::mbar_wait(&a_empty[ab], (use & 1u) ^ 1u, abort_flag, status))) break;
      int *ku = kU + (t & (TC_KU - 1)) * TC_M;
      if (tid < TC_M) ku[tid] = row_exp(__hiloint2double(mxw[tid], 0));
      prod_sync();
      uint8_t *A = Ap + ab * TC_P * aplane;
      // pairs per row; g / JP as (g * jinv) >> 20, exact for g < 2^12, JP <= 32
      const int JP = (NJ + 1) >> 1, np = te * JP;
      const uint32_t jinv = ((1u << 20) + (uint32_t)JP - 1u) / (uint32_t)JP;
      const bool need_b = q.kind != 0;
      TileRows rows{q.a.ptr + e0 * q.a.se, need_b ? q.b.ptr + e0 * q.b.se : q.a.ptr, (int)q.a.se, (int)q.a.sk,
                    (int)q.b.se, (int)q.b.sk};
      // PB pairs per thread per batch (independent chains for the scheduler),
      // the next batch's loads issued before this batch is evaluated
      constexpr int PB = 3;
      double an[4 * PB];                                   // per pair: a0 a1 b0 b1
#pragma unroll
      for (int u = 0; u < PB; ++u) load_pair(rows, need_b, tid + u * NPROD, np, JP, jinv, NJ, an + 4 * u);
      for (int p0 = tid; p0 < np; p0 += PB * NPROD) {
        double av[4 * PB];
#pragma unroll
        for (int u = 0; u < 4 * PB; ++u) av[u] = an[u];
        if (p0 + PB * NPROD < np) {
#pragma unroll
          for (int u = 0; u < PB; ++u) load_pair(rows, need_b, p0 + (PB + u) * NPROD, np, JP, jinv, NJ, an + 4 * u);
        }
        auto batch = [&](auto fast) {
          constexpr bool F = decltype(fast)::value;
#pragma unroll
          for (int u = 0; u < PB; ++u) {
            const int pi = p0 + u * NPROD;
            if (pi < np) {
              const int m = (int)(((uint32_t)pi * jinv) >> 20), j = 2 * (pi - m * JP);
              const float sc = pow2f(-ku[m]);
              float d0[TC_P], d1[TC_P];
              const df u0 = produce_t<F>(q, av[4 * u], av[4 * u + 2], sin_tab);
              const df u1 = produce_t<F>(q, av[4 * u + 1], av[4 * u + 3], sin_tab);   // zero past NJ
              digits_df(u0.hi * sc, u0.lo * sc, d0);
              digits_df(u1.hi * sc, u1.lo * sc, d1);
              uint8_t *dst = A + sw32(TC_M, m, j >> 3) + (j & 7) * 2;
#pragma unroll
              for (int k = 0; k < TC_P; ++k) *(uint32_t *)(dst + k * aplane) = pack_bf16(d0[k], d1[k]);
            }
          }
        };
        bool fast = true;
#pragma unroll
        for (int u = 0; u < PB; ++u)
          fast = fast && produce_fast_ok(q, av[4 * u], av[4 * u + 2]) && produce_fast_ok(q, av[4 * u + 1], av[4 * u + 3]);
        if (fast) batch(std::true_type{});
        else batch(std::false_type{});
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(&a_full[ab]);
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t bbase = tc::smem_u32(Bp);
      const uint64_t adesc0 = tc::sdesc_sw32(tc::smem_u32(Ap));
      int t = 0;
      int64_t cnt = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++t) {
        const int ab = t & 1;
        if (!tc::mbar_wait(&a_full[ab], (uint32_t)(t >> 1) & 1u, abort_flag, status)) break;
        const uint64_t adesc = adesc0 + (uint64_t)((ab * TC_P * aplane) >> 4);
        tc::fence_after();
        for (int cb = 0; cb < tp.ncb; ++cb, ++cnt) {
          const int slot = (int)(cnt % TC_NSLOT);
          const uint32_t use = (uint32_t)(cnt / TC_NSLOT);
          if (!tc::mbar_wait(&s_empty[slot], (use & 1u) ^ 1u, abort_flag, status)) { ok = false; break; }
          tc::fence_after();
          const uint32_t idesc = tc::idesc_bf16(TC_M, tp.ncol[cb]);
          const uint32_t dslot = tmem + (uint32_t)(slot * TC_SLOT);
          // descriptors differ only in the start-address field (bits 0-13,
          // address >> 4), which stays below 2^14 for every operand here
          const uint64_t bblk = tc::sdesc_sw32(bbase + (uint32_t)(tp.n0[cb] * 32));
          // the 21 digit products with p + q <= 5 (p digit of D, q digit of
          // u): level L < 4 into accumulator L, levels 4 and 5 into
          // accumulator 4; the pair filter is resolved at compile time
#pragma unroll
          for (int L = 0; L < TC_LEV; ++L) {
#pragma unroll
            for (int pd = 0; pd < TC_P; ++pd) {
#pragma unroll
              for (int qd = 0; qd < TC_P; ++qd) {
                const int lev = pd + qd;
                if (L < TC_LEV - 1 ? lev != L : (lev < TC_LEV - 1 || lev > TC_LEV)) continue;
                const bool first = pd == 0 && qd == L;     // first pair of accumulator L
                const uint32_t d = dslot + (uint32_t)(L * TC_NCOL);
                const uint64_t da = adesc + (uint64_t)((qd * aplane) >> 4);
                const uint64_t db = bblk + (uint64_t)((pd * bplane) >> 4);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                  if (ks < tp.KS)
                    tc::mma_bf16(d, da + (uint64_t)(ks * (TC_M * 32 >> 4)), db + (uint64_t)(ks * (tp.NBtot * 32 >> 4)), idesc,
                                 (first && ks == 0) ? 0u : 1u);
              }
            }
          }
          tc::mma_commit(&s_full[slot]);
        }
        if (!ok) break;
        tc::mma_commit(&a_empty[ab]);   // this buffer of digit planes may be refilled once these MMAs are done
      }
      tc::mma_commit(fin);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(fin, 0) && clock64() - t0 < tc::TIMEOUT_CYCLES) {
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3, half = (warp - MMA_WARP - 1) >> 2;
    const int m = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * (TC_NCOL / 2));
    const int n_rows = p.n_rows;
    int t = 0;
    int64_t cnt = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++t) {
      const int64_t e = tile * TC_M + m;
      const bool valid = e < p.E;
      // g_k[e, r] of this thread's element as double-float (scaled by
      // 2^(k_e - 16) once the tile's exponents are known)
      df gk[KR][R];
#pragma unroll
      for (int k = 0; k < KR; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r)
          gk[k][r] = dfm::df_from_double(
              (valid && (ROWS || k < n_rows)) ? (p.has_g ? p.rows[k].g.ptr[e * p.rows[k].g.se + r * p.rows[k].g.sk] : 1.0) : 0.0);
      for (int cb = 0; cb < tp.ncb; ++cb, ++cnt) {
        const int slot = (int)(cnt % TC_NSLOT);
        const uint32_t use = (uint32_t)(cnt / TC_NSLOT);
        const bool got = tc::mbar_wait(&s_full[slot], use & 1u, abort_flag, status);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
        tc::fence_after();
        if (cb == 0) {
          const float sg = pow2f(kU[(t & (TC_KU - 1)) * TC_M + m] - 8);
#pragma unroll
          for (int k = 0; k < KR; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) gk[k][r] = df{gk[k][r].hi * sg, gk[k][r].lo * sg};
        }
        const int nI = min(IB, NI - cb * IB);
        const int nIh = max(0, min(H0, nI - half * H0));      // i of this half (warp-uniform)
        const int nch = (nIh * R + 7) >> 3;                      // 8-column chunks holding them
        // t for this half's columns: 5 accumulators per column added in
        // double-float, times 2^k_n of the column's row of D
        float th[16], tl[16];
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          if (ch < nch) {
            uint32_t v[TC_LEV][8];
            __syncwarp();   // tcgen05.ld is .sync.aligned: reconverge after lane-dependent work
#pragma unroll
            for (int L = 0; L < TC_LEV; ++L)
              tc::tmem_ld8(lane_base + (uint32_t)(slot * TC_SLOT + L * TC_NCOL + ch * 8), v[L]);
            tc::tmem_wait_ld();
            if (ch == nch - 1) {                               // this slot is drained
              tc::fence_before();
              tc::mbar_arrive(&s_empty[slot]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              if (ch * 8 + c >= H0 * R) continue;              // padding column of the half
              const df s01 = dfm::two_sum(__uint_as_float(v[0][c]), __uint_as_float(v[1][c]));
              df s23 = dfm::two_sum(__uint_as_float(v[2][c]), __uint_as_float(v[3][c]));
              s23.lo += __uint_as_float(v[4][c]);
              const df x = dfm::df_add(s01, s23);
              const float sc = kDs[min(tp.n0[cb] + half * 16 + ch * 8 + c, tp.NBtot - 1)];
              th[ch * 8 + c] = x.hi * sc;
              tl[ch * 8 + c] = x.lo * sc;
            }
          }
        }
        if (valid) {
#pragma unroll
          for (int il = 0; il < H0; ++il) {
            if (il < nIh) {
              const int i = cb * IB + half * H0 + il;
#pragma unroll
              for (int k = 0; k < KR; ++k) {
                if (ROWS || k < n_rows) {
                  // first term: its exact product starts the pair (s, c)
                  const df g0 = gk[k][0], t0{th[il * R], tl[il * R]};
                  float s = g0.hi * t0.hi;
                  float c = fmaf(g0.hi, t0.lo, fmaf(g0.lo, t0.hi, fmaf(g0.hi, t0.hi, -s)));
#pragma unroll
                  for (int r = 1; r < R; ++r) dfm::dot_acc(s, c, gk[k][r], df{th[il * R + r], tl[il * R + r]});
                  // hi + lo on the FP64 pipe: 3 instructions
                  p.rows[k].out[e * NI + i] = (double)s + (double)c;
                }
              }
            }
          }
        }
        if (nch == 0) {
          tc::fence_before();
          tc::mbar_arrive(&s_empty[slot]);
        }
      }
    }
  }

  // teardown: every MMA of this CTA has completed (fin) before the tensor
  // memory is released
  tc::fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    __syncwarp();   // lane 0 ran the issue loop alone
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

bool build_params(const EParams &p, TcParams &tp, std::string &why) {
  if (p.n_groups != 1) { why = "more than one fused operand"; return false; }
  if (p.NJ0 > 0 || p.groups[0].kind == 3) { why = "stacked producer (divergence / face-mass form)"; return false; }
  if (p.R < 1 || p.R > 4) { why = "R outside 1..4"; return false; }
  if (p.NJ < 1 || p.NJ > 64) { why = "contracted extent outside 1..64"; return false; }
  if (p.NI < 1) { why = "empty output extent"; return false; }
  if (p.n_rows < 1 || p.n_rows > TC_MAXROWS) { why = "more than 4 einsums"; return false; }
  if (!p.has_g && p.R != 1) { why = "no geometric factor with R > 1"; return false; }
  {
    const EProd &q = p.groups[0];
    const int64_t lim = (int64_t)1 << 23;   // in-tile offsets m * se + j * sk stay 32-bit
    if (std::abs(q.a.se) >= lim || std::abs(q.a.sk) >= lim || std::abs(q.b.se) >= lim || std::abs(q.b.sk) >= lim) {
      why = "operand strides too large";
      return false;
    }
  }
  tp.p = p;
  const int h0 = 16 / p.R;
  tp.IB = 2 * h0;
  tp.ncb = (p.NI + tp.IB - 1) / tp.IB;
  if (tp.ncb > 8) { why = "too many column blocks"; return false; }
  int nb = 0;
  for (int cb = 0; cb < tp.ncb; ++cb) {
    const int nI = std::min(tp.IB, p.NI - cb * tp.IB);
    tp.n0[cb] = nb;
    tp.ncol[cb] = nI <= h0 ? 16 : 32;                    // one or two 16-column halves
    nb += tp.ncol[cb];
  }
  if (nb > TC_MAXNB) { why = "R * NI too large for the shared D planes"; return false; }
  tp.NBtot = nb;
  tp.KS = (p.NJ + 15) / 16;
  tp.NG = (p.NJ + 7) / 8;
  return true;
}

size_t smem_bytes(const TcParams &tp) {
  return 1024 + (size_t)TC_P * tp.KS * tp.NBtot * 32 + 2 * (size_t)TC_P * tp.KS * TC_M * 32 +
         sizeof(float2) * dfm::SIN2_N + sizeof(int) * (2 * TC_MAXNB + (TC_KU + 1) * TC_M) + 8 * (5 + 2 * TC_NSLOT) + 16;
}

template <int R, int ROWS>
cudaError_t launch_rr(const TcParams &tp, int grid, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t st =
        cudaFuncSetAttribute(element_tc_kernel<R, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (st != cudaSuccess) return st;
    attr = true;
  }
  element_tc_kernel<R, ROWS><<<grid, TC_THREADS, smem, s>>>(tp);
  return cudaGetLastError();
}
// one einsum per term direction (R einsums, as in a gradient) is
// specialized; other counts take the generic row loop
template <int R>
cudaError_t launch_r(const TcParams &tp, int grid, size_t smem, cudaStream_t s) {
  return tp.p.n_rows == R ? launch_rr<R, R>(tp, grid, smem, s) : launch_rr<R, 0>(tp, grid, smem, s);
}

}  // namespace

bool element_tc_supported(const EParams &p, std::string &why) {
  TcParams tp;
  if (!build_params(p, tp, why)) return false;
  if (smem_bytes(tp) > 227 * 1024) { why = "shared memory"; return false; }
  return true;
}

cudaError_t launch_element_tc(const EParams &p, int *status, cudaStream_t s) {
  TcParams tp;
  std::string why;
  if (!build_params(p, tp, why)) return cudaErrorInvalidValue;
  tp.status = status;
  const size_t smem = smem_bytes(tp);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (p.E <= 0) return cudaSuccess;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (p.E + TC_M - 1) / TC_M;
  const int grid = (int)std::min<int64_t>(tiles, sms);
  switch (p.R) {
    case 1: return launch_r<1>(tp, grid, smem, s);
    case 2: return launch_r<2>(tp, grid, smem, s);
    case 3: return launch_r<3>(tp, grid, smem, s);
    default: return launch_r<4>(tp, grid, smem, s);
  }
}

}  // namespace be

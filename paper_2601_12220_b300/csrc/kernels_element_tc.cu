// Element strategy on the tensor cores: the same batched einsums as
// element_kernel (R_k[e,i] = sum_{r,j} D[r,i,j] g_k[e,r] u[e,j], D shared by
// all elements, Sec. "Batched einsums in DG-FEM Operators"), with the hoisted
// contraction t[e,r,i] = sum_j D[r,i,j] u[e,j] evaluated as a GEMM on
// tcgen05 (M = 128 elements, N = (i, r) columns, K = j) to FP64 accuracy by
// an error-free split of both operands into small integer digits, and a
// per-output check that sends the rare output it cannot certify to an FP64
// recomputation, so that every result is within 1e-12 of the absolute
// contraction S = sum |D| |g| |u| of Eq. (1).
//
//  * u[e, :] (one element, produced by the fused producer in double-float)
//    is scaled by 2^-k_e so that every |v_j| <= 1 and written as six
//    balanced base-512 digits, v = sum_q d_q 2^(-8-9q) with |d_q| <= 256;
//    each d_q 2^(-8-9q) is exact in bf16.  Each row n = (r, i) of D gets its
//    own 2^-k_n and digits c_p (D 2^-k_n = 2^-8 sum_p c_p 2^-9p, c_p 2^-9p
//    stored), from the FP64 bits once per CTA.
//  * sum_j D[n,j] u[e,j] = 2^(k_e + k_n - 8) sum_{p,q} sum_j (c_p 2^-9p)(d_q 2^(-8-9q)).
//    The digit products are grouped by level L = p + q <= 6, one FP32
//    accumulator in tensor memory per level.  Levels 0..3 are exact (every
//    partial sum is an integer multiple of 2^(-8-9L) below 2^24 of that
//    unit: at most 4 pairs x 64 terms x 2^16), levels 4..6 are exact up to
//    K = 42 and nearly so beyond; levels 7 and up are dropped (below
//    2^-52 K of the scale).
//  * Stacked issue: the six planes of D's digits of a column block are
//    contiguous in shared memory, so one MMA with A = u's digit q and
//    B = planes p = 0..P adds d_q c_p into the accumulators of levels
//    q .. q + P at once (its N is (P + 1) x 32 columns, the accumulators of
//    a block sit 32 columns apart).  A block takes 6 MMAs per K-slice of 16
//    (plus one that starts the level-6 accumulator) instead of one per pair.
//  * The epilogue adds the seven accumulators of each column in
//    double-float, applies the scales, contracts with g_k[e, :] in
//    double-float and stores FP64.
//
// Error and the check.  With every level exact, what remains is the
// representation of the operands by six digits (2^-54 of the scale per
// factor), the dropped levels and the double-float roundings: per column,
// |t - t~| <= 2^(k_e+k_n-8) E_n with E_n = 2^-46 (sum_j |D_nj| 2^-k_n + K)
// + 2^-42, plus relative roundings far below 1e-12.  Since
// S >= sum_r |g_r| |t_r|, an output is certified when
//     sum_r |g_r| (F E_n(r) 2^(k_e + k_n - 8) - |t~_r|) <= 0,
// F = (1e-12 - 2^-43)^-1 with margins; the epilogue evaluates this sum for
// every output.  On dense data of moderate range practically every output
// passes (the margin is a factor of about 100 on N(0,1) data).  An element
// with an output that fails, or whose scales leave the window |k| <= 24
// where double-float keeps full precision, is recomputed in FP64 by the
// epilogue warps at the end of its tile (one thread per u_j, per t_ri and
// per output).  Elements that are all zero are exact and never flagged.
//
// Warp roles (512 threads, one CTA per SM, persistent over tiles of 128
// elements):
//  * warps 0-6 produce the digit planes of u (two buffers, so that tile t+1
//    is produced while the MMAs of tile t run) in the 32-byte-swizzle
//    K-major layout, reading a and b with coalesced loads and prefetching
//    the next tile's rows into L2;
//  * warp 7 issues the MMAs (one thread) into two tensor-memory slots of
//    7 accumulators x 32 columns (every accumulator on a 32-column
//    boundary), one column block (two 16-column halves of 16 / R values of
//    i with their R terms) per slot;
//  * warps 8-15 drain a slot (two warps per TMEM lane quarter, one per half
//    of the block) while the next block accumulates, write the outputs and
//    run the per-output check.
// Every wait is bounded (a limit in SM cycles that the caller may lower):
// on expiry the CTA records BE_ETIMEOUT, every role leaves its loop
// collectively, and the tensor memory is freed only after all issued MMAs
// have completed.
//
// The stacked form (the divergence and the face mass: R[e,i] = sum_k
// D[i,k] v[e,k], v = sum_x A_x B_x over the flat k = (s, j), K <= 64) is a
// second instantiation: the producer forms v in double-float with a scale
// from an exponent bound, tiles run over producer groups x element tiles,
// and an eighth accumulator per slot sums bf16(|D|) x bf16(|v|), a lower
// bound of S for the per-output check (with R = 1, |t| alone is a weak one).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <type_traits>

#include <cuda_bf16.h>

#include "df_math.cuh"
#include "exec.hpp"
#include "launch_attr.hpp"
#include "tc_common.cuh"
#include "launch_rec.hpp"

namespace be {

namespace {

using dfm::df;

constexpr int TC_M = 128;                       // elements per tile
constexpr int TC_P = 6;                         // digits per operand
constexpr int TC_LEV = 7;                       // levels 0..6, one accumulator each
constexpr int TC_NCOL = 32;                     // columns of a block (and of an accumulator)
constexpr int TC_SLOT = TC_LEV * TC_NCOL;       // 224 columns per slot, two slots (448 of the 512 tensor-memory columns; 512 in the stacked form)
constexpr int TC_KU = 4;                        // buffers of per-element row scales
constexpr int NPROD = 224, NEPI = 256;
constexpr int MMA_WARP = NPROD / 32;            // 7
constexpr int TC_THREADS = NPROD + 32 + NEPI;   // producer warps 0-6, MMA warp 7, epilogue warps 8-15
constexpr int TC_MAXROWS = 4;                   // einsums (rows) per launch
constexpr int TC_MAXCB = 8;                     // column blocks
constexpr int TC_BPLANE = TC_NCOL * 32;         // bytes of one digit plane of a block and K-slice
constexpr int KU_ZERO = -126;                   // row-scale code of an element that is all zero
constexpr int TC_WIN = 24;                      // scale window |k| <= TC_WIN of the certified path
constexpr size_t TC_SMEM_LIMIT = 227 * 1024;

struct TcParams {
  EParams p;
  int *status;
  long long wait_limit;                         // SM cycles before a wait gives up
  int ncb, IB, KS, NG, NB;                      // column blocks, i per block, K-slices of 16, j groups of 8, B rows
  int G;                                        // producer groups; tiles run over G x element tiles
  int nbuf;                                     // buffers of u's digit planes: 2, or 1 where two do not fit
  int npl;                                      // planes per operand: the six digits (+ |v|, |D| in the stacked form)
  double fcheck;                                // F of the per-output check (margins included)
  int8_t gstart[EM_MAXROWS + 1];                // rows of group g: grow[gstart[g] .. gstart[g + 1])
  int8_t grow[EM_MAXROWS];
};

// byte offsets of the shared-memory regions (from a 256-byte aligned base)
struct TcSmem {
  uint32_t b, a, sin, kD, kDs, zc, kU, mxw, fm, fu, ft, bars, misc, total;
};
__host__ __device__ inline TcSmem tc_smem(const TcParams &tp) {
  TcSmem s;
  uint32_t o = 0;
  s.b = o;    o += (uint32_t)(tp.ncb * tp.KS * tp.npl * TC_BPLANE);
  s.a = o;    o += (uint32_t)(tp.nbuf * tp.npl * tp.KS * TC_M * 32);
  s.sin = o;  o += (uint32_t)(sizeof(float2) * dfm::SINH_N);
  s.kD = o;   o += 4u * tp.NB;
  s.kDs = o;  o += 4u * tp.NB;
  s.zc = o;   o += 4u * tp.NB;
  s.kU = o;   o += 4u * TC_KU * TC_M;
  s.mxw = o;  o += 4u * TC_M;
  s.fm = o;   o += 4u * 8;                      // two 128-bit masks of flagged elements
  s.fu = o;   o += 8u * (uint32_t)((tp.p.NJ + 1) & ~1);
  s.ft = o;   o += 8u * (uint32_t)(tp.p.R * tp.p.NI);
  s.bars = o; o += 8u * 9;
  s.misc = o; o += 16;
  s.total = o;
  return s;
}

// scale exponent k with |x| < 2^k for a row maximum given by the high word
// of its FP64 bits, clamped to [-100, 100] (the scaled values stay in
// FP32's normal range)
__device__ __forceinline__ int row_exp_hw(int hw) {
  const int ex = (hw >> 20) & 0x7FF;
  if (ex == 0) return -100;
  return min(100, max(-100, ex - 1022));
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
// 8-row groups 256 bytes apart; within an 8-row group the two 16-byte halves
// of a row swap places when the row's bit 2 is set.  Byte offset of the
// 16-byte chunk h (values 8h .. 8h+7 of the slice) of row m:
__device__ __forceinline__ uint32_t sw32_row(int m, int h) {
  return (uint32_t)((m >> 3) * 256 + (m & 7) * 32 + (((h & 1) ^ ((m >> 2) & 1)) << 4));
}
// u's planes: plane q holds KS slices of 128 rows; chunk g of row m
__device__ __forceinline__ uint32_t sw32(int rows, int m, int g) {
  return (uint32_t)((g >> 1) * rows * 32) + sw32_row(m, g);
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

// L2 prefetch of the geometric factors g_k[e, r] of elements e1 .. e1+te1-1
// (every row k, every r) when they span at most 64 KB (for the gradient's
// G[e, r, x] the 128 elements' 9 values are one contiguous 9 KB range)
__device__ __forceinline__ void prefetch_g(const EParams &p, int64_t e1, int te1) {
  if (te1 <= 0) return;
  uintptr_t lo = ~(uintptr_t)0, hi = 0;
  for (int k = 0; k < p.n_rows; ++k) {
    const EView &g = p.rows[k].g;
    for (int r = 0; r < p.R; r += max(1, p.R - 1))
      for (int64_t e : {e1, e1 + te1 - 1}) {
        const uintptr_t a = (uintptr_t)(g.ptr + e * g.se + r * g.sk);
        lo = min(lo, a);
        hi = max(hi, a + 8);
      }
  }
  const uintptr_t a = (lo + 15) & ~(uintptr_t)15, b = hi & ~(uintptr_t)15;
  if (b <= a || b - a > 65536) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a)) : "memory");
}

// six balanced base-512 digits of x * 2^-k (|x| < 2^k), each times 2^-9q,
// by integer arithmetic on the bits of x: X = round(x * 2^(53 - k)) is split
// from the bottom, d = ((X + 256) mod 512) - 256, X = (X - d) / 512.  A value
// at or above 2^k (possible only in a row whose scale was clamped; such rows
// never reach a certified output) gives digits of zero.
__device__ __forceinline__ void digits_bits(double x, int k, float *d) {
  const long long b = __double_as_longlong(x);
  int ex = (int)((b >> 52) & 0x7FF);
  long long m = b & 0xFFFFFFFFFFFFFll;
  if (ex == 0) ex = 1;
  else m |= 1ll << 52;
  const int sh = 1022 + k - ex;
  long long X = (sh >= 63 || sh < 0) ? 0 : (sh == 0 ? m : ((m >> (sh - 1)) + 1) >> 1);
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
// conversions stay off the FP64 pipe, which the output sums use); out of
// line, since only batches with an operand outside the fast range take it
static __device__ __noinline__ df produce(const EProd &q, double a, double b, const float2 *sin_tab) {
  if (q.kind == 0) return dfm::df_from_double(a);
  if (q.kind == 2) return dfm::df_mul(dfm::df_from_double(a), dfm::df_from_double(b));
  return dfm::df_mul(dfm::df_sin_half(a, sin_tab), dfm::df_from_double(b));
}

// the producer without range tests or out-of-line calls, for operands that
// produce_fast_ok accepted: a batch whose operands all pass runs as one
// straight-line block
template <bool FAST>
__device__ __forceinline__ df produce_t(const EProd &q, double a, double b, const float2 *sin_tab) {
  if (!FAST) return produce(q, a, b, sin_tab);
  if (q.kind == 0) return dfm::df_from_double_fast(a);
  if (q.kind == 2) return dfm::df_mul(dfm::df_from_double_fast(a), dfm::df_from_double_fast(b));
  return dfm::df_mul(dfm::df_sin_half_fast(a, sin_tab), dfm::df_from_double_fast(b));
}
__device__ __forceinline__ bool produce_fast_ok(const EProd &q, double a, double b) {
  if (q.kind == 0) return dfm::df_fast_ok(a);
  if (q.kind == 2) return dfm::df_fast_ok(a) && dfm::df_fast_ok(b);
  return dfm::sin_fast_ok(a) && dfm::df_fast_ok(b);
}

// digits of the pair (u0, u1) = u[e, j], u[e, j + 1] of pair pi of a tile,
// scaled by the element's row scale, into the six digit planes of u
__device__ __forceinline__ void pair_digits(df u0, df u1, int pi, int JP, uint32_t jinv, const int *ku, uint8_t *A,
                                            int aplane) {
  const int m = (int)(((uint32_t)pi * jinv) >> 20), j = 2 * (pi - m * JP);
  const float sc = pow2f(-ku[m]);
  float d0[TC_P], d1[TC_P];
  digits_df(u0.hi * sc, u0.lo * sc, d0);
  digits_df(u1.hi * sc, u1.lo * sc, d1);
  uint8_t *dst = A + sw32(TC_M, m, j >> 3) + (j & 7) * 2;
#pragma unroll
  for (int k = 0; k < TC_P; ++k) *(uint32_t *)(dst + k * aplane) = pack_bf16(d0[k], d1[k]);
}

// a producer batch with an operand outside the fast range: the operands are
// read again and every value takes the tested producer; out of line, so
// that the hot loop's code stays small
static __device__ __noinline__ void pairs_slow(const EProd &q, TileRows rows, bool need_b, int p0, int pb, int stride,
                                               int np, int JP, uint32_t jinv, int NJ, const int *ku, uint8_t *A,
                                               int aplane, const float2 *sin_tab) {
  for (int u = 0; u < pb; ++u) {
    const int pi = p0 + u * stride;
    if (pi >= np) break;
    double v[4];
    load_pair(rows, need_b, pi, np, JP, jinv, NJ, v);
    pair_digits(produce(q, v[0], v[2], sin_tab), produce(q, v[1], v[3], sin_tab), pi, JP, jinv, ku, A, aplane);
  }
}

// Stacked producer (divergence / face-mass form): v[e, k] = sum_x
// A_x[e, s, j] B_x[e, s, j] at the flat index k = s NJ0 + j; s = k / NJ0 as
// (k * sinv) >> 20 with sinv = ceil(2^20 / NJ0), exact for k, NJ0 <= 64.
__device__ __forceinline__ int64_t stk_off(const ESView &v, int64_t e, int s, int j) {
  return e * v.se + (int64_t)s * v.ss + (int64_t)j * v.sj;
}
// exponent bound at (e, k): the largest ex(A_x) + ex(B_x) over the x whose
// product is nonzero, ex the biased exponent field (at least 1), so that
// |A_x B_x| < 2^(ex(A_x) + ex(B_x) - 2044); 0 when every product is zero
template <int X>
__device__ __forceinline__ int stk_bound(const EProd &q, int64_t e, int k, int NJ, int NJ0, uint32_t sinv) {
  const int s = (int)(((uint32_t)k * sinv) >> 20), j = k - s * NJ0;
  int h = 0;
#pragma unroll
  for (int x = 0; x < X; ++x) {
    const long long a = k < NJ ? __double_as_longlong(q.A[x].ptr[stk_off(q.A[x], e, s, j)]) & 0x7FFFFFFFFFFFFFFFll : 0;
    const long long b = k < NJ ? __double_as_longlong(q.B[x].ptr[stk_off(q.B[x], e, s, j)]) & 0x7FFFFFFFFFFFFFFFll : 0;
    if (a != 0 && b != 0) h = max(h, max(1, (int)(a >> 52)) + max(1, (int)(b >> 52)));
  }
  return h;
}
// the same sum for operands outside the fast conversion range (the tested
// conversion); out of line
static __device__ __noinline__ df stk_slow(const EProd &q, int64_t e, int s, int j) {
  float sh = 0.f, sl = 0.f;
  for (int x = 0; x < q.X; ++x)
    dfm::dot_acc(sh, sl, dfm::df_from_double(q.A[x].ptr[stk_off(q.A[x], e, s, j)]),
                 dfm::df_from_double(q.B[x].ptr[stk_off(q.B[x], e, s, j)]));
  return dfm::two_sum(sh, sl);
}
// operands of v[e, k] (zeros past the row's end) and v in double-float
// (products and their sum through TwoSum, as the double-float element
// kernel forms it); the loads of a batch are issued before any of its
// arithmetic
template <int X>
__device__ __forceinline__ void stk_load(const EProd &q, int64_t e, int k, int NJ0, int NJ, uint32_t sinv, double *a,
                                         double *b) {
  const int s = (int)(((uint32_t)k * sinv) >> 20), j = k - s * NJ0;
#pragma unroll
  for (int x = 0; x < X; ++x) {
    a[x] = k < NJ ? q.A[x].ptr[stk_off(q.A[x], e, s, j)] : 0.0;
    b[x] = k < NJ ? q.B[x].ptr[stk_off(q.B[x], e, s, j)] : 0.0;
  }
}
template <int X>
__device__ __forceinline__ df stk_eval(const EProd &q, int64_t e, int k, int NJ0, uint32_t sinv, const double *a,
                                       const double *b) {
  bool ok = true;
#pragma unroll
  for (int x = 0; x < X; ++x) ok = ok && dfm::df_fast_ok(a[x]) && dfm::df_fast_ok(b[x]);
  if (!ok) {
    const int s = (int)(((uint32_t)k * sinv) >> 20);
    return stk_slow(q, e, s, k - s * NJ0);
  }
  float sh = 0.f, sl = 0.f;
#pragma unroll
  for (int x = 0; x < X; ++x) dfm::dot_acc(sh, sl, dfm::df_from_double_fast(a[x]), dfm::df_from_double_fast(b[x]));
  return dfm::two_sum(sh, sl);
}

// L2 prefetch of the stacked operands of elements e1 .. e1+te1-1: per view
// and value of s, the span between the corners (e1 or the last element, j
// = 0 or NJ0 - 1) when it is at most 64 KB; lane l of the calling warp
// takes (x, operand, s) = l
__device__ __forceinline__ void stk_prefetch(const EProd &q, int64_t e1, int te1, int S, int NJ0, int lane) {
  if (te1 <= 0 || lane >= q.X * 2 * S) return;
  const int x = lane / (2 * S), w = (lane / S) & 1, sv = lane % S;
  const ESView &v = w ? q.B[x] : q.A[x];
  if (v.ss == 0 && sv > 0) return;                      // the same span for every s
  uintptr_t lo = ~(uintptr_t)0, hi = 0;
  for (int64_t e : {e1, e1 + te1 - 1})
    for (int j : {0, NJ0 - 1}) {
      const uintptr_t a = (uintptr_t)(v.ptr + stk_off(v, e, sv, j));
      lo = min(lo, a);
      hi = max(hi, a + 8);
    }
  const uintptr_t a = (lo + 15) & ~(uintptr_t)15, b = hi & ~(uintptr_t)15;
  if (b <= a || b - a > 65536) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(b - a)) : "memory");
}

// pass 1 of the stacked producer: the exponent bound of sum_x |A_x B_x| per
// element into mxw, over the flat items (element, k) of the tile, IB items
// per thread with their loads issued together (item / K as a multiply by
// kinv = ceil(2^20 / K), exact below 2^13 items), the maxima by shared-memory
// atomics
template <int X>
__device__ __forceinline__ void stk_rows_bound(const EProd &q, int64_t e0, int te, int NJ, int NJ0, uint32_t sinv,
                                               int tid, int *mxw) {
  constexpr int IB = X == 1 ? 16 : 8;
  const int n = te * NJ;
  const uint32_t kinv = ((1u << 20) + (uint32_t)NJ - 1u) / (uint32_t)NJ;
  for (int i0 = tid; i0 < n; i0 += IB * NPROD) {
    int h[IB], row[IB];
#pragma unroll
    for (int u = 0; u < IB; ++u) {
      const int it = i0 + u * NPROD;
      row[u] = it < n ? (int)(((uint32_t)it * kinv) >> 20) : 0;
      h[u] = stk_bound<X>(q, e0 + row[u], it < n ? it - row[u] * NJ : NJ, NJ, NJ0, sinv);
    }
#pragma unroll
    for (int u = 0; u < IB; ++u)
      if (h[u] > 0) atomicMax(&mxw[row[u]], h[u]);
  }
}

// pass 2: v over pairs (k, k + 1), PB pairs per thread with their loads
// issued first, written as u's six digit planes and the plane of
// bf16(|v| 2^-k_e)
template <int X>
__device__ __forceinline__ void stk_pairs(const EProd &q, int64_t e0, int np, int JP, uint32_t jinv, int NJ, int NJ0,
                                          uint32_t sinv, const int *ku, uint8_t *A, int aplane, int tid) {
  constexpr int PB = X == 1 ? 4 : 2;
  for (int p0 = tid; p0 < np; p0 += PB * NPROD) {
    double a[PB][2][X], b[PB][2][X];
    int mm[PB], kk[PB];
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int pi = p0 + u * NPROD;
      mm[u] = pi < np ? (int)(((uint32_t)pi * jinv) >> 20) : 0;
      kk[u] = pi < np ? 2 * (pi - mm[u] * JP) : NJ;
      stk_load<X>(q, e0 + mm[u], kk[u], NJ0, NJ, sinv, a[u][0], b[u][0]);
      stk_load<X>(q, e0 + mm[u], kk[u] + 1, NJ0, NJ, sinv, a[u][1], b[u][1]);
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      const int pi = p0 + u * NPROD;
      if (pi >= np) continue;
      const df v0 = stk_eval<X>(q, e0 + mm[u], kk[u], NJ0, sinv, a[u][0], b[u][0]);
      const df v1 = stk_eval<X>(q, e0 + mm[u], kk[u] + 1, NJ0, sinv, a[u][1], b[u][1]);
      pair_digits(v0, v1, pi, JP, jinv, ku, A, aplane);
      const float sc = pow2f(-ku[mm[u]]);
      *(uint32_t *)(A + TC_P * aplane + sw32(TC_M, mm[u], kk[u] >> 3) + (kk[u] & 7) * 2) =
          pack_bf16(fabsf(v0.hi * sc), fabsf(v1.hi * sc));
    }
  }
}

// named barriers: 1 for the producer warps, 2 for the epilogue warps (the
// .red forms return the AND / OR of a predicate over the participants, so
// that a role leaves its loop together)
__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, 224;" ::: "memory"); }
__device__ __forceinline__ bool prod_all(bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, 1, 224, q;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(r)
               : "r"((uint32_t)v)
               : "memory");
  return r != 0;
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }
__device__ __forceinline__ bool epi_any(bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 2, 256, q;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(r)
               : "r"((uint32_t)v)
               : "memory");
  return r != 0;
}

// Columns of a block: two halves of 16, each holding H0 = 16 / R values of
// i with their R terms (column = il * R + r) and zero padding after them, so
// that an epilogue thread's half never splits an i.  B row n (block n / 32,
// column n mod 32) -> (i, r); false for a padding column.
template <int R>
__device__ __forceinline__ bool brow(const TcParams &tp, int n, int &i, int &r) {
  constexpr int H0 = 16 / R;
  const int cb = n >> 5, c = n & 31, h = c >> 4, cc = c & 15;
  r = cc % R;
  const int il = cc / R;
  const int nI = min(2 * H0, tp.p.NI - cb * 2 * H0), h0 = min(H0, (nI + 1) >> 1);
  i = cb * 2 * H0 + h * h0 + il;
  return il < H0 && il < (h == 0 ? h0 : nI - h0);
}

// |k| of a scale outside the certified window
__device__ __forceinline__ bool out_of_window(int k) { return k < -TC_WIN || k > TC_WIN; }

// FP64 recomputation of every output of element e by the 256 epilogue
// threads (et = 0..255): u_j, then t[r, i] = sum_j D[r, i, j] u_j, then
// R_k[e, i] = sum_r g_k[e, r] t[r, i]; each value by one thread in FP64
// (dot products of at most 64 terms, error far below 1e-12 S)
static __device__ __noinline__ void fallback_element(const EParams &p, int64_t e, int et, double *fu, double *ft) {
  const EProd &q = p.groups[0];
  if (et < p.NJ) {
    const double a = q.a.ptr[e * q.a.se + et * q.a.sk];
    double u = a;
    if (q.kind != 0) {
      const double b = q.b.ptr[e * q.b.se + et * q.b.sk];
      u = q.kind == 1 ? sin(a) * b : a * b;
    }
    fu[et] = u;
  }
  epi_sync();
  for (int n = et; n < p.R * p.NI; n += NEPI) {
    const int r = n / p.NI, i = n - r * p.NI;
    const double *d = p.D + r * p.sr + i * p.si;
    double s = 0.0;
    for (int j = 0; j < p.NJ; ++j) s = fma(d[j * p.sj], fu[j], s);
    ft[n] = s;
  }
  epi_sync();
  for (int o = et; o < p.n_rows * p.NI; o += NEPI) {
    const int k = o / p.NI, i = o - k * p.NI;
    double v = ft[i];
    if (p.has_g) {
      const EView &g = p.rows[k].g;
      v = 0.0;
      for (int r = 0; r < p.R; ++r) v = fma(g.ptr[e * g.se + r * g.sk], ft[r * p.NI + i], v);
    }
    p.rows[k].out[e * p.NI + i] = v;
  }
  epi_sync();
}

// the same for the stacked form (group grp, element e): v_k = sum_x A_x B_x
// in FP64 (k < K), t_i = sum_k D[i, k] v_k, written to every row of the
// group
static __device__ __noinline__ void fallback_stacked(const TcParams &tp, int grp, int64_t e, int et, double *fu,
                                                     double *ft) {
  const EParams &p = tp.p;
  const EProd &q = p.groups[grp];
  for (int k = et; k < p.NJ; k += NEPI) {
    const int s = k / p.NJ0, j = k - s * p.NJ0;
    double v = 0.0;
    for (int x = 0; x < q.X; ++x) v = fma(q.A[x].ptr[stk_off(q.A[x], e, s, j)], q.B[x].ptr[stk_off(q.B[x], e, s, j)], v);
    fu[k] = v;
  }
  epi_sync();
  for (int i = et; i < p.NI; i += NEPI) {
    double v = 0.0;
    for (int k = 0; k < p.NJ; ++k) v = fma(p.D[d_offset(p, 0, i, k)], fu[k], v);
    ft[i] = v;
  }
  epi_sync();
  const int r0 = tp.gstart[grp], nr = tp.gstart[grp + 1] - r0;
  for (int o = et; o < nr * p.NI; o += NEPI) {
    const int kk = o / p.NI, i = o - kk * p.NI;
    p.rows[tp.grow[r0 + kk]].out[e * p.NI + i] = ft[i];
  }
  epi_sync();
}

// ROWS: the number of einsums when specialized, 0 for any count up to 4;
// STK: the stacked form (R = 1, no g; tiles over producer groups x element
// tiles, each group's value written to each of its rows); NBUF: buffers of
// u's digit planes (1 where two do not fit in shared memory: the producer
// then waits for the MMAs of the tile before)
template <int R, int ROWS, bool STK, int NBUF>
__global__ void __launch_bounds__(TC_THREADS, 1) element_tc_kernel(const __grid_constant__ TcParams tp) {
  constexpr int H0 = 16 / R;                    // i per 16-column half of a block
  constexpr int KR = ROWS ? ROWS : TC_MAXROWS;  // einsums held per thread
  constexpr int IB = 2 * H0;                    // i per column block
  // planes per operand and tensor-memory columns per slot: the stacked form
  // adds a plane of bf16(|v|) and one of bf16(|D|), whose product sums into
  // an eighth accumulator sum_k |D_ik| |v_k| (a lower bound of S for the
  // per-output check, where one |t| alone would be a weak one)
  constexpr int NPL = STK ? TC_P + 1 : TC_P;
  constexpr int SLOT = STK ? TC_SLOT + TC_NCOL : TC_SLOT;
  const EParams &p = tp.p;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 255) & ~(uintptr_t)255);
  const TcSmem SL = tc_smem(tp);
  uint8_t *Bp = smem + SL.b;                                // [cb][ks][plane p][32 rows][32 B]
  uint8_t *Ap = smem + SL.a;                                // [buffer][plane q][ks][128 rows][32 B]
  float2 *sin_tab = (float2 *)(smem + SL.sin);              // half-circle sine table
  int *kD = (int *)(smem + SL.kD);                          // [NB] scale exponent of each row of D
  float *kDs = (float *)(smem + SL.kDs);                    // [NB] 2^kD
  float *zc = (float *)(smem + SL.zc);                      // [NB] check term F E_n 2^kD
  // Row scales of u for the last TC_KU tiles: the epilogue can trail the
  // producer by up to 2 + ceil(2 / ncb) tiles (two digit buffers ahead of
  // the MMAs, which run at most two column blocks ahead of the epilogue)
  int *kU = (int *)(smem + SL.kU);                          // [TC_KU][TC_M]
  int *mxw = (int *)(smem + SL.mxw);                        // [TC_M] high words of the row bounds
  uint32_t *fmask = (uint32_t *)(smem + SL.fm);             // [2][4] flagged elements of a tile
  double *fu = (double *)(smem + SL.fu);                    // [NJ] FP64 recomputation: u
  double *ft = (double *)(smem + SL.ft);                    // [R * NI] FP64 recomputation: t
  uint64_t *bars = (uint64_t *)(smem + SL.bars);
  uint64_t *a_full = bars, *a_empty = bars + 2, *s_full = bars + 4, *s_empty = bars + 6, *fin = bars + 8;
  uint32_t *tmem_slot = (uint32_t *)(smem + SL.misc);
  volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NJ = p.NJ, NI = p.NI;
  const int aplane = tp.KS * TC_M * 32;                     // bytes per digit plane of u
  const long long limit = tp.wait_limit;

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&a_full[b], NPROD);
      tc::mbar_init(&a_empty[b], 1);
      tc::mbar_init(&s_full[b], 1);
      tc::mbar_init(&s_empty[b], NEPI);
    }
    tc::mbar_init(fin, 1);
    *abort_flag = 0;
    for (int k = 0; k < 8; ++k) fmask[k] = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(tc::smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // zero both operand regions (K padding and padding rows stay zero)
  {
    uint4 *z = (uint4 *)smem;
    const int n16 = (int)(SL.a + NBUF * NPL * aplane) / 16;
    for (int k = tid; k < n16; k += TC_THREADS) z[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (uses_sin(p)) dfm::sin_half_table_fill(sin_tab, tid, TC_THREADS);
  // per row n of D: scale exponent, 2^k, and the check term
  //   zc = F 2^k (2^-46 (sum_j |D_nj| 2^-k + K) + 2^-42) (1 + 2^-20)
  // (0 for a row of zeros, which is exact; infinite for a row whose scale
  // leaves the window, so that every output using it is recomputed)
  for (int n = tid; n < tp.NB; n += TC_THREADS) {
    int i, r;
    int hw = 0;
    double sabs = 0.0;
    if (brow<R>(tp, n, i, r)) {
      for (int j = 0; j < NJ; ++j) {
        const double x = p.D[d_offset(p, r, i, j)];
        hw = max(hw, __double2hiint(x) & 0x7FFFFFFF);
        sabs += fabs(x);
      }
    }
    const int k = row_exp_hw(hw);
    kD[n] = k;
    kDs[n] = pow2f(k);
    float z = 0.0f;
    if (hw != 0) {
      if (out_of_window(k)) {
        z = __int_as_float(0x7F800000);
      } else {
        const double sd = sabs * ldexp(1.0, -k);
        z = (float)(tp.fcheck * ldexp(1.0, k) * (ldexp(sd + NJ, -46) + ldexp(1.0, -42)) * (1.0 + ldexp(1.0, -20)));
      }
    }
    zc[n] = z;
  }
  __syncthreads();
  // digit planes of D: item (row n, group g of 8 values of j)
  for (int item = tid; item < tp.NB * tp.NG; item += TC_THREADS) {
    const int n = item / tp.NG, g = item % tp.NG;
    int i, r;
    if (!brow<R>(tp, n, i, r)) continue;
    const int kn = kD[n];
    uint32_t w[NPL][4];
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) {
      float d0[TC_P], d1[TC_P];
      const int j = g * 8 + 2 * jp;
      const double x0 = j < NJ ? p.D[d_offset(p, r, i, j)] : 0.0, x1 = j + 1 < NJ ? p.D[d_offset(p, r, i, j + 1)] : 0.0;
      digits_bits(x0, kn, d0);
      digits_bits(x1, kn, d1);
#pragma unroll
      for (int q = 0; q < TC_P; ++q) w[q][jp] = pack_bf16(d0[q], d1[q]);
      if constexpr (STK)   // |D| 2^(8 - k_n), in the units of the digits' products
        w[TC_P][jp] = pack_bf16((float)(fabs(x0) * ldexp(1.0, 8 - kn)), (float)(fabs(x1) * ldexp(1.0, 8 - kn)));
    }
    const int cb = n >> 5, nl = n & 31, ks = g >> 1;
    const uint32_t base = (uint32_t)((cb * tp.KS + ks) * NPL) * TC_BPLANE + sw32_row(nl, g & 1);
#pragma unroll
    for (int q = 0; q < NPL; ++q)
      *(uint4 *)(Bp + base + q * TC_BPLANE) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;

  // tiles: element tiles, times the producer groups in the stacked form
  // (tile -> group tile % G, element tile tile / G)
  const int64_t n_tiles = (p.E + TC_M - 1) / TC_M * (STK ? tp.G : 1);
  int *status = tp.status;

  if (STK && warp < MMA_WARP) {
    // ------------------------------------------------------------ producer (stacked form)
    // Pass 1: per element the exponent bound of sum_x |A_x B_x| over k
    // (flat items (element, k) over all producer threads), which gives the
    // row scale 2^k_e (k_e = bound - 2044 + ceil(log2 X)); the a_empty wait
    // (a barrier of the producer warps) orders its atomics before the scales
    // are read.  Pass 2: v over pairs (k, k + 1) in double-float and its
    // digits.  Warp 0 prefetches the next tile's operands into L2.
    const int NJ0 = p.NJ0;
    const uint32_t sinv = ((1u << 20) + (uint32_t)NJ0 - 1u) / (uint32_t)NJ0;
    int t = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
      const int grp = (int)(tile % tp.G);
      const int64_t e0 = tile / tp.G * TC_M;
      const int te = (int)(p.E - e0 < TC_M ? p.E - e0 : TC_M);
      const EProd &q = p.groups[grp];
      const int xlog2 = q.X <= 1 ? 0 : (q.X <= 2 ? 1 : 2);
      if (warp == 0 && tile + gridDim.x < n_tiles) {       // the next tile's operands into L2
        const int64_t t1 = tile + gridDim.x, e1 = t1 / tp.G * TC_M;
        stk_prefetch(p.groups[(int)(t1 % tp.G)], e1, (int)(p.E - e1 < TC_M ? p.E - e1 : TC_M), NJ / NJ0, NJ0, lane);
      }
      if (tid < TC_M) mxw[tid] = 0;
      prod_sync();
      switch (q.X) {
        case 1: stk_rows_bound<1>(q, e0, te, NJ, NJ0, sinv, tid, mxw); break;
        case 2: stk_rows_bound<2>(q, e0, te, NJ, NJ0, sinv, tid, mxw); break;
        case 3: stk_rows_bound<3>(q, e0, te, NJ, NJ0, sinv, tid, mxw); break;
        default: stk_rows_bound<4>(q, e0, te, NJ, NJ0, sinv, tid, mxw); break;
      }
      const int ab = NBUF == 2 ? (t & 1) : 0;
      const uint32_t use = NBUF == 2 ? (uint32_t)(t >> 1) : (uint32_t)t;
      if (!prod_all(tc::mbar_wait(&a_empty[ab], (use & 1u) ^ 1u, abort_flag, status, limit))) break;
      int *ku = kU + (t & (TC_KU - 1)) * TC_M;
      if (tid < TC_M) ku[tid] = mxw[tid] == 0 ? KU_ZERO : min(100, max(-100, mxw[tid] - 2044 + xlog2));
      prod_sync();
      uint8_t *A = Ap + ab * NPL * aplane;
      const int JP = (NJ + 1) >> 1, np = te * JP;
      const uint32_t jinv = ((1u << 20) + (uint32_t)JP - 1u) / (uint32_t)JP;
      switch (q.X) {
        case 1: stk_pairs<1>(q, e0, np, JP, jinv, NJ, NJ0, sinv, ku, A, aplane, tid); break;
        case 2: stk_pairs<2>(q, e0, np, JP, jinv, NJ, NJ0, sinv, ku, A, aplane, tid); break;
        case 3: stk_pairs<3>(q, e0, np, JP, jinv, NJ, NJ0, sinv, ku, A, aplane, tid); break;
        default: stk_pairs<4>(q, e0, np, JP, jinv, NJ, NJ0, sinv, ku, A, aplane, tid); break;
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(&a_full[ab]);
    }
  } else if (warp < MMA_WARP) {
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
        if (p.has_g) prefetch_g(p, e1, te1);
      }
      if (tid < TC_M) mxw[tid] = 0;
      prod_sync();
      // RB rows per warp per round (a larger round, 10, measured 7 % slower)
      constexpr int NPW = NPROD / 32, RB = 4;
      for (int r0 = warp; r0 < te; r0 += NPW * RB) {
        int hw[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const int row = r0 + NPW * u;
          const bool okr = row < te;
          const int h0 = (okr && lane < NJ) ? bound_hw(q, e0 + row, lane) : 0;
          const int h1 = (okr && lane + 32 < NJ) ? bound_hw(q, e0 + row, lane + 32) : 0;
          hw[u] = max(h0, h1);
        }
#pragma unroll
        for (int u = 0; u < RB; ++u) {
          const int h = __reduce_max_sync(0xffffffffu, hw[u]);
          if (lane == 0 && r0 + NPW * u < te) mxw[r0 + NPW * u] = h;
        }
      }
      const int ab = NBUF == 2 ? (t & 1) : 0;
      const uint32_t use = NBUF == 2 ? (uint32_t)(t >> 1) : (uint32_t)t;
      if (!prod_all(tc::mbar_wait(&a_empty[ab], (use & 1u) ^ 1u, abort_flag, status, limit))) break;
      int *ku = kU + (t & (TC_KU - 1)) * TC_M;
      if (tid < TC_M) ku[tid] = mxw[tid] == 0 ? KU_ZERO : row_exp_hw(mxw[tid]);
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
        bool fast = true;
#pragma unroll
        for (int u = 0; u < PB; ++u)
          fast = fast && produce_fast_ok(q, av[4 * u], av[4 * u + 2]) && produce_fast_ok(q, av[4 * u + 1], av[4 * u + 3]);
        if (fast) {
#pragma unroll
          for (int u = 0; u < PB; ++u) {
            const int pi = p0 + u * NPROD;
            if (pi < np)
              pair_digits(produce_t<true>(q, av[4 * u], av[4 * u + 2], sin_tab),
                          produce_t<true>(q, av[4 * u + 1], av[4 * u + 3], sin_tab), pi, JP, jinv, ku, A, aplane);
          }
        } else {
          pairs_slow(q, rows, need_b, p0, PB, NPROD, np, JP, jinv, NJ, ku, A, aplane, sin_tab);
        }
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(&a_full[ab]);
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint64_t adesc0 = tc::sdesc_sw32(tc::smem_u32(Ap));
      const uint64_t bdesc0 = tc::sdesc_sw32(tc::smem_u32(Bp));
      int t = 0;
      int64_t cnt = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++t) {
        const int ab = NBUF == 2 ? (t & 1) : 0;
        const uint32_t use_a = NBUF == 2 ? (uint32_t)(t >> 1) : (uint32_t)t;
        if (!tc::mbar_wait(&a_full[ab], use_a & 1u, abort_flag, status, limit)) break;
        const uint64_t adesc = adesc0 + (uint64_t)((ab * NPL * aplane) >> 4);
        tc::fence_after();
        for (int cb = 0; cb < tp.ncb; ++cb, ++cnt) {
          const int slot = (int)(cnt & 1);
          const uint32_t use = (uint32_t)(cnt >> 1);
          if (!tc::mbar_wait(&s_empty[slot], (use & 1u) ^ 1u, abort_flag, status, limit)) { ok = false; break; }
          tc::fence_after();
          const uint32_t dslot = tmem + (uint32_t)(slot * SLOT);
          // descriptors differ only in the start-address field (bits 0-13,
          // address >> 4), which stays below 2^14 for every operand here
          for (int ks = 0; ks < tp.KS; ++ks) {
            const uint64_t bks = bdesc0 + (uint64_t)(((cb * tp.KS + ks) * NPL * TC_BPLANE) >> 4);
            const uint64_t aks = adesc + (uint64_t)((ks * TC_M * 32) >> 4);
            // u's digit q times D's planes p = 0 .. min(5, 6 - q) into the
            // accumulators of levels q .. q + p (32 columns apart); the first
            // MMA of a block overwrites levels 0..5, the level-6 accumulator
            // is started by its own MMA (q = 1, p = 5)
#pragma unroll
            for (int qd = 0; qd < TC_P; ++qd) {
              const uint64_t aq = aks + (uint64_t)((qd * aplane) >> 4);
              if (qd == 0) {
                tc::mma_bf16(dslot, aq, bks, tc::idesc_bf16(TC_M, 6 * TC_NCOL), ks > 0 ? 1u : 0u);
              } else if (qd == 1 && ks == 0) {
                tc::mma_bf16(dslot + 6 * TC_NCOL, aq, bks + (uint64_t)((5 * TC_BPLANE) >> 4), tc::idesc_bf16(TC_M, TC_NCOL), 0u);
                tc::mma_bf16(dslot + TC_NCOL, aq, bks, tc::idesc_bf16(TC_M, 5 * TC_NCOL), 1u);
              } else {
                const int np_ = qd == 1 ? 6 : 7 - qd;    // planes p = 0 .. np_ - 1
                tc::mma_bf16(dslot + (uint32_t)(qd * TC_NCOL), aq, bks, tc::idesc_bf16(TC_M, np_ * TC_NCOL), 1u);
              }
            }
            // stacked form: bf16(|v|) x bf16(|D|) into the eighth accumulator
            if constexpr (STK)
              tc::mma_bf16(dslot + (uint32_t)(TC_LEV * TC_NCOL), aks + (uint64_t)((TC_P * aplane) >> 4),
                           bks + (uint64_t)((TC_P * TC_BPLANE) >> 4), tc::idesc_bf16(TC_M, TC_NCOL), ks > 0 ? 1u : 0u);
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
    const int et = tid - (NPROD + 32);                      // 0..255
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * (TC_NCOL / 2));
    const int n_rows = p.n_rows;
    int t = 0;
    int64_t cnt = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
      const int grp = STK ? (int)(tile % tp.G) : 0;
      const int64_t e0 = (STK ? tile / tp.G : tile) * TC_M;
      const int64_t e = e0 + m;
      const bool valid = e < p.E;
      // g_k[e, r] of this thread's element as double-float (scaled by
      // 2^(k_e - 8) once the tile's exponents are known); g outside the
      // window flags the element
      df gk[KR][R];
      bool flag = false;
#pragma unroll
      for (int k = 0; k < KR; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const double g =
              (valid && (ROWS || k < n_rows)) ? (p.has_g ? p.rows[k].g.ptr[e * p.rows[k].g.se + r * p.rows[k].g.sk] : 1.0) : 0.0;
          const int hg = __double2hiint(g) & 0x7FFFFFFF;
          flag |= hg != 0 && out_of_window(((hg >> 20) & 0x7FF) - 1023);
          gk[k][r] = dfm::df_from_double(g);
        }
      bool zero_el = false;
      float mx = 0.0f;                                      // largest check value of this thread's outputs
      bool ok = true;
      for (int cb = 0; cb < tp.ncb; ++cb, ++cnt) {
        const int slot = (int)(cnt & 1);
        const uint32_t use = (uint32_t)(cnt >> 1);
        if (ok) ok = __all_sync(0xffffffffu, tc::mbar_wait(&s_full[slot], use & 1u, abort_flag, status, limit));
        if (!ok) continue;                                 // aborting: the tile-end barrier is still reached
        tc::fence_after();
        if (cb == 0) {
          const int ke = kU[(t & (TC_KU - 1)) * TC_M + m];
          zero_el = ke == KU_ZERO;
          flag |= !zero_el && out_of_window(ke);
          const float sg = pow2f(max(ke, -100) - 8);
#pragma unroll
          for (int k = 0; k < KR; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) gk[k][r] = df{gk[k][r].hi * sg, gk[k][r].lo * sg};
        }
        // i of this half (warp-uniform): a block's i split evenly between its
        // halves, the first taking the odd one
        const int nI = min(IB, NI - cb * IB), h0 = min(H0, (nI + 1) >> 1);
        const int nIh = half == 0 ? h0 : nI - h0;
        const int nch = (nIh * R + 7) >> 3;                      // 8-column chunks holding them
        const int nb = cb * TC_NCOL + half * (TC_NCOL / 2);      // first B row of this half
        // t for this half's columns: the 7 level accumulators of a column
        // added in double-float (levels 0-1 and 2-3 by TwoSum, the pairs
        // combined, levels 4-6 into the low part), times 2^k_n
        float th[16], tl[16];
        float sl[STK ? 16 : 1];                              // stacked form: sum_k |D_ik| |v_k|, same units as th
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          if (ch < nch) {
            uint32_t v[TC_LEV][8], vs[8];
            __syncwarp();   // tcgen05.ld is .sync.aligned: reconverge after lane-dependent work
#pragma unroll
            for (int L = 0; L < TC_LEV; ++L)
              tc::tmem_ld8(lane_base + (uint32_t)(slot * SLOT + L * TC_NCOL + ch * 8), v[L]);
            if constexpr (STK) tc::tmem_ld8(lane_base + (uint32_t)(slot * SLOT + TC_LEV * TC_NCOL + ch * 8), vs);
            tc::tmem_wait_ld();
            if (ch == nch - 1) {                               // this slot is drained
              tc::fence_before();
              tc::mbar_arrive(&s_empty[slot]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              if (ch * 8 + c >= H0 * R) continue;              // padding column of the half
              const df s01 = dfm::two_sum(__uint_as_float(v[0][c]), __uint_as_float(v[1][c]));
              const df s23 = dfm::two_sum(__uint_as_float(v[2][c]), __uint_as_float(v[3][c]));
              const float s46 = (__uint_as_float(v[4][c]) + __uint_as_float(v[5][c])) + __uint_as_float(v[6][c]);
              df s = dfm::two_sum(s01.hi, s23.hi);
              s.lo += (s01.lo + s23.lo) + s46;
              const df x = dfm::fast_two_sum(s.hi, s.lo);
              const float sc = kDs[nb + ch * 8 + c];
              th[ch * 8 + c] = x.hi * sc;
              tl[ch * 8 + c] = x.lo * sc;
              if constexpr (STK) sl[ch * 8 + c] = __uint_as_float(vs[c]) * sc;
            }
          }
        }
        if (nch == 0) {
          tc::fence_before();
          tc::mbar_arrive(&s_empty[slot]);
        }
        if (valid) {
#pragma unroll
          for (int il = 0; il < H0; ++il) {
            if (il < nIh) {
              const int i = cb * IB + half * h0 + il;
              // check terms of the R columns of this i
              float z[R];
#pragma unroll
              for (int r = 0; r < R; ++r) {
                // S >= |t|, and in the stacked form S >= sum_k |D_ik| |v_k|,
                // whose bf16 products summed in FP32 are within 2^-7 of it
                float lb = fabsf(th[il * R + r]);
                if constexpr (STK) lb = fmaxf(lb, sl[il * R + r] * (1.0f - 0x1p-6f));
                z[r] = zero_el ? 0.0f : zc[nb + il * R + r] - lb;
              }
#pragma unroll
              for (int k = 0; k < KR; ++k) {
                if (ROWS || k < n_rows) {
                  // first term: its exact product starts the pair (s, c)
                  const df g0 = gk[k][0], t0{th[il * R], tl[il * R]};
                  float s = g0.hi * t0.hi;
                  float c = fmaf(g0.hi, t0.lo, fmaf(g0.lo, t0.hi, fmaf(g0.hi, t0.hi, -s)));
                  float chk = fabsf(g0.hi) * z[0];
#pragma unroll
                  for (int r = 1; r < R; ++r) {
                    dfm::dot_acc(s, c, gk[k][r], df{th[il * R + r], tl[il * R + r]});
                    chk = fmaf(fabsf(gk[k][r].hi), z[r], chk);
                  }
                  mx = fmaxf(mx, chk);
                  // hi + lo: exact conversions by bit moves and one FP64 add
                  // (three FP64-pipe conversions measured 2 % slower: the
                  // pipe is shared with the producer's sine reduction)
                  const double o = dfm::f2d_bits(s) + dfm::f2d_bits(c);
                  if constexpr (STK) {
                    for (int kk = tp.gstart[grp]; kk < tp.gstart[grp + 1]; ++kk) p.rows[tp.grow[kk]].out[e * NI + i] = o;
                  } else {
                    p.rows[k].out[e * NI + i] = o;
                  }
                }
              }
            }
          }
        }
      }
      // tile end: flagged elements of this tile into the mask, then one
      // barrier of the epilogue warps (which also tells every warp whether
      // one of them gave up waiting)
      if (ok && valid && (flag || mx > 0.0f)) atomicOr(&fmask[(t & 1) * 4 + (m >> 5)], 1u << (m & 31));
      if (epi_any(!ok)) break;
      uint32_t fm[4];
#pragma unroll
      for (int w = 0; w < 4; ++w) fm[w] = fmask[(t & 1) * 4 + w];
      if (fm[0] | fm[1] | fm[2] | fm[3]) {
#pragma unroll 1
        for (int w = 0; w < 4; ++w) {
          while (fm[w]) {
            const int b = __ffs(fm[w]) - 1;
            fm[w] &= fm[w] - 1u;
            if constexpr (STK) fallback_stacked(tp, grp, e0 + w * 32 + b, et, fu, ft);
            else fallback_element(p, e0 + w * 32 + b, et, fu, ft);
          }
        }
        // cleared before this thread reaches the next tile-end barrier; the
        // next writer of this mask is two tiles on, past that barrier
        if (et == 0)
          for (int w = 0; w < 4; ++w) fmask[(t & 1) * 4 + w] = 0u;
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
  const bool stk = p.NJ0 > 0;
  if (stk) {
    // the stacked form: one group per distinct pair of per-element operands
    if (p.n_groups < 1 || p.n_groups > EM_MAXROWS) { why = "producer groups outside 1..16"; return false; }
    for (int g = 0; g < p.n_groups; ++g)
      if (p.groups[g].kind != 3 || p.groups[g].X < 1 || p.groups[g].X > EM_MAXX) { why = "stacked producer"; return false; }
    if (p.R != 1 || p.has_g) { why = "stacked form with R > 1 or a geometric factor"; return false; }
    if (p.n_rows < 1 || p.n_rows > EM_MAXROWS) { why = "rows outside 1..16"; return false; }
  } else {
    if (p.n_groups != 1) { why = "more than one fused operand"; return false; }
    if (p.groups[0].kind == 3) { why = "stacked producer without the stacked layout"; return false; }
    if (p.R < 1 || p.R > 4) { why = "R outside 1..4"; return false; }
    if (p.n_rows < 1 || p.n_rows > TC_MAXROWS) { why = "more than 4 einsums"; return false; }
    if (!p.has_g && p.R != 1) { why = "no geometric factor with R > 1"; return false; }
    const EProd &q = p.groups[0];
    const int64_t lim = (int64_t)1 << 23;   // in-tile offsets m * se + j * sk stay 32-bit
    if (std::abs(q.a.se) >= lim || std::abs(q.a.sk) >= lim || std::abs(q.b.se) >= lim || std::abs(q.b.sk) >= lim) {
      why = "operand strides too large";
      return false;
    }
  }
  if (p.NJ < 1 || p.NJ > 64) { why = "contracted extent outside 1..64"; return false; }
  if (p.NI < 1) { why = "empty output extent"; return false; }
  tp.p = p;
  tp.G = stk ? p.n_groups : 1;
  {
    int c = 0;
    for (int g = 0; g < tp.G; ++g) {
      tp.gstart[g] = (int8_t)c;
      for (int k = 0; k < p.n_rows; ++k)
        if (p.rows[k].group == g) tp.grow[c++] = (int8_t)k;
    }
    tp.gstart[tp.G] = (int8_t)c;
    if (c != p.n_rows) { why = "row groups"; return false; }
  }
  const int h0 = 16 / p.R;
  tp.IB = 2 * h0;
  tp.ncb = (p.NI + tp.IB - 1) / tp.IB;
  if (tp.ncb > TC_MAXCB) { why = "too many column blocks"; return false; }
  tp.NB = tp.ncb * TC_NCOL;
  tp.KS = (p.NJ + 15) / 16;
  tp.NG = (p.NJ + 7) / 8;
  // F = (1e-12 - 2^-43)^-1 (2^-43 covers the relative roundings: the
  // producer's double-float value of u, the level sums, the contraction
  // with g and the final conversion) times 1 + 2^-19 for the check's own
  // FP32 roundings and the df -> float view of g
  tp.fcheck = (1.0 + 1e-9) / (1e-12 - std::ldexp(1.0, -43)) * (1.0 + std::ldexp(1.0, -19));
  tp.wait_limit = tc::TIMEOUT_CYCLES;
  tp.status = nullptr;
  // two buffers of u's digit planes where they fit, else one (the stacked
  // form at K > 48: four K-slices of six planes take 96 KB per buffer)
  tp.npl = stk ? TC_P + 1 : TC_P;
  tp.nbuf = 2;
  if (stk && 256 + (size_t)tc_smem(tp).total > TC_SMEM_LIMIT) tp.nbuf = 1;
  return true;
}

size_t smem_bytes(const TcParams &tp) { return 256 + (size_t)tc_smem(tp).total; }

template <int R, int ROWS, bool STK, int NBUF>
cudaError_t launch_rr(const TcParams &tp, int grid, size_t smem, cudaStream_t s) {
  static std::atomic<uint64_t> attr{0};
  const cudaError_t st =
      smem_limit_once((const void *)element_tc_kernel<R, ROWS, STK, NBUF>, (int)TC_SMEM_LIMIT, attr);
  if (st != cudaSuccess) return st;
  return be_launch(element_tc_kernel<R, ROWS, STK, NBUF>, dim3(grid), dim3(TC_THREADS), smem, s, tp);
}
// one einsum per term direction (R einsums, as in a gradient) is
// specialized; other counts take the generic row loop
template <int R>
cudaError_t launch_r(const TcParams &tp, int grid, size_t smem, cudaStream_t s) {
  return tp.p.n_rows == R ? launch_rr<R, R, false, 2>(tp, grid, smem, s) : launch_rr<R, 0, false, 2>(tp, grid, smem, s);
}

}  // namespace

bool element_tc_supported(const EParams &p, std::string &why) {
  TcParams tp;
  if (!build_params(p, tp, why)) return false;
  if (smem_bytes(tp) > TC_SMEM_LIMIT) { why = "shared memory"; return false; }
  return true;
}

cudaError_t launch_element_tc(const EParams &p, int *status, long long wait_limit, cudaStream_t s) {
  TcParams tp;
  std::string why;
  if (!build_params(p, tp, why)) return cudaErrorInvalidValue;
  tp.status = status;
  if (wait_limit > 0) tp.wait_limit = wait_limit;
  const size_t smem = smem_bytes(tp);
  if (smem > TC_SMEM_LIMIT) return cudaErrorInvalidConfiguration;
  if (p.E <= 0) return cudaSuccess;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (p.E + TC_M - 1) / TC_M * tp.G;
  const int grid = (int)std::min<int64_t>(tiles, sms);
  if (p.NJ0 > 0)
    return tp.nbuf == 1 ? launch_rr<1, 1, true, 1>(tp, grid, smem, s) : launch_rr<1, 1, true, 2>(tp, grid, smem, s);
  switch (p.R) {
    case 1: return launch_r<1>(tp, grid, smem, s);
    case 2: return launch_r<2>(tp, grid, smem, s);
    case 3: return launch_r<3>(tp, grid, smem, s);
    default: return launch_r<4>(tp, grid, smem, s);
  }
}

}  // namespace be

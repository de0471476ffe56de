// Double-float ("df") arithmetic on the FP32 pipe: a value is an unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48 significant
// bits.  On B300 the FP64 pipe runs near 1.1 TFLOP/s while FP32 runs near
// 66 TFLOP/s, so FP64-accuracy work is done here in df.
//
// Building blocks (published error-free transformations): TwoSum (Knuth),
// Fast2Sum (Dekker, 1971) for |a| >= |b|, and TwoProd through a fused
// multiply-add (the product's rounding error is exactly fma(a, b, -p)).
// Sine (df_sin, used to fill the tables): Cody-Waite reduction by pi/2
// (pi/2 held in three floats; x - k*p1 with one FP64 fma, k*p2 formed
// exactly with TwoProd) followed by the Taylor series of sin or cos on
// |r| <= pi/4, the small high-order terms in plain float and the leading
// ones in df.  The constants are 1/k! and pi/2 rounded into float pairs
// (hex literals, derived with exact rational arithmetic).  The kernels use
// df_sin_tab2: reduction to a grid of pi/512 and the angle-addition formula
// with a full-circle table of sin(n pi/512).
#pragma once

#include <cstdint>

namespace be {
namespace dfm {

struct df {
  float hi, lo;
};

constexpr float PIO2_1 = 0x1.921fb60000000p+0f, PIO2_2 = -0x1.777a5c0000000p-25f, PIO2_3 = -0x1.ee59da0000000p-50f;
constexpr float TWO_OVER_PI = 0x1.45f3060000000p-1f;
// (-1)^n / (2n+1)!, n = 0..11, as (hi, lo)
static __device__ __constant__ float SIN_C[12][2] = {{0x1.0000000000000p+0f, 0.0f}, {-0x1.5555560000000p-3f, 0x1.5555560000000p-28f}, {0x1.1111120000000p-7f, -0x1.ddddde0000000p-32f}, {-0x1.a01a020000000p-13f, 0x1.7f97fa0000000p-39f}, {0x1.71de3a0000000p-19f, 0x1.55b1cc0000000p-45f}, {-0x1.ae64560000000p-26f, -0x1.fd51380000000p-52f}, {0x1.6124620000000p-33f, -0x1.8af25e0000000p-58f}, {-0x1.ae7f3e0000000p-41f, -0x1.ccee080000000p-67f}, {0x1.952c780000000p-49f, -0x1.f9ea560000000p-74f}, {-0x1.2f49b40000000p-57f, -0x1.a050560000000p-83f}, {0x1.71b8f00000000p-66f, -0x1.2461520000000p-91f}, {-0x1.761b420000000p-75f, 0x1.9d38fc0000000p-100f}};
// (-1)^n / (2n)!, n = 0..11, as (hi, lo)
static __device__ __constant__ float COS_C[12][2] = {{0x1.0000000000000p+0f, 0.0f}, {-0x1.0000000000000p-1f, 0.0f}, {0x1.5555560000000p-5f, -0x1.5555560000000p-30f}, {-0x1.6c16c20000000p-10f, 0x1.27d27e0000000p-35f}, {0x1.a01a020000000p-16f, -0x1.7f97fa0000000p-42f}, {-0x1.27e4fc0000000p-22f, 0x1.10ec140000000p-47f}, {0x1.1eed8e0000000p-29f, 0x1.ff1b120000000p-54f}, {-0x1.93974a0000000p-37f, -0x1.180f940000000p-62f}, {0x1.ae7f3e0000000p-45f, 0x1.ccee080000000p-71f}, {-0x1.6827860000000p-53f, -0x1.dcbecc0000000p-80f}, {0x1.e542ba0000000p-62f, 0x1.00808a0000000p-88f}, {-0x1.0ce3960000000p-70f, -0x1.b6ff0a0000000p-95f}};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b, bp = s - a;
  return df{s, (a - (s - bp)) + (b - bp)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = a + b;
  return df{s, b - (s - a)};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return df{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df x, df y) {
  df p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }

// x * y accumulated into the unnormalized pair (s, c): s carries the running
// sum of the leading products exactly through TwoSum, c the rounding errors
// and the cross terms; normalize with fast_two_sum(s, c) at the end
__device__ __forceinline__ void dot_acc(float &s, float &c, df x, df y) {
  const float p = x.hi * y.hi;
  const float pe = fmaf(x.hi, y.hi, -p);
  const float cr = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, pe));
  const float ns = s + p, bp = ns - s;
  c += ((s - (ns - bp)) + (p - bp)) + cr;
  s = ns;
}

// exact float -> double for normal floats and zero (integer bit moves, no
// FP64 instruction); other encodings go through the hardware conversion
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ef = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)(u >> 31) << 63);   // signed zero
  if (ef == 0u || ef == 0xFFu) return (double)f;
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  const uint64_t e = (uint64_t)(ef - 127u + 1023u);
  return __longlong_as_double((long long)(s | (e << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

// hi + lo as a double, by integer operations on the bits (no FP64
// instruction): hi's 24-bit significand fills the top of the 53-bit one and
// lo's is aligned below it and added or subtracted; bits of lo below the
// double's last place are dropped, so the result is within one unit in the
// last place of hi + lo.  Zeros and non-normal parts use the FP64 path.
__device__ __forceinline__ double df_to_double(df x) {
  const uint32_t uh = __float_as_uint(x.hi), ul = __float_as_uint(x.lo);
  const int eh = (int)((uh >> 23) & 0xFFu), el = (int)((ul >> 23) & 0xFFu);
  if (eh == 0 || eh == 0xFF || (ul & 0x7FFFFFFFu) == 0u) return f2d(x.hi) + f2d(x.lo);
  if (el == 0 || el == 0xFF) return f2d(x.hi) + f2d(x.lo);
  const int64_t mh = (int64_t)((uh & 0x7FFFFFu) | 0x800000u) << 29;   // value mh * 2^(eh-127-52)
  const int sh = 29 - (eh - el);                                       // lo's alignment
  int64_t ml = (int64_t)((ul & 0x7FFFFFu) | 0x800000u);
  ml = sh >= 0 ? (ml << sh) : (sh > -40 ? (ml >> (-sh)) : 0);
  int64_t m = ((uh ^ ul) >> 31) ? mh - ml : mh + ml;
  int e = eh - 127 + 1023;
  if (m >= (1ll << 53)) {
    m >>= 1;
    ++e;
  } else if (m < (1ll << 52)) {
    m <<= 1;
    --e;
  }
  const uint64_t sign = (uint64_t)(uh >> 31) << 63;
  return __longlong_as_double((long long)(sign | ((uint64_t)e << 52) | ((uint64_t)m & 0xFFFFFFFFFFFFFull)));
}

// double -> df for zeros, non-normal parts and out-of-range exponents: the
// FP64 conversions, kept out of line so that callers' hot code stays small
static __device__ __noinline__ df df_from_double_slow(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}

// double -> df with |x - hi - lo| <= 2^-48 |x|, by 32-bit integer operations
// on the two halves of the bits when both parts land in FP32's normal range
// (2^-70 <= |x| < 2^101): hi keeps the top 24 significand bits rounded half
// up (a carry into the exponent is the exact rounding), lo is the signed
// remainder, rem * 2^(e - 1075), rounded to a float
__device__ __forceinline__ df df_from_double(double x) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const uint32_t ax = hw & 0x7FFFFFFFu;
  if (ax - ((1023u - 70u) << 20) >= (171u << 20)) return df_from_double_slow(x);
  const uint32_t rnd = (lw >> 28) & 1u;
  const uint32_t hb = ((ax - (896u << 20)) << 3) + (lw >> 29) + rnd;
  const float hi = __uint_as_float(hb | (hw & 0x80000000u));
  const int rem = (int)(lw & 0x1FFFFFFFu) - (int)(rnd << 29);
  const float lo = (float)rem * __uint_as_float((uint32_t)((int)(ax >> 20) - 948) << 23);
  return df{hi, (int)hw < 0 ? -lo : lo};
}

// the same without the range test, for callers that tested the range
// beforehand (df_fast_ok): valid for zero and 2^-70 <= |x| < 2^101; zero is
// handled by selects, so the code has no branch
__device__ __forceinline__ df df_from_double_fast(double x) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const uint32_t ax = hw & 0x7FFFFFFFu;
  const uint32_t rnd = (lw >> 28) & 1u;
  const uint32_t hb = ((ax - (896u << 20)) << 3) + (lw >> 29) + rnd;
  const float hi = __uint_as_float(hb | (hw & 0x80000000u));
  const int rem = (int)(lw & 0x1FFFFFFFu) - (int)(rnd << 29);
  const float lo = (float)rem * __uint_as_float((uint32_t)((int)(ax >> 20) - 948) << 23);
  const bool z = ax == 0u;
  return df{z ? 0.f : hi, z ? 0.f : ((int)hw < 0 ? -lo : lo)};
}
// x is zero or in df_from_double's exact range
__device__ __forceinline__ bool df_fast_ok(double x) {
  const uint32_t ax = (uint32_t)__double2hiint(x) & 0x7FFFFFFFu;
  return ax == 0u || ax - ((1023u - 70u) << 20) < (171u << 20);
}

// sin(x) as df; |x| < 2^20 (the reduction's exact range), else FP64 sin
__device__ __forceinline__ df df_sin(double x) {
  // |x| < 2^20 (and finite), tested on the exponent bits
  if ((int)((__double_as_longlong(x) >> 52) & 0x7FF) >= 1023 + 20) return df_from_double(sin(x));
  const float k = rintf(df_from_double(x).hi * TWO_OVER_PI);
  // r = x - k * (p1 + p2 + p3): k * p1 is exact in FP64 (45 bits), so one FP64
  // fma gives x - k p1 rounded once; the smaller pieces follow in df
  df r = df_from_double(fma(-f2d(k), f2d(PIO2_1), x));
  r = df_add(r, df_neg(two_prod(k, PIO2_2)));
  r = df_add(r, df{-k * PIO2_3, 0.f});
  const int q = ((int)k) & 3;
  const df x2 = df_mul(r, r);
  df p;
  if (q & 1) {               // cos(r) = sum (-1)^n r^(2n) / (2n)!
    float t = COS_C[11][0];
    for (int n = 10; n >= 6; --n) t = fmaf(t, x2.hi, COS_C[n][0]);
    p = df{t, 0.f};
    for (int n = 5; n >= 0; --n) p = df_add(df_mul(p, x2), df{COS_C[n][0], COS_C[n][1]});
  } else {                   // sin(r) = r * sum (-1)^n r^(2n) / (2n+1)!
    float t = SIN_C[11][0];
    for (int n = 10; n >= 5; --n) t = fmaf(t, x2.hi, SIN_C[n][0]);
    p = df{t, 0.f};
    for (int n = 4; n >= 0; --n) p = df_add(df_mul(p, x2), df{SIN_C[n][0], SIN_C[n][1]});
    p = df_mul(p, r);
  }
  return (q & 2) ? df_neg(p) : p;
}

// FP64 sine of an argument outside the double-float range, kept out of line
// so that the callers' hot code stays small
static __device__ __noinline__ df sin_far(double x) { return df_from_double(sin(x)); }

// Full-circle table: sin(n pi / 512) for n = 0..1023 as (hi, lo); cos of a
// grid point is the entry a quarter turn (256) ahead.  Filled from the first
// quadrant by symmetry, so every entry comes from an argument in [0, pi/2].
constexpr int SIN2_N = 1024;
constexpr double PI512_HI = 0x1.921fb54442d18p-8;                // pi / 512, leading double
constexpr double PI512_LO = 0x1.1a62633145c07p-62;               // pi / 512 - PI512_HI
__device__ __forceinline__ void sin2_table_fill(float2 *tab) {
  for (int n = threadIdx.x; n < SIN2_N; n += blockDim.x) {
    const int m = n & 511, mm = m <= 256 ? m : 512 - m;
    const df s = df_sin((double)mm * PI512_HI);
    tab[n] = n < 512 ? make_float2(s.hi, s.lo) : make_float2(-s.hi, -s.lo);
  }
}

// sin(x) as df from the full-circle table (|x| < 2^20, else FP64 sin):
// x = n pi / 512 + d with |d| <= pi / 1024 (two FP64 fmas), then
// sin x = sin(n pi/512) cos d + cos(n pi/512) sin d with short series in d
__device__ __forceinline__ df df_sin_tab2(double x, const float2 *tab) {
  if ((int)((__double_as_longlong(x) >> 52) & 0x7FF) >= 1023 + 20) return sin_far(x);
  // n = round(x * 512 / pi): adding 1.5 * 2^52 rounds to an integer held in
  // the low word of the sum (|x| < 2^20 keeps |n| far below 2^31)
  const double nm = fma(x, 162.97466172610083, 6755399441055744.0);
  const int n = __double2loint(nm);
  const double nd = nm - 6755399441055744.0;
  const double dr = fma(-nd, PI512_LO, fma(-nd, PI512_HI, x));
  const df d = df_from_double(dr);
  const float d2 = d.hi * d.hi;
  // sin d = d - d^3/6 + d^5/120 (the cubic and quintic terms in float are
  // below 2^-28 and 2^-48 of one)
  const df sd = fast_two_sum(d.hi, fmaf(d.hi * d2, fmaf(d2, 1.f / 120.f, -1.f / 6.f), d.lo));
  // cos d = 1 - d^2/2 + d^4/24 with d^2 exact as a pair
  const df p = two_prod(d.hi, d.hi);
  const df c1 = fast_two_sum(1.f, -0.5f * p.hi);
  const df cd = fast_two_sum(c1.hi, c1.lo + fmaf(-d.hi, d.lo, fmaf(p.hi, p.hi * (1.f / 24.f), -0.5f * p.lo)));
  const float2 s0 = tab[n & (SIN2_N - 1)], c0 = tab[(n + SIN2_N / 4) & (SIN2_N - 1)];
  return df_add(df_mul(df{s0.x, s0.y}, cd), df_mul(df{c0.x, c0.y}, sd));
}

// df_sin_tab2 without the range test: |x| < 2^20 (sin_fast_ok), and the
// reduced argument converted without its range test (it is zero or at least
// 2^-70 whenever it matters: a reduced argument below 2^-70 is replaced by
// zero, an absolute change far below the result's rounding)
__device__ __forceinline__ df df_sin_tab2_fast(double x, const float2 *tab) {
  const double nm = fma(x, 162.97466172610083, 6755399441055744.0);
  const int n = __double2loint(nm);
  const double nd = nm - 6755399441055744.0;
  const double dr = fma(-nd, PI512_LO, fma(-nd, PI512_HI, x));
  const uint32_t adr = (uint32_t)__double2hiint(dr) & 0x7FFFFFFFu;
  const df d = df_from_double_fast(adr < ((1023u - 70u) << 20) ? 0.0 : dr);
  const float d2 = d.hi * d.hi;
  const df sd = fast_two_sum(d.hi, fmaf(d.hi * d2, fmaf(d2, 1.f / 120.f, -1.f / 6.f), d.lo));
  const df p = two_prod(d.hi, d.hi);
  const df c1 = fast_two_sum(1.f, -0.5f * p.hi);
  const df cd = fast_two_sum(c1.hi, c1.lo + fmaf(-d.hi, d.lo, fmaf(p.hi, p.hi * (1.f / 24.f), -0.5f * p.lo)));
  const float2 s0 = tab[n & (SIN2_N - 1)], c0 = tab[(n + SIN2_N / 4) & (SIN2_N - 1)];
  return df_add(df_mul(df{s0.x, s0.y}, cd), df_mul(df{c0.x, c0.y}, sd));
}
// Half-circle table: sin(n pi / 512) for n = 0..511 as (hi, lo); an index
// n of the full circle reads entry n mod 512 and negates it when bit 9 of n
// is set (sin(x + pi) = -sin x).  Half the shared memory of the full table
// for two extra logic operations per lookup.
constexpr int SINH_N = 512;
__device__ __forceinline__ void sin_half_table_fill(float2 *tab, int tid, int nthreads) {
  for (int n = tid; n < SINH_N; n += nthreads) {
    const int mm = n <= 256 ? n : 512 - n;
    const df s = df_sin((double)mm * PI512_HI);
    tab[n] = make_float2(s.hi, s.lo);
  }
}
__device__ __forceinline__ df sin_half_entry(const float2 *tab, int n) {
  const float2 v = tab[n & (SINH_N - 1)];
  const uint32_t sg = ((uint32_t)n << 22) & 0x80000000u;   // bit 9 of n -> sign
  return df{__uint_as_float(__float_as_uint(v.x) ^ sg), __uint_as_float(__float_as_uint(v.y) ^ sg)};
}
// df_sin_tab2_fast on the half-circle table (|x| < 2^20, sin_fast_ok)
__device__ __forceinline__ df df_sin_half_fast(double x, const float2 *tab) {
  const double nm = fma(x, 162.97466172610083, 6755399441055744.0);
  const int n = __double2loint(nm);
  const double nd = nm - 6755399441055744.0;
  const double dr = fma(-nd, PI512_LO, fma(-nd, PI512_HI, x));
  const uint32_t adr = (uint32_t)__double2hiint(dr) & 0x7FFFFFFFu;
  const df d = df_from_double_fast(adr < ((1023u - 70u) << 20) ? 0.0 : dr);
  const float d2 = d.hi * d.hi;
  const df sd = fast_two_sum(d.hi, fmaf(d.hi * d2, fmaf(d2, 1.f / 120.f, -1.f / 6.f), d.lo));
  const df p = two_prod(d.hi, d.hi);
  const df c1 = fast_two_sum(1.f, -0.5f * p.hi);
  const df cd = fast_two_sum(c1.hi, c1.lo + fmaf(-d.hi, d.lo, fmaf(p.hi, p.hi * (1.f / 24.f), -0.5f * p.lo)));
  const df s0 = sin_half_entry(tab, n), c0 = sin_half_entry(tab, n + SINH_N / 2);
  return df_add(df_mul(s0, cd), df_mul(c0, sd));
}
// the tested form: FP64 sine beyond the reduction's exact range
__device__ __forceinline__ df df_sin_half(double x, const float2 *tab) {
  if ((int)((__double_as_longlong(x) >> 52) & 0x7FF) >= 1023 + 20) return sin_far(x);
  const double nm = fma(x, 162.97466172610083, 6755399441055744.0);
  const int n = __double2loint(nm);
  const double nd = nm - 6755399441055744.0;
  const double dr = fma(-nd, PI512_LO, fma(-nd, PI512_HI, x));
  const df d = df_from_double(dr);
  const float d2 = d.hi * d.hi;
  const df sd = fast_two_sum(d.hi, fmaf(d.hi * d2, fmaf(d2, 1.f / 120.f, -1.f / 6.f), d.lo));
  const df p = two_prod(d.hi, d.hi);
  const df c1 = fast_two_sum(1.f, -0.5f * p.hi);
  const df cd = fast_two_sum(c1.hi, c1.lo + fmaf(-d.hi, d.lo, fmaf(p.hi, p.hi * (1.f / 24.f), -0.5f * p.lo)));
  const df s0 = sin_half_entry(tab, n), c0 = sin_half_entry(tab, n + SINH_N / 2);
  return df_add(df_mul(s0, cd), df_mul(c0, sd));
}

// exact float -> double of a normal float or zero by integer operations
// (the 8-bit exponent rebased by 1023 - 127 = 896 in the high word, the
// significand's low 3 bits moved to the top of the low word); subnormal,
// infinite and NaN floats take the hardware conversion
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f), a = u & 0x7FFFFFFFu;
  const uint32_t ef = a >> 23;
  if (ef == 0u || ef == 0xFFu) return a == 0u ? __hiloint2double((int)(u & 0x80000000u), 0) : (double)f;
  return __hiloint2double((int)((u & 0x80000000u) | ((a >> 3) + (896u << 20))), (int)(u << 29));
}

// |x| < 2^20 (and finite): the range of df_sin_tab2_fast
__device__ __forceinline__ bool sin_fast_ok(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF) < 1023 + 20;
}

}  // namespace dfm
}  // namespace be
